// Build-time generator of the bitsliced encode kernels (bitslice.cu).
//
// For each code listed in kSpecs it builds the encode matrix with the
// library's own construction (code.cpp: G for the non-systematic form, the
// parity rows G'' of G' = G G~^-1 for the systematic form, Sec. 3.1-3.3) and
// writes, for every dense block of rows sharing the same inputs (at most 8
// rows), a straight-line XOR schedule:
//
//   multiplication by a constant c is the 8x8 bit matrix M_c whose column j
//   holds the bits of c * 2^j; with the input byte column cut into eight bit
//   planes p0..p7, output plane i of c*x is the XOR of the planes j with
//   M_c[i][j] = 1.  Splitting j into 0..3 and 4..7, every such XOR is
//   Q[a] ^ R[b] where Q (R) holds the XORs of all subsets of p0..p3
//   (p4..p7) and a, b are the two nibbles of row i of M_c.
//
// The output is a header of __device__ functions, one per block, plus a
// table mapping (n, k, construction, form) to its kernel.  Usage:
//   gen_bitslice <main.cuh> <k12.cuh> <k16.cuh>
#include <algorithm>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "bs_emit.h"
#include "code.h"
#include "gf256.h"

using namespace pmrc;

namespace {

struct Spec {
  int n, k, construction, form, d;
};

// the codes of the benchmarked workloads (n = 2k, d = 2k-2 for the PM codes;
// construction 2 is PM-MBR, 3 the Reed-Solomon baseline with d = k).  Group 0
// goes to the main header; the two large sparse systematic codes (k = 12 and
// 16, thousands of coefficients each) get headers of their own, compiled as
// separate translation units in parallel with the rest.
const Spec kSpecs[] = {
    {16, 8, 1, 1, 14}, {16, 8, 0, 0, 14}, {8, 4, 1, 1, 6}, {6, 3, 1, 1, 4},
    {6, 3, 0, 0, 4},   {16, 8, 2, 1, 14}, {16, 8, 3, 1, 8}, {24, 12, 1, 1, 22},
    {32, 16, 1, 1, 30},
};
const int kGroup[] = {0, 0, 0, 0, 0, 0, 0, 1, 2};
constexpr int kGroups = 3;


uint64_t fnv(const std::vector<uint8_t> &v) {
  uint64_t h = 1469598103934665603ull;
  for (uint8_t b : v) {
    h ^= b;
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

int main(int argc, char **argv) {
  if (argc != 1 + kGroups) {
    fprintf(stderr, "usage: gen_bitslice <main.cuh> <group1.cuh> <group2.cuh>\n");
    return 2;
  }
  std::vector<FILE *> out(kGroups);
  for (int g = 0; g < kGroups; g++) {
    out[g] = fopen(argv[1 + g], "w");
    if (!out[g]) return 1;
    fprintf(out[g], "// generated by gen_bitslice.cpp -- do not edit\n#pragma once\n\n");
  }
  FILE *f = out[0];
  std::string table;
  int nspec = 0;
  for (size_t si = 0; si < sizeof kSpecs / sizeof kSpecs[0]; si++) {
    const Spec &s = kSpecs[si];
    FILE *fg = out[kGroup[si]];
    CodeMatrices c;
    std::string err;
    if (build_code(s.n, s.k, s.d, s.construction, s.form, c, err)) {
      fprintf(stderr, "gen_bitslice: %s\n", err.c_str());
      return 1;
    }
    // K data blocks (k alpha for PM-MSR, k Delta for PM-MBR); the systematic
    // form encodes the rows of the nodes after the first k
    const int a = c.alpha, K = c.K, N = c.N;
    const int first = s.form ? s.k * a : 0;
    const int rows = N - first;
    std::vector<uint8_t> M((size_t)rows * K);
    for (int r = 0; r < rows; r++)
      for (int q = 0; q < K; q++) M[(size_t)r * K + q] = c.Gcode.at(first + r, q);
    // blocks: rows grouped by identical support, cut into <= 8 rows
    const std::vector<BsBlock> blks = bs_blocks_by_support(M.data(), rows, K);
    if (blks.size() > (size_t)kBsEmitMaxBlocks) {
      fprintf(stderr, "gen_bitslice: code %d/%d has %zu blocks (at most %d)\n", s.n, s.k,
              blks.size(), kBsEmitMaxBlocks);
      return 1;
    }
    const std::string name = "bs_n" + std::to_string(s.n) + "_k" + std::to_string(s.k) + "_c" +
                             std::to_string(s.construction) + "_f" + std::to_string(s.form);
    const BsEmitted em = bs_emit_kernel(M.data(), rows, K, blks, name, false);
    fputs(em.code.c_str(), fg);
    fprintf(fg, "extern const int %s_cost[] = {", name.c_str());
    for (size_t i = 0; i < em.cost.size(); i++) fprintf(fg, "%s%d", i ? ", " : "", em.cost[i]);
    fprintf(fg, "};\n\n");
    if (kGroup[si] != 0)  // defined in its own translation unit
      fprintf(f, "__global__ void %s(const __grid_constant__ BsArgs a);\nextern const int %s_cost[];\n\n",
              name.c_str(), name.c_str());
    const long long xors = em.xors;
    char buf[256];
    snprintf(buf, sizeof buf, "    {%d, %d, %d, %d, %zu, %d, %d, 0x%016llxull, %lldll, %s, %s_cost},\n",
             s.n, s.k, s.construction, s.form, blks.size(), K, rows,
             (unsigned long long)fnv(M), xors, name.c_str(), name.c_str());
    table += buf;
    nspec++;
  }
  fprintf(f, "static const BsKernel kBsKernels[] = {\n%s};\nstatic const int kBsNumKernels = %d;\n",
          table.c_str(), nspec);
  for (FILE *fg : out) fclose(fg);
  return 0;
}
