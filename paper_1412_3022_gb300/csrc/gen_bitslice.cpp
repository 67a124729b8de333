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
//   gen_bitslice <out.cuh>
#include <algorithm>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "code.h"
#include "gf256.h"

using namespace pmrc;

namespace {

struct Spec {
  int n, k, construction, form, d;
};

// the codes of the benchmarked workloads (n = 2k, d = 2k-2 for the PM codes;
// construction 2 is PM-MBR, 3 the Reed-Solomon baseline with d = k)
const Spec kSpecs[] = {
    {16, 8, 1, 1, 14}, {16, 8, 0, 0, 14}, {8, 4, 1, 1, 6}, {6, 3, 1, 1, 4},
    {6, 3, 0, 0, 4},   {16, 8, 2, 1, 14}, {16, 8, 3, 1, 8},
};

constexpr int kRows = 8;    // rows per block (8 x 8 bit-plane accumulators)
constexpr int kAhead = 4;   // inputs prefetched ahead (bitslice.cu: kBsAhead)
constexpr int kSlots = 5;   // staging ring slots (bitslice.cu: kBsSlots)
constexpr int kMaxBlocks = 32;  // bitslice.cu: kBsMaxBlocks

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
  if (argc != 2) {
    fprintf(stderr, "usage: gen_bitslice <out.cuh>\n");
    return 2;
  }
  FILE *f = fopen(argv[1], "w");
  if (!f) return 1;
  fprintf(f, "// generated by gen_bitslice.cpp -- do not edit\n#pragma once\n\n");
  std::string table;
  int nspec = 0;
  for (const Spec &s : kSpecs) {
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
    // blocks: rows grouped by identical support, cut into <= kRows rows
    std::map<std::vector<int>, std::vector<int>> groups;
    std::vector<std::vector<int>> order;
    for (int r = 0; r < rows; r++) {
      std::vector<int> sup;
      for (int q = 0; q < K; q++)
        if (M[(size_t)r * K + q]) sup.push_back(q);
      if (!groups.count(sup)) order.push_back(sup);
      groups[sup].push_back(r);
    }
    struct Blk {
      std::vector<int> rows, inputs;
    };
    std::vector<Blk> blks;
    for (auto &sup : order) {
      auto &rs = groups[sup];
      const int nb = (int)((rs.size() + kRows - 1) / kRows);
      for (int b = 0; b < nb; b++) {
        Blk B;
        B.rows.assign(rs.begin() + rs.size() * b / nb, rs.begin() + rs.size() * (b + 1) / nb);
        B.inputs = sup;
        blks.push_back(B);
      }
    }
    const std::string name = "bs_n" + std::to_string(s.n) + "_k" + std::to_string(s.k) + "_c" +
                             std::to_string(s.construction) + "_f" + std::to_string(s.form);
    int64_t xors = 0;
    std::vector<int> blk_ops(blks.size(), 0);  // accumulate instructions per block
    for (size_t b = 0; b < blks.size(); b++) {
      const Blk &B = blks[b];
      fprintf(f, "// %s block %zu: %zu rows x %zu inputs\n", name.c_str(), b, B.rows.size(),
              B.inputs.size());
      {  // the block's input columns, read by the prefetch in the loop below
        std::string cols;
        for (size_t i = 0; i < B.inputs.size(); i++) cols += (i ? ", " : "") + std::to_string(B.inputs[i]);
        fprintf(f, "__constant__ uint8_t %s_b%zu_in[%zu] = {%s};\n", name.c_str(), b, B.inputs.size(), cols.c_str());
      }
      fprintf(f,
              "__device__ __forceinline__ void %s_b%zu(const BsCtx &x, uint32_t (&acc)[8][8]) "
              "{\n",
              name.c_str(), b);
      fprintf(f, "  uint32_t Q[16], R[16];\n");
      const int C = (int)B.inputs.size();
      // one loop over the inputs: prefetch, transpose and subset tables are
      // emitted once; only the accumulate XORs differ per input (a switch),
      // which keeps a block's code at about half its fully unrolled size.
      // Short blocks commit empty groups so the wait count stays kAhead - 1.
      fprintf(f, "  const uint8_t *in = %s_b%zu_in;\n", name.c_str(), b);
      for (int i = 0; i < kAhead; i++)
        if (i < C) fprintf(f, "  bs_prefetch(x, %d, %d);\n", B.inputs[i], i % kSlots);
        else fprintf(f, "  bs_commit_empty();\n");
      fprintf(f, "#pragma unroll 1\n  for (int i = 0; i < %d; i++) {\n", C);
      fprintf(f, "    bs_wait<%d>();\n    bs_planes(x, i %% %d, Q, R);\n", kAhead - 1, kSlots);
      fprintf(f, "    if (i + %d < %d) bs_prefetch(x, in[i + %d], (i + %d) %% %d); else bs_commit_empty();\n",
              kAhead, C, kAhead, kAhead, kSlots);
      fprintf(f, "    switch (i) {\n");
      for (int i = 0; i < C; i++) {
        fprintf(f, "    case %d:\n", i);
        const int col = B.inputs[i];
        for (size_t q = 0; q < B.rows.size(); q++) {
          const uint8_t cf = M[(size_t)B.rows[q] * K + col];
          for (int bit = 0; bit < 8; bit++) {
            int lo = 0, hi = 0;  // row `bit` of M_cf, split in two nibbles
            for (int j = 0; j < 8; j++) {
              const uint8_t colj = gf_mul_sr(cf, (uint8_t)(1u << j));
              if ((colj >> bit) & 1) {
                if (j < 4)
                  lo |= 1 << j;
                else
                  hi |= 1 << (j - 4);
              }
            }
            if (lo && hi) {
              fprintf(f, "      acc[%zu][%d] ^= Q[%d] ^ R[%d];\n", q, bit, lo, hi);
              xors += 2;
              blk_ops[b]++;
            } else if (lo) {
              fprintf(f, "      acc[%zu][%d] ^= Q[%d];\n", q, bit, lo);
              xors += 1;
              blk_ops[b]++;
            } else if (hi) {
              fprintf(f, "      acc[%zu][%d] ^= R[%d];\n", q, bit, hi);
              xors += 1;
              blk_ops[b]++;
            }
          }
        }
        fprintf(f, "      break;\n");
      }
      fprintf(f, "    default: break;\n    }\n  }\n");
      fprintf(f, "}\n\n");
    }
    // persistent kernel, one CTA per SM: CTAs [cta_start[b], cta_start[b+1])
    // all run block b, so an SM only ever holds one block's straight-line
    // code, fetched once and then re-executed from its instruction caches;
    // inside the group the warps take 1 KiB column tiles in turn
    fprintf(f, "__global__ void __launch_bounds__(kBsThreads, 1) %s(const __grid_constant__ BsArgs a) {\n",
            name.c_str());
    fprintf(f, "  int b = 0;\n  while (b + 1 < %zu && blockIdx.x >= a.cta_start[b + 1]) b++;\n",
            blks.size());
    fprintf(f, "  const uint32_t c = blockIdx.x - a.cta_start[b], cnt = a.cta_start[b + 1] - a.cta_start[b];\n");
    fprintf(f, "  const uint32_t nunits = (uint32_t)((a.nbytes + kBsUnit - 1) / kBsUnit);\n");
    fprintf(f, "  for (uint32_t u = (threadIdx.x / 32) * cnt + c; u < nunits; u += cnt * (kBsThreads / 32)) {\n");
    fprintf(f, "    BsCtx x;\n    if (!bs_ctx(a, x, u)) continue;\n    uint32_t acc[8][8];\n");
    fprintf(f, "    bs_zero(acc);\n    switch (b) {\n");
    for (size_t b = 0; b < blks.size(); b++) {
      const Blk &B = blks[b];
      fprintf(f, "      case %zu: {\n        %s_b%zu(x, acc);\n", b, name.c_str(), b);
      for (size_t q = 0; q < B.rows.size(); q++)
        fprintf(f, "        bs_store(x, %d, acc[%zu]);\n", K + B.rows[q], q);
      fprintf(f, "      } break;\n");
    }
    fprintf(f, "      default: break;\n    }\n  }\n}\n\n");
    // relative cost of each block (instructions per tile, roughly): input
    // transposes and subset tables, output transposes, accumulate XORs
    fprintf(f, "static const int %s_cost[] = {", name.c_str());
    for (size_t b = 0; b < blks.size(); b++)
      fprintf(f, "%s%d", b ? ", " : "", (int)(blk_ops[b] + 100 * blks[b].inputs.size() + 70 * blks[b].rows.size()));
    fprintf(f, "};\n\n");
    if (blks.size() > (size_t)kMaxBlocks) {
      fprintf(stderr, "gen_bitslice: %s has %zu blocks (at most %d)\n", name.c_str(), blks.size(), kMaxBlocks);
      return 1;
    }
    char buf[256];
    snprintf(buf, sizeof buf, "    {%d, %d, %d, %d, %zu, %d, %d, 0x%016llxull, %lldll, %s, %s_cost},\n",
             s.n, s.k, s.construction, s.form, blks.size(), K, rows,
             (unsigned long long)fnv(M), (long long)xors, name.c_str(), name.c_str());
    table += buf;
    nspec++;
  }
  fprintf(f, "static const BsKernel kBsKernels[] = {\n%s};\nstatic const int kBsNumKernels = %d;\n",
          table.c_str(), nspec);
  fclose(f);
  return 0;
}
