// Bitsliced schedule emitter (see bs_emit.h).
#include "bs_emit.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>

#include "gf256.h"

namespace pmrc {

namespace {

constexpr int kAhead = 4;  // inputs prefetched ahead (bitslice_dev.cuh: kBsAhead)
constexpr int kSlots = 5;  // staging ring slots (bitslice_dev.cuh: kBsSlots)

void appendf(std::string &s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  const int n = vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (n > 0) s.append(buf, std::min<size_t>((size_t)n, sizeof buf - 1));
}

}  // namespace

std::vector<BsBlock> bs_blocks_by_support(const uint8_t *M, int rows, int cols) {
  std::map<std::vector<int>, std::vector<int>> groups;
  std::vector<std::vector<int>> order;
  for (int r = 0; r < rows; r++) {
    std::vector<int> sup;
    for (int q = 0; q < cols; q++)
      if (M[(size_t)r * cols + q]) sup.push_back(q);
    if (!groups.count(sup)) order.push_back(sup);
    groups[sup].push_back(r);
  }
  std::vector<BsBlock> blks;
  for (auto &sup : order) {
    auto &rs = groups[sup];
    const int nb = (int)((rs.size() + kBsEmitRows - 1) / kBsEmitRows);
    for (int b = 0; b < nb; b++) {
      BsBlock B;
      B.rows.assign(rs.begin() + rs.size() * b / nb, rs.begin() + rs.size() * (b + 1) / nb);
      B.inputs = sup;
      blks.push_back(B);
    }
  }
  return blks;
}

std::vector<BsBlock> bs_blocks_chunked(const uint8_t *M, int rows, int cols) {
  std::vector<BsBlock> blks;
  const int nb = (rows + kBsEmitRows - 1) / kBsEmitRows;
  for (int b = 0; b < nb; b++) {  // balance rows over the blocks
    BsBlock B;
    std::vector<char> used(cols, 0);
    for (int r = rows * b / nb; r < rows * (b + 1) / nb; r++) {
      B.rows.push_back(r);
      for (int q = 0; q < cols; q++) used[q] |= M[(size_t)r * cols + q] != 0;
    }
    for (int q = 0; q < cols; q++)
      if (used[q]) B.inputs.push_back(q);
    blks.push_back(B);
  }
  return blks;
}

void bs_cta_ranges(int nblocks, const int *cost, uint64_t ntiles, int ncta, uint32_t *cta_g) {
  double total = 0;
  for (int i = 0; i < nblocks; i++) total += (double)cost[i] * (double)ntiles;
  const uint64_t items = (uint64_t)nblocks * ntiles;
  cta_g[0] = 0;
  int b = 0;
  double before = 0;  // cost of the blocks before b
  for (int c = 1; c < ncta; c++) {
    const double target = total * c / ncta;
    while (b + 1 < nblocks && before + (double)cost[b] * ntiles < target)
      before += (double)cost[b++] * ntiles;
    const double t = std::ceil((target - before) / (double)cost[b]);
    const uint64_t g =
        (uint64_t)b * ntiles + (uint64_t)std::min<double>(std::max(t, 0.0), (double)ntiles);
    cta_g[c] = (uint32_t)std::max<uint64_t>(g, cta_g[c - 1]);
  }
  cta_g[ncta] = (uint32_t)items;
}

BsEmitted bs_emit_kernel(const uint8_t *M, int rows, int cols, const std::vector<BsBlock> &blks,
                         const std::string &name, bool extern_c) {
  BsEmitted e;
  std::string &f = e.code;
  const int K = cols;
  (void)rows;
  std::vector<int> blk_ops(blks.size(), 0);  // accumulate instructions per block
  for (size_t b = 0; b < blks.size(); b++) {
    const BsBlock &B = blks[b];
    appendf(f, "// %s block %zu: %zu rows x %zu inputs\n", name.c_str(), b, B.rows.size(),
            B.inputs.size());
    {  // the block's input columns, read by the prefetch in the loop below
      std::string colsl;
      for (size_t i = 0; i < B.inputs.size(); i++) colsl += (i ? ", " : "") + std::to_string(B.inputs[i]);
      f += "__constant__ uint8_t " + name + "_b" + std::to_string(b) + "_in[" +
           std::to_string(std::max<size_t>(B.inputs.size(), 1)) + "] = {" +
           (colsl.empty() ? std::string("0") : colsl) + "};\n";
    }
    appendf(f, "__device__ __forceinline__ void %s_b%zu(const BsCtx &x, uint32_t (&acc)[8][8]) {\n",
            name.c_str(), b);
    f += "  uint32_t Q[16], R[16];\n";
    const int C = (int)B.inputs.size();
    // one loop over the inputs: prefetch, transpose and subset tables are
    // emitted once; only the accumulate XORs differ per input (a switch),
    // which keeps a block's code at about half its fully unrolled size.
    // Short blocks commit empty groups so the wait count stays kAhead - 1.
    appendf(f, "  const uint8_t *in = %s_b%zu_in;\n", name.c_str(), b);
    for (int i = 0; i < kAhead; i++)
      if (i < C)
        appendf(f, "  bs_prefetch(x, %d, %d);\n", B.inputs[i], i % kSlots);
      else
        f += "  bs_commit_empty();\n";
    appendf(f, "#pragma unroll 1\n  for (int i = 0; i < %d; i++) {\n", C);
    appendf(f, "    bs_wait<%d>();\n    bs_planes(x, i %% %d, Q, R);\n", kAhead - 1, kSlots);
    appendf(f, "    if (i + %d < %d) bs_prefetch(x, in[i + %d], (i + %d) %% %d); else bs_commit_empty();\n",
            kAhead, C, kAhead, kAhead, kSlots);
    f += "    switch (i) {\n";
    for (int i = 0; i < C; i++) {
      appendf(f, "    case %d:\n", i);
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
            appendf(f, "      acc[%zu][%d] ^= Q[%d] ^ R[%d];\n", q, bit, lo, hi);
            e.xors += 2;
            blk_ops[b]++;
          } else if (lo) {
            appendf(f, "      acc[%zu][%d] ^= Q[%d];\n", q, bit, lo);
            e.xors += 1;
            blk_ops[b]++;
          } else if (hi) {
            appendf(f, "      acc[%zu][%d] ^= R[%d];\n", q, bit, hi);
            e.xors += 1;
            blk_ops[b]++;
          }
        }
      }
      f += "      break;\n";
    }
    f += "    default: break;\n    }\n  }\n";
    f += "}\n\n";
  }
  // persistent kernel, one CTA per SM: the host splits the sequence of
  // (block, 1 KiB column tile) items into equal-cost ranges, one per CTA, so
  // an SM runs one block's straight-line code (two at a range boundary),
  // fetched into its instruction caches once and then re-executed; the
  // warps take the range's tiles in turn
  appendf(f, "%s__global__ void __launch_bounds__(kBsThreads, 1) %s(const __grid_constant__ BsArgs a) {\n",
          extern_c ? "extern \"C\" " : "", name.c_str());
  f += "  const uint32_t g1 = a.cta_g[blockIdx.x + 1];\n";
  f += "  for (uint32_t g = a.cta_g[blockIdx.x] + threadIdx.x / 32; g < g1; g += kBsThreads / 32) {\n";
  f += "    const uint32_t b = g / a.ntiles, u = g - b * a.ntiles;\n";
  f += "    BsCtx x;\n    if (!bs_ctx(a, x, u)) continue;\n    uint32_t acc[8][8];\n";
  f += "    bs_zero(acc);\n    switch (b) {\n";
  for (size_t b = 0; b < blks.size(); b++) {
    const BsBlock &B = blks[b];
    appendf(f, "      case %zu: {\n        %s_b%zu(x, acc);\n", b, name.c_str(), b);
    for (size_t q = 0; q < B.rows.size(); q++)
      appendf(f, "        bs_store(x, %d, acc[%zu]);\n", K + B.rows[q], q);
    f += "      } break;\n";
  }
  f += "      default: break;\n    }\n  }\n}\n\n";
  // relative cost of each block (instructions per tile, roughly): input
  // transposes and subset tables, output transposes, accumulate XORs
  for (size_t b = 0; b < blks.size(); b++)
    e.cost.push_back((int)(blk_ops[b] + 100 * blks[b].inputs.size() + 70 * blks[b].rows.size()));
  return e;
}

}  // namespace pmrc
