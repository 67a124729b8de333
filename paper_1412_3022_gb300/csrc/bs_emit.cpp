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

std::vector<BsBlock> bs_blocks_grouped(const uint8_t *M, int rows, int cols,
                                       const std::vector<int> &own, int max_inputs) {
  std::map<std::vector<int>, std::vector<int>> groups;
  std::vector<std::vector<int>> order;
  for (int r = 0; r < rows; r++) {
    std::vector<int> key;
    for (int q = 0; q < cols; q++)
      if (M[(size_t)r * cols + q] && q != own[r]) key.push_back(q);
    if (!groups.count(key)) order.push_back(key);
    groups[key].push_back(r);
  }
  auto union_size = [&](const std::vector<int> &rs) {
    std::vector<char> used(cols, 0);
    int u = 0;
    for (int r : rs)
      for (int q = 0; q < cols; q++)
        if (M[(size_t)r * cols + q] && !used[q]) used[q] = 1, u++;
    return u;
  };
  std::vector<std::vector<int>> row_sets;  // rows of each block
  std::vector<int> cur;
  for (auto &key : order) {
    const auto &rs = groups[key];
    if (rs.size() > (size_t)kBsEmitRows) {  // a large group: balanced blocks of its own
      const int nb = (int)((rs.size() + kBsEmitRows - 1) / kBsEmitRows);
      for (int b = 0; b < nb; b++)
        row_sets.emplace_back(rs.begin() + rs.size() * b / nb, rs.begin() + rs.size() * (b + 1) / nb);
      continue;
    }
    std::vector<int> grown(cur);
    grown.insert(grown.end(), rs.begin(), rs.end());
    if (!cur.empty() && (grown.size() > (size_t)kBsEmitRows || union_size(grown) > max_inputs)) {
      row_sets.push_back(cur);
      cur.assign(rs.begin(), rs.end());
    } else {
      cur = grown;
    }
  }
  if (!cur.empty()) row_sets.push_back(cur);
  std::vector<BsBlock> blks;
  for (auto &rs : row_sets) {
    BsBlock B;
    B.rows = rs;
    std::vector<char> used(cols, 0);
    for (int r : rs)
      for (int q = 0; q < cols; q++) used[q] |= M[(size_t)r * cols + q] != 0;
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

namespace {

// The accumulate statements of input column `col` into the block's rows:
// one logic instruction per (row, plane) with a non-zero term, acc ^ Q[lo] ^
// R[hi] for the two nibbles of row `plane` of the coefficient's bit matrix.
// Returns the instructions emitted.
int emit_accumulate(std::string &f, const uint8_t *M, int K, const BsBlock &B, int col,
                    long long &xors) {
  int ops = 0;
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
        appendf(f, "      acc[%zu][%d] = bs_x3(acc[%zu][%d], Q[%d], R[%d]);\n", q, bit, q, bit, lo, hi);
        xors += 2;
        ops++;
      } else if (lo) {
        appendf(f, "      acc[%zu][%d] = bs_x2(acc[%zu][%d], Q[%d]);\n", q, bit, q, bit, lo);
        xors += 1;
        ops++;
      } else if (hi) {
        appendf(f, "      acc[%zu][%d] = bs_x2(acc[%zu][%d], R[%d]);\n", q, bit, q, bit, hi);
        xors += 1;
        ops++;
      }
    }
  }
  return ops;
}

// One block function: the loop over `ins` (a block's inputs, or half of
// them) accumulating M's coefficients of the block's rows into acc; with
// in_planes the inputs are plane-layout blocks (no transpose).  Returns the
// accumulate instructions emitted.
int emit_block_fn(std::string &f, const uint8_t *M, int K, const BsBlock &B,
                  const std::vector<int> &ins, const std::string &fname, bool in_planes,
                  long long &xors) {
  int ops = 0;
  {  // the inputs' columns, read by the prefetch in the loop below
    std::string colsl;
    for (size_t i = 0; i < ins.size(); i++) colsl += (i ? ", " : "") + std::to_string(ins[i]);
    f += "__constant__ uint8_t " + fname + "_in[" + std::to_string(std::max<size_t>(ins.size(), 1)) +
         "] = {" + (colsl.empty() ? std::string("0") : colsl) + "};\n";
  }
  appendf(f, "__device__ __forceinline__ void %s(const BsCtx &x, uint32_t (&acc)[8][8]) {\n",
          fname.c_str());
  f += "  uint32_t Q[16], R[16];\n";
  const int C = (int)ins.size();
  // one loop over the inputs: prefetch, transpose and subset tables are
  // emitted once; only the accumulate XORs differ per input (a switch),
  // which keeps a block's code at about half its fully unrolled size.
  // The ring's read and write slots advance by one slot per input and wrap
  // (no slot index arithmetic).  Short blocks commit empty groups so the
  // wait count stays kAhead - 1.
  appendf(f, "  const uint8_t *in = %s_in;\n", fname.c_str());
  f += "  const uint32_t base = bs_ring_base(), end = base + kBsSlots * kBsSlotStep;\n";
  for (int i = 0; i < kAhead; i++)
    if (i < C)
      appendf(f, "  bs_prefetch(x, %d, base + %d * kBsSlotStep);\n", ins[i], i % kSlots);
    else
      f += "  bs_commit_empty();\n";
  appendf(f, "  uint32_t rd = base, wr = base + %d * kBsSlotStep;\n", kAhead % kSlots);
  appendf(f, "#pragma unroll 1\n  for (int i = 0; i < %d; i++) {\n", C);
  appendf(f, in_planes ? "    bs_wait<%d>();\n    bs_planes_direct(rd, Q, R);\n"
                       : "    bs_wait<%d>();\n    bs_planes(x, rd, Q, R);\n",
          kAhead - 1);
  appendf(f, "    if (i + %d < %d) bs_prefetch(x, in[i + %d], wr); else bs_commit_empty();\n",
          kAhead, C, kAhead);
  f += "    rd += kBsSlotStep;\n    rd = rd == end ? base : rd;\n";
  f += "    wr += kBsSlotStep;\n    wr = wr == end ? base : wr;\n";
  f += "    switch (i) {\n";
  for (int i = 0; i < C; i++) {
    appendf(f, "    case %d:\n", i);
    ops += emit_accumulate(f, M, K, B, ins[i], xors);
    f += "      break;\n";
  }
  f += "    default: break;\n    }\n  }\n";
  f += "}\n\n";
  return ops;
}

}  // namespace

BsEmitted bs_emit_kernel(const uint8_t *M, int rows, int cols, const std::vector<BsBlock> &blks,
                         const std::string &name, bool extern_c, bool pair_split, bool in_planes,
                         bool out_planes) {
  BsEmitted e;
  std::string &f = e.code;
  const char *store = out_planes ? "bs_store_planes" : "bs_store";
  const int K = cols;
  (void)rows;
  std::vector<int> blk_ops(blks.size(), 0);  // accumulate instructions per block
  for (size_t b = 0; b < blks.size(); b++) {
    const BsBlock &B = blks[b];
    appendf(f, "// %s block %zu: %zu rows x %zu inputs\n", name.c_str(), b, B.rows.size(),
            B.inputs.size());
    const std::string fn = name + "_b" + std::to_string(b);
    if (!pair_split) {
      blk_ops[b] = emit_block_fn(f, M, K, B, B.inputs, fn, in_planes, e.xors);
    } else {  // the inputs cut in two halves, one per warp of a pair
      const size_t h = (B.inputs.size() + 1) / 2;
      const std::vector<int> i0(B.inputs.begin(), B.inputs.begin() + h), i1(B.inputs.begin() + h,
                                                                           B.inputs.end());
      blk_ops[b] = emit_block_fn(f, M, K, B, i0, fn + "_h0", in_planes, e.xors);
      blk_ops[b] += emit_block_fn(f, M, K, B, i1, fn + "_h1", in_planes, e.xors);
    }
  }
  appendf(f, "%s__global__ void __launch_bounds__(kBsThreads, 1) %s(const __grid_constant__ BsArgs a) {\n",
          extern_c ? "extern \"C\" " : "", name.c_str());
  // a two-launch product: the first kernel lets the second be placed at
  // once (programmatic dependent launch); the second waits for the first's
  // completion and memory before it reads the intermediate (both are no-ops
  // in a plain launch)
  if (out_planes) f += "  asm volatile(\"griddepcontrol.launch_dependents;\" ::: \"memory\");\n";
  if (in_planes) f += "  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");\n";
  f += "  const uint32_t g1 = a.cta_g[blockIdx.x + 1];\n";
  if (!pair_split) {
    // persistent kernel, one CTA per SM: the host splits the sequence of
    // (block, 1 KiB column tile) items into equal-cost ranges, one per CTA,
    // so an SM runs one block's straight-line code (two at a range
    // boundary), fetched into its instruction caches once and then
    // re-executed; the warps take the range's tiles in turn
    f += "  for (uint32_t g = a.cta_g[blockIdx.x] + threadIdx.x / 32; g < g1; g += kBsThreads / 32) {\n";
    f += "    const uint32_t b = g / a.ntiles, u = g - b * a.ntiles;\n";
    f += "    BsCtx x;\n    if (!bs_ctx(a, x, u)) continue;\n    uint32_t acc[8][8];\n";
    f += "    bs_zero(acc);\n    switch (b) {\n";
    for (size_t b = 0; b < blks.size(); b++) {
      const BsBlock &B = blks[b];
      appendf(f, "      case %zu: {\n        %s_b%zu(x, acc);\n", b, name.c_str(), b);
      for (size_t q = 0; q < B.rows.size(); q++)
        appendf(f, "        %s(x, %d, acc[%zu]);\n", store, K + B.rows[q], q);
      f += "      } break;\n";
    }
    f += "      default: break;\n    }\n  }\n}\n\n";
  } else {
    // the same ranges, taken by warp pairs: both warps of a pair work on the
    // same item, each over half of the block's inputs; the partial sums meet
    // in shared memory (one exchange area of 8 rows x 8 planes x 32 lanes
    // per pair) and each warp stores half of the block's rows
    f += "  extern __shared__ __align__(16) uint8_t bs_smem[];\n";
    f += "  const uint32_t warp = threadIdx.x / 32, lane = threadIdx.x % 32, pair = warp / 2, half = warp % 2;\n";
    f += "  uint32_t *xs = reinterpret_cast<uint32_t *>(bs_smem + kBsSlots * kBsSlotStep) + pair * 8 * 8 * 32;\n";
    f += "  for (uint32_t g = a.cta_g[blockIdx.x] + pair; g < g1; g += kBsThreads / 64) {\n";
    f += "    const uint32_t b = g / a.ntiles, u = g - b * a.ntiles;\n";
    f += "    BsCtx x;\n    const bool live = bs_ctx(a, x, u);\n";
    f += "    if (!live) x.off = 0;  // lanes past the end read in-range bytes and store nothing\n";
    f += "    uint32_t acc[8][8];\n    bs_zero(acc);\n    switch (b) {\n";
    for (size_t b = 0; b < blks.size(); b++) {
      const BsBlock &B = blks[b];
      const int R = (int)B.rows.size(), rs = (R + 1) / 2;
      appendf(f, "      case %zu: {\n        if (half == 0) %s_b%zu_h0(x, acc); else %s_b%zu_h1(x, acc);\n",
              b, name.c_str(), b, name.c_str(), b);
      appendf(f, "#pragma unroll\n        for (int r = 0; r < %d; r++)\n          if ((r < %d) != (half == 0))\n"
                 "#pragma unroll\n            for (int i = 0; i < 8; i++) xs[(r * 8 + i) * 32 + lane] = acc[r][i];\n",
              R, rs);
      f += "        bs_pair_sync(pair);\n";
      for (int q = 0; q < R; q++) {
        appendf(f, "        if ((%d < %d) == (half == 0)) {\n", q, rs);
        appendf(f, "#pragma unroll\n          for (int i = 0; i < 8; i++) acc[%d][i] = bs_x2(acc[%d][i], xs[(%d * 8 + i) * 32 + lane]);\n",
                q, q, q);
        appendf(f, "          if (live) %s(x, %d, acc[%d]);\n        }\n", store, K + B.rows[q], q);
      }
      f += "        bs_pair_sync(pair);  // the exchange area is reused by the next item\n";
      f += "      } break;\n";
    }
    f += "      default: break;\n    }\n  }\n}\n\n";
  }
  // relative cost of each block (instructions per tile, roughly): input
  // transposes and subset tables, output transposes, accumulate XORs
  for (size_t b = 0; b < blks.size(); b++)
    e.cost.push_back((int)(blk_ops[b] + 100 * blks[b].inputs.size() + 70 * blks[b].rows.size()));
  return e;
}

namespace {

// dst[i] = (or ^=) the XOR of the planes src[jj] whose bit i of c * 2^jj is
// set: output plane i of c * x, for a constant c != 0.  Terms fold into the
// destination two at a time (3-input XOR).
void emit_mul_planes(std::string &f, uint8_t c, const char *dst, const char *src, bool assign,
                     const char *ind, long long &ops) {
  for (int i = 0; i < 8; i++) {
    std::vector<std::string> t;
    for (int jj = 0; jj < 8; jj++)
      if ((gf_mul_sr(c, (uint8_t)(1u << jj)) >> i) & 1)
        t.push_back(std::string(src) + "[" + std::to_string(jj) + "]");
    const std::string d = std::string(dst) + "[" + std::to_string(i) + "]";
    size_t k = 0;
    if (assign) {
      if (t.empty()) {
        f += ind + d + " = 0u;\n";
        continue;
      }
      if (t.size() == 1) {
        f += ind + d + " = " + t[0] + ";\n";
        continue;
      }
      if (t.size() == 2) {
        f += ind + d + " = bs_x2(" + t[0] + ", " + t[1] + ");\n";
        ops++;
        continue;
      }
      f += ind + d + " = bs_x3(" + t[0] + ", " + t[1] + ", " + t[2] + ");\n";
      ops++;
      k = 3;
    }
    for (; k < t.size(); k += 2) {
      if (k + 1 < t.size())
        f += ind + d + " = bs_x3(" + d + ", " + t[k] + ", " + t[k + 1] + ");\n";
      else
        f += ind + d + " = bs_x2(" + d + ", " + t[k] + ");\n";
      ops++;
    }
  }
}

std::vector<int> nonzeros(const uint8_t *phi, int alpha) {
  std::vector<int> nz;
  for (int j = 0; j < alpha; j++)
    if (phi[j]) nz.push_back(j);
  return nz;
}

// The loop over helpers [h0, h1) of one warp task: each helper's blocks read
// by phi (its non-zeros, in order) stream through the shared-memory ring, are
// turned into planes and multiplied into p; `epilogue` follows each helper
// with p holding its projection.  Input i of the task is block nz[i % NZ] of
// helper h0 + i / NZ, prefetched kAhead inputs ahead across helpers.
void emit_helper_loop(std::string &f, const uint8_t *phi, int alpha, const std::string &h0,
                      const std::string &h1, const std::string &epilogue, long long &ops) {
  const std::vector<int> nz = nonzeros(phi, alpha);
  const int NZ = (int)nz.size();
  f += "  const uint32_t base = bs_ring_base(), end = base + kBsSlots * kBsSlotStep;\n";
  for (int i = 0; i < kAhead; i++)
    appendf(f, "  if (%s + %d < %s) bs_prefetch(x, (%s + %d) * %d + %d, base + %d * kBsSlotStep); "
               "else bs_commit_empty();\n",
            h0.c_str(), i / NZ, h1.c_str(), h0.c_str(), i / NZ, alpha, nz[i % NZ], i % kSlots);
  appendf(f, "  uint32_t rd = base, wr = base + %d * kBsSlotStep;\n", kAhead % kSlots);
  appendf(f, "#pragma unroll 1\n  for (uint32_t h = %s; h < %s; h++) {\n", h0.c_str(), h1.c_str());
  for (int jj = 0; jj < NZ; jj++) {
    appendf(f, "    bs_wait<%d>();\n    bs_load(rd, w);\n    bs_transpose(w, *x.a);\n", kAhead - 1);
    emit_mul_planes(f, phi[nz[jj]], "p", "w", jj == 0, "    ", ops);
    const int t = jj + kAhead, dh = t / NZ, jn = nz[t % NZ];
    appendf(f, "    if (h + %d < %s) bs_prefetch(x, (h + %d) * %d + %d, wr); else bs_commit_empty();\n",
            dh, h1.c_str(), dh, alpha, jn);
    f += "    rd += kBsSlotStep;\n    rd = rd == end ? base : rd;\n";
    f += "    wr += kBsSlotStep;\n    wr = wr == end ? base : wr;\n";
  }
  f += epilogue;
  f += "  }\n";
}

}  // namespace

BsEmitted bs_emit_projection(const uint8_t *phi, int alpha, const std::string &name) {
  BsEmitted e;
  std::string &f = e.code;
  appendf(f, "// %s: helper projections p_h = sum_j phi[j] Y[alpha h + j], alpha = %d\n",
          name.c_str(), alpha);
  appendf(f, "extern \"C\" __global__ void __launch_bounds__(kBsThreads, 1) %s(const __grid_constant__ BsArgs a) {\n",
          name.c_str());
  f += "  const uint32_t warps = gridDim.x * (kBsThreads / 32);\n";
  f += "  for (uint32_t g = blockIdx.x * (kBsThreads / 32) + threadIdx.x / 32; g < a.ntasks; g += warps) {\n";
  f += "    const uint32_t grp = g % a.ngroups, u = g / a.ngroups;\n";
  appendf(f, "    const uint32_t h0 = grp * %d, h1 = h0 + %d < a.nh ? h0 + %d : a.nh;\n",
          kBsHelpersPerTask, kBsHelpersPerTask, kBsHelpersPerTask);
  f += "    BsCtx x;\n    const bool live = bs_ctx(a, x, u);\n";
  f += "    if (!live) x.off = 0;  // lanes past the end read in-range bytes and store nothing\n";
  f += "    uint32_t w[8], p[8];\n";
  std::string body;
  appendf(body, "    if (live) bs_store(x, (int)(a.nh * %d + h), p);\n", alpha);
  std::string loop;
  emit_helper_loop(loop, phi, alpha, "h0", "h1", body, e.xors);
  // indent the loop one level into the task loop
  for (size_t pos = 0; pos < loop.size();) {
    const size_t nl = loop.find('\n', pos);
    const std::string line = loop.substr(pos, nl - pos);
    f += (line.rfind("#pragma", 0) == 0 ? "" : "  ") + line + "\n";
    pos = nl + 1;
  }
  f += "  }\n}\n";
  return e;
}

BsEmitted bs_emit_fused_repair(const uint8_t *phi, int alpha, const uint8_t *D, int d,
                               const std::string &name) {
  BsEmitted e;
  std::string &f = e.code;
  const int d0 = (d + 1) / 2;     // group 0: helpers [0, d0), group 1: [d0, d)
  const int rs = (alpha + 1) / 2;  // group 0 stores rows [0, rs), group 1 rows [rs, alpha)
  appendf(f, "// %s: fused repair, alpha = %d, d = %d\n", name.c_str(), alpha, d);
  for (int g = 0; g < 2; g++) {
    const int h0 = g ? d0 : 0, h1 = g ? d : d0;
    appendf(f, "__device__ __forceinline__ void %s_g%d(const BsCtx &x, uint32_t (&acc)[%d][8]) {\n",
            name.c_str(), g, alpha);
    f += "  uint32_t Q[16], R[16], w[8], p[8];\n";
    std::string epi = "    bs_tables(p, Q, R);\n    switch (h) {\n";
    for (int q = h0; q < h1; q++) {
      appendf(epi, "    case %d:\n", q);
      for (int r = 0; r < alpha; r++) {
        const uint8_t cf = D[(size_t)r * d + q];
        if (!cf) continue;
        for (int bit = 0; bit < 8; bit++) {
          int lo = 0, hi = 0;  // row `bit` of M_cf, split in two nibbles
          for (int j = 0; j < 8; j++)
            if ((gf_mul_sr(cf, (uint8_t)(1u << j)) >> bit) & 1) {
              if (j < 4)
                lo |= 1 << j;
              else
                hi |= 1 << (j - 4);
            }
          if (lo && hi)
            appendf(epi, "      acc[%d][%d] = bs_x3(acc[%d][%d], Q[%d], R[%d]);\n", r, bit, r, bit, lo, hi);
          else if (lo)
            appendf(epi, "      acc[%d][%d] = bs_x2(acc[%d][%d], Q[%d]);\n", r, bit, r, bit, lo);
          else
            appendf(epi, "      acc[%d][%d] = bs_x2(acc[%d][%d], R[%d]);\n", r, bit, r, bit, hi);
          e.xors++;
        }
      }
      epi += "      break;\n";
    }
    epi += "    default: break;\n    }\n";
    emit_helper_loop(f, phi, alpha, std::to_string(h0), std::to_string(h1), epi, e.xors);
    f += "}\n\n";
  }
  appendf(f, "extern \"C\" __global__ void __launch_bounds__(kBsThreads, 1) %s(const __grid_constant__ BsArgs a) {\n",
          name.c_str());
  f += "  extern __shared__ __align__(16) uint8_t bs_smem[];\n";
  f += "  const uint32_t warp = threadIdx.x / 32, lane = threadIdx.x % 32, pair = warp / 2, grp = warp % 2;\n";
  appendf(f, "  uint32_t *xs = reinterpret_cast<uint32_t *>(bs_smem + kBsSlots * kBsSlotStep) + pair * %d;\n",
          alpha * 8 * 32);
  // tile u goes to CTA u % gridDim.x: consecutive tiles spread over every
  // SM, whatever the tile count
  f += "  for (uint32_t u = pair * gridDim.x + blockIdx.x; u < a.ntiles; u += gridDim.x * (kBsThreads / 64)) {\n";
  f += "    BsCtx x;\n    const bool live = bs_ctx(a, x, u);\n";
  f += "    if (!live) x.off = 0;  // lanes past the end read in-range bytes and store nothing\n";
  appendf(f, "    uint32_t acc[%d][8];\n#pragma unroll\n    for (int r = 0; r < %d; r++)\n#pragma unroll\n"
             "      for (int i = 0; i < 8; i++) acc[r][i] = 0;\n", alpha, alpha);
  appendf(f, "    if (grp == 0) %s_g0(x, acc); else %s_g1(x, acc);\n", name.c_str(), name.c_str());
  f += "    // each warp hands the other the partial sums of the rows that warp stores\n";
  appendf(f, "#pragma unroll\n    for (int r = 0; r < %d; r++)\n      if ((r < %d) != (grp == 0))\n#pragma unroll\n"
             "        for (int i = 0; i < 8; i++) xs[(r * 8 + i) * 32 + lane] = acc[r][i];\n", alpha, rs);
  f += "    bs_pair_sync(pair);\n";
  appendf(f, "#pragma unroll\n    for (int r = 0; r < %d; r++)\n      if ((r < %d) == (grp == 0)) {\n#pragma unroll\n"
             "        for (int i = 0; i < 8; i++) acc[r][i] = bs_x2(acc[r][i], xs[(r * 8 + i) * 32 + lane]);\n"
             "        if (live) bs_store(x, (int)(a.nh * %d + r), acc[r]);\n      }\n", alpha, rs, alpha);
  f += "    bs_pair_sync(pair);  // the exchange area is reused by the next tile\n";
  f += "  }\n}\n";
  return e;
}

}  // namespace pmrc
