// Region plan construction (see plan.h).
#include "plan.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "gf256.h"

namespace pmrc {

Plan::~Plan() {
  for (auto &kv : dev) {
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(kv.first);
    cudaFree(kv.second);
    if (cur >= 0) cudaSetDevice(cur);
  }
}

int Plan::device_image(const void **out, std::string &err) {
  int devid = -1;
  cudaError_t e = cudaGetDevice(&devid);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return kECuda;
  }
  std::lock_guard<std::mutex> g(mu);
  auto it = dev.find(devid);
  if (it != dev.end()) {
    *out = it->second;
    return kOk;
  }
  void *p = nullptr;
  e = cudaMalloc(&p, image.size());
  if (e != cudaSuccess) {
    err = std::string("cudaMalloc(plan): ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? kENoMem : kECuda;
  }
  e = cudaMemcpy(p, image.data(), image.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p);
    err = std::string("cudaMemcpy(plan): ") + cudaGetErrorString(e);
    return kECuda;
  }
  dev[devid] = p;
  *out = p;
  return kOk;
}

static int round_rows(int r) {
  int R = 1;
  while (R < r) R <<= 1;
  return R;
}

// A plan above kMaxSlots slots, or with a block of more split tables than
// shared memory holds (see plan.h): the wanted rows, in the order
// of their support groups, are packed into sets of at most kPartRows rows.
// A set of rows with at most kPartCols non-zero columns each grows while the
// union of its columns stays within kPartCols (block-diagonal and sparse
// matrices then need no accumulation); a set holding a wider row takes rows
// up to kPartRows and its columns are cut into balanced chunks of at most
// kPartCols.  One part per (row set, column chunk): the first chunk of a set
// writes its outputs, the later ones accumulate into them.
static std::shared_ptr<Plan> make_parts(const Mat &M, const std::vector<int> &out_slot, int nout) {
  auto plan = std::make_shared<Plan>();
  plan->nin = M.cols;
  plan->nout = nout;
  std::map<std::vector<int>, std::vector<int>> groups;
  std::vector<std::vector<int>> order;
  for (int r = 0; r < M.rows; r++) {
    if (out_slot[r] < 0) continue;
    std::vector<int> sup;
    for (int c = 0; c < M.cols; c++)
      if (M.at(r, c)) sup.push_back(c);
    auto it = groups.find(sup);
    if (it == groups.end()) {
      order.push_back(sup);
      groups[sup].push_back(r);
    } else {
      it->second.push_back(r);
    }
  }
  std::vector<int> set;
  std::vector<char> used(M.cols, 0);
  int nused = 0;
  bool wide = false;
  auto flush = [&]() {
    std::vector<int> cols;
    for (int c = 0; c < M.cols; c++)
      if (used[c]) cols.push_back(c);
    const size_t nch = std::max<size_t>(1, (cols.size() + kPartCols - 1) / kPartCols);
    for (size_t j = 0; j < nch; j++) {
      PlanPart pt;
      pt.in_cols.assign(cols.begin() + cols.size() * j / nch, cols.begin() + cols.size() * (j + 1) / nch);
      pt.accumulate = j > 0;
      Mat S((int)set.size(), (int)pt.in_cols.size());
      std::vector<int> slot(set.size());
      for (size_t q = 0; q < set.size(); q++) {
        bool any = false;
        for (size_t i = 0; i < pt.in_cols.size(); i++) {
          S.at((int)q, (int)i) = M.at(set[q], pt.in_cols[i]);
          any = any || S.at((int)q, (int)i) != 0;
        }
        slot[q] = (pt.accumulate && !any) ? -1 : (int)q;  // nothing to add from this chunk
        pt.out_slots.push_back(out_slot[set[q]]);
      }
      pt.plan = make_plan(S, slot, (int)set.size());
      plan->nnz += pt.plan->nnz;
      plan->parts.push_back(std::move(pt));
    }
    set.clear();
    std::fill(used.begin(), used.end(), 0);
    nused = 0;
    wide = false;
  };
  for (auto &sup : order)
    for (int r : groups[sup]) {
      const bool w = (int)sup.size() > kPartCols;
      if (!set.empty()) {
        int grown = nused;
        for (int c : sup) grown += !used[c];
        if ((int)set.size() == kPartRows || (!wide && (w || grown > kPartCols))) flush();
      }
      set.push_back(r);
      for (int c : sup) nused += !used[c], used[c] = 1;
      wide = wide || w;
    }
  if (!set.empty()) flush();
  return plan;
}

std::shared_ptr<Plan> make_plan(const Mat &M, const std::vector<int> &out_slot, int nout) {
  if (M.cols + nout > kMaxSlots) return make_parts(M, out_slot, nout);
  auto plan = std::make_shared<Plan>();
  plan->nin = M.cols;
  plan->nout = nout;
  // 1. group wanted rows by their set of non-zero columns
  std::map<std::vector<uint16_t>, std::vector<int>> groups;
  std::vector<std::vector<uint16_t>> order;  // supports in first-seen order
  for (int r = 0; r < M.rows; r++) {
    if (out_slot[r] < 0) continue;
    std::vector<uint16_t> sup;
    for (int c = 0; c < M.cols; c++)
      if (M.at(r, c)) sup.push_back((uint16_t)c);
    plan->nnz += (int64_t)sup.size();
    auto it = groups.find(sup);
    if (it == groups.end()) {
      order.push_back(sup);
      groups[sup].push_back(r);
    } else {
      it->second.push_back(r);
    }
  }
  // 2. merge groups into blocks of at most kMaxBlockRows rows.  A block
  // costs kSplitCost per input (load + bit-field split, shared by its rows)
  // plus one product per (row, input) -- zero coefficients included, since
  // the kernel does not branch on them.  Pairs of blocks are merged greedily
  // while that lowers the total cost, so rows with the same or largely
  // overlapping inputs share the input splits, and rows with disjoint
  // inputs (block-diagonal matrices) stay apart.
  struct Proto {
    std::vector<int> rows;
    std::vector<char> used;  // input columns
    int ninputs = 0;
  };
  constexpr double kSplitCost = 1.5;
  auto cost = [&](int rows, int inputs) { return inputs * kSplitCost + (double)rows * inputs; };
  std::vector<Proto> protos;
  for (auto &sup : order) {
    auto &rows = groups[sup];
    const int nblk = (int)((rows.size() + kMaxBlockRows - 1) / kMaxBlockRows);
    for (int b = 0; b < nblk; b++) {  // balance rows over the blocks of a group
      Proto p;
      size_t lo = rows.size() * b / nblk, hi = rows.size() * (b + 1) / nblk;
      p.rows.assign(rows.begin() + lo, rows.begin() + hi);
      p.used.assign(M.cols, 0);
      for (uint16_t c : sup) p.used[c] = 1;
      p.ninputs = (int)sup.size();
      protos.push_back(std::move(p));
    }
  }
  for (;;) {
    double best = 0;
    int bi = -1, bj = -1;
    for (size_t i = 0; i < protos.size(); i++)
      for (size_t j = i + 1; j < protos.size(); j++) {
        const int r = (int)(protos[i].rows.size() + protos[j].rows.size());
        if (r > kMaxBlockRows) continue;
        int u = 0;
        for (int c = 0; c < M.cols; c++) u += protos[i].used[c] | protos[j].used[c];
        const double gain = cost((int)protos[i].rows.size(), protos[i].ninputs) +
                            cost((int)protos[j].rows.size(), protos[j].ninputs) - cost(r, u);
        if (gain > best) {
          best = gain;
          bi = (int)i;
          bj = (int)j;
        }
      }
    if (bi < 0) break;
    Proto &A = protos[bi], &Bp = protos[bj];
    A.rows.insert(A.rows.end(), Bp.rows.begin(), Bp.rows.end());
    A.ninputs = 0;
    for (int c = 0; c < M.cols; c++) A.ninputs += (A.used[c] |= Bp.used[c]);
    protos.erase(protos.begin() + bj);
  }
  int maxr = 1;
  for (auto &p : protos) maxr = std::max(maxr, (int)p.rows.size());
  plan->R = round_rows(maxr);
  const int R = plan->R;
  for (auto &p : protos) {
    PlanBlock b;
    for (int r : p.rows) b.rows.push_back((uint16_t)(M.cols + out_slot[r]));
    for (int c = 0; c < M.cols; c++)
      if (p.used[c]) b.inputs.push_back((uint16_t)c);
    plan->max_inputs = std::max(plan->max_inputs, (int)b.inputs.size());
    b.coef.assign(b.inputs.size() * R, 0);
    for (size_t i = 0; i < b.inputs.size(); i++)
      for (size_t q = 0; q < p.rows.size(); q++) b.coef[i * R + q] = M.at(p.rows[q], b.inputs[i]);
    plan->blocks.push_back(std::move(b));
  }
  // 3. device image: descriptors, uint16 slots, per-entry split tables
  static const SplitTables split = make_split_tables();
  const size_t nb = plan->blocks.size();
  size_t nidx = 0, nent = 0;
  for (auto &b : plan->blocks) {
    nidx += b.inputs.size() + b.rows.size();
    nent += b.coef.size();
    plan->max_entries = std::max(plan->max_entries, (int)b.coef.size());
  }
  // a block's split tables are staged in shared memory (20 bytes an entry)
  if (plan->max_entries > kPartCols * kMaxBlockRows) return make_parts(M, out_slot, nout);
  plan->idx_base = nb * sizeof(BlockDesc);
  plan->tab4_base = (plan->idx_base + nidx * 2 + 15) & ~(size_t)15;
  plan->tab1_base = plan->tab4_base + nent * sizeof(TabEntry);
  plan->image.assign(plan->tab1_base + nent * 4 + 16, 0);
  uint8_t *img = plan->image.data();
  uint32_t io = 0, eo = 0;
  for (size_t i = 0; i < nb; i++) {
    auto &b = plan->blocks[i];
    BlockDesc d{};
    d.in_off = io;
    memcpy(img + plan->idx_base + (size_t)io * 2, b.inputs.data(), b.inputs.size() * 2);
    io += (uint32_t)b.inputs.size();
    d.out_off = io;
    memcpy(img + plan->idx_base + (size_t)io * 2, b.rows.data(), b.rows.size() * 2);
    io += (uint32_t)b.rows.size();
    d.tab_off = eo;
    for (size_t e = 0; e < b.coef.size(); e++) {
      const uint32_t *w = split.w[b.coef[e]];
      TabEntry t{w[0], w[1], w[2], w[3]};
      memcpy(img + plan->tab4_base + (size_t)(eo + e) * sizeof(TabEntry), &t, sizeof t);
      memcpy(img + plan->tab1_base + (size_t)(eo + e) * 4, &w[4], 4);
    }
    eo += (uint32_t)b.coef.size();
    d.nrows = (uint16_t)b.rows.size();
    d.ninputs = (uint16_t)b.inputs.size();
    memcpy(img + i * sizeof(BlockDesc), &d, sizeof d);
  }
  return plan;
}

std::vector<int> plan_reads(const Plan &p) {
  std::vector<char> r(p.nin, 0);
  for (const auto &b : p.blocks)
    for (uint16_t s : b.inputs) r[s] = 1;
  for (const auto &pt : p.parts)
    for (const auto &b : pt.plan->blocks)
      for (uint16_t s : b.inputs) r[pt.in_cols[s]] = 1;
  std::vector<int> out;
  for (int i = 0; i < p.nin; i++)
    if (r[i]) out.push_back(i);
  return out;
}

}  // namespace pmrc
