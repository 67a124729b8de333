// Region plan construction (see plan.h).
#include "plan.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

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

std::shared_ptr<Plan> make_plan(const Mat &M, const std::vector<int> &out_slot, int nout) {
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
  // 2. cut groups into blocks of at most kMaxBlockRows rows.  Groups of a
  // single row or two (sparse, unstructured matrices) are merged with their
  // neighbours: a shared input is then split once for several rows, and a
  // zero coefficient costs only a skipped branch in the kernel.
  struct Proto {
    std::vector<int> rows;
    std::vector<uint16_t> inputs;
  };
  std::vector<Proto> protos;
  size_t total_rows = 0;
  for (auto &s : order) total_rows += groups[s].size();
  const bool merge = !order.empty() && total_rows < 3 * order.size();
  if (!merge) {
    for (auto &s : order) {
      auto &rows = groups[s];
      const int nblk = (int)((rows.size() + kMaxBlockRows - 1) / kMaxBlockRows);
      // balance rows over the blocks of a group
      for (int b = 0; b < nblk; b++) {
        Proto p;
        size_t lo = rows.size() * b / nblk, hi = rows.size() * (b + 1) / nblk;
        p.rows.assign(rows.begin() + lo, rows.begin() + hi);
        p.inputs = s;
        protos.push_back(std::move(p));
      }
    }
  } else {
    std::vector<int> rows;
    for (auto &s : order)
      for (int r : groups[s]) rows.push_back(r);
    for (size_t lo = 0; lo < rows.size(); lo += kMaxBlockRows) {
      Proto p;
      size_t hi = std::min(rows.size(), lo + kMaxBlockRows);
      p.rows.assign(rows.begin() + lo, rows.begin() + hi);
      std::vector<char> used(M.cols, 0);
      for (int r : p.rows)
        for (int c = 0; c < M.cols; c++)
          if (M.at(r, c)) used[c] = 1;
      for (int c = 0; c < M.cols; c++)
        if (used[c]) p.inputs.push_back((uint16_t)c);
      protos.push_back(std::move(p));
    }
  }
  int maxr = 1;
  for (auto &p : protos) maxr = std::max(maxr, (int)p.rows.size());
  plan->R = round_rows(maxr);
  const int R = plan->R;
  for (auto &p : protos) {
    PlanBlock b;
    for (int r : p.rows) b.rows.push_back((uint16_t)(M.cols + out_slot[r]));
    plan->max_inputs = std::max(plan->max_inputs, (int)p.inputs.size());
    b.inputs = p.inputs;
    b.coef.assign(p.inputs.size() * R, 0);
    for (size_t i = 0; i < p.inputs.size(); i++)
      for (size_t q = 0; q < p.rows.size(); q++) b.coef[i * R + q] = M.at(p.rows[q], p.inputs[i]);
    plan->blocks.push_back(std::move(b));
  }
  // 3. device image: descriptors, uint16 slots, coefficients
  const size_t nb = plan->blocks.size();
  size_t nidx = 0, ncoef = 0;
  for (auto &b : plan->blocks) {
    nidx += b.inputs.size() + b.rows.size();
    ncoef += b.coef.size();
  }
  plan->idx_base = nb * sizeof(BlockDesc);
  plan->coef_base = (plan->idx_base + nidx * 2 + 15) & ~(size_t)15;
  plan->image.assign(plan->coef_base + ncoef + 16, 0);
  uint8_t *img = plan->image.data();
  uint32_t io = 0, co = 0;
  for (size_t i = 0; i < nb; i++) {
    auto &b = plan->blocks[i];
    BlockDesc d{};
    d.in_off = io;
    memcpy(img + plan->idx_base + (size_t)io * 2, b.inputs.data(), b.inputs.size() * 2);
    io += (uint32_t)b.inputs.size();
    d.out_off = io;
    memcpy(img + plan->idx_base + (size_t)io * 2, b.rows.data(), b.rows.size() * 2);
    io += (uint32_t)b.rows.size();
    d.coef_off = co;
    memcpy(img + plan->coef_base + co, b.coef.data(), b.coef.size());
    co += (uint32_t)b.coef.size();
    d.nrows = (uint16_t)b.rows.size();
    d.ninputs = (uint16_t)b.inputs.size();
    memcpy(img + i * sizeof(BlockDesc), &d, sizeof d);
  }
  return plan;
}

}  // namespace pmrc
