// Batched execution: many stripes of uneven code size and block size in one
// persistent launch, replayed from a CUDA graph.
//
// Every stripe operation is cut into work items: (dense block of its plan x
// range of 4 KiB byte tiles) for encode and decode, (fused repair x range of
// tiles) for repair.  A persistent grid pulls items from an atomic counter
// (reset by a memset node in the same graph), stages the item's split tables
// in shared memory and runs the same inner loop as the single-stripe
// kernels (region_dev.cuh).  Items are listed biggest stripe first so the
// dynamic pull balances the tail.  Item size and CTAs per SM are tunable
// (pmrc_batch_tune times candidates on the device and keeps the fastest).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pmrc.h"
#include "api_internal.h"
#include "gf256.h"
#include "plan.h"
#include "repair.h"

namespace pmrc {
namespace {

#include "region_dev.cuh"
#include "repair_dev.cuh"

constexpr int kBatchR = 16;  // rows in registers: covers alpha <= 16 and plans with R <= 16

struct BatchItem {
  const uint8_t *image;   // region plan image, or fused repair image
  uint8_t *const *ptrs;   // this stripe's pointers: inputs, then outputs
  uint64_t nbytes;        // block size of the stripe
  uint32_t tile0, ntiles; // tile range
  uint32_t idx_base, tab4_base, tab1_base;  // region image offsets
  uint16_t type;          // 0 region block, 1 fused repair
  uint16_t block;         // region: block index
  uint16_t nin;           // region: input slots (outputs follow)
  uint16_t stride;        // region: table stride (the plan's R)
  uint16_t aligned;
  uint16_t pad[3];
};

struct BatchArgs {
  const BatchItem *items;
  int nitems;
  unsigned *counter;
  MulConsts k;
};

template <int R>
__global__ void __launch_bounds__(kThreads) batch_kernel(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int s_item;
  const MulConsts k = a.k;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= a.nitems) break;
    const BatchItem w = a.items[it];
    const bool vec = w.aligned != 0;
    if (w.type == 0) {
      const BlockDesc d = reinterpret_cast<const BlockDesc *>(w.image)[w.block];
      const int nin = d.ninputs, nrows = d.nrows, nent = nin * w.stride;
      uint4 *t4 = reinterpret_cast<uint4 *>(smem);
      uint32_t *t1 = reinterpret_cast<uint32_t *>(smem + (size_t)nent * 16);
      uint16_t *slot = reinterpret_cast<uint16_t *>(smem + (size_t)nent * 20);
      const uint4 *g4 = reinterpret_cast<const uint4 *>(w.image + w.tab4_base) + d.tab_off;
      const uint32_t *g1 = reinterpret_cast<const uint32_t *>(w.image + w.tab1_base) + d.tab_off;
      const uint16_t *idx = reinterpret_cast<const uint16_t *>(w.image + w.idx_base);
      for (int i = threadIdx.x; i < nent; i += kThreads) {
        t4[i] = g4[i];
        t1[i] = g1[i];
      }
      for (int i = threadIdx.x; i < nin; i += kThreads) slot[i] = idx[d.in_off + i];
      for (int i = threadIdx.x; i < nrows; i += kThreads) slot[nin + i] = idx[d.out_off + i];
      __syncthreads();
      for (uint32_t tile = w.tile0; tile < w.tile0 + w.ntiles; tile++) {
        const uint64_t off = ((uint64_t)tile * kThreads + threadIdx.x) * kVec;
        if (off >= w.nbytes) continue;
        uint32_t acc[R][4];
        mac_block<R>(acc, nin, nrows, w.stride, t4, t1, k,
                     [&](int i) { return load16(w.ptrs[slot[i]], off, w.nbytes, vec); });
#pragma unroll
        for (int r = 0; r < R; r++)
          if (r < nrows) {
            uint8_t *o = w.ptrs[slot[nin + r]];
            if (o) store16(o, off, w.nbytes, vec, acc_bytes(acc[r]));
          }
      }
    } else {
      const FusedRepairHeader *hp = reinterpret_cast<const FusedRepairHeader *>(w.image);
      const int d = hp->d, alpha = hp->alpha, nz = hp->nz, rl = hp->rl;
      const bool direct = hp->direct != 0;
      const int n1 = nz, n2 = d * 4 * rl;
      uint4 *proj = reinterpret_cast<uint4 *>(smem);
      uint4 *t1a = proj + (size_t)d * kRepCols;
      uint4 *t2a = t1a + n1;
      uint32_t *t1b = reinterpret_cast<uint32_t *>(t2a + n2);
      uint32_t *t2b = t1b + n1;
      uint16_t *s_nz = reinterpret_cast<uint16_t *>(t2b + n2);
      const uint4 *g4 = reinterpret_cast<const uint4 *>(w.image + hp->tab4_off);
      const uint32_t *g1 = reinterpret_cast<const uint32_t *>(w.image + hp->tab1_off);
      for (int i = threadIdx.x; i < n1 + n2; i += kThreads) {
        t1a[i] = g4[i];
        t1b[i] = g1[i];
      }
      if (threadIdx.x < 16) s_nz[threadIdx.x] = hp->nzidx[threadIdx.x];
      __syncthreads();
      const uint64_t span_end = (uint64_t)(w.tile0 + w.ntiles) * kThreads * kVec;
      const uint64_t end = span_end < w.nbytes ? span_end : w.nbytes;
      for (uint64_t t = (uint64_t)w.tile0 * kThreads * kVec; t < end; t += kRepTile)
        fused_repair_tile<0>(w.ptrs, t, w.nbytes, vec, d, alpha, nz, direct, s_nz, t1a, t1b, t2a,
                             t2b, rl, proj, k);
    }
    __syncthreads();
  }
}

struct Stripe {
  int type = 0;  // 0 region plan, 1 fused repair
  std::shared_ptr<Plan> plan;
  std::shared_ptr<FusedRepairPlan> fplan;
  std::vector<uint8_t *> ptrs;
  size_t nbytes = 0;
  int64_t user_bytes = 0;
  int64_t work = 0;  // products per byte column (cost model)
  bool aligned = true;
};


std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;  // signature -> (work_bytes, ctas_per_sm)

const char *kErrBuilt = "batch already built: create a new batch to add stripes";

}  // namespace
}  // namespace pmrc

using namespace pmrc;

struct pmrc_batch {
  std::vector<Stripe> stripes;
  int device = -1;
  bool built = false;
  // device state
  uint8_t **d_ptrs = nullptr;
  BatchItem *d_items = nullptr;
  unsigned *d_counter = nullptr;
  int nitems = 0;
  unsigned grid = 0;
  size_t smem = 0;
  int work_bytes = 0, ctas_per_sm = 0;
  int64_t user_bytes = 0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;

  void release_device() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    cudaFree(d_ptrs);
    cudaFree(d_items);
    cudaFree(d_counter);
    exec = nullptr;
    graph = nullptr;
    cap = nullptr;
    d_ptrs = nullptr;
    d_items = nullptr;
    d_counter = nullptr;
    built = false;
  }
  ~pmrc_batch() { release_device(); }
};

namespace {

int bfail(int rc, const std::string &msg) {
  pmrc::set_last_error(msg);
  return rc;
}

bool ptr_aligned(const void *p) { return ((uintptr_t)p % 16) == 0; }

std::string signature(const pmrc_batch *b) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  // k mix and size buckets of the batch
  std::map<std::string, int> cnt;
  for (auto &s : b->stripes) {
    int lg = 0;
    while ((1ull << lg) < s.nbytes) lg++;
    cnt[std::to_string(s.type) + "/" + std::to_string(s.work) + "/" + std::to_string(lg / 2)]++;
  }
  std::string sig = std::string(prop.name) + "|" + std::to_string(prop.multiProcessorCount);
  for (auto &kv : cnt) sig += "|" + kv.first + ":" + std::to_string(kv.second > 0);
  return sig;
}

int build_device(pmrc_batch *b, int work_bytes, int ctas_per_sm, std::string &err) {
  b->release_device();
  cudaError_t e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return kECuda;
  }
  b->device = dev;
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t tile = (uint64_t)kThreads * kVec;
  const uint32_t tiles_per_item = (uint32_t)std::max<uint64_t>(1, (uint64_t)work_bytes / tile);
  // pointer array
  std::vector<uint8_t *> hp;
  std::vector<size_t> base(b->stripes.size());
  for (size_t s = 0; s < b->stripes.size(); s++) {
    base[s] = hp.size();
    hp.insert(hp.end(), b->stripes[s].ptrs.begin(), b->stripes[s].ptrs.end());
  }
  e = cudaMalloc(&b->d_ptrs, std::max<size_t>(1, hp.size()) * sizeof(uint8_t *));
  if (e == cudaSuccess && !hp.empty())
    e = cudaMemcpy(b->d_ptrs, hp.data(), hp.size() * sizeof(uint8_t *), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    err = std::string("batch pointer upload: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? kENoMem : kECuda;
  }
  // items: biggest stripes first; the blocks of one tile range adjacent
  std::vector<size_t> order(b->stripes.size());
  for (size_t s = 0; s < order.size(); s++) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
    const auto &X = b->stripes[x], &Y = b->stripes[y];
    return (double)X.work * X.nbytes > (double)Y.work * Y.nbytes;
  });
  std::vector<BatchItem> items;
  size_t smem = 64;
  for (size_t s : order) {
    const Stripe &S = b->stripes[s];
    const uint32_t ntiles = (uint32_t)((S.nbytes + tile - 1) / tile);
    const void *image = nullptr;
    int rc = S.type == 0 ? S.plan->device_image(&image, err) : S.fplan->device_image(&image, err);
    if (rc) return rc;
    for (uint32_t t0 = 0; t0 < ntiles; t0 += tiles_per_item) {
      BatchItem w{};
      w.image = static_cast<const uint8_t *>(image);
      w.ptrs = b->d_ptrs + base[s];
      w.nbytes = S.nbytes;
      w.tile0 = t0;
      w.ntiles = std::min(tiles_per_item, ntiles - t0);
      w.aligned = S.aligned ? 1 : 0;
      if (S.type == 0) {
        const Plan &P = *S.plan;
        w.type = 0;
        w.nin = (uint16_t)P.nin;
        w.stride = (uint16_t)P.R;
        w.idx_base = (uint32_t)P.idx_base;
        w.tab4_base = (uint32_t)P.tab4_base;
        w.tab1_base = (uint32_t)P.tab1_base;
        for (size_t blk = 0; blk < P.blocks.size(); blk++) {
          w.block = (uint16_t)blk;
          items.push_back(w);
        }
        smem = std::max(smem, (size_t)P.max_entries * 20 + (size_t)(P.max_inputs + P.R) * 2 + 16);
      } else {
        const FusedRepairHeader &h = S.fplan->header;
        w.type = 1;
        items.push_back(w);
        smem = std::max(smem, fused_repair_smem(h) + 64);
      }
    }
  }
  b->nitems = (int)items.size();
  e = cudaMalloc(&b->d_items, std::max<size_t>(1, items.size()) * sizeof(BatchItem));
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned));
  if (e != cudaSuccess) {
    err = std::string("batch work list upload: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? kENoMem : kECuda;
  }
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(batch_kernel<kBatchR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) {
      err = std::string("batch smem opt-in: ") + cudaGetErrorString(e);
      return kECuda;
    }
  }
  int fit = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, batch_kernel<kBatchR>, kThreads, smem);
  if (fit < 1) fit = 1;
  const int per_sm = std::max(1, std::min(ctas_per_sm, fit));
  b->grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, std::max(1, b->nitems)));
  b->smem = smem;
  // graph: counter reset + persistent kernel
  BatchArgs args;
  args.items = b->d_items;
  args.nitems = b->nitems;
  args.counter = b->d_counter;
  args.k = MulConsts{2u, 16u, 1u << 16, 1u << 26, 1u << 29, 1u << 30};
  e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), b->cap);
    batch_kernel<kBatchR><<<b->grid, kThreads, smem, b->cap>>>(args);
    e = cudaStreamEndCapture(b->cap, &b->graph);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    err = std::string("batch graph capture: ") + cudaGetErrorString(e);
    return kECuda;
  }
  b->work_bytes = work_bytes;
  b->ctas_per_sm = per_sm;
  b->built = true;
  return kOk;
}

int add_stripe(pmrc_batch *b, Stripe &&s) {
  if (b->built) return bfail(PMRC_EBUSY, kErrBuilt);
  for (auto *p : s.ptrs)
    if (p && !ptr_aligned(p)) s.aligned = false;
  b->user_bytes += s.user_bytes;
  b->stripes.push_back(std::move(s));
  return (int)b->stripes.size() - 1;
}

}  // namespace

extern "C" {

int pmrc_batch_create(pmrc_batch **out) {
  if (!out) return bfail(PMRC_EINVAL, "out is NULL");
  *out = new (std::nothrow) pmrc_batch();
  return *out ? PMRC_OK : bfail(PMRC_ENOMEM, "out of host memory");
}

void pmrc_batch_destroy(pmrc_batch *b) { delete b; }

int pmrc_batch_add_encode(pmrc_batch *b, const pmrc_code *c, const uint8_t *const *data,
                          uint8_t *const *out, size_t nbytes) {
  if (!b || !c || !data || !out) return bfail(PMRC_EINVAL, "NULL argument");
  Stripe s;
  s.type = 0;
  s.plan = c->encode;
  for (int i = 0; i < s.plan->nin; i++) {
    if (!data[i]) return bfail(PMRC_EINVAL, "data block is NULL");
    s.ptrs.push_back(const_cast<uint8_t *>(data[i]));
  }
  for (int j = 0; j < s.plan->nout; j++) s.ptrs.push_back(out[j]);
  s.nbytes = nbytes;
  s.user_bytes = (int64_t)c->m.k * c->m.alpha * nbytes;
  s.work = s.plan->nnz;
  return add_stripe(b, std::move(s));
}

int pmrc_batch_add_repair(pmrc_batch *b, const pmrc_code *c, int f, const int *helpers,
                          const uint8_t *const *blocks, uint8_t *const *out, size_t nbytes) {
  if (!b || !c || !helpers || !blocks || !out) return bfail(PMRC_EINVAL, "NULL argument");
  if (c->m.alpha > 16) return bfail(PMRC_EUNSUPPORTED, "batched repair needs alpha <= 16");
  Stripe s;
  s.type = 1;
  std::string err;
  int rc = fused_repair_plan(c, f, helpers, s.fplan, err);
  if (rc) return bfail(rc, err);
  const FusedRepairHeader &h = s.fplan->header;
  for (uint32_t q = 0; q < h.d; q++)
    for (uint32_t j = 0; j < h.alpha; j++) {
      const uint8_t *p = blocks[q * h.alpha + j];
      bool used = false;
      for (uint32_t i = 0; i < h.nz; i++) used |= h.nzidx[i] == j;
      if (used && !p) return bfail(PMRC_EINVAL, "a helper block the repair reads is NULL");
      s.ptrs.push_back(const_cast<uint8_t *>(p));
    }
  for (uint32_t r = 0; r < h.alpha; r++) {
    if (!out[r]) return bfail(PMRC_EINVAL, "output block is NULL");
    s.ptrs.push_back(out[r]);
  }
  s.nbytes = nbytes;
  s.user_bytes = (int64_t)c->m.alpha * nbytes;
  s.work = (int64_t)h.d * (h.direct ? 0 : h.nz) + (int64_t)h.d * h.alpha;
  return add_stripe(b, std::move(s));
}

int pmrc_batch_add_decode(pmrc_batch *b, const pmrc_code *c, const int *nodes,
                          const uint8_t *const *node_blocks, uint8_t *const *data_out,
                          size_t nbytes) {
  if (!b || !c || !nodes || !node_blocks || !data_out) return bfail(PMRC_EINVAL, "NULL argument");
  {
    std::vector<char> seen(c->m.n, 0);
    for (int i = 0; i < c->m.k; i++) {
      if (nodes[i] < 0 || nodes[i] >= c->m.n || seen[nodes[i]])
        return bfail(PMRC_EINVAL, "nodes: out of range or repeated node id");
      seen[nodes[i]] = 1;
    }
  }
  std::vector<char> want;
  decode_wanted(c, nodes, node_blocks, data_out, want);
  Stripe s;
  s.type = 0;
  std::string err;
  int rc = decode_plan(c, nodes, want, s.plan, err);
  if (rc) return bfail(rc, err);
  const int K = c->m.k * c->m.alpha;
  for (int i = 0; i < K; i++) s.ptrs.push_back(const_cast<uint8_t *>(node_blocks[i]));
  for (int r = 0; r < K; r++) s.ptrs.push_back(want[r] ? data_out[r] : nullptr);
  for (const auto &blk : s.plan->blocks)
    for (uint16_t in : blk.inputs)
      if (!node_blocks[in]) return bfail(PMRC_EINVAL, "a block the decode reads is NULL");
  s.nbytes = nbytes;
  s.user_bytes = (int64_t)K * nbytes;
  s.work = s.plan->nnz;
  return add_stripe(b, std::move(s));
}

int pmrc_batch_build(pmrc_batch *b, int work_bytes, int ctas_per_sm) {
  if (!b) return bfail(PMRC_EINVAL, "NULL batch");
  if (b->stripes.empty()) return bfail(PMRC_EINVAL, "empty batch");
  if (work_bytes <= 0 || ctas_per_sm <= 0) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(signature(b));
    const std::pair<int, int> def{64 << 10, 2};
    const auto &p = it != g_tune.end() ? it->second : def;
    if (work_bytes <= 0) work_bytes = p.first;
    if (ctas_per_sm <= 0) ctas_per_sm = p.second;
  }
  std::string err;
  int rc = build_device(b, work_bytes, ctas_per_sm, err);
  return rc ? bfail(rc, err) : PMRC_OK;
}

int pmrc_batch_launch(pmrc_batch *b, pmrc_stream_t stream) {
  if (!b || !b->built) return bfail(PMRC_EINVAL, "batch not built");
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess)
    return bfail(PMRC_ECUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
  return PMRC_OK;
}

int pmrc_batch_tune(pmrc_batch *b, pmrc_stream_t stream, int *best_out) {
  if (!b || b->stripes.empty()) return bfail(PMRC_EINVAL, "empty batch");
  const int work[] = {16 << 10, 64 << 10, 256 << 10};
  const int ctas[] = {1, 2};
  cudaStream_t st = (cudaStream_t)stream;
  float best_ms = 1e30f;
  int bw = 64 << 10, bc = 2;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return bfail(PMRC_ECUDA, "cudaEventCreate");
  std::string err;
  int rc = PMRC_OK;
  for (int w : work)
    for (int c : ctas) {
      rc = build_device(b, w, c, err);
      if (rc) break;
      cudaGraphLaunch(b->exec, st);  // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3; r++) cudaGraphLaunch(b->exec, st);
      cudaEventRecord(e1, st);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        rc = PMRC_ECUDA;
        err = std::string("batch tune: ") + cudaGetErrorString(e);
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        bw = w;
        bc = c;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return bfail(rc, err);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[signature(b)] = {bw, bc};
  }
  rc = build_device(b, bw, bc, err);
  if (rc) return bfail(rc, err);
  if (best_out) {
    best_out[0] = bw;
    best_out[1] = b->ctas_per_sm;
  }
  return PMRC_OK;
}

int pmrc_batch_info(const pmrc_batch *b, int64_t *info) {
  if (!b || !info) return bfail(PMRC_EINVAL, "NULL argument");
  info[0] = (int64_t)b->stripes.size();
  info[1] = b->nitems;
  info[2] = b->grid;
  info[3] = b->work_bytes;
  info[4] = b->ctas_per_sm;
  info[5] = b->user_bytes;
  info[6] = 0;
  info[7] = (int64_t)b->smem;
  return PMRC_OK;
}

}  // extern "C"
