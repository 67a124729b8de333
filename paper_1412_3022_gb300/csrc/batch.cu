// Batched execution: many stripes of uneven code size and block size in one
// persistent launch, replayed from a CUDA graph.
//
// Every stripe operation is cut into work items: (dense block of its plan x
// range of 4 KiB byte tiles) for encode and decode, (fused repair x range of
// 1 KiB tiles) for repair; no item costs more than a fixed share of the
// list, so a stripe with short blocks and many products still spreads over
// the grid.  A persistent grid pulls items from an atomic counter
// (reset by a memset node in the same graph), stages the item's split tables
// in shared memory and runs the same inner loops as the single-stripe
// kernels (region_dev.cuh, repair_dev.cuh).  Items are listed biggest stripe
// first so the dynamic pull balances the tail.  Item size and CTAs per SM
// are tunable (pmrc_batch_tune times candidates on the device and keeps the
// fastest).  The serving loop (serve.cu) launches the same kernel on work
// lists it rebuilds every iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/pmrc.h"
#include "api_internal.h"
#include "batch_internal.h"
#include "bitslice.h"
#include "device_info.h"
#include "trace.h"
#include "gf256.h"

namespace pmrc {
namespace {

#include "region_dev.cuh"
#include "repair_dev.cuh"

constexpr int kBatchR = 16;  // rows in registers: covers alpha <= 16 and plans with R <= 16

struct BatchArgs {
  const WorkItem *items;
  int nitems;
  uint8_t *const *ptrs;  // pointer table of the launch
  unsigned *counter;
  uint32_t ptr_area;     // leading shared-memory bytes: the item's stripe pointers
  MulConsts k;
};

template <int R>
__global__ void __launch_bounds__(kThreads) batch_kernel(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(16) uint8_t dsm[];
  __shared__ int s_item;
  __shared__ uint4 s_w[sizeof(WorkItem) / 16];
  const MulConsts k = a.k;
  // the item's stripe pointers stay in shared memory for the whole item:
  // the list and the pointer table are read once per item, wherever they sit
  uint8_t **ptrs = reinterpret_cast<uint8_t **>(dsm);
  uint8_t *const smem = dsm + a.ptr_area;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= a.nitems) break;
    if (threadIdx.x < sizeof(WorkItem) / 16)
      s_w[threadIdx.x] = reinterpret_cast<const uint4 *>(a.items + it)[threadIdx.x];
    __syncthreads();
    const WorkItem w = *reinterpret_cast<const WorkItem *>(s_w);
    for (uint32_t i = threadIdx.x; i < w.nptrs; i += kThreads) ptrs[i] = a.ptrs[w.ptr_off + i];
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
                     [&](int i) { return load16(ptrs[slot[i]], off, w.nbytes, vec); });
#pragma unroll
        for (int r = 0; r < R; r++)
          if (r < nrows) {
            uint8_t *o = ptrs[slot[nin + r]];
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
      const uint64_t span_end = (uint64_t)(w.tile0 + w.ntiles) * kRepTile;
      const uint64_t end = span_end < w.nbytes ? span_end : w.nbytes;
      for (uint64_t t = (uint64_t)w.tile0 * kRepTile; t < end; t += kRepTile)
        fused_repair_tile<0>(ptrs, t, w.nbytes, vec, d, alpha, nz, direct, s_nz, t1a, t1b, t2a,
                             t2b, rl, proj, k);
    }
    __syncthreads();
  }
}

bool ptr_aligned(const void *p) { return ((uintptr_t)p % 16) == 0; }

void finish_stripe(WorkStripe &s) {
  for (auto *p : s.ptrs)
    if (p && !ptr_aligned(p)) s.aligned = false;
}

}  // namespace

int stripe_encode(const pmrc_code *c, const uint8_t *const *data, uint8_t *const *out,
                  size_t nbytes, WorkStripe &s, std::string &err) {
  s = WorkStripe();
  if (c->m.w != 8) {
    err = "batched and served operations take GF(2^8) codes";
    return kEUnsupported;
  }
  s.type = 0;
  s.plan = c->encode;
  if (!s.plan->parts.empty()) {
    err = "code too large for the batched kernel (its encode runs as several launches)";
    return kEUnsupported;
  }
  for (int i = 0; i < s.plan->nin; i++) {
    if (!data[i]) {
      err = "data block is NULL";
      return kEInval;
    }
    s.ptrs.push_back(const_cast<uint8_t *>(data[i]));
  }
  for (int j = 0; j < s.plan->nout; j++) s.ptrs.push_back(out[j]);
  s.nbytes = nbytes;
  s.user_bytes = (int64_t)c->m.K * nbytes;
  s.work = s.plan->nnz;
  finish_stripe(s);
  return kOk;
}

bool bitsliced_encode_split(const pmrc_code *c, const uint8_t *const *data, uint8_t *const *out,
                            size_t nbytes, BitslicedEncode &e) {
  if (c->m.w != 8 || c->bs_id < 0 || c->encode_kernel == PMRC_KERNEL_GENERIC || nbytes < 32 ||
      (size_t)c->m.K * nbytes < kBatchBitslicedMinBytes || !c->encode->parts.empty())
    return false;
  const Plan &P = *c->encode;
  for (int i = 0; i < P.nin; i++)
    if (!data[i] || (uintptr_t)data[i] % 16) return false;
  for (int j = 0; j < P.nout; j++)
    if (!out[j] || (uintptr_t)out[j] % 16) return false;
  e.id = c->bs_id;
  e.in.assign(data, data + P.nin);
  e.out.assign(out, out + P.nout);
  e.nbytes = nbytes & ~(size_t)31;
  return true;
}

int stripe_repair(const pmrc_code *c, int f, const int *helpers, const uint8_t *const *blocks,
                  uint8_t *const *out, size_t nbytes, WorkStripe &s, std::string &err) {
  s = WorkStripe();
  if (c->m.w != 8) {
    err = "batched and served operations take GF(2^8) codes";
    return kEUnsupported;
  }
  if (c->m.alpha > 16) {
    err = "batched repair needs alpha <= 16";
    return kEUnsupported;
  }
  s.type = 1;
  int rc = fused_repair_plan(c, f, helpers, s.fplan, err);
  if (rc) return rc;
  const FusedRepairHeader &h = s.fplan->header;
  for (uint32_t q = 0; q < h.d; q++)
    for (uint32_t j = 0; j < h.alpha; j++) {
      const uint8_t *p = blocks[q * h.alpha + j];
      bool used = false;
      for (uint32_t i = 0; i < h.nz; i++) used |= h.nzidx[i] == j;
      if (used && !p) {
        err = "a helper block the repair reads is NULL";
        return kEInval;
      }
      s.ptrs.push_back(const_cast<uint8_t *>(p));
    }
  for (uint32_t r = 0; r < h.alpha; r++) {
    if (!out[r]) {
      err = "output block is NULL";
      return kEInval;
    }
    s.ptrs.push_back(out[r]);
  }
  s.nbytes = nbytes;
  s.user_bytes = (int64_t)c->m.alpha * nbytes;
  s.work = (int64_t)h.d * (h.direct ? 0 : h.nz) + (int64_t)h.d * h.alpha;
  finish_stripe(s);
  return kOk;
}

int stripe_decode(const pmrc_code *c, const int *nodes, const uint8_t *const *node_blocks,
                  uint8_t *const *data_out, size_t nbytes, WorkStripe &s, std::string &err) {
  s = WorkStripe();
  if (c->m.w != 8) {
    err = "batched and served operations take GF(2^8) codes";
    return kEUnsupported;
  }
  {
    std::vector<char> seen(c->m.n, 0);
    for (int i = 0; i < c->m.k; i++) {
      if (nodes[i] < 0 || nodes[i] >= c->m.n || seen[nodes[i]]) {
        err = "nodes: out of range or repeated node id";
        return kEInval;
      }
      seen[nodes[i]] = 1;
    }
  }
  std::vector<char> want;
  decode_wanted(c, nodes, node_blocks, data_out, want);
  s.type = 0;
  int rc = decode_plan(c, nodes, want, s.plan, err);
  if (rc) return rc;
  if (!s.plan->parts.empty()) {
    err = "code too large for the batched kernel (its reconstruction runs as several launches)";
    return kEUnsupported;
  }
  const int KA = c->m.k * c->m.alpha, K = c->m.K;  // node blocks read, data blocks out
  for (int i = 0; i < KA; i++) s.ptrs.push_back(const_cast<uint8_t *>(node_blocks[i]));
  for (int r = 0; r < K; r++) s.ptrs.push_back(want[r] ? data_out[r] : nullptr);
  for (const auto &blk : s.plan->blocks)
    for (uint16_t in : blk.inputs)
      if (!node_blocks[in]) {
        err = "a block the decode reads is NULL";
        return kEInval;
      }
  s.nbytes = nbytes;
  s.user_bytes = (int64_t)K * nbytes;
  s.work = s.plan->nnz;
  finish_stripe(s);
  return kOk;
}

int worklist_build(const std::vector<const WorkStripe *> &stripes, int work_bytes,
                   int target_items, WorkList &wl, std::string &err) {
  const uint64_t tile = (uint64_t)kThreads * kVec;  // region items: 4 KiB tiles
  const uint64_t rtile = (uint64_t)kRepTile;        // fused repair items: 1 KiB tiles
  std::vector<const WorkStripe *> order(stripes);
  std::stable_sort(order.begin(), order.end(), [](const WorkStripe *x, const WorkStripe *y) {
    return (double)x->work * x->nbytes > (double)y->work * y->nbytes;
  });
  // No item may cost more than 1/target_items of the whole list (products
  // per item = bytes of its range x products per byte column): a stripe
  // with few byte columns but many products (a large-k repair or
  // reconstruction over short blocks) is cut into finer ranges, down to one
  // tile, so that it spreads over the grid instead of a few CTAs.
  double total = 0;
  for (const WorkStripe *S : order) total += (double)S->work * (double)S->nbytes;
  const double cap = target_items > 0 ? total / target_items : 0;
  for (const WorkStripe *S : order) {
    if (S->nbytes == 0) continue;
    const uint32_t base = (uint32_t)wl.ptrs.size();
    wl.ptrs.insert(wl.ptrs.end(), S->ptrs.begin(), S->ptrs.end());
    wl.user_bytes += S->user_bytes;
    const uint64_t unit = S->type == 0 ? tile : rtile;
    const uint32_t nunits = (uint32_t)((S->nbytes + unit - 1) / unit);
    uint32_t span = (uint32_t)std::max<uint64_t>(1, (uint64_t)work_bytes / unit);
    double per_unit = (double)unit * (double)S->work;  // products of one unit of the stripe
    if (S->type == 0) {
      size_t widest = 1;
      for (const PlanBlock &b : S->plan->blocks)
        widest = std::max(widest, b.inputs.size() * b.rows.size());
      per_unit = (double)unit * (double)widest;
    }
    if (cap > 0 && per_unit * span > cap)
      span = (uint32_t)std::max(1.0, std::floor(cap / per_unit));
    const void *image = nullptr;
    int rc = S->type == 0 ? S->plan->device_image(&image, err) : S->fplan->device_image(&image, err);
    if (rc) return rc;
    wl.ptr_area = std::max(wl.ptr_area, (S->ptrs.size() * sizeof(uint8_t *) + 15) & ~(size_t)15);
    for (uint32_t t0 = 0; t0 < nunits; t0 += span) {
      WorkItem w{};
      w.image = static_cast<const uint8_t *>(image);
      w.nbytes = S->nbytes;
      w.ptr_off = base;
      w.nptrs = (uint32_t)S->ptrs.size();
      w.tile0 = t0;
      w.ntiles = std::min(span, nunits - t0);
      w.aligned = S->aligned ? 1 : 0;
      if (S->type == 0) {
        const Plan &P = *S->plan;
        w.type = 0;
        w.stride = (uint16_t)P.R;
        w.idx_base = (uint32_t)P.idx_base;
        w.tab4_base = (uint32_t)P.tab4_base;
        w.tab1_base = (uint32_t)P.tab1_base;
        for (size_t blk = 0; blk < P.blocks.size(); blk++) {
          w.block = (uint16_t)blk;
          wl.items.push_back(w);
        }
        wl.smem = std::max(wl.smem,
                           (size_t)P.max_entries * 20 + (size_t)(P.max_inputs + P.R) * 2 + 16);
      } else {
        w.type = 1;
        wl.items.push_back(w);
        wl.smem = std::max(wl.smem, fused_repair_smem(S->fplan->header) + 64);
      }
    }
  }
  wl.smem += wl.ptr_area;
  return kOk;
}

static std::atomic<uint64_t> g_batch_smem_set[kMaxDevices];

int worklist_ctas_per_sm(size_t smem) {
  if (smem > 48 * 1024)
    allow_max_smem(reinterpret_cast<const void *>(batch_kernel<kBatchR>), g_batch_smem_set, 0);
  int fit = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, batch_kernel<kBatchR>, kThreads, smem);
  return fit < 1 ? 1 : fit;
}

cudaError_t worklist_launch(const WorkItem *items, int nitems, uint8_t *const *ptrs,
                            unsigned *d_counter, unsigned grid, size_t smem, size_t ptr_area,
                            cudaStream_t stream) {
  if (smem > 48 * 1024) {
    const cudaError_t e =
        allow_max_smem(reinterpret_cast<const void *>(batch_kernel<kBatchR>), g_batch_smem_set, 0);
    if (e != cudaSuccess) return e;
  }
  BatchArgs args;
  args.items = items;
  args.nitems = nitems;
  args.ptrs = ptrs;
  args.counter = d_counter;
  args.ptr_area = (uint32_t)ptr_area;
  args.k = MulConsts{2u, 16u, 1u << 16, 1u << 26, 1u << 29, 1u << 30};
  cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  batch_kernel<kBatchR><<<grid, kThreads, smem, stream>>>(args);
  return cudaGetLastError();
}

}  // namespace pmrc

using namespace pmrc;

struct pmrc_batch {
  std::vector<WorkStripe> stripes;        // items of the batched kernel
  std::vector<BitslicedEncode> bitsliced;  // large encodes: own launches in the graph
  int count = 0;                           // stripes added
  bool built = false;
  // device state
  uint8_t **d_ptrs = nullptr;
  WorkItem *d_items = nullptr;
  unsigned *d_counter = nullptr;
  int nitems = 0;
  unsigned grid = 0;
  size_t smem = 0, ptr_area = 0;
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

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;  // shape -> (work_bytes, ctas_per_sm)

int bfail(int rc, const std::string &msg) {
  pmrc::set_last_error(msg);
  return rc;
}

std::string signature(const pmrc_batch *b) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  // operation kinds, work per column and size buckets present in the batch
  std::map<std::string, int> cnt;
  for (auto &s : b->stripes) {
    int lg = 0;
    while ((1ull << lg) < s.nbytes) lg++;
    cnt[std::to_string(s.type) + "/" + std::to_string(s.work) + "/" + std::to_string(lg / 2)]++;
  }
  std::string sig = std::string(prop.name) + "|" + std::to_string(prop.multiProcessorCount);
  for (auto &kv : cnt) sig += "|" + kv.first;
  return sig;
}

int build_device(pmrc_batch *b, int work_bytes, int ctas_per_sm, std::string &err) {
  b->release_device();
  int dev = 0, sms = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return kECuda;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  std::vector<const WorkStripe *> sp;
  for (auto &s : b->stripes) sp.push_back(&s);
  WorkList wl;
  if (!sp.empty()) {
    int rc = worklist_build(sp, work_bytes, kItemsPerCta * sms * std::max(1, ctas_per_sm), wl, err);
    if (rc) return rc;
  }
  // the bitsliced kernels' shared-memory setting is made before the capture
  for (const auto &be : b->bitsliced) {
    const cudaError_t pe = bitslice_prepare(be.id);
    if (pe != cudaSuccess) {
      err = std::string("bitsliced encode setup: ") + cudaGetErrorString(pe);
      return kECuda;
    }
  }
  e = cudaMalloc(&b->d_ptrs, std::max<size_t>(1, wl.ptrs.size()) * sizeof(uint8_t *));
  if (e == cudaSuccess && !wl.ptrs.empty())
    e = cudaMemcpy(b->d_ptrs, wl.ptrs.data(), wl.ptrs.size() * sizeof(uint8_t *),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMalloc(&b->d_items, std::max<size_t>(1, wl.items.size()) * sizeof(WorkItem));
  if (e == cudaSuccess && !wl.items.empty())
    e = cudaMemcpy(b->d_items, wl.items.data(), wl.items.size() * sizeof(WorkItem),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned));
  if (e != cudaSuccess) {
    err = std::string("batch work list upload: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? kENoMem : kECuda;
  }
  b->nitems = (int)wl.items.size();
  b->smem = wl.smem;
  b->ptr_area = wl.ptr_area;
  const int per_sm = std::max(1, std::min(ctas_per_sm, worklist_ctas_per_sm(wl.smem)));
  b->grid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((int64_t)sms * per_sm, std::max(1, b->nitems)));
  // graph: counter reset + persistent kernel, then one launch of the
  // built-in bitsliced kernel per large encode
  e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t le = cudaSuccess;
    if (b->nitems > 0)
      le = worklist_launch(b->d_items, b->nitems, b->d_ptrs, b->d_counter, b->grid, b->smem, b->ptr_area,
                           b->cap);
    for (const auto &be : b->bitsliced)
      if (le == cudaSuccess)
        le = bitslice_launch(be.id, be.in.data(), be.out.data(), be.nbytes, b->cap);
    e = cudaStreamEndCapture(b->cap, &b->graph);
    if (le != cudaSuccess) e = le;
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

int add(pmrc_batch *b, int rc, WorkStripe &&s, const std::string &err) {
  if (rc) return bfail(rc, err);
  b->user_bytes += s.user_bytes;
  b->stripes.push_back(std::move(s));
  return b->count++;
}

const char *kErrBuilt = "batch already built: create a new batch to add stripes";

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
  if (b->built) return bfail(PMRC_EBUSY, kErrBuilt);
  WorkStripe s;
  std::string err;
  BitslicedEncode be;
  if (bitsliced_encode_split(c, data, out, nbytes, be)) {
    if (be.nbytes < nbytes) {  // the ragged tail joins the batched kernel's items
      std::vector<const uint8_t *> in2(be.in.size());
      std::vector<uint8_t *> out2(be.out.size());
      for (size_t i = 0; i < in2.size(); i++) in2[i] = be.in[i] + be.nbytes;
      for (size_t j = 0; j < out2.size(); j++) out2[j] = be.out[j] + be.nbytes;
      int rc = stripe_encode(c, in2.data(), out2.data(), nbytes - be.nbytes, s, err);
      if (rc) return bfail(rc, err);
      s.user_bytes = 0;  // counted with the stripe below
      b->stripes.push_back(std::move(s));
    }
    b->user_bytes += (int64_t)c->m.K * nbytes;
    b->bitsliced.push_back(std::move(be));
    return b->count++;
  }
  int rc = stripe_encode(c, data, out, nbytes, s, err);
  return add(b, rc, std::move(s), err);
}

int pmrc_batch_add_repair(pmrc_batch *b, const pmrc_code *c, int f, const int *helpers,
                          const uint8_t *const *blocks, uint8_t *const *out, size_t nbytes) {
  if (!b || !c || !helpers || !blocks || !out) return bfail(PMRC_EINVAL, "NULL argument");
  if (b->built) return bfail(PMRC_EBUSY, kErrBuilt);
  WorkStripe s;
  std::string err;
  int rc = stripe_repair(c, f, helpers, blocks, out, nbytes, s, err);
  return add(b, rc, std::move(s), err);
}

int pmrc_batch_add_decode(pmrc_batch *b, const pmrc_code *c, const int *nodes,
                          const uint8_t *const *node_blocks, uint8_t *const *data_out,
                          size_t nbytes) {
  if (!b || !c || !nodes || !node_blocks || !data_out) return bfail(PMRC_EINVAL, "NULL argument");
  if (b->built) return bfail(PMRC_EBUSY, kErrBuilt);
  WorkStripe s;
  std::string err;
  int rc = stripe_decode(c, nodes, node_blocks, data_out, nbytes, s, err);
  return add(b, rc, std::move(s), err);
}

int pmrc_batch_build(pmrc_batch *b, int work_bytes, int ctas_per_sm) {
  PMRC_TRACE("pmrc_batch_build");
  if (!b) return bfail(PMRC_EINVAL, "NULL batch");
  if (b->stripes.empty() && b->bitsliced.empty()) return bfail(PMRC_EINVAL, "empty batch");
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
  PMRC_TRACE("pmrc_batch_launch");
  if (!b || !b->built) return bfail(PMRC_EINVAL, "batch not built");
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess)
    return bfail(PMRC_ECUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
  return PMRC_OK;
}

int pmrc_batch_tune(pmrc_batch *b, pmrc_stream_t stream, int *best_out) {
  PMRC_TRACE("pmrc_batch_tune");
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
  info[0] = b->count;
  info[1] = b->nitems;
  info[2] = b->grid;
  info[3] = b->work_bytes;
  info[4] = b->ctas_per_sm;
  info[5] = b->user_bytes;
  info[6] = (int64_t)b->bitsliced.size();
  info[7] = (int64_t)b->smem;
  return PMRC_OK;
}

}  // extern "C"
