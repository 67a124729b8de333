// Fused single-node repair on one GPU: the d helper projections
// p_h = sum_j phi_f[j] Y[alpha h + j] and the newcomer apply
// node_f = D p (D = [I | lambda_f I] Psi_H^-1) in one kernel.
//
// In the paper's system the helpers send p_h over the network (Sec. 2, 3.3).
// When helpers and newcomer share a GPU, the projections need not visit
// device memory at all: a CTA covers 1 KiB of byte column with 4 lanes of 64
// threads, the lanes split the d projections (stage 1, all of a helper's
// loads issued before they are used), park them in shared memory, and then
// split the alpha output rows (stage 2, repair_dev.cuh).  When phi_f has a
// single non-zero equal to 1 (sparse code, failed node among the alpha
// first) p_h is a block the helper already stores, and the newcomer reads it
// in place.
#include <cuda_runtime.h>

#include <cstring>

#include "device_info.h"
#include "gf256.h"
#include "plan.h"
#include "repair.h"

namespace pmrc {
namespace {

#include "region_dev.cuh"
#include "repair_dev.cuh"

constexpr int kRepMaxPtr = 512;

struct RepairArgs {
  const uint8_t *image;  // FusedRepairHeader + split tables (device)
  uint64_t nbytes;
  uint32_t ntiles;       // 1 KiB tiles
  int aligned;
  MulConsts k;
  uint8_t *ptr[kRepMaxPtr];  // d*alpha helper blocks, then alpha outputs
};

// Shared memory: split tables, then the d x 64 projection vectors.
template <int NZ>
__global__ void __launch_bounds__(kThreads, 2) fused_repair_kernel(const __grid_constant__ RepairArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint16_t s_nz[16];
  const FusedRepairHeader *hp = reinterpret_cast<const FusedRepairHeader *>(a.image);
  const int d = hp->d, alpha = hp->alpha, nz = hp->nz, rl = hp->rl;
  const bool direct = hp->direct != 0;
  const uint32_t tab4_off = hp->tab4_off, tab1_off = hp->tab1_off;
  if (threadIdx.x < 16) s_nz[threadIdx.x] = hp->nzidx[threadIdx.x];
  const int n1 = nz, n2 = d * 4 * rl;
  uint4 *proj = reinterpret_cast<uint4 *>(smem);
  uint4 *t1a = proj + (size_t)d * kRepCols;
  uint4 *t2a = t1a + n1;
  uint32_t *t1b = reinterpret_cast<uint32_t *>(t2a + n2);
  uint32_t *t2b = t1b + n1;
  {
    const uint4 *g4 = reinterpret_cast<const uint4 *>(a.image + tab4_off);
    const uint32_t *g1 = reinterpret_cast<const uint32_t *>(a.image + tab1_off);
    for (int i = threadIdx.x; i < n1 + n2; i += kThreads) {
      t1a[i] = g4[i];  // t2a follows t1a contiguously, as in the image
      t1b[i] = g1[i];
    }
  }
  __syncthreads();
  const MulConsts k = a.k;
  const bool vec = a.aligned != 0;
  for (uint32_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x)
    fused_repair_tile<NZ>(a.ptr, (uint64_t)tile * kRepTile, a.nbytes, vec, d, alpha, nz, direct,
                          s_nz, t1a, t1b, t2a, t2b, rl, proj, k);
}

// Fills the pointer table of a launch; checks NULL blocks and alignment.
int repair_pointers(const FusedRepairHeader &h, const uint8_t *const *helper_blocks,
                    uint8_t *const *out, RepairArgs &a, std::string &err) {
  const int d = h.d, alpha = h.alpha;
  memset(a.ptr, 0, sizeof a.ptr);
  bool aligned = true;
  for (int q = 0; q < d; q++)
    for (int j = 0; j < alpha; j++) {
      const uint8_t *p = helper_blocks[q * alpha + j];
      a.ptr[q * alpha + j] = const_cast<uint8_t *>(p);
      bool used = false;
      for (uint32_t i = 0; i < h.nz; i++) used |= (h.nzidx[i] == j);
      if (used && !p) {
        err = "a helper block the repair reads is NULL";
        return kEInval;
      }
      if (p) aligned = aligned && ((uintptr_t)p % kVec == 0);
    }
  for (int r = 0; r < alpha; r++) {
    if (!out[r]) {
      err = "output block is NULL";
      return kEInval;
    }
    a.ptr[d * alpha + r] = out[r];
    aligned = aligned && ((uintptr_t)out[r] % kVec == 0);
  }
  a.aligned = aligned ? 1 : 0;
  return kOk;
}

cudaError_t repair_launch(const FusedRepairHeader &h, RepairArgs &a, const void *image,
                          size_t nbytes, cudaStream_t stream) {
  a.image = static_cast<const uint8_t *>(image);
  a.nbytes = nbytes;
  a.ntiles = (uint32_t)((nbytes + kRepTile - 1) / kRepTile);
  a.k = MulConsts{2u, 16u, 1u << 16, 1u << 26, 1u << 29, 1u << 30};
  const unsigned grid = fused_repair_grid(a.ntiles);
  const size_t smem = fused_repair_smem(h);
  if (h.nz <= 8)
    fused_repair_kernel<8><<<grid, kThreads, smem, stream>>>(a);
  else
    fused_repair_kernel<16><<<grid, kThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

// Fixed scratch of pmrc_repair_noalloc: room for the repair's header and
// split tables.  Every GPU that loads the library holds it until the
// process exits.
constexpr size_t kNoAllocTableBytes = 64u << 10;
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocTableBytes];

std::shared_ptr<FusedRepairPlan> make_fused_repair_plan(const std::vector<uint8_t> &phi,
                                                        const Mat &D) {
  static const SplitTables split = make_split_tables();
  auto p = std::make_shared<FusedRepairPlan>();
  const int alpha = D.rows, d = D.cols;
  FusedRepairHeader h{};
  h.d = (uint32_t)d;
  h.alpha = (uint32_t)alpha;
  std::vector<int> nzl;
  for (int j = 0; j < (int)phi.size(); j++)
    if (phi[j]) nzl.push_back(j);
  h.nz = (uint32_t)nzl.size();
  for (size_t i = 0; i < nzl.size(); i++) h.nzidx[i] = (uint16_t)nzl[i];
  h.direct = (nzl.size() == 1 && phi[nzl[0]] == 1) ? 1u : 0u;
  h.rl = (uint32_t)((alpha + 3) / 4);
  const size_t n1 = nzl.size(), n2 = (size_t)d * 4 * h.rl;
  h.tab4_off = (uint32_t)((sizeof(FusedRepairHeader) + 15) & ~(size_t)15);
  h.tab1_off = h.tab4_off + (uint32_t)((n1 + n2) * sizeof(TabEntry));
  p->image.assign(h.tab1_off + (n1 + n2) * 4 + 16, 0);
  auto put = [&](size_t e, uint8_t c) {
    const uint32_t *w = split.w[c];
    TabEntry t{w[0], w[1], w[2], w[3]};
    memcpy(p->image.data() + h.tab4_off + e * sizeof(TabEntry), &t, sizeof t);
    memcpy(p->image.data() + h.tab1_off + e * 4, &w[4], 4);
  };
  for (size_t i = 0; i < n1; i++) put(i, phi[nzl[i]]);
  for (int q = 0; q < d; q++)  // entry (input q, lane l, m) holds row l + 4m
    for (int l = 0; l < 4; l++)
      for (uint32_t m = 0; m < h.rl; m++) {
        const int r = l + 4 * (int)m;
        put(n1 + ((size_t)q * 4 + l) * h.rl + m, r < alpha ? D.at(r, q) : 0);
      }
  memcpy(p->image.data(), &h, sizeof h);
  p->header = h;
  return p;
}

size_t fused_repair_smem(const FusedRepairHeader &h) {
  return (size_t)h.d * kRepCols * kVec + (size_t)(h.nz + (size_t)h.d * 4 * h.rl) * 20;
}

static int check_repair_size(const FusedRepairHeader &h, std::string &err) {
  if ((h.d + 1) * h.alpha > (uint32_t)kRepMaxPtr || h.alpha > 16 || h.nz > 16) {
    err = "code too large for the fused repair kernel";
    return kEUnsupported;
  }
  return kOk;
}

int launch_fused_repair(FusedRepairPlan &plan, const uint8_t *const *helper_blocks,
                        uint8_t *const *out, size_t nbytes, cudaStream_t stream,
                        std::string &err) {
  const FusedRepairHeader &h = plan.header;
  int rc = check_repair_size(h, err);
  if (rc) return rc;
  RepairArgs a;
  rc = repair_pointers(h, helper_blocks, out, a, err);
  if (rc) return rc;
  if (nbytes == 0) return kOk;
  const void *image = nullptr;
  rc = plan.device_image(&image, err);
  if (rc) return rc;
  cudaError_t e = repair_launch(h, a, image, nbytes, stream);
  if (e != cudaSuccess) {
    err = std::string("fused repair launch: ") + cudaGetErrorString(e);
    return kECuda;
  }
  return kOk;
}

int launch_fused_repair_noalloc(const FusedRepairPlan &plan, const uint8_t *const *helper_blocks,
                                uint8_t *const *out, size_t nbytes, cudaStream_t stream,
                                std::string &err) {
  const FusedRepairHeader &h = plan.header;
  int rc = check_repair_size(h, err);
  if (rc) return rc;
  if (plan.image.size() > kNoAllocTableBytes) {
    err = "repair tables exceed the 64 KiB fixed scratch";
    return kEUnsupported;
  }
  RepairArgs a;
  rc = repair_pointers(h, helper_blocks, out, a, err);
  if (rc) return rc;
  if (nbytes == 0) return kOk;
  // device address of the fixed scratch on the calling thread's current
  // device, looked up on every call (a host-side query): the host-side name
  // is not a device address, and a cached address would go stale if the
  // device's context were torn down and the module loaded again
  uint8_t *base = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void **)&base, g_noalloc_scratch);
  if (e != cudaSuccess) {
    err = std::string("cudaGetSymbolAddress(fixed scratch): ") + cudaGetErrorString(e);
    return kECuda;
  }
  e = cudaMemcpyAsync(base, plan.image.data(), plan.image.size(), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = repair_launch(h, a, base, nbytes, stream);
  if (e != cudaSuccess) {
    err = std::string("fused repair (fixed scratch): ") + cudaGetErrorString(e);
    return kECuda;
  }
  return kOk;
}

unsigned fused_repair_grid(uint32_t ntiles) {
  const uint32_t cap = (uint32_t)current_sm_count() * 2;
  return ntiles < cap ? (ntiles ? ntiles : 1) : cap;
}

int FusedRepairPlan::device_image(const void **out, std::string &err) {
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
    err = std::string("cudaMalloc(repair plan): ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? kENoMem : kECuda;
  }
  e = cudaMemcpy(p, image.data(), image.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p);
    err = std::string("cudaMemcpy(repair plan): ") + cudaGetErrorString(e);
    return kECuda;
  }
  dev[devid] = p;
  *out = p;
  return kOk;
}

FusedRepairPlan::~FusedRepairPlan() {
  for (auto &kv : dev) {
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(kv.first);
    cudaFree(kv.second);
    if (cur >= 0) cudaSetDevice(cur);
  }
}

}  // namespace pmrc
