// GF(2^8) region multiply-XOR over dense row blocks (sm_103a).
//
// Every operation of a linearized product-matrix code -- generator encode,
// systematic encode, helper projection, newcomer repair and reconstruction --
// is out[r] = sum_c M[r][c] * in[c] over byte blocks (Sec. 2 and 3.1 of the
// paper).  This kernel computes one dense block of M (up to R rows that
// share the same inputs) over one byte tile:
//
//   * each thread owns 16 consecutive bytes of every block of the tile;
//   * each input is read once (16 B, coalesced), cut into three bit fields
//     and then multiplied into all R rows held in registers;
//   * multiplication by a constant c is a GF(2)-linear map, so
//     c*x = T0[x & 7] ^ T1[(x >> 3) & 7] ^ T2[x >> 6] with 8-, 8- and 4-entry
//     tables; each table lookup of four bytes is one PRMT (byte permute)
//     whose selector nibbles are the bit fields (the GPU form of the split
//     tables the paper's CPU code uses, Sec. 4);
//   * the accumulators hold bytes in an interleaved lane order that makes
//     the selector construction cheap; two PRMTs per word restore byte order
//     before the 16-byte store;
//   * the split tables of every (input, row) coefficient of the block are
//     precomputed in the plan and staged in shared memory; a zero
//     coefficient has all-zero tables, so no coefficient needs a branch;
//   * for blocks of one or two rows a CTA loops over several byte tiles (the
//     tables are staged once per CTA), and blocks of few inputs load all of a
//     tile's inputs before using the first.
#include "device_info.h"
#include "gf256.h"
#include "region.h"

namespace pmrc {

namespace {

#include "region_dev.cuh"

template <int MAXP>
struct RegionArgs {
  const uint8_t *image;  // plan device image
  uint64_t nbytes;       // block size
  uint32_t idx_base;     // byte offset of the uint16 slot array in image
  uint32_t tab4_base;    // byte offset of the TabEntry array
  uint32_t tab1_base;    // byte offset of the T2 word array
  uint32_t ntiles;       // ceil(nbytes / (blockDim.x * kVec))
  int aligned;           // every pointer is 16-byte aligned
  int accumulate;        // XOR the results into the outputs (a later input chunk)
  MulConsts k;
  uint8_t *ptr[MAXP];    // input slots, then output slots
};

template <int R, int MAXP>
__global__ void __launch_bounds__(kThreads)
    region_kernel(const __grid_constant__ RegionArgs<MAXP> a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const BlockDesc d = reinterpret_cast<const BlockDesc *>(a.image)[blockIdx.x];
  const int nin = d.ninputs, nrows = d.nrows, nent = nin * R;
  uint4 *s_tab4 = reinterpret_cast<uint4 *>(smem);
  uint32_t *s_tab1 = reinterpret_cast<uint32_t *>(smem + (size_t)nent * 16);
  uint16_t *s_slot = reinterpret_cast<uint16_t *>(smem + (size_t)nent * 20);
  {
    const uint4 *g4 = reinterpret_cast<const uint4 *>(a.image + a.tab4_base) + d.tab_off;
    const uint32_t *g1 = reinterpret_cast<const uint32_t *>(a.image + a.tab1_base) + d.tab_off;
    const uint16_t *idx = reinterpret_cast<const uint16_t *>(a.image + a.idx_base);
    for (int i = threadIdx.x; i < nent; i += blockDim.x) {
      s_tab4[i] = g4[i];
      s_tab1[i] = g1[i];
    }
    for (int i = threadIdx.x; i < nin; i += blockDim.x) s_slot[i] = idx[d.in_off + i];
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) s_slot[nin + i] = idx[d.out_off + i];
  }
  __syncthreads();

  const MulConsts k = a.k;
  const bool vec = a.aligned != 0;
  for (uint32_t tile = blockIdx.y; tile < a.ntiles; tile += gridDim.y) {
    const uint64_t off = ((uint64_t)tile * blockDim.x + threadIdx.x) * kVec;
    if (off >= a.nbytes) continue;
    uint32_t acc[R][4];
    auto fetch = [&](int i) { return load16(a.ptr[s_slot[i]], off, a.nbytes, vec); };
    if (R <= 2 && nin <= 8)
      mac_block_preload<R>(acc, nin, nrows, R, s_tab4, s_tab1, k, fetch);
    else
      mac_block<R>(acc, nin, nrows, R, s_tab4, s_tab1, k, fetch);
#pragma unroll
    for (int r = 0; r < R; r++) {
      if (r < nrows) {
        uint8_t *o = a.ptr[s_slot[nin + r]];
        if (!o) continue;
        uint4 v = acc_bytes(acc[r]);
        if (a.accumulate) {
          const uint4 p = load16(o, off, a.nbytes, vec);
          v = make_uint4(v.x ^ p.x, v.y ^ p.y, v.z ^ p.z, v.w ^ p.w);
        }
        store16(o, off, a.nbytes, vec, v);
      }
    }
  }
}

template <int R, int MAXP>
cudaError_t launch_t(const Plan &plan, const void *image, const uint8_t *const *in,
                     uint8_t *const *out, size_t nbytes, bool aligned, bool accumulate,
                     cudaStream_t st) {
  RegionArgs<MAXP> a;
  a.image = static_cast<const uint8_t *>(image);
  a.nbytes = nbytes;
  a.idx_base = (uint32_t)plan.idx_base;
  a.tab4_base = (uint32_t)plan.tab4_base;
  a.tab1_base = (uint32_t)plan.tab1_base;
  const int sms = current_sm_count();
  const uint64_t nb = plan.blocks.size();
  // 128-thread CTAs on 2 KiB tiles for blocks of one or two rows (their
  // tiles are mostly loads, and smaller CTAs leave a shorter tail) and for
  // launches of few blocks on short columns (a newcomer apply, say), which
  // would leave most SMs idle with 4 KiB tiles
  unsigned threads = kThreads;
  if (R <= 2 || nb * ((nbytes + (uint64_t)kThreads * kVec - 1) / ((uint64_t)kThreads * kVec)) <
                    (uint64_t)sms * 4)
    threads = kThreads / 2;
  const uint64_t tile = (uint64_t)threads * kVec;
  a.ntiles = (uint32_t)((nbytes + tile - 1) / tile);
  a.aligned = aligned ? 1 : 0;
  a.accumulate = accumulate ? 1 : 0;
  a.k = MulConsts{2u, 16u, 1u << 16, 1u << 26, 1u << 29, 1u << 30};
  for (int i = 0; i < plan.nin; i++) a.ptr[i] = const_cast<uint8_t *>(in[i]);
  for (int j = 0; j < plan.nout; j++) a.ptr[plan.nin + j] = out[j];
  for (int j = plan.nin + plan.nout; j < MAXP; j++) a.ptr[j] = nullptr;
  // blocks of one or two rows do little work per tile: their CTAs loop over
  // several tiles (about two waves of CTAs in all) so the block's tables are
  // staged once per CTA; bigger blocks keep one tile per CTA, which balances
  // the tail better
  uint64_t gy = a.ntiles;
  if (R <= 2) {
    const uint64_t target = (uint64_t)sms * 16;  // 8 resident CTAs per SM, two waves
    gy = (target + nb - 1) / nb;
    if (gy > a.ntiles) gy = a.ntiles;
  }
  if (gy > 65535u) gy = 65535u;
  if (gy < 1) gy = 1;
  const dim3 grid((unsigned)nb, (unsigned)gy);
  const size_t smem = (size_t)plan.max_entries * 20 + (size_t)(plan.max_inputs + R) * 2 + 16;
  if (smem > 48 * 1024) {  // once per device for this kernel
    static std::atomic<uint64_t> smem_set[kMaxDevices];
    const cudaError_t e =
        allow_max_smem(reinterpret_cast<const void *>(region_kernel<R, MAXP>), smem_set, 0);
    if (e != cudaSuccess) return e;
  }
  region_kernel<R, MAXP><<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int MAXP>
cudaError_t launch_p(const Plan &plan, const void *image, const uint8_t *const *in,
                     uint8_t *const *out, size_t nbytes, bool aligned, bool acc, cudaStream_t st) {
  switch (plan.R) {
    case 1: return launch_t<1, MAXP>(plan, image, in, out, nbytes, aligned, acc, st);
    case 2: return launch_t<2, MAXP>(plan, image, in, out, nbytes, aligned, acc, st);
    case 4: return launch_t<4, MAXP>(plan, image, in, out, nbytes, aligned, acc, st);
    case 8: return launch_t<8, MAXP>(plan, image, in, out, nbytes, aligned, acc, st);
    default: return launch_t<16, MAXP>(plan, image, in, out, nbytes, aligned, acc, st);
  }
}

int launch_one(Plan &plan, const uint8_t *const *in, uint8_t *const *out, size_t nbytes,
               bool accumulate, cudaStream_t stream, std::string &err) {
  if (plan.nin + plan.nout > kMaxSlots) {
    err = "too many blocks for one launch (input + output pointers > 1024)";
    return kEUnsupported;
  }
  if (nbytes == 0 || plan.blocks.empty()) return kOk;
  bool aligned = true;
  for (const auto &b : plan.blocks)
    for (uint16_t s : b.inputs) {
      if (!in[s]) {
        err = "a block the operation reads is NULL";
        return kEInval;
      }
      aligned = aligned && ((uintptr_t)in[s] % kVec == 0);
    }
  for (int j = 0; j < plan.nout; j++) aligned = aligned && ((uintptr_t)out[j] % kVec == 0);
  const void *image = nullptr;
  int rc = plan.device_image(&image, err);
  if (rc) return rc;
  cudaError_t e =
      (plan.nin + plan.nout <= 256)
          ? launch_p<256>(plan, image, in, out, nbytes, aligned, accumulate, stream)
          : launch_p<kMaxSlots>(plan, image, in, out, nbytes, aligned, accumulate, stream);
  if (e != cudaSuccess) {
    err = std::string("region kernel launch: ") + cudaGetErrorString(e);
    return kECuda;
  }
  return kOk;
}

}  // namespace

int launch_region(Plan &plan, const uint8_t *const *in, uint8_t *const *out, size_t nbytes,
                  cudaStream_t stream, std::string &err) {
  if (plan.parts.empty()) return launch_one(plan, in, out, nbytes, false, stream, err);
  // a plan too large for one launch: its parts in order, on the same stream
  // (an accumulating part follows the part that wrote its outputs); the
  // inputs are checked before the first part runs
  if (nbytes == 0) return kOk;
  for (int s : plan_reads(plan))
    if (!in[s]) {
      err = "a block the operation reads is NULL";
      return kEInval;
    }
  std::vector<const uint8_t *> in2;
  std::vector<uint8_t *> out2;
  for (auto &pt : plan.parts) {
    in2.resize(pt.in_cols.size());
    out2.resize(pt.out_slots.size());
    for (size_t i = 0; i < pt.in_cols.size(); i++) in2[i] = in[pt.in_cols[i]];
    for (size_t j = 0; j < pt.out_slots.size(); j++) out2[j] = out[pt.out_slots[j]];
    const int rc = launch_one(*pt.plan, in2.data(), out2.data(), nbytes, pt.accumulate, stream, err);
    if (rc) return rc;
  }
  return kOk;
}

}  // namespace pmrc
