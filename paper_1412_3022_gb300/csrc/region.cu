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
//     before the 16-byte store.
//
// Zero coefficients are skipped and a coefficient of 1 is a plain XOR, both
// on warp-uniform branches.
#include "gf256.h"
#include "region.h"

namespace pmrc {

__constant__ SplitTables c_split = make_split_tables();

namespace {

constexpr int kThreads = 256;
constexpr int kVec = 16;  // bytes per thread per tile

template <int MAXP>
struct RegionArgs {
  const uint8_t *image;  // plan device image
  uint64_t nbytes;       // block size
  uint32_t idx_base;     // byte offset of the uint16 slot array in image
  uint32_t coef_base;    // byte offset of the coefficient array in image
  uint32_t ntiles;       // ceil(nbytes / (kThreads * kVec))
  int aligned;           // every pointer is 16-byte aligned
  uint8_t *ptr[MAXP];    // input slots, then output slots
};

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t s) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
  return d;
}

// Selectors for 8 bytes (w0 = bytes 0-3, w1 = bytes 4-7).  Nibble 2m of the
// field word holds the field of byte m of w0, nibble 2m+1 that of byte m of
// w1; s[2q] feeds lanes (w0.b0, w1.b0, w0.b1, w1.b1), s[2q+1] lanes
// (w0.b2, w1.b2, w0.b3, w1.b3).
__device__ __forceinline__ void split_fields(uint32_t w0, uint32_t w1, uint32_t *s) {
  const uint32_t f0 = (w0 & 0x07070707u) | ((w1 & 0x07070707u) << 4);
  const uint32_t f1 = ((w0 >> 3) & 0x07070707u) | ((w1 << 1) & 0x70707070u);
  const uint32_t f2 = ((w0 >> 6) & 0x03030303u) | ((w1 >> 2) & 0x30303030u);
  s[0] = f0;
  s[1] = f0 >> 16;
  s[2] = f1;
  s[3] = f1 >> 16;
  s[4] = f2;
  s[5] = f2 >> 16;
}

template <int R>
__device__ __forceinline__ void mac_input(uint32_t (&acc)[R][4], const uint4 x,
                                          const uint8_t *coefs, int nrows) {
  uint32_t s[12];
  split_fields(x.x, x.y, s);
  split_fields(x.z, x.w, s + 6);
#pragma unroll
  for (int r = 0; r < R; r++) {
    if (r < nrows) {
      const uint32_t c = coefs[r];
      if (c > 1) {
        const uint32_t *T = c_split.w[c];
        const uint32_t t0 = T[0], t1 = T[1], t2 = T[2], t3 = T[3], t4 = T[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const uint32_t *sq = s + 6 * (q >> 1) + (q & 1);
          acc[r][q] ^= prmt(t0, t1, sq[0]) ^ prmt(t2, t3, sq[2]) ^ prmt(t4, t4, sq[4]);
        }
      } else if (c == 1) {
        acc[r][0] ^= prmt(x.x, x.y, 0x5140);
        acc[r][1] ^= prmt(x.x, x.y, 0x7362);
        acc[r][2] ^= prmt(x.z, x.w, 0x5140);
        acc[r][3] ^= prmt(x.z, x.w, 0x7362);
      }
    }
  }
}

__device__ __forceinline__ uint4 load16(const uint8_t *p, uint64_t off, uint64_t nbytes,
                                        bool vec) {
  if (vec && off + kVec <= nbytes) return __ldg(reinterpret_cast<const uint4 *>(p + off));
  uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
  for (int b = 0; b < kVec; b++)
    if (off + b < nbytes) w[b >> 2] |= (uint32_t)p[off + b] << (8 * (b & 3));
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void store16(uint8_t *p, uint64_t off, uint64_t nbytes, bool vec,
                                        uint4 v) {
  if (vec && off + kVec <= nbytes) {
    __stcs(reinterpret_cast<uint4 *>(p + off), v);
    return;
  }
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int b = 0; b < kVec; b++)
    if (off + b < nbytes) p[off + b] = (uint8_t)(w[b >> 2] >> (8 * (b & 3)));
}

template <int R, int MAXP>
__global__ void __launch_bounds__(kThreads)
    region_kernel(const __grid_constant__ RegionArgs<MAXP> a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const BlockDesc d = reinterpret_cast<const BlockDesc *>(a.image)[blockIdx.x];
  const int nin = d.ninputs, nrows = d.nrows;
  uint8_t *s_coef = smem;
  uint16_t *s_slot = reinterpret_cast<uint16_t *>(smem + ((nin * R + 15) & ~15));
  const uint16_t *idx = reinterpret_cast<const uint16_t *>(a.image + a.idx_base);
  const uint8_t *coef = a.image + a.coef_base + d.coef_off;
  for (int i = threadIdx.x; i < nin * R; i += kThreads) s_coef[i] = coef[i];
  for (int i = threadIdx.x; i < nin; i += kThreads) s_slot[i] = idx[d.in_off + i];
  for (int i = threadIdx.x; i < nrows; i += kThreads) s_slot[nin + i] = idx[d.out_off + i];
  __syncthreads();

  const bool vec = a.aligned != 0;
  for (uint32_t tile = blockIdx.y; tile < a.ntiles; tile += gridDim.y) {
    const uint64_t off = ((uint64_t)tile * kThreads + threadIdx.x) * kVec;
    if (off >= a.nbytes) continue;
    uint32_t acc[R][4];
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[r][q] = 0;
    if (nin > 0) {
      uint4 x = load16(a.ptr[s_slot[0]], off, a.nbytes, vec);
      for (int i = 0; i < nin; i++) {
        uint4 xn = x;
        if (i + 1 < nin) xn = load16(a.ptr[s_slot[i + 1]], off, a.nbytes, vec);
        mac_input<R>(acc, x, s_coef + i * R, nrows);
        x = xn;
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      if (r < nrows) {
        uint8_t *o = a.ptr[s_slot[nin + r]];
        if (o) {
          const uint4 v = make_uint4(prmt(acc[r][0], acc[r][1], 0x6420),
                                     prmt(acc[r][0], acc[r][1], 0x7531),
                                     prmt(acc[r][2], acc[r][3], 0x6420),
                                     prmt(acc[r][2], acc[r][3], 0x7531));
          store16(o, off, a.nbytes, vec, v);
        }
      }
    }
  }
}

template <int R, int MAXP>
cudaError_t launch_t(const Plan &plan, const void *image, const uint8_t *const *in,
                     uint8_t *const *out, size_t nbytes, bool aligned, cudaStream_t st) {
  RegionArgs<MAXP> a;
  a.image = static_cast<const uint8_t *>(image);
  a.nbytes = nbytes;
  a.idx_base = (uint32_t)plan.idx_base;
  a.coef_base = (uint32_t)plan.coef_base;
  const uint64_t tile = (uint64_t)kThreads * kVec;
  a.ntiles = (uint32_t)((nbytes + tile - 1) / tile);
  a.aligned = aligned ? 1 : 0;
  for (int i = 0; i < plan.nin; i++) a.ptr[i] = const_cast<uint8_t *>(in[i]);
  for (int j = 0; j < plan.nout; j++) a.ptr[plan.nin + j] = out[j];
  for (int j = plan.nin + plan.nout; j < MAXP; j++) a.ptr[j] = nullptr;
  const dim3 grid((unsigned)plan.blocks.size(), a.ntiles < 65535u ? a.ntiles : 65535u);
  const size_t smem = (size_t)((plan.max_inputs * R + 15) & ~15) +
                      (size_t)(plan.max_inputs + R) * sizeof(uint16_t);
  region_kernel<R, MAXP><<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int MAXP>
cudaError_t launch_p(const Plan &plan, const void *image, const uint8_t *const *in,
                     uint8_t *const *out, size_t nbytes, bool aligned, cudaStream_t st) {
  switch (plan.R) {
    case 1: return launch_t<1, MAXP>(plan, image, in, out, nbytes, aligned, st);
    case 2: return launch_t<2, MAXP>(plan, image, in, out, nbytes, aligned, st);
    case 4: return launch_t<4, MAXP>(plan, image, in, out, nbytes, aligned, st);
    case 8: return launch_t<8, MAXP>(plan, image, in, out, nbytes, aligned, st);
    default: return launch_t<16, MAXP>(plan, image, in, out, nbytes, aligned, st);
  }
}

}  // namespace

int launch_region(Plan &plan, const uint8_t *const *in, uint8_t *const *out, size_t nbytes,
                  cudaStream_t stream, std::string &err) {
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
  cudaError_t e = (plan.nin + plan.nout <= 256)
                      ? launch_p<256>(plan, image, in, out, nbytes, aligned, stream)
                      : launch_p<kMaxSlots>(plan, image, in, out, nbytes, aligned, stream);
  if (e != cudaSuccess) {
    err = std::string("region kernel launch: ") + cudaGetErrorString(e);
    return kECuda;
  }
  return kOk;
}

}  // namespace pmrc
