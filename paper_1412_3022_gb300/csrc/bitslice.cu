// Bitsliced encode kernels for the codes listed in gen_bitslice.cpp.
//
// Same operation as region.cu (out[r] = sum_c M[r][c] * in[c], Sec. 2/3.1),
// for an encode matrix fixed at build time, with a different inner loop:
//
//   * each thread owns 32 consecutive bytes of every block of a tile and
//     turns them into eight 32-bit bit planes (plane i = bit i of the 32
//     bytes) with a 3-stage delta-swap transpose of the 8 words;
//   * from the planes it forms Q[s] (XOR of the subset s of planes 0-3) and
//     R[s] (subset of planes 4-7);
//   * output plane i of a row gains Q[a] ^ R[b] per input, where a and b are
//     the nibbles of row i of the coefficient's 8x8 bit matrix -- one 3-input
//     XOR per (row, plane, input), against three table lookups and two XORs
//     per 4 bytes in region.cu;
//   * accumulated planes go back to bytes with the same transpose (it is its
//     own inverse) and are stored with 16-byte streaming stores.
//
// The XOR schedules are generated at build time from the library's own
// construction (gen_bitslice.cpp); the launcher only uses a kernel whose
// matrix checksum equals the code's encode matrix.
#include <cuda_runtime.h>

#include <cstring>

#include "bitslice.h"

namespace pmrc {
namespace {

constexpr int kBsThreads = 256;
constexpr int kBsBytes = 32;          // bytes per thread per tile
constexpr int kBsMaxPtr = 256;

struct BsArgs {
  uint64_t nbytes;  // bytes covered by this launch (multiple of kBsBytes)
  uint32_t hi28, hi30, hi31;  // 2^28, 2^30, 2^31: right shifts as multiply-high
  uint32_t x16, x4, x2;       // left shifts as multiplies
  uint8_t *ptr[kBsMaxPtr];    // K input blocks, then the output blocks
};

struct BsCtx {
  const BsArgs *a;
  uint64_t off;
};

__device__ __forceinline__ bool bs_ctx(const BsArgs &a, BsCtx &x) {
  x.a = &a;
  x.off = ((uint64_t)blockIdx.x * kBsThreads + threadIdx.x) * kBsBytes;
  return x.off < a.nbytes;
}

__device__ __forceinline__ void bs_zero(uint32_t (&acc)[8][8]) {
#pragma unroll
  for (int r = 0; r < 8; r++)
#pragma unroll
    for (int i = 0; i < 8; i++) acc[r][i] = 0;
}

// 8x8 bit transpose inside each byte lane of 8 words: afterwards word i
// holds bit i of the 32 bytes (bit 8m+j = bit i of byte m of word j).  The
// transform is an involution.  Shifts run as multiplies on the FMA pipe.
__device__ __forceinline__ void bs_transpose(uint32_t (&w)[8], const BsArgs &a) {
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const uint32_t t = (__umulhi(w[j], a.hi28) ^ w[j + 4]) & 0x0F0F0F0Fu;
    w[j + 4] ^= t;
    w[j] ^= t * a.x16;
  }
#pragma unroll
  for (int j = 0; j < 8; j += 4)
#pragma unroll
    for (int q = 0; q < 2; q++) {
      const uint32_t t = (__umulhi(w[j + q], a.hi30) ^ w[j + q + 2]) & 0x33333333u;
      w[j + q + 2] ^= t;
      w[j + q] ^= t * a.x4;
    }
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    const uint32_t t = (__umulhi(w[j], a.hi31) ^ w[j + 1]) & 0x55555555u;
    w[j + 1] ^= t;
    w[j] ^= t * a.x2;
  }
}

__device__ __forceinline__ void bs_planes(const BsCtx &x, int col, uint32_t (&Q)[16],
                                          uint32_t (&R)[16]) {
  const uint4 *p = reinterpret_cast<const uint4 *>(x.a->ptr[col] + x.off);
  const uint4 u = __ldg(p), v = __ldg(p + 1);
  uint32_t w[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
  bs_transpose(w, *x.a);
  Q[0] = 0;
  Q[1] = w[0];
  Q[2] = w[1];
  Q[3] = w[0] ^ w[1];
  Q[4] = w[2];
  Q[5] = w[2] ^ w[0];
  Q[6] = w[2] ^ w[1];
  Q[7] = w[2] ^ Q[3];
  Q[8] = w[3];
#pragma unroll
  for (int s = 9; s < 16; s++) Q[s] = w[3] ^ Q[s - 8];
  R[0] = 0;
  R[1] = w[4];
  R[2] = w[5];
  R[3] = w[4] ^ w[5];
  R[4] = w[6];
  R[5] = w[6] ^ w[4];
  R[6] = w[6] ^ w[5];
  R[7] = w[6] ^ R[3];
  R[8] = w[7];
#pragma unroll
  for (int s = 9; s < 16; s++) R[s] = w[7] ^ R[s - 8];
}

__device__ __forceinline__ void bs_store(const BsCtx &x, int slot, uint32_t (&planes)[8]) {
  uint32_t w[8];
#pragma unroll
  for (int i = 0; i < 8; i++) w[i] = planes[i];
  bs_transpose(w, *x.a);
  uint4 *p = reinterpret_cast<uint4 *>(x.a->ptr[slot] + x.off);
  __stcs(p, make_uint4(w[0], w[1], w[2], w[3]));
  __stcs(p + 1, make_uint4(w[4], w[5], w[6], w[7]));
}

struct BsKernel {
  int n, k, construction, form;
  int nblocks, ninputs, noutputs;
  unsigned long long checksum;
  long long xors;
  void (*fn)(BsArgs);
};

#include "bitslice_gen.cuh"

}  // namespace

uint64_t bitslice_checksum(const uint8_t *m, size_t len) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < len; i++) {
    h ^= m[i];
    h *= 1099511628211ull;
  }
  return h;
}

int bitslice_find(int n, int k, int construction, int form, uint64_t checksum) {
  for (int i = 0; i < kBsNumKernels; i++) {
    const BsKernel &b = kBsKernels[i];
    if (b.n == n && b.k == k && b.construction == construction && b.form == form)
      return b.checksum == checksum ? i : -1;
  }
  return -1;
}

long long bitslice_xors(int id) { return id >= 0 && id < kBsNumKernels ? kBsKernels[id].xors : 0; }

cudaError_t bitslice_launch(int id, const uint8_t *const *in, uint8_t *const *out, size_t nbytes,
                            cudaStream_t stream) {
  const BsKernel &b = kBsKernels[id];
  BsArgs a;
  a.nbytes = nbytes;
  a.hi28 = 1u << 28;
  a.hi30 = 1u << 30;
  a.hi31 = 1u << 31;
  a.x16 = 16;
  a.x4 = 4;
  a.x2 = 2;
  memset(a.ptr, 0, sizeof a.ptr);
  for (int i = 0; i < b.ninputs; i++) a.ptr[i] = const_cast<uint8_t *>(in[i]);
  for (int j = 0; j < b.noutputs; j++) a.ptr[b.ninputs + j] = out[j];
  const uint64_t tile = (uint64_t)kBsThreads * kBsBytes;
  const dim3 grid((unsigned)((nbytes + tile - 1) / tile), (unsigned)b.nblocks);
  b.fn<<<grid, kBsThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

int bitslice_max_pointers() { return kBsMaxPtr; }

}  // namespace pmrc
