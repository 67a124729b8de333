// Bitsliced encode kernels for the codes listed in gen_bitslice.cpp.
//
// Same operation as region.cu (out[r] = sum_c M[r][c] * in[c], Sec. 2/3.1),
// for an encode matrix fixed at build time, with a different inner loop:
//
//   * each thread owns 32 consecutive bytes of every block of a tile; it
//     streams its inputs through a 5-slot shared-memory ring with cp.async,
//     four inputs ahead of the one in use (the XOR work per input is short,
//     so the loads must be in flight well before they are needed), and
//     turns each into eight 32-bit bit planes (plane i = bit i of the 32
//     bytes) with a 3-stage transpose of the 8 words, each stage a pair of
//     bit-field selects (one 3-input logic op each) on shifted copies;
//   * from the planes it forms Q[s] (XOR of the subset s of planes 0-3) and
//     R[s] (subset of planes 4-7);
//   * output plane i of a row gains Q[a] ^ R[b] per input, where a and b are
//     the nibbles of row i of the coefficient's 8x8 bit matrix -- one 3-input
//     XOR per (row, plane, input), against three table lookups and two XORs
//     per 4 bytes in region.cu;
//   * accumulated planes go back to bytes with the same transpose (it is its
//     own inverse) and are stored with 16-byte streaming stores;
//   * the inputs of a block are walked by a loop whose body switches on the
//     input only for the accumulate XORs, halving the code of a block;
//   * the grid is persistent, one 512-thread CTA per SM: each CTA stays on
//     one block of the matrix and its warps loop over that block's 1 KiB
//     column tiles, so an SM holds one block's straight-line code (tens of
//     KiB), fetched into its instruction caches once and then re-executed;
//     blocks get CTAs in proportion to their cost.
//
// The XOR schedules are generated at build time from the library's own
// construction (gen_bitslice.cpp); the launcher only uses a kernel whose
// matrix checksum equals the code's encode matrix.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "bitslice.h"
#include "device_info.h"

namespace pmrc {
namespace {

constexpr int kBsThreads = 512;       // one CTA per SM (128 registers a thread)
constexpr int kBsBytes = 32;          // bytes per thread per tile
constexpr int kBsMaxPtr = 256;
constexpr int kBsAhead = 4;           // inputs prefetched ahead of the one in use
constexpr int kBsSlots = kBsAhead + 1;  // shared-memory ring (never the slot being read)
constexpr uint32_t kBsUnit = 32 * kBsBytes;  // bytes of column per warp tile
constexpr int kBsMaxBlocks = 32;

struct BsArgs {
  uint64_t nbytes;  // bytes covered by this launch (multiple of kBsBytes)
  uint32_t hi28, hi30, hi31;  // 2^28, 2^30, 2^31: right shifts as multiply-high
  uint32_t x16, x4, x2;       // left shifts as multiplies
  uint16_t cta_start[kBsMaxBlocks + 1];  // CTAs [cta_start[b], cta_start[b+1]) run block b
  uint8_t *ptr[kBsMaxPtr];    // K input blocks, then the output blocks
};

struct BsCtx {
  const BsArgs *a;
  uint64_t off;
};

__device__ __forceinline__ bool bs_ctx(const BsArgs &a, BsCtx &x, uint32_t unit) {
  x.a = &a;
  x.off = (uint64_t)unit * kBsUnit + (threadIdx.x % 32) * kBsBytes;
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
// transform is an involution.  Each stage exchanges the bit fields `mask` of
// the lower word with the fields `mask << s` of the upper one: both words are
// rebuilt as a select between the word and a shifted copy of its partner (one
// 3-input logic op each); the shifts run as multiplies on the FMA pipe.
__device__ __forceinline__ void bs_transpose(uint32_t (&w)[8], const BsArgs &a) {
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const uint32_t sl = __umulhi(w[j], a.hi28), sh = w[j + 4] * a.x16;
    w[j + 4] = (sl & 0x0F0F0F0Fu) | (w[j + 4] & ~0x0F0F0F0Fu);
    w[j] = (sh & 0xF0F0F0F0u) | (w[j] & ~0xF0F0F0F0u);
  }
#pragma unroll
  for (int j = 0; j < 8; j += 4)
#pragma unroll
    for (int q = 0; q < 2; q++) {
      const uint32_t sl = __umulhi(w[j + q], a.hi30), sh = w[j + q + 2] * a.x4;
      w[j + q + 2] = (sl & 0x33333333u) | (w[j + q + 2] & ~0x33333333u);
      w[j + q] = (sh & 0xCCCCCCCCu) | (w[j + q] & ~0xCCCCCCCCu);
    }
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    const uint32_t sl = __umulhi(w[j], a.hi31), sh = w[j + 1] * a.x2;
    w[j + 1] = (sl & 0x55555555u) | (w[j + 1] & ~0x55555555u);
    w[j] = (sh & 0xAAAAAAAAu) | (w[j] & ~0xAAAAAAAAu);
  }
}

// Asynchronous copy of this thread's 32 bytes of input `col` into ring slot
// `slot` of the shared-memory staging area (cp.async, one commit group per
// input).  Each thread reads back only what it copied, so no barrier is
// needed; cp.async.wait_group orders the read after the copy.
__device__ __forceinline__ void bs_prefetch(const BsCtx &x, int col, int slot) {
  extern __shared__ __align__(16) uint8_t bs_smem[];
  const uint8_t *src = x.a->ptr[col] + x.off;
  const uint32_t dst = (uint32_t)__cvta_generic_to_shared(
      bs_smem + ((size_t)slot * kBsThreads + threadIdx.x) * kBsBytes);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16), "l"(src + 16)
               : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// An empty commit group: keeps the number of groups in flight the same for
// every input of a block shorter than the prefetch distance.
__device__ __forceinline__ void bs_commit_empty() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void bs_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void bs_planes(const BsCtx &x, int slot, uint32_t (&Q)[16],
                                          uint32_t (&R)[16]) {
  extern __shared__ __align__(16) uint8_t bs_smem[];
  const uint4 *p = reinterpret_cast<const uint4 *>(
      bs_smem + ((size_t)slot * kBsThreads + threadIdx.x) * kBsBytes);
  const uint4 u = p[0], v = p[1];
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
  const int *cost;  // relative cost of each block per tile
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
  // one CTA per SM; each block gets CTAs in proportion to its cost, at
  // least one, and no more than it has warp tiles to hand out
  static std::atomic<uint64_t> smem_set[kMaxDevices];
  const int sms = current_sm_count();
  const size_t smem = (size_t)kBsSlots * kBsThreads * kBsBytes;  // 80 KiB
  if (first_on_device(smem_set, id)) {
    cudaError_t e = cudaFuncSetAttribute(b.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const uint64_t units = (nbytes + kBsUnit - 1) / kBsUnit;
  const uint64_t cap = std::max<uint64_t>(1, (units + kBsThreads / 32 - 1) / (kBsThreads / 32));
  double total = 0;
  for (int i = 0; i < b.nblocks; i++) total += b.cost[i];
  int cnt[kBsMaxBlocks];
  int used = 0;
  for (int i = 0; i < b.nblocks; i++) {
    cnt[i] = std::max(1, (int)(sms * b.cost[i] / total));
    cnt[i] = (int)std::min<uint64_t>(cnt[i], cap);
    used += cnt[i];
  }
  for (; used < sms; used++) {  // hand out the rest to the slowest block
    int best = -1;
    double worst = 0;
    for (int i = 0; i < b.nblocks; i++) {
      const double t = (double)b.cost[i] / cnt[i];
      if ((uint64_t)cnt[i] < cap && t > worst) worst = t, best = i;
    }
    if (best < 0) break;
    cnt[best]++;
  }
  a.cta_start[0] = 0;
  for (int i = 0; i < b.nblocks; i++) a.cta_start[i + 1] = (uint16_t)(a.cta_start[i] + cnt[i]);
  for (int i = b.nblocks + 1; i <= kBsMaxBlocks; i++) a.cta_start[i] = a.cta_start[b.nblocks];
  b.fn<<<a.cta_start[b.nblocks], kBsThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

int bitslice_max_pointers() { return kBsMaxPtr; }

}  // namespace pmrc
