// Device side of the bitsliced kernels (bitslice.cu): constants, the launch
// arguments and the per-thread building blocks the generated block functions
// call.  Self-contained (no includes): the library compiles it with nvcc,
// and its text is also compiled at run time (jit.cpp) together with
// schedules generated for matrices known only then.  Expects uint8_t,
// uint16_t, uint32_t and uint64_t to be defined.
constexpr int kBsThreads = 512;       // one CTA per SM (128 registers a thread)
constexpr int kBsBytes = 32;          // bytes per thread per tile
constexpr int kBsMaxPtr = 512;       // block pointers per launch
constexpr int kBsAhead = 4;           // inputs prefetched ahead of the one in use
constexpr int kBsSlots = kBsAhead + 1;  // shared-memory ring (never the slot being read)
constexpr uint32_t kBsUnit = 32 * kBsBytes;  // bytes of column per warp tile
constexpr int kBsMaxBlocks = 64;     // dense blocks per schedule
constexpr int kBsMaxCtas = 256;      // CTAs per launch (one per SM)

struct BsArgs {
  uint64_t nbytes;  // bytes covered by this launch (multiple of kBsBytes)
  uint32_t hi28, hi30, hi31;  // 2^28, 2^30, 2^31: right shifts as multiply-high
  uint32_t x16, x4, x2;       // left shifts as multiplies
  // the launch's work is the sequence of warp tiles g = b * ntiles + t
  // (block b, 1 KiB column tile t); CTA c takes tiles [cta_g[c], cta_g[c+1])
  uint32_t ntiles;
  // repair kernels (bs_emit_projection / bs_emit_fused_repair): helpers in
  // the launch, helper groups per tile, and warp tasks (tiles x groups)
  uint32_t nh, ngroups, ntasks;
  uint32_t cta_g[kBsMaxCtas + 1];
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

// Three-input XOR and two-input XOR as single logic instructions (lop3 with
// the truth table of a ^ b ^ c, 0x96), so that every accumulate of a
// schedule is exactly one instruction whatever the compiler would otherwise
// fuse or split.
__device__ __forceinline__ uint32_t bs_x3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t bs_x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("xor.b32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// Bit-field select (a & M) | (b & ~M) for a constant mask M: one lop3
// (truth table 0xE4 with M as the third operand).
template <uint32_t M>
__device__ __forceinline__ uint32_t bs_sel(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0xE4;" : "=r"(d) : "r"(a), "r"(b), "n"(M));
  return d;
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
    w[j + 4] = bs_sel<0x0F0F0F0Fu>(sl, w[j + 4]);
    w[j] = bs_sel<0xF0F0F0F0u>(sh, w[j]);
  }
#pragma unroll
  for (int j = 0; j < 8; j += 4)
#pragma unroll
    for (int q = 0; q < 2; q++) {
      const uint32_t sl = __umulhi(w[j + q], a.hi30), sh = w[j + q + 2] * a.x4;
      w[j + q + 2] = bs_sel<0x33333333u>(sl, w[j + q + 2]);
      w[j + q] = bs_sel<0xCCCCCCCCu>(sh, w[j + q]);
    }
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    const uint32_t sl = __umulhi(w[j], a.hi31), sh = w[j + 1] * a.x2;
    w[j + 1] = bs_sel<0x55555555u>(sl, w[j + 1]);
    w[j] = bs_sel<0xAAAAAAAAu>(sh, w[j]);
  }
}

// Shared-memory staging ring of the per-thread input copies: slot s of
// thread t is at byte (s * kBsThreads + t) * kBsBytes of the dynamic shared
// memory.  bs_ring_base() is this thread's slot 0 as a shared-space address;
// the emitted loops advance a read and a write address by one slot per input
// and wrap them, so no slot index is recomputed per input.
constexpr uint32_t kBsSlotStep = kBsThreads * kBsBytes;

__device__ __forceinline__ uint32_t bs_ring_base() {
  extern __shared__ __align__(16) uint8_t bs_smem[];
  return (uint32_t)__cvta_generic_to_shared(bs_smem + threadIdx.x * kBsBytes);
}

// Asynchronous copy of this thread's 32 bytes of an input block into the
// ring slot at shared address `dst` (cp.async, one commit group per input).
// Each thread reads back only what it copied, so no barrier is needed;
// cp.async.wait_group orders the read after the copy.
__device__ __forceinline__ void bs_prefetch(const BsCtx &x, int col, uint32_t dst) {
  const uint8_t *src = x.a->ptr[col] + x.off;
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

// The 32 staged bytes at shared address `src`, as eight words.
__device__ __forceinline__ void bs_load(uint32_t src, uint32_t (&w)[8]) {
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
               : "r"(src)
               : "memory");
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
               : "r"(src + 16)
               : "memory");
}

// Subset tables of eight bit planes: Q[s] is the XOR of the planes 0-3
// selected by the bits of s, R[s] the same over planes 4-7.
__device__ __forceinline__ void bs_tables(const uint32_t (&w)[8], uint32_t (&Q)[16],
                                          uint32_t (&R)[16]) {
  Q[0] = 0;
  Q[1] = w[0];
  Q[2] = w[1];
  Q[3] = bs_x2(w[0], w[1]);
  Q[4] = w[2];
  Q[5] = bs_x2(w[2], w[0]);
  Q[6] = bs_x2(w[2], w[1]);
  Q[7] = bs_x3(w[2], w[0], w[1]);
  Q[8] = w[3];
#pragma unroll
  for (int s = 9; s < 16; s++) Q[s] = bs_x2(w[3], Q[s - 8]);
  R[0] = 0;
  R[1] = w[4];
  R[2] = w[5];
  R[3] = bs_x2(w[4], w[5]);
  R[4] = w[6];
  R[5] = bs_x2(w[6], w[4]);
  R[6] = bs_x2(w[6], w[5]);
  R[7] = bs_x3(w[6], w[4], w[5]);
  R[8] = w[7];
#pragma unroll
  for (int s = 9; s < 16; s++) R[s] = bs_x2(w[7], R[s - 8]);
}

// The 32 staged bytes at shared address `src` as bit planes, and their
// subset tables.
__device__ __forceinline__ void bs_planes(const BsCtx &x, uint32_t src, uint32_t (&Q)[16],
                                          uint32_t (&R)[16]) {
  uint32_t w[8];
  bs_load(src, w);
  bs_transpose(w, *x.a);
  bs_tables(w, Q, R);
}

// Plane-layout input: the 32 staged bytes at shared address `src` are
// already the eight bit planes of the lane's 32 bytes (an intermediate a
// plane-layout store wrote); their subset tables, no transpose.
__device__ __forceinline__ void bs_planes_direct(uint32_t src, uint32_t (&Q)[16],
                                                 uint32_t (&R)[16]) {
  uint32_t w[8];
  bs_load(src, w);
  bs_tables(w, Q, R);
}

// Barrier of the two warps of pair `pair` (named barrier 1 + pair, 64
// threads); the fused repair kernels exchange partial sums through shared
// memory between them.
__device__ __forceinline__ void bs_pair_sync(uint32_t pair) {
  asm volatile("bar.sync %0, 64;" ::"r"(1 + pair) : "memory");
}

// Plane-layout output: the eight planes stored as they are (an
// intermediate for a later launch that reads it with bs_planes_direct), with
// ordinary stores so that the next launch finds it in L2.
__device__ __forceinline__ void bs_store_planes(const BsCtx &x, int slot, const uint32_t (&planes)[8]) {
  uint4 *p = reinterpret_cast<uint4 *>(x.a->ptr[slot] + x.off);
  p[0] = make_uint4(planes[0], planes[1], planes[2], planes[3]);
  p[1] = make_uint4(planes[4], planes[5], planes[6], planes[7]);
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

