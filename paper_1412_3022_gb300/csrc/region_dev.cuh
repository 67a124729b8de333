// Device routines shared by the region kernels (region.cu, repair.cu,
// batch.cu): nibble-field selectors, PRMT split-table lookups, 16-byte
// loads and stores with a byte path for ragged tails and unaligned blocks.
// Included inside an anonymous namespace of each translation unit.
#pragma once

constexpr int kThreads = 256;
constexpr int kVec = 16;  // bytes per thread per tile

// Multipliers passed at run time so that the selector construction below is
// issued as integer multiply-adds (FMA pipe) rather than shifts (ALU pipe),
// which the table lookups keep busy.
struct MulConsts {
  uint32_t x2, x16, hi16, hi26, hi29, hi30;  // 2, 16, 2^16, 2^26, 2^29, 2^30
};


__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t s) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
  return d;
}

// Selectors for 8 bytes (w0 = bytes 0-3, w1 = bytes 4-7).  Nibble 2m of a
// field word holds the field of byte m of w0, nibble 2m+1 that of byte m of
// w1 (fields: x&7, (x>>3)&7, x>>6).  s[2q] feeds lanes (w0.b0, w1.b0, w0.b1,
// w1.b1) of field q, s[2q+1] lanes (w0.b2, w1.b2, w0.b3, w1.b3).  The
// fields of w0 and w1 never overlap, so they are combined by addition.
__device__ __forceinline__ void split_fields(uint32_t w0, uint32_t w1, const MulConsts &k,
                                             uint32_t *s) {
  const uint32_t f0 = (w1 & 0x07070707u) * k.x16 + (w0 & 0x07070707u);
  const uint32_t f1 = (w1 & 0x38383838u) * k.x2 + __umulhi(w0 & 0x38383838u, k.hi29);
  const uint32_t f2 = __umulhi(w1 & 0xC0C0C0C0u, k.hi30) + __umulhi(w0 & 0xC0C0C0C0u, k.hi26);
  s[0] = f0;
  s[1] = __umulhi(f0, k.hi16);
  s[2] = f1;
  s[3] = __umulhi(f1, k.hi16);
  s[4] = f2;
  s[5] = __umulhi(f2, k.hi16);
}

// product of the 16 bytes behind selectors s with the coefficient whose split
// tables are (t, t2), lane word q (see split_fields)
__device__ __forceinline__ uint32_t lookup(const uint4 &t, uint32_t t2, const uint32_t *s, int q) {
  const uint32_t *sq = s + 6 * (q >> 1) + (q & 1);
  return prmt(t.x, t.y, sq[0]) ^ prmt(t.z, t.w, sq[2]) ^ prmt(t2, t2, sq[4]);
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


// Bytes of an accumulator (interleaved lanes, see split_fields) in order.
__device__ __forceinline__ uint4 acc_bytes(const uint32_t (&a)[4]) {
  return make_uint4(prmt(a[0], a[1], 0x6420), prmt(a[0], a[1], 0x7531), prmt(a[2], a[3], 0x6420),
                    prmt(a[2], a[3], 0x7531));
}

// acc[r] = sum over the nin inputs of coef(i, r) * input_i for r < nrows,
// on the 16 bytes each thread owns.  The split tables of coefficient (i, r)
// are tab4[i * stride + r], tab1[i * stride + r]; fetch(i) returns the 16
// input bytes of input i.  Two inputs per step: their six lookups per lane
// word fold into three 3-input XORs with the accumulator.
template <int R, class Fetch>
__device__ __forceinline__ void mac_block(uint32_t (&acc)[R][4], int nin, int nrows, int stride,
                                          const uint4 *tab4, const uint32_t *tab1,
                                          const MulConsts &k, Fetch fetch) {
#pragma unroll
  for (int r = 0; r < R; r++)
#pragma unroll
    for (int q = 0; q < 4; q++) acc[r][q] = 0;
  int i = 0;
  uint4 x0 = make_uint4(0, 0, 0, 0), x1 = x0;
  if (nin > 0) x0 = fetch(0);
  if (nin > 1) x1 = fetch(1);
  for (; i + 1 < nin; i += 2) {
    uint4 n0 = x0, n1 = x1;
    if (i + 2 < nin) n0 = fetch(i + 2);
    if (i + 3 < nin) n1 = fetch(i + 3);
    uint32_t s0[12], s1[12];
    split_fields(x0.x, x0.y, k, s0);
    split_fields(x0.z, x0.w, k, s0 + 6);
    split_fields(x1.x, x1.y, k, s1);
    split_fields(x1.z, x1.w, k, s1 + 6);
    const uint4 *ta = tab4 + i * stride;
    const uint32_t *tb = tab1 + i * stride;
#pragma unroll
    for (int r = 0; r < R; r++) {
      if (r < nrows) {
        const uint4 u = ta[r], v = ta[stride + r];
        const uint32_t u2 = tb[r], v2 = tb[stride + r];
#pragma unroll
        for (int q = 0; q < 4; q++) acc[r][q] ^= lookup(u, u2, s0, q) ^ lookup(v, v2, s1, q);
      }
    }
    x0 = n0;
    x1 = n1;
  }
  if (i < nin) {
    uint32_t s0[12];
    split_fields(x0.x, x0.y, k, s0);
    split_fields(x0.z, x0.w, k, s0 + 6);
#pragma unroll
    for (int r = 0; r < R; r++) {
      if (r < nrows) {
        const uint4 u = tab4[i * stride + r];
        const uint32_t u2 = tab1[i * stride + r];
#pragma unroll
        for (int q = 0; q < 4; q++) acc[r][q] ^= lookup(u, u2, s0, q);
      }
    }
  }
}

// mac_block for blocks of few inputs (nin <= 8): every input of the tile is
// loaded before the first is used, so the tile waits for one round trip to
// memory instead of one per pair of inputs.  Same arithmetic and result.
template <int R, typename Fetch>
__device__ __forceinline__ void mac_block_preload(uint32_t (&acc)[R][4], int nin, int nrows,
                                                  int stride, const uint4 *tab4,
                                                  const uint32_t *tab1, const MulConsts &k,
                                                  Fetch fetch) {
#pragma unroll
  for (int r = 0; r < R; r++)
#pragma unroll
    for (int q = 0; q < 4; q++) acc[r][q] = 0;
  uint4 x[8];
#pragma unroll
  for (int i = 0; i < 8; i++) x[i] = i < nin ? fetch(i) : make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int i = 0; i < 8; i += 2) {
    if (i < nin) {
      uint32_t s0[12], s1[12];
      split_fields(x[i].x, x[i].y, k, s0);
      split_fields(x[i].z, x[i].w, k, s0 + 6);
      split_fields(x[i + 1].x, x[i + 1].y, k, s1);
      split_fields(x[i + 1].z, x[i + 1].w, k, s1 + 6);
      const bool two = i + 1 < nin;
#pragma unroll
      for (int r = 0; r < R; r++) {
        if (r < nrows) {
          const uint4 u = tab4[i * stride + r];
          const uint32_t u2 = tab1[i * stride + r];
          if (two) {
            const uint4 v = tab4[(i + 1) * stride + r];
            const uint32_t v2 = tab1[(i + 1) * stride + r];
#pragma unroll
            for (int q = 0; q < 4; q++) acc[r][q] ^= lookup(u, u2, s0, q) ^ lookup(v, v2, s1, q);
          } else {
#pragma unroll
            for (int q = 0; q < 4; q++) acc[r][q] ^= lookup(u, u2, s0, q);
          }
        }
      }
    }
  }
}

__device__ __forceinline__ MulConsts mul_consts_default() {
  return MulConsts{2u, 16u, 1u << 16, 1u << 26, 1u << 29, 1u << 30};
}
