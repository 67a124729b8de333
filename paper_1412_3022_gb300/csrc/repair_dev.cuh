// One 1 KiB byte tile of a fused repair (repair.cu, batch.cu), for a CTA of
// 256 threads arranged as 64 columns x 4 lanes (thread = lane * 64 + column;
// a column is 16 bytes).  Included after region_dev.cuh inside an anonymous
// namespace.
//
//   stage 1: lane l computes the projections p_q of helpers q = l, l+4, ...
//            for its column and parks them in the CTA's projection area
//            (d x 64 vectors); a barrier makes them visible to the CTA;
//   stage 2: lane l computes newcomer rows r = l, l+4, ... (< alpha) over
//            the d projections of its column.
// When phi_f is a single 1 the projections are the helpers' stored blocks:
// stage 1 is skipped and stage 2 reads them in place.
//
// Tables: stage 1 t1a/t1b (nz entries: the non-zero helper coefficients),
// stage 2 t2a/t2b lane-major: entry (q, lane l, m) at q*4*rl + l*rl + m holds
// D[l + 4m][q] (rl = ceil(alpha / 4)).
#pragma once

constexpr int kRepCols = 64;                      // columns per 1 KiB tile
constexpr int kRepTile = kRepCols * kVec;         // bytes of column per tile

// acc = sum_i coef_i * x_i over nz inputs already in registers (nz <= NZ),
// two inputs per step as in mac_block.
template <int NZ>
__device__ __forceinline__ void mac_loaded(uint32_t (&acc)[4], int nz, const uint4 (&x)[NZ],
                                           const uint4 *t4, const uint32_t *t1,
                                           const MulConsts &k) {
#pragma unroll
  for (int q = 0; q < 4; q++) acc[q] = 0;
#pragma unroll
  for (int i = 0; i < NZ; i += 2) {
    if (i + 1 < nz) {
      uint32_t s0[12], s1[12];
      split_fields(x[i].x, x[i].y, k, s0);
      split_fields(x[i].z, x[i].w, k, s0 + 6);
      split_fields(x[i + 1].x, x[i + 1].y, k, s1);
      split_fields(x[i + 1].z, x[i + 1].w, k, s1 + 6);
      const uint4 u = t4[i], v = t4[i + 1];
      const uint32_t u2 = t1[i], v2 = t1[i + 1];
#pragma unroll
      for (int q = 0; q < 4; q++) acc[q] ^= lookup(u, u2, s0, q) ^ lookup(v, v2, s1, q);
    } else if (i < nz) {
      uint32_t s0[12];
      split_fields(x[i].x, x[i].y, k, s0);
      split_fields(x[i].z, x[i].w, k, s0 + 6);
      const uint4 u = t4[i];
      const uint32_t u2 = t1[i];
#pragma unroll
      for (int q = 0; q < 4; q++) acc[q] ^= lookup(u, u2, s0, q);
    }
  }
}

// NZ > 0: stage 1 loads all of a helper's inputs before using them (NZ >= nz
// registers of 16 bytes); NZ == 0: it streams them two at a time.
// proj: the CTA's projection area, d x 64 vectors (shared or global memory).
template <int NZ>
__device__ __forceinline__ void fused_repair_tile(uint8_t *const *ptrs, uint64_t tile_off,
                                                  uint64_t nbytes, bool vec, int d, int alpha,
                                                  int nz, bool direct, const uint16_t *s_nz,
                                                  const uint4 *t1a, const uint32_t *t1b,
                                                  const uint4 *t2a, const uint32_t *t2b, int rl,
                                                  uint4 *proj, const MulConsts &k) {
  const int col = threadIdx.x & (kRepCols - 1), lane = threadIdx.x / kRepCols;
  const uint64_t off = tile_off + (uint64_t)col * kVec;
  const bool live = off < nbytes;
  if (!direct) {
    if (live)
      for (int q = lane; q < d; q += 4) {
        uint32_t acc1[4];
        if constexpr (NZ > 0) {
          uint4 x[NZ];
#pragma unroll
          for (int i = 0; i < NZ; i++)
            if (i < nz) x[i] = load16(ptrs[q * alpha + s_nz[i]], off, nbytes, vec);
          mac_loaded<NZ>(acc1, nz, x, t1a, t1b, k);
        } else {
          uint32_t a1[1][4];
          mac_block<1>(a1, nz, 1, 1, t1a, t1b, k, [&](int i) {
            return load16(ptrs[q * alpha + s_nz[i]], off, nbytes, vec);
          });
#pragma unroll
          for (int w = 0; w < 4; w++) acc1[w] = a1[0][w];
        }
        proj[q * kRepCols + col] = acc_bytes(acc1);
      }
    __syncthreads();
  }
  const int nrows = (alpha - lane + 3) / 4;  // rows lane, lane + 4, ... below alpha
  if (live && nrows > 0) {
    uint32_t acc[4][4];
    const uint4 *ta = t2a + lane * rl;
    const uint32_t *tb = t2b + lane * rl;
    if (direct) {
      const int j0 = s_nz[0];
      mac_block<4>(acc, d, nrows, 4 * rl, ta, tb, k,
                   [&](int q) { return load16(ptrs[q * alpha + j0], off, nbytes, vec); });
    } else {
      mac_block<4>(acc, d, nrows, 4 * rl, ta, tb, k,
                   [&](int q) { return proj[q * kRepCols + col]; });
    }
#pragma unroll
    for (int m = 0; m < 4; m++)
      if (m < nrows) store16(ptrs[d * alpha + lane + 4 * m], off, nbytes, vec, acc_bytes(acc[m]));
  }
  if (!direct) __syncthreads();  // the projection area is reused by the next tile
}
