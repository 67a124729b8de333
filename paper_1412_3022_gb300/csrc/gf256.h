// GF(2^8) arithmetic for the library (host and device).
//
// The field is GF(2)[x]/(x^8 + x^4 + x^3 + x^2 + 1) (0x11D), the default
// 8-bit field of the paper's GF-Complete setup (Sec. 4); g = 2 generates its
// multiplicative group.  Products are computed by shift-and-reduce, so the
// same constexpr function builds host tables and the device split tables.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define PMRC_HD __host__ __device__
#else
#define PMRC_HD
#endif

namespace pmrc {

constexpr unsigned kPoly = 0x11D;

// a*b by shift-and-reduce (carry-less multiply with on-the-fly reduction).
PMRC_HD constexpr uint8_t gf_mul_sr(uint8_t a, uint8_t b) {
  unsigned x = a, r = 0;
  for (int i = 0; i < 8; i++) {
    if (b & (1u << i)) r ^= x;
    x <<= 1;
    if (x & 0x100u) x ^= kPoly;
  }
  return (uint8_t)r;
}

// a^e by square-and-multiply.
PMRC_HD constexpr uint8_t gf_pow(uint8_t a, unsigned e) {
  uint8_t r = 1, s = a;
  while (e) {
    if (e & 1u) r = gf_mul_sr(r, s);
    s = gf_mul_sr(s, s);
    e >>= 1;
  }
  return r;
}

// a^-1 = a^254 (the multiplicative group has order 255); 0 maps to 0.
PMRC_HD constexpr uint8_t gf_inv(uint8_t a) { return a ? gf_pow(a, 254) : 0; }

// Host-side 256x256 product table, filled once.
struct MulTable {
  uint8_t t[256][256];
  MulTable() {
    for (int a = 0; a < 256; a++)
      for (int b = 0; b < 256; b++) t[a][b] = gf_mul_sr((uint8_t)a, (uint8_t)b);
  }
};

inline const MulTable &mul_table() {
  static const MulTable tab;
  return tab;
}

inline uint8_t gmul(uint8_t a, uint8_t b) { return mul_table().t[a][b]; }

// Split tables for the region kernels.  A byte x is cut into three bit
// fields: x[2:0], x[5:3] and x[7:6].  Because multiplication by a constant c
// is GF(2)-linear, c*x = T0[x&7] ^ T1[(x>>3)&7] ^ T2[x>>6] with
// Tq[y] = c * (y << 3q).  Each 8-entry table is two 32-bit words (entries
// 0-3 and 4-7), the operand pair of one byte-permute (PRMT) lookup; T2 has 4
// entries and needs one word.  Layout per coefficient:
//   w[0], w[1] = T0;  w[2], w[3] = T1;  w[4] = T2;  w[5] = 0 (pad).
struct SplitTables {
  uint32_t w[256][6];
};

PMRC_HD constexpr uint32_t split_word(uint8_t c, int shift, int first) {
  uint32_t v = 0;
  for (int e = 0; e < 4; e++)
    v |= (uint32_t)gf_mul_sr(c, (uint8_t)(((first + e) << shift) & 0xFF)) << (8 * e);
  return v;
}

constexpr SplitTables make_split_tables() {
  SplitTables s{};
  for (int c = 0; c < 256; c++) {
    s.w[c][0] = split_word((uint8_t)c, 0, 0);
    s.w[c][1] = split_word((uint8_t)c, 0, 4);
    s.w[c][2] = split_word((uint8_t)c, 3, 0);
    s.w[c][3] = split_word((uint8_t)c, 3, 4);
    s.w[c][4] = split_word((uint8_t)c, 6, 0);
    s.w[c][5] = 0;
  }
  return s;
}

}  // namespace pmrc
