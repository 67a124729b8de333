// GF(2^16) for the PM-MSR codes of Sec. 3.3 over the larger field (the
// paper checks the sparse construction in GF(2^16) up to k = 64).
//
// The field is the quadratic extension GF(2^8)[y]/(y^2 + y + w) of the
// library's GF(2^8), w the smallest element of absolute trace 1 (for which
// the polynomial has no root).  The element a + b y is the value a | b << 8;
// g is the smallest value of multiplicative order 65535.  Multiplying by
// c = c0 + c1 y is GF(2^8)-linear on the pair (a, b):
//     [c0     w c1   ] [a]
//     [c1   c0 + c1  ] [b]
// so a GF(2^16) region operation on blocks stored as two byte planes (low
// bytes, then high bytes) is a GF(2^8) region operation with every
// coefficient expanded to this 2 x 2 block (code16.cpp).
#pragma once
#include <cstdint>
#include <vector>

#include "gf256.h"

namespace pmrc {

struct Gf16 {
  uint8_t w = 0;
  uint16_t g = 0;
  std::vector<uint16_t> exp;  // 2 * 65535 entries
  std::vector<int> log;       // 65536 entries
};

// (a0 + a1 y)(b0 + b1 y) with y^2 = y + w, from GF(2^8) products
inline uint16_t g16_mul_direct(uint8_t w, uint16_t x, uint16_t z) {
  const uint8_t a0 = (uint8_t)x, a1 = (uint8_t)(x >> 8), b0 = (uint8_t)z, b1 = (uint8_t)(z >> 8);
  const uint8_t hh = gmul(a1, b1);
  const uint8_t lo = gmul(a0, b0) ^ gmul(w, hh);
  const uint8_t hi = gmul(a1, b0) ^ gmul(a0, b1) ^ hh;
  return (uint16_t)(lo | (hi << 8));
}

inline const Gf16 &gf16() {
  static const Gf16 F = [] {
    Gf16 f;
    for (int a = 1; a < 256 && !f.w; a++) {  // absolute trace a + a^2 + ... + a^128
      uint8_t t = (uint8_t)a, s = (uint8_t)a;
      for (int i = 1; i < 8; i++) {
        t = gmul(t, t);
        s ^= t;
      }
      if (s == 1) f.w = (uint8_t)a;
    }
    auto pw = [&](uint16_t x, uint32_t e) {
      uint16_t r = 1;
      while (e) {
        if (e & 1) r = g16_mul_direct(f.w, r, x);
        x = g16_mul_direct(f.w, x, x);
        e >>= 1;
      }
      return r;
    };
    for (uint32_t v = 2; v < 65536 && !f.g; v++) {  // order 65535 = 3 * 5 * 17 * 257
      bool prim = true;
      for (uint32_t p : {3u, 5u, 17u, 257u}) prim = prim && pw((uint16_t)v, 65535u / p) != 1;
      if (prim) f.g = (uint16_t)v;
    }
    f.exp.assign(2 * 65535, 0);
    f.log.assign(65536, -1);
    uint16_t p = 1;
    for (int i = 0; i < 65535; i++) {
      f.exp[i] = f.exp[i + 65535] = p;
      f.log[p] = i;
      p = g16_mul_direct(f.w, p, f.g);
    }
    return f;
  }();
  return F;
}

inline uint16_t g16mul(uint16_t a, uint16_t b) {
  if (!a || !b) return 0;
  const Gf16 &f = gf16();
  return f.exp[f.log[a] + f.log[b]];
}

inline uint16_t g16inv(uint16_t a) {
  const Gf16 &f = gf16();
  return a ? f.exp[(65535 - f.log[a]) % 65535] : 0;
}

inline uint16_t g16pow(uint32_t e) { return gf16().exp[e % 65535]; }

}  // namespace pmrc
