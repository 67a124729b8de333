// PM-MSR codes over GF(2^16) (gf16.h), expanded to GF(2^8) region matrices.
//
// The constructions are those of code.cpp (Sec. 3.1-3.3) with the GF(2^16)
// arithmetic and generator.  A user block of B bytes holds B/2 symbols as
// two byte planes, so block r is the pair of GF(2^8) sub-blocks 2r (low
// bytes) and 2r + 1 (high bytes), and every GF(2^16) matrix M becomes the
// GF(2^8) matrix with M[r][c] replaced by its 2 x 2 block (gf16.h).  The
// expanded code (alpha, K, N doubled; beta = 2 sub-blocks per helper
// projection) then runs on the GF(2^8) planner and kernels unchanged.
#include <algorithm>

#include "code.h"
#include "gf16.h"

namespace pmrc {

namespace {

using V16 = std::vector<uint16_t>;

bool inverse16(const V16 &A, int m, V16 &out) {
  V16 W((size_t)m * 2 * m, 0);
  for (int i = 0; i < m; i++) {
    for (int j = 0; j < m; j++) W[(size_t)i * 2 * m + j] = A[(size_t)i * m + j];
    W[(size_t)i * 2 * m + m + i] = 1;
  }
  for (int c = 0; c < m; c++) {
    int p = c;
    while (p < m && W[(size_t)p * 2 * m + c] == 0) p++;
    if (p == m) return false;
    if (p != c)
      for (int j = 0; j < 2 * m; j++) std::swap(W[(size_t)p * 2 * m + j], W[(size_t)c * 2 * m + j]);
    const uint16_t s = g16inv(W[(size_t)c * 2 * m + c]);
    for (int j = 0; j < 2 * m; j++) W[(size_t)c * 2 * m + j] = g16mul(W[(size_t)c * 2 * m + j], s);
    for (int r = 0; r < m; r++) {
      const uint16_t f = W[(size_t)r * 2 * m + c];
      if (r == c || !f) continue;
      for (int j = 0; j < 2 * m; j++) W[(size_t)r * 2 * m + j] ^= g16mul(f, W[(size_t)c * 2 * m + j]);
    }
  }
  out.assign((size_t)m * m, 0);
  for (int i = 0; i < m; i++)
    for (int j = 0; j < m; j++) out[(size_t)i * m + j] = W[(size_t)i * 2 * m + m + j];
  return true;
}

}  // namespace

void expand16(const std::vector<uint16_t> &M, int rows, int cols, Mat &out) {
  const uint8_t w = gf16().w;
  out = Mat(2 * rows, 2 * cols);
  for (int r = 0; r < rows; r++)
    for (int c = 0; c < cols; c++) {
      const uint16_t v = M[(size_t)r * cols + c];
      if (!v) continue;
      const uint8_t c0 = (uint8_t)v, c1 = (uint8_t)(v >> 8);
      out.at(2 * r, 2 * c) = c0;
      out.at(2 * r, 2 * c + 1) = gmul(w, c1);
      out.at(2 * r + 1, 2 * c) = c1;
      out.at(2 * r + 1, 2 * c + 1) = c0 ^ c1;
    }
}

int build_code16(int n, int k, int d, int construction, int systematic, CodeMatrices &c,
                 std::string &err) {
  if (k < 2 || d != 2 * k - 2) {
    err = "PM-MSR needs k >= 2 and d = 2k-2";
    return kEInval;
  }
  if (n < d + 1 || n > 254) {
    err = "n must satisfy 2k-1 <= n <= 254";
    return kEInval;
  }
  if (construction != 0 && construction != 1) {
    err = "GF(2^16) codes: construction must be PMRC_VANILLA or PMRC_SPARSE";
    return kEInval;
  }
  const int a = k - 1, K = k * a, N = n * a;
  auto &f = c.f16;
  f.alpha = a;
  f.K = K;
  f.N = N;
  f.phi.assign((size_t)n * a, 0);
  f.lambda.assign(n, 0);
  if (construction == 0) {  // Vandermonde, lambda_i = g^(i alpha)
    for (int i = 0; i < n; i++) {
      for (int j = 0; j < a; j++) f.phi[(size_t)i * a + j] = g16pow((uint32_t)(i * j));
      f.lambda[i] = g16pow((uint32_t)(i * a));
    }
  } else {  // identity + Cauchy, 1-based i, j as in Sec. 3.3
    for (int i = 1; i <= n; i++) {
      const uint16_t z = g16pow((uint32_t)(i + a));
      for (int j = 1; j <= a; j++)
        f.phi[(size_t)(i - 1) * a + j - 1] =
            i <= a ? (uint16_t)(i == j) : g16inv((uint16_t)(z ^ g16pow((uint32_t)(j - 1))));
      f.lambda[i - 1] = g16mul((uint16_t)(z ^ 1), g16inv((uint16_t)(z ^ g16pow((uint32_t)a))));
    }
  }
  {
    V16 s = f.lambda;
    std::sort(s.begin(), s.end());
    if (std::adjacent_find(s.begin(), s.end()) != s.end()) {
      err = "construction has repeated lambda values at this (n, k) in GF(2^16)";
      return kEUnsupported;
    }
  }
  f.psi.assign((size_t)n * d, 0);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < a; j++) {
      f.psi[(size_t)i * d + j] = f.phi[(size_t)i * a + j];
      f.psi[(size_t)i * d + a + j] = g16mul(f.lambda[i], f.phi[(size_t)i * a + j]);
    }
  // index matrix: upper triangles of S1 then S2, row by row (Sec. 3.1)
  std::vector<int> L((size_t)d * a);
  {
    std::vector<int> tri((size_t)a * a);
    int next = 0;
    for (int r = 0; r < a; r++)
      for (int q = r; q < a; q++) tri[(size_t)r * a + q] = tri[(size_t)q * a + r] = next++;
    for (int r = 0; r < a; r++)
      for (int q = 0; q < a; q++) {
        L[(size_t)r * a + q] = tri[(size_t)r * a + q];
        L[(size_t)(a + r) * a + q] = next + tri[(size_t)r * a + q];
      }
  }
  V16 G((size_t)N * K, 0);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < a; j++)
      for (int l = 0; l < d; l++) G[(size_t)(a * i + j) * K + L[(size_t)l * a + j]] = f.psi[(size_t)i * d + l];
  if (!systematic) {
    f.Gcode = G;
  } else {
    V16 top(G.begin(), G.begin() + (size_t)K * K), ti;
    if (!inverse16(top, K, ti)) {
      err = "the first k nodes do not determine the data: no systematic form";
      return kEUnsupported;
    }
    f.Gcode.assign((size_t)N * K, 0);
    for (int r = 0; r < N; r++)
      for (int q = 0; q < K; q++) {
        const uint16_t g = G[(size_t)r * K + q];
        if (!g) continue;
        for (int col = 0; col < K; col++) f.Gcode[(size_t)r * K + col] ^= g16mul(g, ti[(size_t)q * K + col]);
      }
  }
  // the expanded GF(2^8) code the planner and kernels run
  c.w = 16;
  c.beta = 2;
  c.n = n;
  c.k = k;
  c.d = d;
  c.alpha = 2 * a;
  c.K = 2 * K;
  c.N = 2 * N;
  c.construction = construction;
  c.systematic = systematic;
  c.L = L;
  expand16(G, N, K, c.G);
  expand16(f.Gcode, N, K, c.Gcode);
  c.phi = Mat();
  c.lambda.clear();
  c.psi = Mat();
  mark_unit_rows(c);
  return kOk;
}

void helper_matrix16(const CodeMatrices &c, int f, Mat &P) {
  const int a = c.f16.alpha;
  V16 row(c.f16.phi.begin() + (size_t)f * a, c.f16.phi.begin() + (size_t)(f + 1) * a);
  expand16(row, 1, a, P);
}

static bool psi_h_inverse16(const CodeMatrices &c, const int *helpers, V16 &inv) {
  const int d = c.d;
  V16 PH((size_t)d * d);
  for (int i = 0; i < d; i++)
    for (int l = 0; l < d; l++) PH[(size_t)i * d + l] = c.f16.psi[(size_t)helpers[i] * d + l];
  return inverse16(PH, d, inv);
}

bool helpers_invertible16(const CodeMatrices &c, const int *helpers) {
  V16 inv;
  return psi_h_inverse16(c, helpers, inv);
}

int newcomer_matrix16(const CodeMatrices &c, int f, const int *helpers, Mat &D, std::string &err) {
  V16 inv;
  if (!psi_h_inverse16(c, helpers, inv)) {
    err = "the helpers' rows of Psi are singular for this failed node";
    return kESingular;
  }
  const int a = c.f16.alpha, d = c.d;
  V16 D16((size_t)a * d);
  const uint16_t lf = c.f16.lambda[f];
  for (int j = 0; j < a; j++)
    for (int q = 0; q < d; q++)
      D16[(size_t)j * d + q] = inv[(size_t)j * d + q] ^ g16mul(lf, inv[(size_t)(a + j) * d + q]);
  expand16(D16, a, d, D);
  return kOk;
}

int decode_matrix16(const CodeMatrices &c, const int *nodes, Mat &Rinv, std::string &err) {
  const int a = c.f16.alpha, K = c.f16.K;
  V16 GR((size_t)K * K), inv;
  for (int i = 0; i < c.k; i++)
    for (int j = 0; j < a; j++)
      std::copy(c.f16.Gcode.begin() + (size_t)(a * nodes[i] + j) * K,
                c.f16.Gcode.begin() + (size_t)(a * nodes[i] + j + 1) * K,
                GR.begin() + (size_t)(a * i + j) * K);
  if (!inverse16(GR, K, inv)) {
    err = "these k nodes do not determine the data";
    return kESingular;
  }
  expand16(inv, K, K, Rinv);
  return kOk;
}

}  // namespace pmrc
