// Host construction of PM-MSR and PM-MBR codes (see code.h for the paper
// sections).
#include "code.h"

#include <algorithm>

#include "gf256.h"

namespace pmrc {

Mat mat_mul(const Mat &A, const Mat &B) {
  Mat C(A.rows, B.cols);
  const auto &T = mul_table().t;
  for (int i = 0; i < A.rows; i++)
    for (int l = 0; l < A.cols; l++) {
      uint8_t a = A.at(i, l);
      if (!a) continue;
      const uint8_t *row = T[a];
      for (int j = 0; j < B.cols; j++) C.at(i, j) ^= row[B.at(l, j)];
    }
  return C;
}

bool mat_inverse(const Mat &A, Mat &out) {
  const int m = A.rows;
  if (m != A.cols || m <= 0) return false;
  const auto &T = mul_table().t;
  Mat W(m, 2 * m);
  for (int i = 0; i < m; i++) {
    for (int j = 0; j < m; j++) W.at(i, j) = A.at(i, j);
    W.at(i, m + i) = 1;
  }
  for (int c = 0; c < m; c++) {
    int p = c;
    while (p < m && W.at(p, c) == 0) p++;
    if (p == m) return false;
    if (p != c)
      for (int j = 0; j < 2 * m; j++) std::swap(W.at(p, j), W.at(c, j));
    const uint8_t *s = T[gf_inv(W.at(c, c))];
    for (int j = 0; j < 2 * m; j++) W.at(c, j) = s[W.at(c, j)];
    for (int r = 0; r < m; r++) {
      uint8_t f = W.at(r, c);
      if (r == c || !f) continue;
      const uint8_t *fr = T[f];
      for (int j = 0; j < 2 * m; j++) W.at(r, j) ^= fr[W.at(c, j)];
    }
  }
  out = Mat(m, m);
  for (int i = 0; i < m; i++)
    for (int j = 0; j < m; j++) out.at(i, j) = W.at(i, m + j);
  return true;
}

static uint8_t gpow(unsigned e) { return gf_pow(2, e % 255); }

// Rows of Gcode that are unit vectors copy one data block verbatim.
void mark_unit_rows(CodeMatrices &c) {
  c.unit_col.assign(c.N, -1);
  for (int r = 0; r < c.N; r++) {
    int col = -1, cnt = 0;
    for (int q = 0; q < c.K && cnt < 2; q++)
      if (c.Gcode.at(r, q)) {
        cnt++;
        col = c.Gcode.at(r, q) == 1 ? q : -2;
      }
    if (cnt == 1 && col >= 0) c.unit_col[r] = col;
  }
}

// PM-MBR (Sec. 2: alpha = d, Delta = (2d-k+1)/2).  M = [S T; T^t 0] with S
// symmetric k x k and T k x (d-k); the upper triangle of S is numbered row
// by row, then T row by row.  Psi = [I_k 0; C] (the systematic form of
// Sec. 3.2, Psi = [I; Psi'']) with C_ij = (g^(d+i) + g^j)^-1 a Cauchy matrix
// (0-based i < n-k, j < d): every square sub-matrix of C is invertible, so
// any d rows of Psi, and any k rows of its first k columns, are independent.
static int build_mbr(int n, int k, int d, int systematic, CodeMatrices &c, std::string &err) {
  if (k < 1 || d < k || d > n - 1) {
    err = "PM-MBR needs 1 <= k <= d <= n-1";
    return kEInval;
  }
  if (n > 254 || d + n - k > 255) {
    err = "PM-MBR needs d + n - k <= 255 (distinct Cauchy points in GF(2^8))";
    return kEInval;
  }
  c.n = n;
  c.k = k;
  c.d = d;
  c.alpha = d;
  c.K = k * (2 * d - k + 1) / 2;
  c.N = n * d;
  c.construction = kConsMbr;
  c.systematic = systematic;
  c.psi = Mat(n, d);
  for (int i = 0; i < k; i++) c.psi.at(i, i) = 1;
  for (int i = 0; i < n - k; i++)
    for (int j = 0; j < d; j++)
      c.psi.at(k + i, j) = gf_inv(gpow((unsigned)(d + i)) ^ gpow((unsigned)j));
  c.phi = c.psi;  // helper h projects its d blocks on psi_f
  c.lambda.assign(n, 0);
  c.L.assign((size_t)d * d, -1);
  int next = 0;
  for (int i = 0; i < k; i++)
    for (int j = i; j < k; j++, next++) c.L[(size_t)i * d + j] = c.L[(size_t)j * d + i] = next;
  for (int i = 0; i < k; i++)
    for (int m = 0; m < d - k; m++, next++)
      c.L[(size_t)i * d + k + m] = c.L[(size_t)(k + m) * d + i] = next;
  c.G = Mat(c.N, c.K);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < d; j++)
      for (int l = 0; l < d; l++) {
        const int s = c.L[(size_t)l * d + j];
        if (s >= 0) c.G.at(d * i + j, s) = c.psi.at(i, l);
      }
  c.Gcode = c.G;  // already systematic: node i < k stores row i of M
  mark_unit_rows(c);
  return kOk;
}

// Reed-Solomon (the comparison code of Sec. 4): node i stores the message
// polynomial evaluated at g^i, Y = V Z with V[i][j] = g^(ij); any k of the
// n <= 255 distinct points determine Z.  Systematic form G' = V V~^-1
// (Sec. 3.2).  One block per node; node f is repaired from k helpers by
// decoding and re-encoding its row, so Psi := G' (the rows the newcomer
// inverts) and every helper sends its block (phi = 1).
static int build_rs(int n, int k, int d, int systematic, CodeMatrices &c, std::string &err) {
  if (k < 1 || n <= k || n > 255) {
    err = "Reed-Solomon needs 1 <= k < n <= 255";
    return kEInval;
  }
  if (d != k) {
    err = "Reed-Solomon repair reads d = k helpers";
    return kEInval;
  }
  c.n = n;
  c.k = k;
  c.d = k;
  c.alpha = 1;
  c.K = k;
  c.N = n;
  c.construction = kConsRs;
  c.systematic = systematic;
  c.G = Mat(n, k);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < k; j++) c.G.at(i, j) = gpow((unsigned)(i * j));
  if (!systematic) {
    c.Gcode = c.G;
  } else {
    Mat top(k, k), topinv;
    std::copy(c.G.v.begin(), c.G.v.begin() + (size_t)k * k, top.v.begin());
    if (!mat_inverse(top, topinv)) {
      err = "the first k points do not determine the message";
      return kEUnsupported;
    }
    c.Gcode = mat_mul(c.G, topinv);
  }
  c.psi = c.Gcode;
  c.phi = Mat(n, 1);
  for (int i = 0; i < n; i++) c.phi.at(i, 0) = 1;
  c.lambda.assign(n, 0);
  c.L.clear();
  mark_unit_rows(c);
  return kOk;
}

int build_code(int n, int k, int d, int construction, int systematic, CodeMatrices &c,
               std::string &err) {
  if (systematic != 0 && systematic != 1) {
    err = "form must be PMRC_NONSYSTEMATIC or PMRC_SYSTEMATIC";
    return kEInval;
  }
  if (construction == kConsMbr) return build_mbr(n, k, d, systematic, c, err);
  if (construction == kConsRs) return build_rs(n, k, d, systematic, c, err);
  if (k < 2 || d != 2 * k - 2) {
    err = "PM-MSR needs k >= 2 and d = 2k-2";
    return kEInval;
  }
  if (n < d + 1 || n > 254) {
    err = "n must satisfy 2k-1 <= n <= 254";
    return kEInval;
  }
  if (construction != 0 && construction != 1) {
    err = "construction must be PMRC_VANILLA, PMRC_SPARSE, PMRC_MBR or PMRC_RS";
    return kEInval;
  }
  const int a = k - 1;
  c.n = n;
  c.k = k;
  c.d = d;
  c.alpha = a;
  c.construction = construction;
  c.systematic = systematic;
  c.phi = Mat(n, a);
  c.lambda.assign(n, 0);
  if (construction == 0) {
    // Vandermonde: Phi_ij = g^(i j), lambda_i = g^(i alpha) (0-based), so
    // that Psi_il = g^(i l) (Sec. 3.3, printed n=5 example).
    for (int i = 0; i < n; i++) {
      for (int j = 0; j < a; j++) c.phi.at(i, j) = gpow((unsigned)(i * j));
      c.lambda[i] = gpow((unsigned)(i * a));
    }
  } else {
    // Sparse: identity on the first alpha rows, Cauchy below; 1-based
    // i, j as in Sec. 3.3:  Phi_ij = (g^(i+alpha) + g^(j-1))^-1 for i > alpha,
    // lambda_i = (g^(i+alpha) + 1) / (g^(i+alpha) + g^alpha).
    for (int i = 1; i <= n; i++) {
      const uint8_t z = gpow((unsigned)(i + a));
      for (int j = 1; j <= a; j++)
        c.phi.at(i - 1, j - 1) = (i <= a) ? (uint8_t)(i == j) : gf_inv(z ^ gpow((unsigned)(j - 1)));
      c.lambda[i - 1] = gmul(z ^ 1, gf_inv(z ^ gpow((unsigned)a)));
    }
  }
  {
    std::vector<uint8_t> s = c.lambda;
    std::sort(s.begin(), s.end());
    if (std::adjacent_find(s.begin(), s.end()) != s.end()) {
      err = "construction has repeated lambda values at this (n, k): not an MSR code in GF(2^8)";
      return kEUnsupported;
    }
  }
  c.psi = Mat(n, d);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < a; j++) {
      c.psi.at(i, j) = c.phi.at(i, j);
      c.psi.at(i, a + j) = gmul(c.lambda[i], c.phi.at(i, j));
    }
  // Index matrix (Sec. 3.1): upper triangles of S1 then S2 numbered row by
  // row; M = [S1; S2] is d x alpha with symmetric blocks.
  c.L.assign((size_t)d * a, 0);
  {
    std::vector<int> tri((size_t)a * a, 0);
    int next = 0;
    for (int r = 0; r < a; r++)
      for (int q = r; q < a; q++) tri[(size_t)r * a + q] = tri[(size_t)q * a + r] = next++;
    const int half = next;
    for (int r = 0; r < a; r++)
      for (int q = 0; q < a; q++) {
        c.L[(size_t)r * a + q] = tri[(size_t)r * a + q];
        c.L[(size_t)(a + r) * a + q] = half + tri[(size_t)r * a + q];
      }
  }
  const int K = k * a, N = n * a;
  c.K = K;
  c.N = N;
  c.G = Mat(N, K);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < a; j++)
      for (int l = 0; l < d; l++) c.G.at(a * i + j, c.L[(size_t)l * a + j]) = c.psi.at(i, l);
  if (!systematic) {
    c.Gcode = c.G;
  } else {
    Mat top(K, K), topinv;
    std::copy(c.G.v.begin(), c.G.v.begin() + (size_t)K * K, top.v.begin());
    if (!mat_inverse(top, topinv)) {
      err = "the first k nodes do not determine the data: no systematic form";
      return kEUnsupported;
    }
    c.Gcode = mat_mul(c.G, topinv);
  }
  mark_unit_rows(c);
  return kOk;
}

void helper_matrix(const CodeMatrices &c, int f, Mat &P) {
  if (c.w == 16) {
    helper_matrix16(c, f, P);
    return;
  }
  P = Mat(1, c.alpha);
  for (int j = 0; j < c.alpha; j++) P.at(0, j) = c.phi.at(f, j);
}

void helper_coefficients(const CodeMatrices &c, int f, std::vector<uint8_t> &coef) {
  coef.assign(c.phi.v.begin() + (size_t)f * c.alpha, c.phi.v.begin() + (size_t)(f + 1) * c.alpha);
}

static int check_distinct(const int *ids, int cnt, int n, int exclude, std::string &err,
                          const char *what) {
  std::vector<char> seen(n, 0);
  for (int i = 0; i < cnt; i++) {
    if (ids[i] < 0 || ids[i] >= n) {
      err = std::string(what) + ": node id out of range";
      return kEInval;
    }
    if (ids[i] == exclude) {
      err = std::string(what) + ": the failed node cannot help";
      return kEInval;
    }
    if (seen[ids[i]]) {
      err = std::string(what) + ": repeated node id";
      return kEInval;
    }
    seen[ids[i]] = 1;
  }
  return kOk;
}

int newcomer_matrix(const CodeMatrices &c, int f, const int *helpers, Mat &D, std::string &err) {
  if (f < 0 || f >= c.n) {
    err = "failed node out of range";
    return kEInval;
  }
  int rc = check_distinct(helpers, c.d, c.n, f, err, "helpers");
  if (rc) return rc;
  if (c.w == 16) return newcomer_matrix16(c, f, helpers, D, err);
  Mat PH(c.d, c.d), inv;
  for (int i = 0; i < c.d; i++)
    for (int l = 0; l < c.d; l++) PH.at(i, l) = c.psi.at(helpers[i], l);
  if (!mat_inverse(PH, inv)) {
    err = "the helpers' rows of Psi are singular for this failed node";
    return kESingular;
  }
  if (c.construction == kConsRs) {
    // X = G'_H^-1 y_H, so node f's block is G'[f] G'_H^-1 y_H
    D = Mat(1, c.d);
    const auto &T = mul_table().t;
    for (int q = 0; q < c.d; q++) {
      uint8_t s = 0;
      for (int l = 0; l < c.d; l++) s ^= T[c.psi.at(f, l)][inv.at(l, q)];
      D.at(0, q) = s;
    }
    return kOk;
  }
  if (c.construction == kConsMbr) {
    // Psi_H M psi_f = p  =>  M psi_f = Psi_H^-1 p, and node f stores
    // psi_f^t M = (M psi_f)^t (M symmetric): D = Psi_H^-1.
    D = inv;
    return kOk;
  }
  // Psi_H M phi_f = p  =>  M phi_f = Psi_H^-1 p = [S1 phi_f; S2 phi_f];
  // node f stores phi_f^t S1 + lambda_f phi_f^t S2 (S1, S2 symmetric).
  const int a = c.alpha;
  D = Mat(a, c.d);
  const uint8_t lf = c.lambda[f];
  for (int j = 0; j < a; j++)
    for (int q = 0; q < c.d; q++) D.at(j, q) = inv.at(j, q) ^ gmul(lf, inv.at(a + j, q));
  return kOk;
}

// MBR reconstruction: the k alpha rows of the listed nodes span the K data
// blocks.  Rows are taken in order of preference -- rows copying a data
// block first, then the others in node order -- and kept when independent
// of those already kept (incremental elimination); the K kept rows are
// inverted and every other row gets coefficient zero.
static int decode_matrix_mbr(const CodeMatrices &c, const int *nodes, Mat &Rinv,
                             std::string &err) {
  const int a = c.alpha, K = c.K, KA = c.k * a;
  const auto &T = mul_table().t;
  std::vector<int> order;
  for (int pass = 0; pass < 2; pass++)
    for (int p = 0; p < KA; p++) {
      const bool unit = c.unit_col[a * nodes[p / a] + p % a] >= 0;
      if (unit == (pass == 0)) order.push_back(p);
    }
  Mat E(K, K), picked(K, K);      // reduced rows (pivot 1, pivots cleared) and originals
  std::vector<int> pivot, kept;
  std::vector<uint8_t> v(K);
  for (int p : order) {
    if ((int)kept.size() == K) break;
    const int row = a * nodes[p / a] + p % a;
    for (int q = 0; q < K; q++) v[q] = c.Gcode.at(row, q);
    for (size_t e = 0; e < kept.size(); e++) {
      const uint8_t f = v[pivot[e]];
      if (!f) continue;
      for (int q = 0; q < K; q++) v[q] ^= T[f][E.at((int)e, q)];
    }
    int pc = 0;
    while (pc < K && !v[pc]) pc++;
    if (pc == K) continue;
    const uint8_t *s = T[gf_inv(v[pc])];
    for (int q = 0; q < K; q++) v[q] = s[v[q]];
    for (size_t e = 0; e < kept.size(); e++) {
      const uint8_t f = E.at((int)e, pc);
      if (!f) continue;
      for (int q = 0; q < K; q++) E.at((int)e, q) ^= T[f][v[q]];
    }
    const int e = (int)kept.size();
    for (int q = 0; q < K; q++) {
      E.at(e, q) = v[q];
      picked.at(e, q) = c.Gcode.at(row, q);
    }
    pivot.push_back(pc);
    kept.push_back(p);
  }
  Mat inv;
  if ((int)kept.size() < K || !mat_inverse(picked, inv)) {
    err = "these k nodes do not determine the data";
    return kESingular;
  }
  Rinv = Mat(K, KA);
  for (int x = 0; x < K; x++)
    for (int t = 0; t < K; t++) Rinv.at(x, kept[t]) = inv.at(x, t);
  return kOk;
}

namespace {

// The systematic form's reconstruction, factored: a present data block is
// its own row of G' (a unit row), so only the missing data columns M need
// solving.  With Q the parity rows received, y_Q = A x_P + B x_M (A =
// G'[Q][present columns], B = G'[Q][M], |Q| = |M|) and x_P = y_P, hence
// x_M = B^-1 (y_Q + A y_P) (characteristic 2), an |M|^3 elimination instead
// of a K^3 one.  qpos[i]: input slot of the i-th received parity block;
// pcols / ppos: present data columns and their input slots; mcols: the
// missing data columns, in order.
struct SysFactors {
  std::vector<int> qpos, pcols, ppos, mcols;
  Mat A, Binv;
};

int systematic_factors(const CodeMatrices &c, const int *nodes, SysFactors &F,
                       std::string &err) {
  const int a = c.alpha, K = c.k * a;
  std::vector<int> pos_of_col(K, -1);
  for (int i = 0; i < c.k; i++)
    for (int j = 0; j < a; j++) {
      if (nodes[i] < c.k)
        pos_of_col[a * nodes[i] + j] = a * i + j;
      else
        F.qpos.push_back(a * i + j);
    }
  for (int col = 0; col < K; col++) {
    if (pos_of_col[col] < 0) {
      F.mcols.push_back(col);
    } else {
      F.pcols.push_back(col);
      F.ppos.push_back(pos_of_col[col]);
    }
  }
  const int m = (int)F.mcols.size();
  if (m == 0) return kOk;
  Mat B(m, m);
  F.A = Mat(m, (int)F.pcols.size());
  for (int qi = 0; qi < m; qi++) {
    const int row = a * nodes[F.qpos[qi] / a] + F.qpos[qi] % a;  // row of G'
    for (int mi = 0; mi < m; mi++) B.at(qi, mi) = c.Gcode.at(row, F.mcols[mi]);
    for (size_t pi = 0; pi < F.pcols.size(); pi++) F.A.at(qi, (int)pi) = c.Gcode.at(row, F.pcols[pi]);
  }
  if (!mat_inverse(B, F.Binv)) {
    err = "these k nodes do not determine the data";
    return kESingular;
  }
  return kOk;
}

}  // namespace

int decode_matrix(const CodeMatrices &c, const int *nodes, Mat &Rinv, std::string &err) {
  int rc = check_distinct(nodes, c.k, c.n, -1, err, "nodes");
  if (rc) return rc;
  if (c.construction == kConsMbr) return decode_matrix_mbr(c, nodes, Rinv, err);
  if (c.w == 16) return decode_matrix16(c, nodes, Rinv, err);
  const int a = c.alpha, K = c.k * a;
  if (!c.systematic) {
    Mat GR(K, K);
    for (int i = 0; i < c.k; i++)
      for (int j = 0; j < a; j++)
        std::copy(c.Gcode.v.begin() + (size_t)(a * nodes[i] + j) * K,
                  c.Gcode.v.begin() + (size_t)(a * nodes[i] + j + 1) * K,
                  GR.v.begin() + (size_t)(a * i + j) * K);
    if (!mat_inverse(GR, Rinv)) {
      err = "these k nodes do not determine the data";
      return kESingular;
    }
    return kOk;
  }
  SysFactors F;
  rc = systematic_factors(c, nodes, F, err);
  if (rc) return rc;
  Rinv = Mat(K, K);
  for (size_t pi = 0; pi < F.pcols.size(); pi++) Rinv.at(F.pcols[pi], F.ppos[pi]) = 1;
  const int m = (int)F.mcols.size();
  if (m == 0) return kOk;
  Mat BA = F.pcols.empty() ? Mat(m, 0) : mat_mul(F.Binv, F.A);
  for (int mi = 0; mi < m; mi++) {
    const int col = F.mcols[mi];
    for (int qi = 0; qi < m; qi++) Rinv.at(col, F.qpos[qi]) = F.Binv.at(mi, qi);
    for (size_t pi = 0; pi < F.pcols.size(); pi++) Rinv.at(col, F.ppos[pi]) = BA.at(mi, (int)pi);
  }
  return kOk;
}

int decode_factors(const CodeMatrices &c, const int *nodes, Mat &Z, Mat &W,
                   std::vector<int> &mcols, std::vector<int> &zslot, std::string &err) {
  int rc = check_distinct(nodes, c.k, c.n, -1, err, "nodes");
  if (rc) return rc;
  if (c.construction == kConsMbr || c.w != 8 || !c.systematic) {
    err = "factored reconstruction: systematic GF(2^8) MSR and Reed-Solomon codes only";
    return kEUnsupported;
  }
  SysFactors F;
  rc = systematic_factors(c, nodes, F, err);
  if (rc) return rc;
  const int m = (int)F.mcols.size(), KA = c.k * c.alpha;
  mcols = F.mcols;
  zslot = F.qpos;
  Z = Mat(m, KA);
  for (int qi = 0; qi < m; qi++) {
    Z.at(qi, F.qpos[qi]) = 1;
    for (size_t pi = 0; pi < F.pcols.size(); pi++) Z.at(qi, F.ppos[pi]) = F.A.at(qi, (int)pi);
  }
  W = F.Binv;
  return kOk;
}

int default_helpers(const CodeMatrices &c, int f, int *out, std::string &err) {
  if (f < 0 || f >= c.n) {
    err = "failed node out of range";
    return kEInval;
  }
  std::vector<int> surv;
  for (int i = 0; i < c.n; i++)
    if (i != f) surv.push_back(i);
  const int m = (int)surv.size(), d = c.d;
  // Combinations of d survivors in lexicographic order: the first is the d
  // lowest-index survivors.
  std::vector<int> idx(d);
  for (int i = 0; i < d; i++) idx[i] = i;
  for (int tries = 0; tries < 100000; tries++) {
    bool ok;
    if (c.w == 16) {
      std::vector<int> h(d);
      for (int i = 0; i < d; i++) h[i] = surv[idx[i]];
      ok = helpers_invertible16(c, h.data());
    } else {
      Mat PH(d, d), inv;
      for (int i = 0; i < d; i++)
        for (int l = 0; l < d; l++) PH.at(i, l) = c.psi.at(surv[idx[i]], l);
      ok = mat_inverse(PH, inv);
    }
    if (ok) {
      for (int i = 0; i < d; i++) out[i] = surv[idx[i]];
      return kOk;
    }
    int p = d - 1;
    while (p >= 0 && idx[p] == m - d + p) p--;
    if (p < 0) break;
    idx[p]++;
    for (int q = p + 1; q < d; q++) idx[q] = idx[q - 1] + 1;
  }
  err = "no invertible helper set found for this failed node";
  return kESingular;
}

}  // namespace pmrc
