// Stage matrices of the product-matrix data collector and of the systematic
// encode by decoding then encoding (Sec. 3.2, Sec. 4 "specific" algorithms).
//
// With DC the k listed nodes (in list order), Y_DC their k x alpha contents,
// Phi_DC and Lambda_DC their rows of Phi and Lambda (Sec. 3.3):
//   Y_DC = Phi_DC S1 + Lambda_DC Phi_DC S2, so A = Y_DC Phi_DC^t = P + Lambda_DC Q
//   with P = Phi_DC S1 Phi_DC^t and Q = Phi_DC S2 Phi_DC^t symmetric.
//   stage A : A_ij = sum_l Y_i[l] phi_j[l]                      (i != j)
//   stage PQ: Q_ij = (A_ij + A_ji) / (lambda_i + lambda_j),
//             P_ij = A_ij + lambda_i Q_ij                        (i < j)
//   stage UV: for the first alpha listed nodes i, the alpha values P_ij
//             (j != i) are phi_i^t S1 phi_j; with F_i the matrix of those
//             columns phi_j, u_i = phi_i^t S1 = [P_ij]_j F_i^-1, and v_i
//             likewise from Q
//   stage S : Phi_sub S1 = U and Phi_sub S2 = V (Phi_sub = rows phi_i of those
//             alpha nodes), so S1 = Phi_sub^-1 U, S2 = Phi_sub^-1 V; the
//             message symbols are the upper triangles, placed through L
//   stage X : systematic codes hold G~ Z on nodes 0..k-1 (Z the precoded
//             message): decode re-encodes the missing data rows with G,
//             precode encode produces the parity rows G[k alpha..] Z.
#include "specific.h"

#include <algorithm>

#include "gf256.h"

namespace pmrc {

size_t specific_pitch(size_t block_bytes) { return (block_bytes + 255) & ~(size_t)255; }

size_t specific_workspace_blocks(const CodeMatrices &c) {
  const int k = c.k, a = c.alpha;
  const int nA = k * (k - 1), nUV = 2 * a * a;
  return (size_t)std::max(nA, nUV) + nA + (c.systematic ? (size_t)k * a : 0);
}

int build_specific(const CodeMatrices &c, const int *nodes, bool precode,
                   const std::vector<char> &want, SpecificPlan &out, std::string &err) {
  const int k = c.k, a = c.alpha, K = k * a, N = c.n * a;
  if ((c.construction != 0 && c.construction != 1) || k - 1 != a) {
    err = "the data collector is the PM-MSR one (alpha = k - 1)";
    return kEUnsupported;
  }
  const int nA = k * (k - 1), np = nA / 2, nUV = 2 * a * a;
  out = SpecificPlan();
  out.k = k;
  out.alpha = a;
  out.npair = np;
  out.w0 = std::max(nA, nUV);
  out.w1 = nA;
  out.w2 = c.systematic ? K : 0;
  auto rowA = [&](int i, int j) { return i * (k - 1) + (j < i ? j : j - 1); };
  std::vector<int> pair((size_t)k * k, -1);  // pair index of {i, j}, i != j
  for (int i = 0, p = 0; i < k; i++)
    for (int j = i + 1; j < k; j++, p++) pair[(size_t)i * k + j] = pair[(size_t)j * k + i] = p;

  // stage A (k(k-1) x k alpha): row (i, j) reads node i's alpha blocks
  Mat MA(nA, K);
  for (int i = 0; i < k; i++)
    for (int j = 0; j < k; j++) {
      if (i == j) continue;
      for (int l = 0; l < a; l++) MA.at(rowA(i, j), a * i + l) = c.phi.at(nodes[j], l);
    }
  // stage PQ (k(k-1) x k(k-1)): P_ij rows 0..np-1, Q_ij rows np..2np-1
  Mat MPQ(nA, nA);
  for (int i = 0; i < k; i++)
    for (int j = i + 1; j < k; j++) {
      const uint8_t li = c.lambda[nodes[i]], s = li ^ c.lambda[nodes[j]];
      if (!s) {
        err = "two listed nodes share lambda";
        return kESingular;
      }
      const uint8_t q = gf_inv(s), lq = gmul(li, q);
      const int p = pair[(size_t)i * k + j];
      MPQ.at(np + p, rowA(i, j)) = q;
      MPQ.at(np + p, rowA(j, i)) = q;
      MPQ.at(p, rowA(i, j)) = (uint8_t)(1 ^ lq);
      MPQ.at(p, rowA(j, i)) = lq;
    }
  // stage UV (2 alpha^2 x k(k-1)): u_t[b] rows t*alpha+b, v_t[b] after them
  Mat MUV(nUV, nA);
  for (int t = 0; t < a; t++) {
    std::vector<int> J;
    for (int j = 0; j < k; j++)
      if (j != t) J.push_back(j);
    Mat F(a, a), Finv;
    for (int l = 0; l < a; l++)
      for (int q = 0; q < a; q++) F.at(l, q) = c.phi.at(nodes[J[q]], l);
    if (!mat_inverse(F, Finv)) {
      err = "alpha rows of Phi are dependent";
      return kESingular;
    }
    for (int b = 0; b < a; b++)
      for (int q = 0; q < a; q++) {
        const int p = pair[(size_t)t * k + J[q]];
        MUV.at(t * a + b, p) = Finv.at(q, b);
        MUV.at(a * a + t * a + b, np + p) = Finv.at(q, b);
      }
  }
  // stage S (k alpha x 2 alpha^2): message symbol L[x][b] (x <= b) of S1, S2
  Mat Psub(a, a), Psinv;
  for (int t = 0; t < a; t++)
    for (int l = 0; l < a; l++) Psub.at(t, l) = c.phi.at(nodes[t], l);
  if (!mat_inverse(Psub, Psinv)) {
    err = "alpha rows of Phi are dependent";
    return kESingular;
  }
  Mat MS(K, nUV);
  for (int x = 0; x < a; x++)
    for (int b = x; b < a; b++) {
      const int s1 = c.L[(size_t)x * a + b], s2 = c.L[(size_t)(a + x) * a + b];
      for (int t = 0; t < a; t++) {
        MS.at(s1, t * a + b) = Psinv.at(x, t);
        MS.at(s2, a * a + t * a + b) = Psinv.at(x, t);
      }
    }

  std::vector<int> all(nA), allUV(nUV);
  for (int r = 0; r < nA; r++) all[r] = r;
  for (int r = 0; r < nUV; r++) allUV[r] = r;
  out.A = make_plan(MA, all, nA);
  out.PQ = make_plan(MPQ, all, nA);
  out.UV = make_plan(MUV, allUV, nUV);
  std::vector<int> sslot(K);
  for (int r = 0; r < K; r++) sslot[r] = (c.systematic || precode || want[r]) ? r : -1;
  out.S = make_plan(MS, sslot, K);

  if (precode) {  // parity = rows k alpha .. n alpha - 1 of G applied to Z
    Mat MX(N - K, K);
    for (int r = 0; r < N - K; r++)
      for (int q = 0; q < K; q++) MX.at(r, q) = c.G.at(K + r, q);
    std::vector<int> slot(N - K);
    for (int r = 0; r < N - K; r++) slot[r] = r;
    out.X = make_plan(MX, slot, N - K);
  } else if (c.systematic) {  // data rows: copy from a listed node, or G~ Z
    std::vector<int> pos(c.n, -1);
    for (int i = 0; i < k; i++) pos[nodes[i]] = i;
    Mat MX(K, K);
    std::vector<int> slot(K, -1);
    bool any = false;
    for (int r = 0; r < K; r++) {
      if (!want[r]) continue;
      if (pos[r / a] >= 0) {
        out.copy_rows.push_back(r);
        continue;
      }
      for (int q = 0; q < K; q++) MX.at(r, q) = c.G.at(r, q);
      slot[r] = r;
      any = true;
    }
    if (any) out.X = make_plan(MX, slot, K);
  }
  if (!out.A || !out.PQ || !out.UV || !out.S || ((precode) && !out.X)) {
    err = "out of host memory";
    return kENoMem;
  }
  return kOk;
}

}  // namespace pmrc
