// The product-matrix algorithms that Sec. 4 evaluates as "specific" (beside
// the linearized ones): the data collector of the seminal PM paper, which
// recovers the message matrix from any k nodes through alpha x alpha solves,
// and the systematic encode of Sec. 3.2 built from it by decoding the data
// as nodes 0..k-1 and encoding the parity nodes.
//
// Every stage is linear with constant coefficients, so each runs as one
// region launch over a small matrix built here; intermediate blocks live in
// a caller-supplied device workspace.
#pragma once
#include <cstddef>
#include <memory>
#include <string>
#include <vector>

#include "code.h"
#include "plan.h"

namespace pmrc {

// Workspace layout, in blocks of `pitch` bytes (block size rounded up to 256):
//   W0  max(k(k-1), 2 alpha^2) blocks: the k(k-1) entries A_ij (i != j) of
//       A = Y_DC Phi_DC^t, later overwritten by U and V (2 alpha^2)
//   W1  k(k-1) blocks: P_ij then Q_ij for the pairs i < j
//   W2  k alpha blocks: the precoded message Z (systematic codes only)
struct SpecificPlan {
  int k = 0, alpha = 0;
  int npair = 0;       // k(k-1)/2
  int w0 = 0, w1 = 0, w2 = 0;
  std::shared_ptr<Plan> A, PQ, UV, S;  // data collector stages
  std::shared_ptr<Plan> X;             // re-encode: data rows (decode) or parity (precode)
  std::vector<int> copy_rows;          // data rows copied from a listed node (decode)
};

size_t specific_pitch(size_t block_bytes);
size_t specific_workspace_blocks(const CodeMatrices &c);

// Builds the stage plans for node list `nodes` (k ids).  precode: nodes are
// 0..k-1 and X produces the parity rows.  Otherwise `want[r]` marks the data
// rows to produce; for the systematic code rows held by a listed node are
// copied (copy_rows) instead of re-encoded.
int build_specific(const CodeMatrices &c, const int *nodes, bool precode,
                   const std::vector<char> &want, SpecificPlan &out, std::string &err);

}  // namespace pmrc
