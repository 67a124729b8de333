// Host-side construction of product-matrix MSR codes and of the small
// matrices each region operation applies.
//
//   Sec. 2    erasure code as a linear map, MSR point alpha = d-k+1
//   Sec. 3.1  linearization: generator G from Psi and the index matrix L
//   Sec. 3.2  systematic form G' = G * G~^-1 = [I; G'']
//   Sec. 3.3  Psi = [Phi  Lambda*Phi], vanilla (Vandermonde) and sparse
//             (identity + Cauchy) constructions; helper read reduction
//
//   Sec. 4    Vandermonde Reed-Solomon baseline (construction 3): Y = V Z,
//             V[i][j] = g^(ij), systematic G' = V V~^-1; one block per node
//   Sec. 2    MBR point alpha = d, Delta = (2d-k+1)/2 (construction 2):
//             M = [S T; T^t 0] symmetric d x d, Psi = [I_k 0; Cauchy]
//             (Sec. 3.2: a systematic Psi = [I; Psi''] given directly)
//
// All matrices are row-major uint8 over GF(2^8) (modulus 0x11D).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace pmrc {

enum Status {
  kOk = 0,
  kEInval = -1,
  kESingular = -2,
  kEUnsupported = -3,
  kENoMem = -4,
  kECuda = -5,
  kETimeout = -6,
  kEBusy = -7,
};

struct Mat {
  int rows = 0, cols = 0;
  std::vector<uint8_t> v;
  Mat() = default;
  Mat(int r, int c) : rows(r), cols(c), v((size_t)r * c, 0) {}
  uint8_t &at(int r, int c) { return v[(size_t)r * cols + c]; }
  uint8_t at(int r, int c) const { return v[(size_t)r * cols + c]; }
};

Mat mat_mul(const Mat &A, const Mat &B);
// Gauss-Jordan inverse; returns false if A is singular.
bool mat_inverse(const Mat &A, Mat &out);

constexpr int kConsMbr = 2;  // construction id of the PM-MBR code
constexpr int kConsRs = 3;   // Reed-Solomon baseline (Sec. 4), alpha = 1, d = k

struct CodeMatrices {
  int n = 0, k = 0, d = 0, alpha = 0;
  int K = 0, N = 0;      // data blocks (k alpha for MSR, k Delta for MBR), n alpha
  int construction = 0;  // 0 vanilla MSR, 1 sparse MSR, 2 MBR, 3 Reed-Solomon
  int systematic = 0;
  Mat phi;      // n x alpha: the helper projection vectors (Phi for MSR, Psi for MBR)
  std::vector<uint8_t> lambda;  // n (MSR)
  Mat psi;      // n x d
  std::vector<int> L;           // d x alpha index matrix (-1: zero entry of M, MBR)
  Mat G;        // N x K, linearized generator (Sec. 3.1)
  Mat Gcode;    // the code's generator: G, or G' = G G~^-1 when systematic (MSR)
  std::vector<int> unit_col;    // per row of Gcode: the data block it copies, or -1
  // GF(2^16) codes (code16.cpp): the matrices above are the GF(2^8)
  // expansion (two byte planes per user block, alpha/K/N doubled); the
  // GF(2^16) originals are kept here.  beta = sub-blocks per helper projection.
  int w = 8, beta = 1;
  struct {
    int alpha = 0, K = 0, N = 0;
    std::vector<uint16_t> phi, lambda, psi, Gcode;
  } f16;
};

void mark_unit_rows(CodeMatrices &c);

// GF(2^16) (code16.cpp): construction and its expansion to GF(2^8) region
// matrices; the repair and decode matrices of such a code, expanded.
int build_code16(int n, int k, int d, int construction, int systematic, CodeMatrices &c,
                 std::string &err);
void expand16(const std::vector<uint16_t> &M, int rows, int cols, Mat &out);
void helper_matrix16(const CodeMatrices &c, int f, Mat &P);
bool helpers_invertible16(const CodeMatrices &c, const int *helpers);
int newcomer_matrix16(const CodeMatrices &c, int f, const int *helpers, Mat &D, std::string &err);
int decode_matrix16(const CodeMatrices &c, const int *nodes, Mat &Rinv, std::string &err);

// The helper projection of node f as a beta x alpha matrix (1 x alpha
// phi_f for GF(2^8) codes, its 2 x 2 expansion for GF(2^16)).
void helper_matrix(const CodeMatrices &c, int f, Mat &P);

// Builds every matrix of the code.  Returns kEInval for bad parameters,
// kEUnsupported when the construction is not an MSR code in GF(2^8) at this
// size (repeated lambda, or G~ singular for the systematic form).
int build_code(int n, int k, int d, int construction, int systematic, CodeMatrices &out,
               std::string &err);

// Repair (Sec. 3.3 read pattern; product-matrix repair): the helper
// coefficients are phi_f; the newcomer applies D = [I | lambda_f I] Psi_H^-1.
void helper_coefficients(const CodeMatrices &c, int f, std::vector<uint8_t> &coef);
int newcomer_matrix(const CodeMatrices &c, int f, const int *helpers, Mat &D, std::string &err);

// Reconstruction from k nodes (Sec. 2): Rinv (K x k alpha) with
// X = Rinv Y_nodes.  MSR: the inverse of the nodes' rows of Gcode.  MBR: the
// nodes' k alpha rows have rank K; K independent ones (rows that copy a data
// block first) are inverted and the others get zero coefficients.
int decode_matrix(const CodeMatrices &c, const int *nodes, Mat &Rinv, std::string &err);
// The reconstruction of a systematic GF(2^8) MSR or Reed-Solomon code in
// factored form: the missing data rows mcols (W's rows, in order) are
// x_M = W z with z = Z y, y the k alpha received blocks.  Z (|M| x k alpha)
// is the received parity blocks plus their present-data terms (sparse: a
// parity row's non-zeros on present columns; row i starts from the parity
// block in input slot zslot[i], coefficient 1), W = B^-1 (|M| x |M|).  The
// product W Z equals decode_matrix's rows mcols.  |M| = 0 when every data
// node is among the k; kEUnsupported for other codes.
int decode_factors(const CodeMatrices &c, const int *nodes, Mat &Z, Mat &W,
                   std::vector<int> &mcols, std::vector<int> &zslot, std::string &err);

// Default helper set for node f: the d lowest-index survivors, or the first
// set (in that order of preference) whose Psi rows are invertible.
int default_helpers(const CodeMatrices &c, int f, int *helpers_out, std::string &err);

}  // namespace pmrc
