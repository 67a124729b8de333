/*
 * pmrc_oracle.c -- plain CPU statement of product-matrix MSR regenerating
 * codes (Le Scouarnec, "Fast Product-Matrix Regenerating Codes").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the bench's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the library under paper_1412_3022_gb300/, and the library never calls
 * it.
 *
 * Everything here is deliberately slow and literal:
 *   - GF(2^8) arithmetic through log/antilog tables (modulus x^8+x^4+x^3+x^2+1,
 *     i.e. 0x11D, generator g = 2);
 *   - every matrix is built entry by entry from its definition in the paper;
 *   - inverses are plain Gauss-Jordan elimination;
 *   - region work is the definition Y[r][t] = sum_c G[r][c] * X[c][t],
 *     one byte at a time.
 *
 * Notation (0-based throughout; the paper is 1-based in Sec. 3.3 and 0-based
 * in the Y_{alpha i + j} indexing of Sec. 3.1):
 *   k data nodes, d = 2k-2 helpers, alpha = d-k+1 = k-1 blocks per node,
 *   n nodes in total, k*alpha data blocks X, n*alpha coded blocks Y.
 *
 * Error codes: 0 ok, -1 bad argument, -2 singular matrix.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ESINGULAR (-2)

#define OR_VANILLA 0
#define OR_SPARSE 1

/* ------------------------------------------------------------------------ */
/* GF(2^8), log/antilog tables (Sec. 4: the paper works in GF(2^8) through   */
/* GF-Complete; modulus 0x11D, generator g = 2).                            */
/* ------------------------------------------------------------------------ */

static uint8_t or_exp[255]; /* or_exp[i] = g^i                         */
static int or_log[256];     /* or_log[g^i] = i; or_log[0] unused (-1)   */
static int or_ready = 0;

static void or_init(void)
{
    if (or_ready)
        return;
    int x = 1;
    for (int i = 0; i < 256; i++)
        or_log[i] = -1;
    for (int i = 0; i < 255; i++) {
        or_exp[i] = (uint8_t)x;
        or_log[x] = i;
        x <<= 1;              /* multiply by g = 2 ...              */
        if (x & 0x100)
            x ^= 0x11D;       /* ... and reduce modulo the polynomial */
    }
    or_ready = 1;
}

uint8_t or_gf_mul(uint8_t a, uint8_t b)
{
    or_init();
    if (a == 0 || b == 0)
        return 0;
    return or_exp[(or_log[a] + or_log[b]) % 255];
}

/* a^-1 for a != 0; returns 0 for a == 0 (callers never ask for it). */
uint8_t or_gf_inv(uint8_t a)
{
    or_init();
    if (a == 0)
        return 0;
    return or_exp[(255 - or_log[a]) % 255];
}

/* g^e for any integer e >= 0. */
uint8_t or_gf_pow_g(int e)
{
    or_init();
    return or_exp[e % 255];
}

int or_gf_log(uint8_t a)
{
    or_init();
    return or_log[a];
}

/* Addition and subtraction in GF(2^8) are both XOR. */
static uint8_t or_add(uint8_t a, uint8_t b) { return (uint8_t)(a ^ b); }

/* ------------------------------------------------------------------------ */
/* Small dense matrices over GF(2^8), row-major.                             */
/* ------------------------------------------------------------------------ */

/* C (m x p) = A (m x q) * B (q x p) */
void or_mat_mul(int m, int q, int p, const uint8_t *A, const uint8_t *B, uint8_t *C)
{
    for (int i = 0; i < m; i++)
        for (int j = 0; j < p; j++) {
            uint8_t s = 0;
            for (int l = 0; l < q; l++)
                s = or_add(s, or_gf_mul(A[i * q + l], B[l * p + j]));
            C[i * p + j] = s;
        }
}

/* Gauss-Jordan inverse of the m x m matrix A.  Returns OR_ESINGULAR if A has
 * no inverse (Sec. 2: decoding is X = G~^-1 Y~). */
int or_invert(int m, const uint8_t *A, uint8_t *Ainv)
{
    if (m <= 0)
        return OR_EINVAL;
    uint8_t *W = (uint8_t *)malloc((size_t)m * 2 * m);
    if (!W)
        return OR_EINVAL;
    int w = 2 * m;
    for (int i = 0; i < m; i++)
        for (int j = 0; j < w; j++)
            W[i * w + j] = j < m ? A[i * m + j] : (uint8_t)(j - m == i);
    for (int col = 0; col < m; col++) {
        int piv = -1;
        for (int i = col; i < m; i++)
            if (W[i * w + col] != 0) {
                piv = i;
                break;
            }
        if (piv < 0) {
            free(W);
            return OR_ESINGULAR;
        }
        if (piv != col)
            for (int j = 0; j < w; j++) {
                uint8_t t = W[col * w + j];
                W[col * w + j] = W[piv * w + j];
                W[piv * w + j] = t;
            }
        uint8_t s = or_gf_inv(W[col * w + col]);
        for (int j = 0; j < w; j++)
            W[col * w + j] = or_gf_mul(s, W[col * w + j]);
        for (int i = 0; i < m; i++) {
            if (i == col || W[i * w + col] == 0)
                continue;
            uint8_t f = W[i * w + col];
            for (int j = 0; j < w; j++)
                W[i * w + j] = or_add(W[i * w + j], or_gf_mul(f, W[col * w + j]));
        }
    }
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++)
            Ainv[i * m + j] = W[i * w + m + j];
    free(W);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Code parameters and the encoding matrix Psi = [Phi  Lambda*Phi]           */
/* (Sec. 3.3).                                                              */
/* ------------------------------------------------------------------------ */

/* MSR point with d = 2k-2: alpha = Delta = d-k+1 = k-1 (Sec. 2). */
int or_params(int n, int k, int *d, int *alpha)
{
    if (k < 2 || n < 2 * k - 1 || n > 254)
        return OR_EINVAL;
    *d = 2 * k - 2;
    *alpha = k - 1;
    return OR_OK;
}

/* Phi (n x alpha) and the diagonal of Lambda (n).
 *
 * Vanilla (Sec. 3.3, the Vandermonde construction): Phi_{i,j} = g^{ij}
 * (0-based) and, from the printed n=5 example whose Lambda is
 * diag(1, g^2, g^4, g^6, g^8) at alpha = 2, lambda_i = g^{i*alpha}; then
 * Psi_{i,l} = g^{il} is the Vandermonde matrix printed beside it.
 *
 * Sparse (Sec. 3.3, the paper's construction), in the paper's 1-based
 * indices i = 1..n, j = 1..alpha:
 *   Phi_{i,j} = delta_{ij}                        for i <= alpha,
 *   Phi_{i,j} = (g^{i+alpha} - g^{j-1})^-1          for i > alpha,
 *   lambda_i  = (g^{i+alpha} - g^0) / (g^{i+alpha} - g^alpha).
 */
int or_phi_lambda(int n, int k, int construction, uint8_t *phi, uint8_t *lambda)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    if (construction == OR_VANILLA) {
        for (int i = 0; i < n; i++) {
            for (int j = 0; j < a; j++)
                phi[i * a + j] = or_gf_pow_g(i * j);
            lambda[i] = or_gf_pow_g(i * a);
        }
        return OR_OK;
    }
    if (construction == OR_SPARSE) {
        for (int i1 = 1; i1 <= n; i1++) {
            int i = i1 - 1;
            for (int j1 = 1; j1 <= a; j1++) {
                int j = j1 - 1;
                if (i1 <= a)
                    phi[i * a + j] = (uint8_t)(i1 == j1);
                else
                    phi[i * a + j] =
                        or_gf_inv(or_add(or_gf_pow_g(i1 + a), or_gf_pow_g(j1 - 1)));
            }
            uint8_t num = or_add(or_gf_pow_g(i1 + a), or_gf_pow_g(0));
            uint8_t den = or_add(or_gf_pow_g(i1 + a), or_gf_pow_g(a));
            lambda[i] = or_gf_mul(num, or_gf_inv(den));
        }
        return OR_OK;
    }
    return OR_EINVAL;
}

/* Psi (n x d) = [Phi  Lambda*Phi] (Sec. 3.3, first constraint). */
int or_psi(int n, int k, int construction, uint8_t *psi)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    uint8_t *phi = (uint8_t *)malloc((size_t)n * a);
    uint8_t *lam = (uint8_t *)malloc((size_t)n);
    int rc = or_phi_lambda(n, k, construction, phi, lam);
    if (rc == OR_OK)
        for (int i = 0; i < n; i++)
            for (int j = 0; j < a; j++) {
                psi[i * d + j] = phi[i * a + j];
                psi[i * d + a + j] = or_gf_mul(lam[i], phi[i * a + j]);
            }
    free(phi);
    free(lam);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Message matrix and its index matrix L (Sec. 3.1).                         */
/* ------------------------------------------------------------------------ */

/* L (d x alpha): M_{l,j} = X_{L[l][j]}.  M = [S1; S2] with S1 and S2
 * symmetric alpha x alpha.  The upper triangle of S1 is numbered row by row
 * (0 .. alpha(alpha+1)/2 - 1), S2 continues the numbering; the lower triangle
 * mirrors the upper one.  For k = 3 this is the paper's printed example
 * L^t = [[1,2,4,5],[2,3,5,6]] (1-based). */
int or_index_matrix(int k, int *L)
{
    int a = k - 1, d = 2 * k - 2;
    if (k < 2)
        return OR_EINVAL;
    int half = a * (a + 1) / 2;
    for (int s = 0; s < 2; s++) {
        int base = s * half;
        for (int r = 0; r < a; r++)
            for (int c = 0; c < a; c++) {
                int i = r < c ? r : c, j = r < c ? c : r; /* upper-triangle cell */
                int num = 0;                              /* row-major rank of (i, j) */
                for (int rr = 0; rr < i; rr++)
                    num += a - rr;
                num += j - i;
                L[(s * a + r) * a + c] = base + num;
            }
    }
    (void)d;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Linearized generator (Sec. 3.1) and systematic form (Sec. 3.2).           */
/* ------------------------------------------------------------------------ */

/* G (n*alpha x k*alpha): G[alpha i + j][L[l][j]] = Psi[i][l] for l < d, and
 * zero elsewhere.  (The paper's sum runs "l = 1..n"; M has d rows, so it runs
 * over l < d.) */
int or_generator(int n, int k, int construction, uint8_t *G)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    int K = k * a;
    uint8_t *psi = (uint8_t *)malloc((size_t)n * d);
    int *L = (int *)malloc(sizeof(int) * d * a);
    int rc = or_psi(n, k, construction, psi);
    if (rc == OR_OK) {
        or_index_matrix(k, L);
        memset(G, 0, (size_t)n * a * K);
        for (int i = 0; i < n; i++)
            for (int j = 0; j < a; j++)
                for (int l = 0; l < d; l++)
                    G[(size_t)(a * i + j) * K + L[l * a + j]] = psi[i * d + l];
    }
    free(psi);
    free(L);
    return rc;
}

/* G' = G * G~^-1 with G~ the first k*alpha rows of G (Sec. 3.2).  The first
 * k*alpha rows of G' are the identity; the rest is G''. */
int or_systematic_generator(int n, int k, int construction, uint8_t *Gp)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    int K = k * a, N = n * a;
    uint8_t *G = (uint8_t *)malloc((size_t)N * K);
    uint8_t *Ginv = (uint8_t *)malloc((size_t)K * K);
    int rc = or_generator(n, k, construction, G);
    if (rc == OR_OK)
        rc = or_invert(K, G, Ginv); /* G~ = first K rows of G */
    if (rc == OR_OK)
        or_mat_mul(N, K, K, G, Ginv, Gp);
    free(G);
    free(Ginv);
    return rc;
}

/* The code's generator: G (non-systematic) or G' (systematic). */
int or_code_generator(int n, int k, int construction, int systematic, uint8_t *Gout)
{
    return systematic ? or_systematic_generator(n, k, construction, Gout)
                      : or_generator(n, k, construction, Gout);
}

/* ------------------------------------------------------------------------ */
/* Region work: Y = M X over byte blocks (Sec. 2: Y = GX, blockwise).        */
/* ------------------------------------------------------------------------ */

/* out[r][t] = sum_c M[r][c] * in[c][t] for t < nbytes.  Block c of the input
 * starts at in + c*in_stride, block r of the output at out + r*out_stride. */
void or_region_apply(int rows, int cols, const uint8_t *M, const uint8_t *in,
                     size_t in_stride, uint8_t *out, size_t out_stride, size_t nbytes)
{
    for (int r = 0; r < rows; r++) {
        uint8_t *y = out + (size_t)r * out_stride;
        memset(y, 0, nbytes);
        for (int c = 0; c < cols; c++) {
            uint8_t m = M[(size_t)r * cols + c];
            if (m == 0)
                continue; /* a zero coefficient adds nothing (Sec. 3.3) */
            const uint8_t *x = in + (size_t)c * in_stride;
            for (size_t t = 0; t < nbytes; t++)
                y[t] = or_add(y[t], or_gf_mul(m, x[t]));
        }
    }
}

/* Encode (Sec. 3.1/3.2): out receives all n*alpha coded blocks, node-major
 * (block alpha*i + j is slot j of node i).  For the systematic code the first
 * k*alpha blocks equal the data. */
int or_encode(int n, int k, int construction, int systematic, const uint8_t *data,
              uint8_t *out, size_t nbytes)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    int K = k * a, N = n * a;
    uint8_t *G = (uint8_t *)malloc((size_t)N * K);
    int rc = or_code_generator(n, k, construction, systematic, G);
    if (rc == OR_OK)
        or_region_apply(N, K, G, data, nbytes, out, nbytes, nbytes);
    free(G);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Repair of node f from d helpers (product-matrix MSR repair; Sec. 3.3      */
/* describes which helper blocks are read).                                 */
/* ------------------------------------------------------------------------ */

/* Helper coefficients: the helper sends p_h = sum_j phi_f[j] * Y[alpha h + j],
 * i.e. its stored row C_h = psi_h^t M projected on phi_f. */
int or_helper_coefficients(int n, int k, int construction, int f, uint8_t *coef)
{
    int d, a;
    if (or_params(n, k, &d, &a) || f < 0 || f >= n)
        return OR_EINVAL;
    uint8_t *phi = (uint8_t *)malloc((size_t)n * a);
    uint8_t *lam = (uint8_t *)malloc((size_t)n);
    int rc = or_phi_lambda(n, k, construction, phi, lam);
    if (rc == OR_OK)
        memcpy(coef, phi + (size_t)f * a, (size_t)a);
    free(phi);
    free(lam);
    return rc;
}

int or_repair_helper(int n, int k, int construction, int f, const uint8_t *blocks,
                     uint8_t *out, size_t nbytes)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    uint8_t *coef = (uint8_t *)malloc((size_t)a);
    int rc = or_helper_coefficients(n, k, construction, f, coef);
    if (rc == OR_OK)
        or_region_apply(1, a, coef, blocks, nbytes, out, nbytes, nbytes);
    free(coef);
    return rc;
}

/* Newcomer matrix D (alpha x d).  With Psi_H the rows of Psi for the helpers
 * (in list order), the received vector is p = Psi_H M phi_f, so
 * M phi_f = Psi_H^-1 p = [S1 phi_f; S2 phi_f].  By symmetry of S1 and S2 the
 * lost row is C_f = phi_f^t S1 + lambda_f phi_f^t S2, hence
 *   D[j][c] = Psi_H^-1[j][c] + lambda_f * Psi_H^-1[alpha + j][c]. */
int or_newcomer_matrix(int n, int k, int construction, int f, const int *helpers,
                       uint8_t *D)
{
    int d, a;
    if (or_params(n, k, &d, &a) || f < 0 || f >= n)
        return OR_EINVAL;
    for (int i = 0; i < d; i++) {
        if (helpers[i] < 0 || helpers[i] >= n || helpers[i] == f)
            return OR_EINVAL;
        for (int j = 0; j < i; j++)
            if (helpers[j] == helpers[i])
                return OR_EINVAL;
    }
    uint8_t *psi = (uint8_t *)malloc((size_t)n * d);
    uint8_t *PH = (uint8_t *)malloc((size_t)d * d);
    uint8_t *PHinv = (uint8_t *)malloc((size_t)d * d);
    uint8_t *phi = (uint8_t *)malloc((size_t)n * a);
    uint8_t *lam = (uint8_t *)malloc((size_t)n);
    int rc = or_psi(n, k, construction, psi);
    if (rc == OR_OK)
        rc = or_phi_lambda(n, k, construction, phi, lam);
    if (rc == OR_OK) {
        for (int i = 0; i < d; i++)
            memcpy(PH + (size_t)i * d, psi + (size_t)helpers[i] * d, (size_t)d);
        rc = or_invert(d, PH, PHinv);
    }
    if (rc == OR_OK)
        for (int j = 0; j < a; j++)
            for (int c = 0; c < d; c++)
                D[j * d + c] = or_add(PHinv[j * d + c],
                                      or_gf_mul(lam[f], PHinv[(a + j) * d + c]));
    free(psi);
    free(PH);
    free(PHinv);
    free(phi);
    free(lam);
    return rc;
}

/* recv: d blocks, in the order of helpers; out: the alpha blocks of node f. */
int or_repair_newcomer(int n, int k, int construction, int f, const int *helpers,
                       const uint8_t *recv, uint8_t *out, size_t nbytes)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    uint8_t *D = (uint8_t *)malloc((size_t)a * d);
    int rc = or_newcomer_matrix(n, k, construction, f, helpers, D);
    if (rc == OR_OK)
        or_region_apply(a, d, D, recv, nbytes, out, nbytes, nbytes);
    free(D);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Reconstruction from any k nodes (Sec. 2: X = G~^-1 Y~).                   */
/* ------------------------------------------------------------------------ */

/* Inverse of the k*alpha rows of the code generator that belong to nodes[]
 * (node-major, slots in order). */
int or_decode_matrix(int n, int k, int construction, int systematic, const int *nodes,
                     uint8_t *Rinv)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    for (int i = 0; i < k; i++) {
        if (nodes[i] < 0 || nodes[i] >= n)
            return OR_EINVAL;
        for (int j = 0; j < i; j++)
            if (nodes[j] == nodes[i])
                return OR_EINVAL;
    }
    int K = k * a, N = n * a;
    uint8_t *G = (uint8_t *)malloc((size_t)N * K);
    uint8_t *GR = (uint8_t *)malloc((size_t)K * K);
    int rc = or_code_generator(n, k, construction, systematic, G);
    if (rc == OR_OK) {
        for (int i = 0; i < k; i++)
            for (int j = 0; j < a; j++)
                memcpy(GR + (size_t)(a * i + j) * K,
                       G + (size_t)(a * nodes[i] + j) * K, (size_t)K);
        rc = or_invert(K, GR, Rinv);
    }
    free(G);
    free(GR);
    return rc;
}

/* node_blocks: the k*alpha blocks of nodes[] (node-major); data: k*alpha
 * data blocks X. */
int or_decode(int n, int k, int construction, int systematic, const int *nodes,
              const uint8_t *node_blocks, uint8_t *data, size_t nbytes)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    int K = k * a;
    uint8_t *Rinv = (uint8_t *)malloc((size_t)K * K);
    int rc = or_decode_matrix(n, k, construction, systematic, nodes, Rinv);
    if (rc == OR_OK)
        or_region_apply(K, K, Rinv, node_blocks, nbytes, data, nbytes, nbytes);
    free(Rinv);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* The product-matrix algorithms that Sec. 4 calls "specific" (as opposed    */
/* to linearized): the data collector of the seminal PM paper, and the      */
/* systematic encode built from it by decoding then encoding (Sec. 3.2).    */
/* The paper defers the data collector to the seminal paper; the steps      */
/* below are restated from the definitions of Sec. 2-3.                     */
/* ------------------------------------------------------------------------ */

/* Message recovery from the k*alpha blocks of nodes[] (node-major, in list
 * order), one byte column at a time.  With DC the listed nodes:
 *   1. Y_DC = Phi_DC S1 + Lambda_DC Phi_DC S2 (k x alpha), so
 *      A = Y_DC Phi_DC^t = P + Lambda_DC Q, where P = Phi_DC S1 Phi_DC^t and
 *      Q = Phi_DC S2 Phi_DC^t are symmetric k x k;
 *   2. for i != j:  A_ij = P_ij + lambda_i Q_ij  and  A_ji = P_ij + lambda_j Q_ij,
 *      so Q_ij = (A_ij + A_ji) / (lambda_i + lambda_j), P_ij = A_ij + lambda_i Q_ij
 *      (the diagonals of P and Q are never needed);
 *   3. for each of the first alpha listed nodes i, the alpha values P_ij
 *      (j != i, in list order) are phi_i^t S1 phi_j: with F_i the alpha x
 *      alpha matrix whose columns are those phi_j, phi_i^t S1 = [P_ij]_j F_i^-1;
 *      likewise phi_i^t S2 = [Q_ij]_j F_i^-1;
 *   4. stacking these rows, Phi_sub S1 = U and Phi_sub S2 = V with Phi_sub the
 *      rows phi_i of those alpha nodes, so S1 = Phi_sub^-1 U, S2 = Phi_sub^-1 V;
 *   5. the message symbols are read out of S1 and S2 through L (Sec. 3.1).
 * msg receives the k*alpha message blocks. */
int or_dc_decode(int n, int k, int construction, const int *nodes, const uint8_t *node_blocks,
                 uint8_t *msg, size_t nbytes)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    for (int i = 0; i < k; i++) {
        if (nodes[i] < 0 || nodes[i] >= n)
            return OR_EINVAL;
        for (int j = 0; j < i; j++)
            if (nodes[j] == nodes[i])
                return OR_EINVAL;
    }
    uint8_t *phi = (uint8_t *)malloc((size_t)n * a);
    uint8_t *lam = (uint8_t *)malloc((size_t)n);
    int *L = (int *)malloc(sizeof(int) * d * a);
    uint8_t *Finv = (uint8_t *)malloc((size_t)a * a * a);   /* F_i^-1, i < alpha */
    uint8_t *F = (uint8_t *)malloc((size_t)a * a);
    uint8_t *Psub = (uint8_t *)malloc((size_t)a * a);
    uint8_t *Psubinv = (uint8_t *)malloc((size_t)a * a);
    uint8_t *Y = (uint8_t *)malloc((size_t)k * a);
    uint8_t *A = (uint8_t *)malloc((size_t)k * k);
    uint8_t *P = (uint8_t *)malloc((size_t)k * k);
    uint8_t *Q = (uint8_t *)malloc((size_t)k * k);
    uint8_t *U = (uint8_t *)malloc((size_t)a * a);
    uint8_t *V = (uint8_t *)malloc((size_t)a * a);
    int rc = or_phi_lambda(n, k, construction, phi, lam);
    if (rc == OR_OK)
        or_index_matrix(k, L);
    /* lambda_i + lambda_j must be invertible for every listed pair */
    for (int i = 0; i < k && rc == OR_OK; i++)
        for (int j = 0; j < i && rc == OR_OK; j++)
            if (or_add(lam[nodes[i]], lam[nodes[j]]) == 0)
                rc = OR_ESINGULAR;
    /* F_i: column c is phi of the c-th listed node other than i */
    for (int i = 0; i < a && rc == OR_OK; i++) {
        for (int c = 0, j = 0; j < k; j++) {
            if (j == i)
                continue;
            for (int l = 0; l < a; l++)
                F[l * a + c] = phi[(size_t)nodes[j] * a + l];
            c++;
        }
        rc = or_invert(a, F, Finv + (size_t)i * a * a);
    }
    if (rc == OR_OK) {
        for (int i = 0; i < a; i++)
            memcpy(Psub + (size_t)i * a, phi + (size_t)nodes[i] * a, (size_t)a);
        rc = or_invert(a, Psub, Psubinv);
    }
    for (size_t t = 0; t < nbytes && rc == OR_OK; t++) {
        for (int i = 0; i < k; i++)
            for (int l = 0; l < a; l++)
                Y[i * a + l] = node_blocks[(size_t)(a * i + l) * nbytes + t];
        /* step 1 */
        for (int i = 0; i < k; i++)
            for (int j = 0; j < k; j++) {
                uint8_t s = 0;
                for (int l = 0; l < a; l++)
                    s = or_add(s, or_gf_mul(Y[i * a + l], phi[(size_t)nodes[j] * a + l]));
                A[i * k + j] = s;
            }
        /* step 2 */
        for (int i = 0; i < k; i++)
            for (int j = 0; j < k; j++) {
                if (i == j)
                    continue;
                uint8_t q = or_gf_mul(or_add(A[i * k + j], A[j * k + i]),
                                      or_gf_inv(or_add(lam[nodes[i]], lam[nodes[j]])));
                Q[i * k + j] = q;
                P[i * k + j] = or_add(A[i * k + j], or_gf_mul(lam[nodes[i]], q));
            }
        /* step 3 */
        for (int i = 0; i < a; i++)
            for (int b = 0; b < a; b++) {
                uint8_t u = 0, v = 0;
                for (int c = 0, j = 0; j < k; j++) {
                    if (j == i)
                        continue;
                    uint8_t f = Finv[(size_t)i * a * a + c * a + b];
                    u = or_add(u, or_gf_mul(P[i * k + j], f));
                    v = or_add(v, or_gf_mul(Q[i * k + j], f));
                    c++;
                }
                U[i * a + b] = u;
                V[i * a + b] = v;
            }
        /* steps 4 and 5 */
        for (int x = 0; x < a; x++)
            for (int b = 0; b < a; b++) {
                uint8_t s1 = 0, s2 = 0;
                for (int i = 0; i < a; i++) {
                    s1 = or_add(s1, or_gf_mul(Psubinv[x * a + i], U[i * a + b]));
                    s2 = or_add(s2, or_gf_mul(Psubinv[x * a + i], V[i * a + b]));
                }
                msg[(size_t)L[x * a + b] * nbytes + t] = s1;
                msg[(size_t)L[(a + x) * a + b] * nbytes + t] = s2;
            }
    }
    free(phi);
    free(lam);
    free(L);
    free(Finv);
    free(F);
    free(Psub);
    free(Psubinv);
    free(Y);
    free(A);
    free(P);
    free(Q);
    free(U);
    free(V);
    return rc;
}

/* Specific decode.  For the non-systematic code the message is the data.
 * The systematic code stores, on nodes 0..k-1, the PM codeword of the
 * precoded message Z (Sec. 3.2), so the data is X = G~ Z: the data collector
 * finds Z and the first k*alpha rows of G re-encode it. */
int or_decode_specific(int n, int k, int construction, int systematic, const int *nodes,
                       const uint8_t *node_blocks, uint8_t *data, size_t nbytes)
{
    if (!systematic)
        return or_dc_decode(n, k, construction, nodes, node_blocks, data, nbytes);
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    int K = k * a, N = n * a;
    uint8_t *Z = (uint8_t *)malloc((size_t)K * (nbytes ? nbytes : 1));
    uint8_t *G = (uint8_t *)malloc((size_t)N * K);
    int rc = or_dc_decode(n, k, construction, nodes, node_blocks, Z, nbytes);
    if (rc == OR_OK)
        rc = or_generator(n, k, construction, G);
    if (rc == OR_OK)
        or_region_apply(K, K, G, Z, nbytes, data, nbytes, nbytes);
    free(Z);
    free(G);
    return rc;
}

/* Systematic encode by decoding then encoding (Sec. 3.2): the data blocks
 * are taken as the contents of nodes 0..k-1, the data collector recovers the
 * precoded message Z from them, and the remaining (n-k)*alpha rows of G
 * encode Z into the parity blocks. */
int or_encode_precode(int n, int k, int construction, const uint8_t *data, uint8_t *parity,
                      size_t nbytes)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    int K = k * a, N = n * a;
    int *nodes = (int *)malloc(sizeof(int) * k);
    uint8_t *Z = (uint8_t *)malloc((size_t)K * (nbytes ? nbytes : 1));
    uint8_t *G = (uint8_t *)malloc((size_t)N * K);
    for (int i = 0; i < k; i++)
        nodes[i] = i;
    int rc = or_dc_decode(n, k, construction, nodes, data, Z, nbytes);
    if (rc == OR_OK)
        rc = or_generator(n, k, construction, G);
    if (rc == OR_OK)
        or_region_apply(N - K, K, G + (size_t)K * K, Z, nbytes, parity, nbytes, nbytes);
    free(nodes);
    free(Z);
    free(G);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Product-matrix MBR codes (Sec. 2: alpha = d, Delta = (2d-k+1)/2; Sec. 3.2: */
/* a systematic encoding matrix Psi = [I; Psi''] given directly; Sec. 4.2    */
/* evaluates encode, repair and decode).  The message matrix of the seminal  */
/* PM paper, restated:                                                       */
/*     M = [ S    T ]    (d x d, symmetric)                                  */
/*         [ T^t  0 ]                                                        */
/* with S a symmetric k x k matrix and T a k x (d-k) matrix of message      */
/* symbols, k(k+1)/2 + k(d-k) = k Delta in all.  Node i stores psi_i^t M     */
/* (alpha = d blocks).  Psi must have every d rows independent and every k   */
/* rows of its first k columns (Phi) independent.                            */
/* ------------------------------------------------------------------------ */

/* alpha = d, B = k Delta = k(2d-k+1)/2 message blocks; k <= d <= n-1. */
int or_mbr_params(int n, int k, int d, int *alpha, int *B)
{
    if (k < 1 || d < k || d > n - 1 || n > 128)
        return OR_EINVAL;
    *alpha = d;
    *B = k * (2 * d - k + 1) / 2;
    return OR_OK;
}

/* Psi (n x d) = [I_k 0; C]: the first k rows are the unit rows e_i (the
 * systematic nodes store message symbols verbatim), and the other n-k rows
 * are the Cauchy matrix C_{i,j} = (g^{d+i} - g^j)^-1 (0-based i < n-k,
 * j < d), every square sub-matrix of which is invertible.  Then any d rows
 * of Psi, and any k rows of its first k columns, are independent. */
int or_mbr_psi(int n, int k, int d, uint8_t *psi)
{
    int a, B;
    if (or_mbr_params(n, k, d, &a, &B))
        return OR_EINVAL;
    if (d + n - k > 255)
        return OR_EINVAL;
    memset(psi, 0, (size_t)n * d);
    for (int i = 0; i < k; i++)
        psi[(size_t)i * d + i] = 1;
    for (int i = 0; i < n - k; i++)
        for (int j = 0; j < d; j++)
            psi[(size_t)(k + i) * d + j] = or_gf_inv(or_add(or_gf_pow_g(d + i), or_gf_pow_g(j)));
    return OR_OK;
}

/* L (d x d): M_{l,j} = X_{L[l][j]}, or -1 where M is zero.  The upper
 * triangle of S is numbered row by row (0 .. k(k+1)/2 - 1), then T row by
 * row; the rest follows from the symmetry of M. */
int or_mbr_index_matrix(int k, int d, int *L)
{
    if (k < 1 || d < k)
        return OR_EINVAL;
    for (int i = 0; i < d * d; i++)
        L[i] = -1;
    int s = 0;
    for (int i = 0; i < k; i++)
        for (int j = i; j < k; j++, s++) {
            L[i * d + j] = s;
            L[j * d + i] = s;
        }
    for (int i = 0; i < k; i++)
        for (int m = 0; m < d - k; m++, s++) {
            L[i * d + k + m] = s;
            L[(k + m) * d + i] = s;
        }
    return OR_OK;
}

/* G (n*alpha x B): G[alpha i + j][L[l][j]] = Psi[i][l] (Sec. 3.1 applied to
 * the MBR message matrix; zero entries of M contribute nothing). */
int or_mbr_generator(int n, int k, int d, uint8_t *G)
{
    int a, B;
    if (or_mbr_params(n, k, d, &a, &B))
        return OR_EINVAL;
    uint8_t *psi = (uint8_t *)malloc((size_t)n * d);
    int *L = (int *)malloc(sizeof(int) * d * d);
    int rc = or_mbr_psi(n, k, d, psi);
    if (rc == OR_OK) {
        or_mbr_index_matrix(k, d, L);
        memset(G, 0, (size_t)n * a * B);
        for (int i = 0; i < n; i++)
            for (int j = 0; j < a; j++)
                for (int l = 0; l < d; l++)
                    if (L[l * d + j] >= 0)
                        G[(size_t)(a * i + j) * B + L[l * d + j]] = psi[i * d + l];
    }
    free(psi);
    free(L);
    return rc;
}

/* All n*alpha coded blocks (node-major). */
int or_mbr_encode(int n, int k, int d, const uint8_t *data, uint8_t *out, size_t nbytes)
{
    int a, B;
    if (or_mbr_params(n, k, d, &a, &B))
        return OR_EINVAL;
    uint8_t *G = (uint8_t *)malloc((size_t)n * a * B);
    int rc = or_mbr_generator(n, k, d, G);
    if (rc == OR_OK)
        or_region_apply(n * a, B, G, data, nbytes, out, nbytes, nbytes);
    free(G);
    return rc;
}

/* Repair of node f: helper h sends psi_h^t M psi_f, i.e. its alpha blocks
 * projected on psi_f. */
int or_mbr_helper_coefficients(int n, int k, int d, int f, uint8_t *coef)
{
    int a, B;
    if (or_mbr_params(n, k, d, &a, &B) || f < 0 || f >= n)
        return OR_EINVAL;
    uint8_t *psi = (uint8_t *)malloc((size_t)n * d);
    int rc = or_mbr_psi(n, k, d, psi);
    if (rc == OR_OK)
        memcpy(coef, psi + (size_t)f * d, (size_t)d);
    free(psi);
    return rc;
}

/* The received vector is p = Psi_H M psi_f; Psi_H is invertible, so
 * M psi_f = Psi_H^-1 p, and by symmetry of M the lost node psi_f^t M is its
 * transpose: D = Psi_H^-1 (d x d). */
int or_mbr_newcomer_matrix(int n, int k, int d, int f, const int *helpers, uint8_t *D)
{
    int a, B;
    if (or_mbr_params(n, k, d, &a, &B) || f < 0 || f >= n)
        return OR_EINVAL;
    for (int i = 0; i < d; i++) {
        if (helpers[i] < 0 || helpers[i] >= n || helpers[i] == f)
            return OR_EINVAL;
        for (int j = 0; j < i; j++)
            if (helpers[j] == helpers[i])
                return OR_EINVAL;
    }
    uint8_t *psi = (uint8_t *)malloc((size_t)n * d);
    uint8_t *PH = (uint8_t *)malloc((size_t)d * d);
    int rc = or_mbr_psi(n, k, d, psi);
    if (rc == OR_OK) {
        for (int i = 0; i < d; i++)
            memcpy(PH + (size_t)i * d, psi + (size_t)helpers[i] * d, (size_t)d);
        rc = or_invert(d, PH, D);
    }
    free(psi);
    free(PH);
    return rc;
}

/* Reconstruction from k nodes (Sec. 2, X = G~^-1 Y~ with G~ made square):
 * the k*alpha rows of G of the listed nodes have rank B; the first B of them
 * (node-major) that are independent of the rows before them form G~, and
 * R (B x k*alpha) applies G~^-1 to those rows and ignores the others. */
int or_mbr_decode_matrix(int n, int k, int d, const int *nodes, uint8_t *R)
{
    int a, B;
    if (or_mbr_params(n, k, d, &a, &B))
        return OR_EINVAL;
    for (int i = 0; i < k; i++) {
        if (nodes[i] < 0 || nodes[i] >= n)
            return OR_EINVAL;
        for (int j = 0; j < i; j++)
            if (nodes[j] == nodes[i])
                return OR_EINVAL;
    }
    int KA = k * a, N = n * a;
    uint8_t *G = (uint8_t *)malloc((size_t)N * B);
    uint8_t *E = (uint8_t *)malloc((size_t)B * B);   /* echelon copy of picked rows */
    uint8_t *Gt = (uint8_t *)malloc((size_t)B * B);  /* picked rows, unreduced */
    uint8_t *Gti = (uint8_t *)malloc((size_t)B * B);
    uint8_t *v = (uint8_t *)malloc((size_t)B);
    int *pick = (int *)malloc(sizeof(int) * B);
    int *pivcol = (int *)malloc(sizeof(int) * B);
    int rc = or_mbr_generator(n, k, d, G), got = 0;
    for (int r = 0; r < KA && got < B && rc == OR_OK; r++) {
        const uint8_t *row = G + (size_t)(a * nodes[r / a] + r % a) * B;
        memcpy(v, row, (size_t)B);
        /* reduce v by the echelon rows found so far */
        for (int e = 0; e < got; e++) {
            uint8_t f = v[pivcol[e]];
            if (f)
                for (int c = 0; c < B; c++)
                    v[c] = or_add(v[c], or_gf_mul(f, E[(size_t)e * B + c]));
        }
        int pc = -1;
        for (int c = 0; c < B && pc < 0; c++)
            if (v[c])
                pc = c;
        if (pc < 0)
            continue; /* dependent on the rows already picked */
        uint8_t inv = or_gf_inv(v[pc]);
        for (int c = 0; c < B; c++)
            v[c] = or_gf_mul(v[c], inv);
        /* keep the echelon rows reduced at the new pivot column */
        for (int e = 0; e < got; e++) {
            uint8_t f = E[(size_t)e * B + pc];
            if (f)
                for (int c = 0; c < B; c++)
                    E[(size_t)e * B + c] = or_add(E[(size_t)e * B + c], or_gf_mul(f, v[c]));
        }
        memcpy(E + (size_t)got * B, v, (size_t)B);
        memcpy(Gt + (size_t)got * B, row, (size_t)B);
        pivcol[got] = pc;
        pick[got] = r;
        got++;
    }
    if (rc == OR_OK && got < B)
        rc = OR_ESINGULAR;
    if (rc == OR_OK)
        rc = or_invert(B, Gt, Gti);
    if (rc == OR_OK) {
        memset(R, 0, (size_t)B * KA);
        for (int x = 0; x < B; x++)
            for (int t = 0; t < B; t++)
                R[(size_t)x * KA + pick[t]] = Gti[(size_t)x * B + t];
    }
    free(G);
    free(E);
    free(Gt);
    free(Gti);
    free(v);
    free(pick);
    free(pivcol);
    return rc;
}

int or_mbr_decode(int n, int k, int d, const int *nodes, const uint8_t *node_blocks,
                  uint8_t *data, size_t nbytes)
{
    int a, B;
    if (or_mbr_params(n, k, d, &a, &B))
        return OR_EINVAL;
    uint8_t *R = (uint8_t *)malloc((size_t)B * k * a);
    int rc = or_mbr_decode_matrix(n, k, d, nodes, R);
    if (rc == OR_OK)
        or_region_apply(B, k * a, R, node_blocks, nbytes, data, nbytes, nbytes);
    free(R);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Reed-Solomon baseline (Sec. 4: the paper compares every PM code against   */
/* Vandermonde-based Reed-Solomon codes).  Restated from the definitions:    */
/* node i stores the evaluation at x_i = g^i of the polynomial whose k       */
/* coefficients are the message Z, i.e. Y = V Z with V[i][j] = g^(i j)       */
/* (n <= 255 distinct points: any k rows of V are invertible).  The          */
/* systematic form is Sec. 3.2's G' = V V~^-1 with V~ the first k rows.      */
/* One block per node (alpha = 1); repair of node f reads any k nodes.       */
/* ------------------------------------------------------------------------ */

int or_rs_generator(int n, int k, int systematic, uint8_t *G)
{
    if (k < 1 || n <= k || n > 255)
        return OR_EINVAL;
    uint8_t *V = (uint8_t *)malloc((size_t)n * k);
    uint8_t *Vinv = (uint8_t *)malloc((size_t)k * k);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < k; j++)
            V[i * k + j] = or_gf_pow_g(i * j);
    int rc = OR_OK;
    if (!systematic) {
        memcpy(G, V, (size_t)n * k);
    } else {
        rc = or_invert(k, V, Vinv);
        if (rc == OR_OK)
            or_mat_mul(n, k, k, V, Vinv, G);
    }
    free(V);
    free(Vinv);
    return rc;
}

int or_rs_encode(int n, int k, int systematic, const uint8_t *data, uint8_t *out, size_t nbytes)
{
    uint8_t *G = (uint8_t *)malloc((size_t)n * k);
    int rc = or_rs_generator(n, k, systematic, G);
    if (rc == OR_OK)
        or_region_apply(n, k, G, data, nbytes, out, nbytes, nbytes);
    free(G);
    return rc;
}

/* X = G_S^-1 Y_S from the blocks of any k distinct nodes. */
int or_rs_decode(int n, int k, int systematic, const int *nodes, const uint8_t *node_blocks,
                 uint8_t *data, size_t nbytes)
{
    if (k < 1 || n <= k || n > 255)
        return OR_EINVAL;
    for (int i = 0; i < k; i++) {
        if (nodes[i] < 0 || nodes[i] >= n)
            return OR_EINVAL;
        for (int j = 0; j < i; j++)
            if (nodes[j] == nodes[i])
                return OR_EINVAL;
    }
    uint8_t *G = (uint8_t *)malloc((size_t)n * k);
    uint8_t *GS = (uint8_t *)malloc((size_t)k * k);
    uint8_t *R = (uint8_t *)malloc((size_t)k * k);
    int rc = or_rs_generator(n, k, systematic, G);
    if (rc == OR_OK) {
        for (int i = 0; i < k; i++)
            memcpy(GS + (size_t)i * k, G + (size_t)nodes[i] * k, (size_t)k);
        rc = or_invert(k, GS, R);
    }
    if (rc == OR_OK)
        or_region_apply(k, k, R, node_blocks, nbytes, data, nbytes, nbytes);
    free(G);
    free(GS);
    free(R);
    return rc;
}

/* Repair of node f from k helpers: decode, then re-encode row f. */
int or_rs_repair(int n, int k, int systematic, int f, const int *helpers,
                 const uint8_t *helper_blocks, uint8_t *out, size_t nbytes)
{
    if (f < 0 || f >= n)
        return OR_EINVAL;
    for (int i = 0; i < k; i++)
        if (helpers[i] == f)
            return OR_EINVAL;
    uint8_t *X = (uint8_t *)malloc((size_t)k * (nbytes ? nbytes : 1));
    uint8_t *G = (uint8_t *)malloc((size_t)n * k);
    int rc = or_rs_decode(n, k, systematic, helpers, helper_blocks, X, nbytes);
    if (rc == OR_OK)
        rc = or_rs_generator(n, k, systematic, G);
    if (rc == OR_OK)
        or_region_apply(1, k, G + (size_t)f * k, X, nbytes, out, nbytes, nbytes);
    free(X);
    free(G);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* GF(2^16) variant (Sec. 3.3: the validity of the sparse construction is    */
/* also checked in GF(2^16), for k up to 64).  Reading: GF(2^16) is built as */
/* the quadratic extension GF(2^8)[y]/(y^2 + y + w), w the smallest element  */
/* of GF(2^8) of absolute trace 1 (so the polynomial has no root); an        */
/* element a + b y is the 16-bit value a | b << 8, and g is the smallest      */
/* value of multiplicative order 65535.  A block of B bytes holds B/2        */
/* symbols in two byte planes: the low bytes a at [0, B/2), the high bytes b */
/* at [B/2, B).  Constructions and operations are those above with g and the */
/* arithmetic of this field.                                                 */
/* ------------------------------------------------------------------------ */

static uint8_t or16_w;
static uint16_t or16_g;
static uint16_t or16_exp[2 * 65535];
static int or16_log[65536];
static int or16_ready;

static uint8_t or_trace(uint8_t a)
{
    uint8_t t = a, s = a;
    for (int i = 1; i < 8; i++) {
        t = or_gf_mul(t, t);
        s ^= t;
    }
    return s;
}

/* (a0 + a1 y)(b0 + b1 y) with y^2 = y + w */
static uint16_t or16_mul_direct(uint16_t x, uint16_t z)
{
    uint8_t a0 = (uint8_t)x, a1 = (uint8_t)(x >> 8), b0 = (uint8_t)z, b1 = (uint8_t)(z >> 8);
    uint8_t hh = or_gf_mul(a1, b1);
    uint8_t lo = or_add(or_gf_mul(a0, b0), or_gf_mul(or16_w, hh));
    uint8_t hi = or_add(or_add(or_gf_mul(a1, b0), or_gf_mul(a0, b1)), hh);
    return (uint16_t)(lo | (hi << 8));
}

static void or16_init(void)
{
    if (or16_ready)
        return;
    or_init();
    or16_w = 0;
    for (int a = 1; a < 256 && !or16_w; a++)
        if (or_trace((uint8_t)a) == 1)
            or16_w = (uint8_t)a;
    for (int v = 2; v < 65536; v++) {
        uint16_t p = 1;
        int ord = 0;
        for (int i = 1; i <= 65535; i++) {
            p = or16_mul_direct(p, (uint16_t)v);
            if (p == 1) {
                ord = i;
                break;
            }
        }
        if (ord == 65535) {
            or16_g = (uint16_t)v;
            break;
        }
    }
    uint16_t p = 1;
    for (int i = 0; i < 65535; i++) {
        or16_exp[i] = or16_exp[i + 65535] = p;
        or16_log[p] = i;
        p = or16_mul_direct(p, or16_g);
    }
    or16_log[0] = -1;
    or16_ready = 1;
}

uint8_t or16_omega(void) { or16_init(); return or16_w; }
uint16_t or16_primitive(void) { or16_init(); return or16_g; }

uint16_t or16_gf_mul(uint16_t a, uint16_t b)
{
    or16_init();
    if (!a || !b)
        return 0;
    return or16_exp[or16_log[a] + or16_log[b]];
}

uint16_t or16_gf_inv(uint16_t a)
{
    or16_init();
    return a ? or16_exp[(65535 - or16_log[a]) % 65535] : 0;
}

uint16_t or16_gf_pow_g(int e)
{
    or16_init();
    return or16_exp[e % 65535];
}

static int or16_invert(int m, const uint16_t *A, uint16_t *Ainv)
{
    uint16_t *W = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)m * 2 * m);
    for (int i = 0; i < m; i++)
        for (int j = 0; j < 2 * m; j++)
            W[(size_t)i * 2 * m + j] = j < m ? A[(size_t)i * m + j] : (uint16_t)(j - m == i);
    int rc = OR_OK;
    for (int c = 0; c < m && rc == OR_OK; c++) {
        int p = c;
        while (p < m && W[(size_t)p * 2 * m + c] == 0)
            p++;
        if (p == m) {
            rc = OR_ESINGULAR;
            break;
        }
        for (int j = 0; j < 2 * m; j++) {
            uint16_t t = W[(size_t)p * 2 * m + j];
            W[(size_t)p * 2 * m + j] = W[(size_t)c * 2 * m + j];
            W[(size_t)c * 2 * m + j] = t;
        }
        uint16_t inv = or16_gf_inv(W[(size_t)c * 2 * m + c]);
        for (int j = 0; j < 2 * m; j++)
            W[(size_t)c * 2 * m + j] = or16_gf_mul(W[(size_t)c * 2 * m + j], inv);
        for (int r = 0; r < m; r++) {
            uint16_t f = W[(size_t)r * 2 * m + c];
            if (r == c || !f)
                continue;
            for (int j = 0; j < 2 * m; j++)
                W[(size_t)r * 2 * m + j] ^= or16_gf_mul(f, W[(size_t)c * 2 * m + j]);
        }
    }
    if (rc == OR_OK)
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++)
                Ainv[(size_t)i * m + j] = W[(size_t)i * 2 * m + m + j];
    free(W);
    return rc;
}

/* Phi (n x alpha) and lambda (n) over GF(2^16), the same formulas as
 * or_phi_lambda with this field's g. */
int or16_phi_lambda(int n, int k, int construction, uint16_t *phi, uint16_t *lambda)
{
    int d, a;
    if (or_params(n, k, &d, &a) || n > 60000)
        return OR_EINVAL;
    or16_init();
    if (construction == OR_VANILLA) {
        for (int i = 0; i < n; i++) {
            for (int j = 0; j < a; j++)
                phi[i * a + j] = or16_gf_pow_g(i * j);
            lambda[i] = or16_gf_pow_g(i * a);
        }
    } else {
        for (int i = 1; i <= n; i++) {
            uint16_t x = or16_gf_pow_g(i + a);
            for (int j = 1; j <= a; j++)
                phi[(i - 1) * a + (j - 1)] =
                    i <= a ? (uint16_t)(i == j) : or16_gf_inv((uint16_t)(x ^ or16_gf_pow_g(j - 1)));
            lambda[i - 1] = or16_gf_mul((uint16_t)(x ^ 1), or16_gf_inv((uint16_t)(x ^ or16_gf_pow_g(a))));
        }
    }
    return OR_OK;
}

int or16_psi(int n, int k, int construction, uint16_t *psi)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    uint16_t *phi = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n * a);
    uint16_t *lam = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n);
    int rc = or16_phi_lambda(n, k, construction, phi, lam);
    if (rc == OR_OK)
        for (int i = 0; i < n; i++)
            for (int j = 0; j < a; j++) {
                psi[i * d + j] = phi[i * a + j];
                psi[i * d + a + j] = or16_gf_mul(lam[i], phi[i * a + j]);
            }
    free(phi);
    free(lam);
    return rc;
}

/* G (non-systematic) or G' = G G~^-1 (systematic) over GF(2^16). */
int or16_code_generator(int n, int k, int construction, int systematic, uint16_t *Gout)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    int K = k * a, N = n * a;
    uint16_t *psi = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n * d);
    int *L = (int *)malloc(sizeof(int) * d * a);
    uint16_t *G = (uint16_t *)calloc((size_t)N * K, sizeof(uint16_t));
    int rc = or16_psi(n, k, construction, psi);
    if (rc == OR_OK) {
        or_index_matrix(k, L);
        for (int i = 0; i < n; i++)
            for (int j = 0; j < a; j++)
                for (int l = 0; l < d; l++)
                    G[(size_t)(a * i + j) * K + L[l * a + j]] = psi[i * d + l];
    }
    if (rc == OR_OK && !systematic)
        memcpy(Gout, G, sizeof(uint16_t) * (size_t)N * K);
    if (rc == OR_OK && systematic) {
        uint16_t *Ti = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)K * K);
        rc = or16_invert(K, G, Ti);
        if (rc == OR_OK)
            for (int r = 0; r < N; r++)
                for (int c = 0; c < K; c++) {
                    uint16_t s = 0;
                    for (int q = 0; q < K; q++)
                        s ^= or16_gf_mul(G[(size_t)r * K + q], Ti[(size_t)q * K + c]);
                    Gout[(size_t)r * K + c] = s;
                }
        free(Ti);
    }
    free(psi);
    free(L);
    free(G);
    return rc;
}

/* Y = M X over planar GF(2^16) blocks of nbytes (even) bytes. */
void or16_region_apply(int rows, int cols, const uint16_t *M, const uint8_t *in, uint8_t *out,
                       size_t nbytes)
{
    size_t h = nbytes / 2;
    for (int r = 0; r < rows; r++) {
        uint8_t *y = out + (size_t)r * nbytes;
        for (size_t t = 0; t < h; t++) {
            uint16_t s = 0;
            for (int c = 0; c < cols; c++) {
                uint16_t m = M[(size_t)r * cols + c];
                if (!m)
                    continue;
                const uint8_t *x = in + (size_t)c * nbytes;
                s ^= or16_gf_mul(m, (uint16_t)(x[t] | (x[h + t] << 8)));
            }
            y[t] = (uint8_t)s;
            y[h + t] = (uint8_t)(s >> 8);
        }
    }
}

int or16_encode(int n, int k, int construction, int systematic, const uint8_t *data, uint8_t *out,
                size_t nbytes)
{
    int d, a;
    if (or_params(n, k, &d, &a) || nbytes % 2)
        return OR_EINVAL;
    int K = k * a, N = n * a;
    uint16_t *G = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)N * K);
    int rc = or16_code_generator(n, k, construction, systematic, G);
    if (rc == OR_OK)
        or16_region_apply(N, K, G, data, out, nbytes);
    free(G);
    return rc;
}

/* Repair (the PM repair of the section above, over GF(2^16)): helper h
 * sends its alpha blocks projected on phi_f; D = [I | lambda_f I] Psi_H^-1. */
int or16_newcomer_matrix(int n, int k, int construction, int f, const int *helpers, uint16_t *D)
{
    int d, a;
    if (or_params(n, k, &d, &a) || f < 0 || f >= n)
        return OR_EINVAL;
    for (int i = 0; i < d; i++) {
        if (helpers[i] < 0 || helpers[i] >= n || helpers[i] == f)
            return OR_EINVAL;
        for (int j = 0; j < i; j++)
            if (helpers[j] == helpers[i])
                return OR_EINVAL;
    }
    uint16_t *psi = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n * d);
    uint16_t *PH = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)d * d);
    uint16_t *PHi = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)d * d);
    uint16_t *phi = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n * a);
    uint16_t *lam = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n);
    int rc = or16_psi(n, k, construction, psi);
    if (rc == OR_OK)
        rc = or16_phi_lambda(n, k, construction, phi, lam);
    if (rc == OR_OK) {
        for (int i = 0; i < d; i++)
            memcpy(PH + (size_t)i * d, psi + (size_t)helpers[i] * d, sizeof(uint16_t) * d);
        rc = or16_invert(d, PH, PHi);
    }
    if (rc == OR_OK)
        for (int j = 0; j < a; j++)
            for (int c = 0; c < d; c++)
                D[j * d + c] = PHi[j * d + c] ^ or16_gf_mul(lam[f], PHi[(a + j) * d + c]);
    free(psi);
    free(PH);
    free(PHi);
    free(phi);
    free(lam);
    return rc;
}

int or16_helper_coefficients(int n, int k, int construction, int f, uint16_t *coef)
{
    int d, a;
    if (or_params(n, k, &d, &a) || f < 0 || f >= n)
        return OR_EINVAL;
    uint16_t *phi = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n * a);
    uint16_t *lam = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n);
    int rc = or16_phi_lambda(n, k, construction, phi, lam);
    if (rc == OR_OK)
        memcpy(coef, phi + (size_t)f * a, sizeof(uint16_t) * a);
    free(phi);
    free(lam);
    return rc;
}

/* Reconstruction: the inverse of the listed nodes' rows of the code's
 * generator. */
int or16_decode_matrix(int n, int k, int construction, int systematic, const int *nodes,
                       uint16_t *Rinv)
{
    int d, a;
    if (or_params(n, k, &d, &a))
        return OR_EINVAL;
    for (int i = 0; i < k; i++) {
        if (nodes[i] < 0 || nodes[i] >= n)
            return OR_EINVAL;
        for (int j = 0; j < i; j++)
            if (nodes[j] == nodes[i])
                return OR_EINVAL;
    }
    int K = k * a, N = n * a;
    uint16_t *G = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)N * K);
    uint16_t *GR = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)K * K);
    int rc = or16_code_generator(n, k, construction, systematic, G);
    if (rc == OR_OK) {
        for (int i = 0; i < k; i++)
            for (int j = 0; j < a; j++)
                memcpy(GR + (size_t)(a * i + j) * K, G + (size_t)(a * nodes[i] + j) * K,
                       sizeof(uint16_t) * K);
        rc = or16_invert(K, GR, Rinv);
    }
    free(G);
    free(GR);
    return rc;
}
