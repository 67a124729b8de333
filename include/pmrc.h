/*
 * pmrc.h -- C ABI of libpmrc: product-matrix regenerating codes over GF(2^8)
 * on one NVIDIA GB300 GPU (sm_103a): minimum-storage (PM-MSR) codes and,
 * with construction PMRC_MBR, minimum-bandwidth (PM-MBR) codes.
 *
 * Follows N. Le Scouarnec, "Fast Product-Matrix Regenerating Codes":
 *   Sec. 2    the code as a linear map: k*alpha data blocks X, n*alpha coded
 *             blocks Y = G X; decoding X = G~^-1 Y~ from the rows that remain;
 *             MSR point alpha = Delta = d-k+1; repair downloads one block from
 *             each of d helpers.
 *   Sec. 3.1  linearization: G[alpha i + j][L[l][j]] = Psi[i][l].
 *   Sec. 3.2  systematic form G' = G G~^-1 = [I; G''].
 *   Sec. 3.3  Psi = [Phi  Lambda*Phi]: the vanilla (Vandermonde) and the
 *             sparse (identity + Cauchy) constructions; helpers of a failed
 *             node among the alpha first read one block, alpha otherwise.
 *
 * PM-MSR parameters: d = 2k-2, alpha = k-1, 2k-1 <= n <= 254 (PM-MBR: see
 * pmrc_create; there "k*alpha data blocks" below reads "K = k Delta data
 * blocks", and node blocks are still alpha per node).  Field GF(2^8) with
 * modulus x^8+x^4+x^3+x^2+1 (0x11D) and generator g = 2.  Node i stores the
 * alpha blocks Y[alpha*i .. alpha*i + alpha-1] ("node-major").  The message
 * matrix M = [S1; S2] numbers the upper triangle of S1 row by row, then that
 * of S2 (only non-systematic codewords depend on this order).
 *
 * Conventions shared by every call:
 *   - Region pointers (data, out, blocks, ...) are DEVICE pointers owned by
 *     the caller, all blocks of one call have the same size block_bytes
 *     (any value >= 0; 0 does nothing).  16-byte aligned pointers take the
 *     vector path, any other alignment a slower byte path; results are the
 *     same.  Arrays of pointers (const uint8_t *const *) are HOST arrays.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream) on the current CUDA device, return a status, never
 *     throw and never exit.  Input blocks must not overlap output blocks.
 *   - A call may build and upload a small coefficient plan on first use of
 *     an (operation, failure pattern, device) combination (a synchronous
 *     cudaMalloc + cudaMemcpy); make that first call outside CUDA stream
 *     capture.  Later calls with the same pattern allocate nothing.
 *   - An operation over more than 1024 blocks (inputs + outputs, e.g. the
 *     encode of k >= 24 at n = 2k) or with rows over more than 512 inputs
 *     runs as several kernel launches on the stream, later launches XORing
 *     into outputs the first one wrote; the batched and served calls take
 *     only operations of one launch (PMRC_EUNSUPPORTED otherwise).
 *   - One code handle may be used from several threads at once.
 *   - On failure the call returns a negative PMRC_E* status, writes nothing
 *     and pmrc_last_error() describes the problem (thread-local).
 */
#ifndef PMRC_H
#define PMRC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pmrc_code pmrc_code;
typedef struct CUstream_st *pmrc_stream_t; /* same type as cudaStream_t */

enum {
  PMRC_OK = 0,
  PMRC_EINVAL = -1,      /* bad argument (range, NULL, repeated node id)      */
  PMRC_ESINGULAR = -2,   /* helper set / node set does not determine the data */
  PMRC_EUNSUPPORTED = -3,/* parameters outside what the construction supports */
  PMRC_ENOMEM = -4,      /* host or device allocation failed                  */
  PMRC_ECUDA = -5,       /* a CUDA call failed (message in pmrc_last_error)   */
  PMRC_ETIMEOUT = -6,    /* a bounded device wait gave up                     */
  PMRC_EBUSY = -7        /* resource in use (batch/server state)              */
};

enum { PMRC_VANILLA = 0, PMRC_SPARSE = 1 };            /* Sec. 3.3 (PM-MSR)   */
enum { PMRC_MBR = 2 };                                 /* Sec. 2, 3.2, 4.2    */
enum { PMRC_RS = 3 };                                  /* Sec. 4 baseline     */
enum { PMRC_NONSYSTEMATIC = 0, PMRC_SYSTEMATIC = 1 };  /* Sec. 3.1 / Sec. 3.2 */

/* Builds the code (Phi, Lambda, Psi, L, G and, for the systematic form,
 * G' = G G~^-1) on the host and its encode plan.  Host only: works without a
 * GPU.  *out receives a handle owned by the caller (free with pmrc_destroy).
 *
 * PMRC_VANILLA / PMRC_SPARSE: PM-MSR codes (Sec. 3.3), alpha = k-1; d must
 * equal 2k-2 (PMRC_EINVAL otherwise).  Returns PMRC_EUNSUPPORTED when the
 * construction is not an MSR code in GF(2^8) at this size (e.g. vanilla
 * with repeated lambda, k=16 n=32).  Data: K = k alpha blocks.
 *
 * PMRC_MBR: the PM-MBR code (Sec. 2: alpha = d, Delta = (2d-k+1)/2), any
 * 1 <= k <= d <= n-1 with d + n - k <= 255.  Message matrix M = [S T; T^t 0]
 * (S symmetric k x k, T k x (d-k); upper triangle of S then T, row by row,
 * are the data blocks 0..K-1, K = k Delta).  Psi = [I_k 0; C] (the
 * systematic Psi = [I; Psi''] of Sec. 3.2) with C_ij = (g^(d+i) + g^j)^-1,
 * 0-based i < n-k, j < d; node i < k stores row i of M, i.e. data blocks
 * verbatim.  The form only selects what pmrc_encode writes (every node, or
 * the n-k parity nodes).  Repair: helper h sends its d blocks projected on
 * psi_f (pmrc_helper_coefficients), the newcomer applies Psi_H^-1 (any d
 * helpers work).  Decode reads k nodes (k d blocks) and writes the K data
 * blocks.  The specific calls below are PM-MSR only.
 *
 * PMRC_RS: the Reed-Solomon baseline the paper compares against (Sec. 4):
 * node i stores the message polynomial evaluated at g^i (Y = V Z,
 * V[i][j] = g^(ij)), systematic form V V~^-1 (Sec. 3.2); 1 <= k < n <= 255,
 * d must equal k, alpha = 1.  Repair of node f reads one block from each of
 * k helpers (helper coefficient 1) and applies G'[f] G'_H^-1. */
int pmrc_create(int n, int k, int d, int construction, int form, pmrc_code **out);

/* pmrc_create over GF(2^8) (field_bits = 8, the same as pmrc_create) or
 * GF(2^16) (field_bits = 16; PMRC_VANILLA / PMRC_SPARSE only).  GF(2^16) is
 * the quadratic extension GF(2^8)[y]/(y^2 + y + w), w the smallest element
 * of GF(2^8) of absolute trace 1; a + b y is the value a | b << 8 and g the
 * smallest value of order 65535 (Sec. 3.3 checks the sparse construction in
 * GF(2^16) for k up to 64; the vanilla code at k=16, n=32 is valid there).
 * A block of B bytes (B even) holds B/2 symbols as two byte planes: the low
 * bytes at [0, B/2), the high bytes at [B/2, B).  pmrc_encode,
 * pmrc_repair_helper(s), pmrc_repair_newcomer and pmrc_decode take the same
 * arguments as for GF(2^8) codes (B must be even); the other calls return
 * PMRC_EUNSUPPORTED for GF(2^16) codes.  PMRC_EINVAL for another
 * field_bits. */
int pmrc_create_field(int n, int k, int d, int construction, int form, int field_bits,
                      pmrc_code **out);

/* Frees the handle and its device plans.  The caller makes sure no call on
 * it is still running on the GPU.  NULL is ignored. */
void pmrc_destroy(pmrc_code *code);

/* Encode (Sec. 3.1 / 3.2).  data: K device pointers (X; K = k*alpha for
 * PM-MSR, pmrc_code_blocks).  out:
 * non-systematic -> n*alpha pointers, all coded blocks Y = G X;
 * systematic     -> (n-k)*alpha pointers, the parity nodes' blocks (G'' X
 * for PM-MSR; the first k nodes hold the data itself).  NULL entries of out
 * are skipped. */
int pmrc_encode(const pmrc_code *code, const uint8_t *const *data, uint8_t *const *out,
                size_t block_bytes, pmrc_stream_t stream);

/* Helper side of repairing node `failed` (Sec. 3.3): node `helper` sends
 * p = sum_j phi_failed[j] * Y[alpha*helper + j].  helper_blocks: the alpha
 * blocks the helper stores; entries whose coefficient is zero are never
 * read and may be NULL (sparse code: a failed node among the alpha first
 * needs one block).  out: one block. */
int pmrc_repair_helper(const pmrc_code *code, int failed, int helper,
                       const uint8_t *const *helper_blocks, uint8_t *out, size_t block_bytes,
                       pmrc_stream_t stream);

/* The same projection for nhelpers helpers in one launch.  helper_blocks:
 * nhelpers*alpha pointers (helper h's blocks at [h*alpha, h*alpha+alpha)),
 * out: nhelpers pointers.  helpers[] only serves the range checks. */
int pmrc_repair_helpers(const pmrc_code *code, int failed, int nhelpers, const int *helpers,
                        const uint8_t *const *helper_blocks, uint8_t *const *out,
                        size_t block_bytes, pmrc_stream_t stream);

/* Newcomer side of the repair of node `failed` (Sec. 2: exact repair at the
 * MSR point from d = 2k-2 helpers, each sending beta = 1 block; Sec. 3.3:
 * the product-matrix repair the sparse code keeps).  From the d projected
 * blocks received from `helpers` (d distinct node ids != failed, host
 * array, same order as received), rebuild the alpha blocks of node `failed`
 * with D = [I | lambda_f I] Psi_H^-1: Psi_H M phi_f = p gives M phi_f, whose
 * halves S1 phi_f and S2 phi_f give, by the symmetry of S1 and S2, the
 * stored content phi_f^t S1 + lambda_f phi_f^t S2.  received: d device
 * pointers; out: alpha device pointers (never NULL).  PMRC_ESINGULAR when
 * the helpers' rows of Psi are singular (possible at n >= 2k for the sparse
 * code). */
int pmrc_repair_newcomer(const pmrc_code *code, int failed, const int *helpers,
                         const uint8_t *const *received, uint8_t *const *out,
                         size_t block_bytes, pmrc_stream_t stream);

/* Whole repair of node `failed` on one GPU: the d helper projections of
 * pmrc_repair_helper and the newcomer apply of pmrc_repair_newcomer in one
 * launch (same result as the two-step protocol).  The projections stay in
 * on-chip shared memory instead of going through device memory; when
 * phi_failed is a single 1 (sparse code, failed node among the alpha first,
 * Sec. 3.3) the newcomer reads the helpers' blocks directly.
 * helper_blocks: d*alpha pointers (helper i's alpha blocks at
 * [i*alpha, i*alpha + alpha)), entries with a zero helper coefficient may be
 * NULL.  out: alpha pointers.  Requires alpha <= 16.  For PMRC_RS (one
 * block per node, helper coefficient 1) the projections are the helper
 * blocks themselves and the call runs the newcomer row over them. */
int pmrc_repair(const pmrc_code *code, int failed, const int *helpers,
                const uint8_t *const *helper_blocks, uint8_t *const *out, size_t block_bytes,
                pmrc_stream_t stream);

/* Degraded read: bytes [offset, offset + length) of the alpha blocks of a
 * lost systematic node (node < k on a PMRC_SYSTEMATIC handle), rebuilt by
 * the repair above from d helpers instead of a reconstruction from k nodes
 * (the systematic nodes store data verbatim, Sec. 3.2: for PM-MSR node i
 * holds data blocks alpha*i .. alpha*i + alpha-1).  With the sparse code and
 * node < alpha each helper contributes one block (Sec. 3.3), so the read
 * touches d blocks where a reconstruction reads k*alpha.  helper_blocks:
 * d*alpha pointers to the helpers' whole blocks (as for pmrc_repair; the
 * call adds `offset`); out: alpha device pointers receiving `length` bytes
 * each.  PMRC_EINVAL for a non-systematic handle or node >= k; otherwise the
 * conditions and errors of pmrc_repair. */
int pmrc_read_degraded(const pmrc_code *code, int node, const int *helpers,
                       const uint8_t *const *helper_blocks, uint8_t *const *out, size_t offset,
                       size_t length, pmrc_stream_t stream);

/* pmrc_repair_noalloc: the same repair as pmrc_repair (same arguments, same
 * bytes out) for callers that cannot allocate GPU memory -- for example a
 * library running inside a process whose device memory is owned by another
 * allocator (a framework pool that reserves the whole device), or a
 * latency-critical path where an allocation could block, synchronize the
 * device or fail part-way through a repair.  The paper has no counterpart:
 * this is an interface choice of this library.
 *
 * It allocates nothing on the device (no cudaMalloc/cudaFree, no
 * stream-ordered or library allocator): pmrc_repair uploads its repair
 * tables once per (failed node, helpers, device) into device memory it
 * allocates, whereas this entry point copies them, on every call, into one
 * fixed 64 KiB array compiled into the library, which every GPU that loads
 * the library holds until the process exits.  A repair whose tables exceed
 * 64 KiB is rejected with PMRC_EUNSUPPORTED (no code with alpha <= 16 comes
 * close: k = 16 needs about 10 KiB).
 *
 * Every call looks up the array's device address on the calling thread's
 * current device (cudaGetSymbolAddress, a host-side query; the array's
 * host-side name is not a device address).  The first call on a device also
 * loads the library's device code there, so make that first call before any
 * stream capture.  Every call uses the same array and it keeps the last
 * call's contents, so calls that overlap on the GPU (other streams, other
 * host threads) race and corrupt each other's results: issue them one after
 * another on one stream.  For PMRC_RS codes (one block per node, helper
 * coefficient 1) the fused kernel applies the newcomer's 1 x k row to the
 * helper blocks read in place. */
int pmrc_repair_noalloc(const pmrc_code *code, int failed, const int *helpers,
                        const uint8_t *const *helper_blocks, uint8_t *const *out,
                        size_t block_bytes, pmrc_stream_t stream);

/* Reconstruction from any k nodes (Sec. 2: X = G~^-1 Y~).  nodes: k
 * distinct node ids (host array).  node_blocks: their k*alpha blocks,
 * node-major in the order of nodes.  data_out: k*alpha pointers for X; a
 * NULL entry is not produced, and an entry equal to the node block that
 * already holds that data block (systematic code) is left in place, so only
 * the missing blocks are computed (lazy decode, Sec. 3.1). */
int pmrc_decode(const pmrc_code *code, const int *nodes, const uint8_t *const *node_blocks,
                uint8_t *const *data_out, size_t block_bytes, pmrc_stream_t stream);

/* ---- "Specific" product-matrix algorithms (Sec. 4: "PM Spec." codes) ----
 *
 * The linearized calls above apply one matrix per operation (Sec. 3.1).  The
 * two calls below run the seminal PM paper's own algorithms instead, which
 * Sec. 3.2 and Sec. 4 compare against linearization:
 *
 *   data collector (pmrc_decode_specific): with DC the k listed nodes,
 *     A = Y_DC Phi_DC^t = P + Lambda_DC Q with P, Q symmetric; the pairs
 *     (A_ij, A_ji) give P_ij and Q_ij (i != j); alpha x alpha solves give
 *     phi_i^t S1 and phi_i^t S2 for alpha of the nodes, and one more solve
 *     gives S1 and S2, i.e. the message.  Systematic codes then re-encode
 *     the missing data nodes from the precoded message (Sec. 3.2).
 *   precode encode (pmrc_encode_precode): the systematic encode "by
 *     successively decoding and encoding" (Sec. 3.2): the data blocks are
 *     decoded as the contents of nodes 0..k-1 into the precoded message Z,
 *     and Z is encoded into the parity nodes.  Same result as pmrc_encode on
 *     a systematic handle (G'' X), computed the specific way.
 *
 * Each stage is one launch on `stream`; intermediate blocks live in a
 * caller-owned device workspace of at least pmrc_specific_workspace_bytes()
 * bytes (contents undefined afterwards; 256-byte alignment keeps every
 * stage on the vectorized path).  Calls that share a workspace must not
 * overlap on the GPU. */

/* Workspace bytes the specific calls need for blocks of block_bytes bytes:
 * (max(k(k-1), 2 alpha^2) + k(k-1) [+ k alpha if systematic]) blocks, each
 * rounded up to 256 bytes.  0 if code is NULL. */
size_t pmrc_specific_workspace_bytes(const pmrc_code *code, size_t block_bytes);

/* Reconstruction from k nodes by the data collector.  Arguments and the
 * data_out conventions (NULL entries skipped, aliased systematic blocks left
 * in place) are those of pmrc_decode; present systematic blocks that are
 * not aliased are copied.  PMRC_EINVAL for a missing or short workspace. */
int pmrc_decode_specific(const pmrc_code *code, const int *nodes,
                         const uint8_t *const *node_blocks, uint8_t *const *data_out,
                         size_t block_bytes, void *workspace, size_t workspace_bytes,
                         pmrc_stream_t stream);

/* Systematic encode by decoding then encoding.  data: k*alpha device
 * pointers; parity: (n-k)*alpha device pointers (none NULL).  The handle
 * must be systematic (PMRC_EINVAL otherwise). */
int pmrc_encode_precode(const pmrc_code *code, const uint8_t *const *data,
                        uint8_t *const *parity, size_t block_bytes, void *workspace,
                        size_t workspace_bytes, pmrc_stream_t stream);

/* Encode kernel of a handle.  A bitsliced kernel runs when the call's
 * pointers are 16-byte aligned with no NULL output: the one generated at
 * build time for this code, or one compiled at run time (NVRTC) for its
 * encode matrix on the first such encode and cached in the handle.  A
 * run-time schedule fits when inputs + outputs <= 512 blocks, in at most 64
 * blocks of 8 rows (rows of identical support, else consecutive rows) of at
 * most 64 inputs each -- e.g. the sparse systematic codes up to k = 16 at
 * n = 2k; its compilation takes seconds to minutes as the matrix grows (the
 * per-code initialization Sec. 4 reports apart from throughput).
 * PMRC_KERNEL_AUTO (default): the built-in kernel; a run-time one for blocks
 * of at least 256 KiB and encode matrices of at most 2048 non-zero
 * coefficients (k <= 10 sparse systematic at n = 2k); the nibble-table
 * kernel otherwise.  PMRC_KERNEL_GENERIC: always the nibble-table kernel.
 * PMRC_KERNEL_BITSLICED: a bitsliced kernel at any size and matrix that
 * fits; PMRC_EUNSUPPORTED here if the code has no built-in kernel and its
 * matrix does not fit a run-time one (or NVRTC is missing), and from
 * pmrc_encode if the compilation fails.  Results are identical; only speed
 * differs.  Do not change it while encodes on the handle are being
 * issued. */
enum { PMRC_KERNEL_AUTO = 0, PMRC_KERNEL_GENERIC = 1, PMRC_KERNEL_BITSLICED = 2 };
int pmrc_set_encode_kernel(pmrc_code *code, int which);

/* Reconstruction kernel of a handle (GF(2^8) codes).  PMRC_KERNEL_AUTO
 * (default): for blocks of at least 256 KiB, a bitsliced kernel generated
 * for the call's decode rows and compiled at run time (NVRTC, loaded on
 * demand) from the first reconstruction of each (node set, wanted rows) --
 * a few seconds in the background, part of the per-failure-pattern
 * initialization that Sec. 4 reports apart from throughput -- then cached
 * in the handle; the split-table kernel until then, otherwise, and whenever
 * the run-time kernel cannot be
 * built (NVRTC missing, blocks not 16-byte aligned, or more than 64 inputs
 * per 8-row block).  For a systematic MSR or Reed-Solomon code whose wanted
 * rows are all missing data rows, the reconstruction may instead run
 * factored, as two launches of run-time kernels: z = the received parity
 * blocks plus their present-data terms, then B^-1 z (B: the parity rows on
 * the missing columns), z held as bit planes in stream-ordered scratch of a
 * memory pool the library keeps per device.  The library picks the form per
 * (node set, wanted rows) from the kernels' instruction counts.
 * PMRC_KERNEL_GENERIC: always the split-table kernel.
 * PMRC_KERNEL_BITSLICED: the run-time kernel at any size, PMRC_EUNSUPPORTED
 * from pmrc_decode when it cannot be built.  Results are identical.  The
 * same choice applies to pmrc_repair_newcomer (its D, per failed node and
 * helper list), where AUTO takes the run-time kernel from 1 MiB blocks and
 * PMRC_KERNEL_BITSLICED falls back to the split-table kernel rather than
 * failing.
 *
 * The same policy governs the repair kernels compiled at run time: the
 * helper projections (pmrc_repair_helper(s), one kernel per failed node) and
 * the fused repair (pmrc_repair, one kernel per failed node and helper set,
 * alpha <= 8), which AUTO takes from 256 KiB blocks.
 *
 * Under PMRC_KERNEL_AUTO the run-time compilations (encode, reconstruction,
 * newcomer, repair) run on background threads: the call that needs one
 * starts it and runs the split-table kernel, as do later calls until it has
 * finished (pmrc_wait_kernels waits for it); the first call after that loads
 * it.  Under PMRC_KERNEL_BITSLICED the call compiles before it launches.
 *
 * Kernels compiled at run time are kept across handles and processes: each
 * compiled cubin is stored on disk under a hash of its source, and a later
 * compilation of the same schedule reads the file instead of running NVRTC.
 * The directory is the environment variable PMRC_KERNEL_CACHE when it is
 * set (empty, "0" or "off" turns the cache off), else $XDG_CACHE_HOME/pmrc,
 * else $HOME/.cache/pmrc (created, mode 0700), read at each compilation. */
int pmrc_set_decode_kernel(pmrc_code *code, int which);

/* Waits until the handle's background compilations have finished, at most
 * timeout_ms milliseconds (negative: no limit); PMRC_ETIMEOUT if some are
 * still running.  Host only. */
int pmrc_wait_kernels(const pmrc_code *code, int timeout_ms);

/* Number of the handle's run-time kernels compiled (*ready) and still
 * compiling (*pending).  Host only. */
int pmrc_runtime_kernels(const pmrc_code *code, int *ready, int *pending);

/* ---- batched execution ---------------------------------------------------
 * Many stripes (any mix of codes, block sizes and operations) run by one
 * persistent kernel replayed from a CUDA graph.  The same per-stripe results
 * as the single calls: encode = pmrc_encode, repair = pmrc_repair,
 * decode = pmrc_decode.  Pointers given to pmrc_batch_add_* are remembered
 * and must stay valid while the batch is launched; pmrc_batch_launch reads
 * and writes them again each time.  Add all stripes, build, then launch any
 * number of times.  A batch is not thread-safe; launches of one batch must
 * not overlap on the GPU (they share a work counter). */
typedef struct pmrc_batch pmrc_batch;

int pmrc_batch_create(pmrc_batch **out);
void pmrc_batch_destroy(pmrc_batch *batch); /* no launch may still be running */

/* Each returns the stripe index (>= 0) or a negative status. */
int pmrc_batch_add_encode(pmrc_batch *batch, const pmrc_code *code, const uint8_t *const *data,
                          uint8_t *const *out, size_t block_bytes);
int pmrc_batch_add_repair(pmrc_batch *batch, const pmrc_code *code, int failed,
                          const int *helpers, const uint8_t *const *helper_blocks,
                          uint8_t *const *out, size_t block_bytes);
int pmrc_batch_add_decode(pmrc_batch *batch, const pmrc_code *code, const int *nodes,
                          const uint8_t *const *node_blocks, uint8_t *const *data_out,
                          size_t block_bytes);

/* Uploads the work list (device allocations) and captures the graph on the
 * current device.  work_bytes: byte-column span of one work item (rounded to
 * 4 KiB tiles); ctas_per_sm: persistent CTAs per SM.  0 for either takes
 * the value pmrc_batch_tune found for a batch of the same shape in this
 * process, else 64 KiB and 2. */
int pmrc_batch_build(pmrc_batch *batch, int work_bytes, int ctas_per_sm);

/* One replay of the graph on `stream` (asynchronous). */
int pmrc_batch_launch(pmrc_batch *batch, pmrc_stream_t stream);

/* Autotuner: times the batch (synchronously, on `stream`) for each candidate
 * item size (16, 64, 256 KiB) and CTAs per SM (1, 2), rebuilds it with the
 * fastest and remembers the choice for batches of the same shape.
 * best_out[2] (optional) = {work_bytes, ctas_per_sm}. */
int pmrc_batch_tune(pmrc_batch *batch, pmrc_stream_t stream, int *best_out);

/* info_out[8] = {stripes, work items, CTAs, work_bytes, ctas_per_sm,
 * user bytes per launch, bitsliced encode launches, shared memory bytes per
 * CTA}.  Encodes of at least 4 MiB of data on codes with a built-in
 * bitsliced kernel (16-byte aligned blocks) run as their own launches of that
 * kernel in the batch's graph, after the persistent kernel (which takes
 * their ragged tails and every other stripe). */
int pmrc_batch_info(const pmrc_batch *batch, int64_t *info_out);

/* ---- serving -------------------------------------------------------------
 * A request loop with continuous batching: a scheduler thread admits
 * requests in arrival order while a slot is free and the device budget has
 * room for the request's inputs and outputs, copies their inputs in while
 * the previous iteration computes, runs every request whose inputs have
 * landed in one persistent launch (the batched kernel, plus the built-in
 * bitsliced kernel for encodes of at least 4 MiB of data), and copies
 * results back, recording submit-to-completion latency.  Copies run on four
 * streams per direction, each copy on the one with the fewest bytes queued;
 * the persistent kernel reads its work list from pinned host memory in
 * place.  Each request gives the same bytes as the corresponding single
 * call.  Requests use HOST buffers (make them pinned, cudaMallocHost /
 * cudaHostRegister, so the copies run asynchronously, and keep them alive
 * until the request is finished), or device blocks with PMRC_REQ_DEVICE.
 * The coefficient plan of a request is built (or found) and uploaded at
 * submission, on the caller's thread. */
typedef struct pmrc_server pmrc_server;

enum { PMRC_OP_ENCODE = 0, PMRC_OP_REPAIR = 1, PMRC_OP_DECODE = 2 };

/* OR'ed into pmrc_request.op: `in` and `out` are DEVICE blocks of the
 * server's device (the same layout as the host buffers below, 16-byte
 * aligned, B a multiple of 16), owned by the caller and alive until the
 * request is finished.  The request takes a slot but no arena space, its
 * blocks are neither copied in nor out, and the batched kernel reads and
 * writes them in place: stripe state kept resident in HBM. */
enum { PMRC_REQ_DEVICE = 0x100 };

typedef struct {
  int op;                 /* PMRC_OP_*                                          */
  const pmrc_code *code;  /* must outlive the request                           */
  size_t block_bytes;     /* B                                                  */
  const uint8_t *in;      /* host, contiguous blocks of B bytes:
                             ENCODE: k*alpha data blocks;
                             REPAIR: d*alpha blocks, helper i's alpha blocks at
                                     [i*alpha, i*alpha + alpha) (all alpha sent);
                             DECODE: k*alpha blocks of `nodes`, node-major      */
  uint8_t *out;           /* host: ENCODE: the pmrc_encode outputs ((n-k)*alpha
                             or n*alpha blocks); REPAIR: alpha blocks of node
                             `failed`; DECODE: k*alpha data blocks             */
  int failed;             /* REPAIR                                             */
  const int *helpers;     /* REPAIR: d node ids (copied at submit)              */
  const int *nodes;       /* DECODE: k node ids (copied at submit)              */
} pmrc_request;

/* Starts a server on the current device with a device arena of
 * budget_bytes (allocated once, the HBM budget of in-flight requests) and at
 * most max_slots requests admitted at a time. */
int pmrc_server_create(size_t budget_bytes, int max_slots, pmrc_server **out);

/* Finishes every submitted request, stops the scheduler and frees the
 * server.  NULL is ignored. */
void pmrc_server_destroy(pmrc_server *server);

/* Queues a request (validated now: PMRC_ENOMEM if it cannot fit the budget
 * even alone, PMRC_ESINGULAR for bad helper/node sets).  *id_out receives
 * its id. */
int pmrc_server_submit(pmrc_server *server, const pmrc_request *request, uint64_t *id_out);

/* 1 if the request finished (status and latency filled in; the record is
 * then dropped and the id becomes unknown), 0 if not yet. */
int pmrc_server_poll(pmrc_server *server, uint64_t id, int *status, double *latency_ms);

/* Waits up to timeout_ms (< 0: forever) for the request; PMRC_ETIMEOUT if it
 * is still running.  On success the record is dropped as in poll. */
int pmrc_server_wait(pmrc_server *server, uint64_t id, int timeout_ms, int *status,
                     double *latency_ms);

/* Withdraws a request that is still queued (PMRC_EBUSY once admitted). */
int pmrc_server_cancel(pmrc_server *server, uint64_t id);

/* stats_out[10] = {completed, failed, p50 latency ms, p99 ms, max ms, user
 * bytes completed, user GB/s from first submit to last completion, peak
 * device bytes in use, iterations launched, budget bytes}. */
int pmrc_server_stats(pmrc_server *server, double *stats_out);
int pmrc_server_reset_stats(pmrc_server *server);

/* Default helpers for node `failed`: the first d-subset of the survivors,
 * in lexicographic order, whose Psi rows are invertible (the d lowest ids
 * when they qualify).  helpers_out: d ints. */
int pmrc_default_helpers(const pmrc_code *code, int failed, int *helpers_out);

/* Thread-local description of the last error on this thread ("" if none). */
const char *pmrc_last_error(void);

/* ---- host-side introspection (no GPU needed) ---------------------------- */

/* params_out[6] = {n, k, d, alpha, construction, form}. */
int pmrc_code_params(const pmrc_code *code, int *params_out);

/* Data blocks K (k alpha for PM-MSR, k Delta for PM-MBR) and coded blocks
 * n alpha: the pointer counts of encode (K in) and decode (K out). */
int pmrc_code_blocks(const pmrc_code *code, int *data_blocks, int *coded_blocks);

/* 8 or 16: the field of the code's symbols (0 if code is NULL). */
int pmrc_code_field_bits(const pmrc_code *code);

/* The generator of a GF(2^16) code (n*alpha x k*alpha, row-major, 16-bit
 * values a | b << 8).  PMRC_EINVAL for a GF(2^8) code. */
int pmrc_code_generator16(const pmrc_code *code, uint16_t *g_out);

/* The code's generator, n*alpha x K, row-major: G (non-systematic) or
 * G' (systematic); for PM-MBR always G (already systematic). */
int pmrc_code_generator(const pmrc_code *code, uint8_t *g_out);

/* phi_failed (alpha bytes): the helper coefficients of pmrc_repair_helper. */
int pmrc_helper_coefficients(const pmrc_code *code, int failed, uint8_t *coef_out);

/* D (alpha x d, row-major) applied by pmrc_repair_newcomer. */
int pmrc_newcomer_matrix(const pmrc_code *code, int failed, const int *helpers, uint8_t *d_out);

/* (K x k*alpha, row-major) matrix applied by pmrc_decode: the inverse of
 * the nodes' rows (PM-MSR; K = k*alpha), or of K independent ones of them
 * with zero columns for the others (PM-MBR). */
int pmrc_decode_matrix(const pmrc_code *code, const int *nodes, uint8_t *r_out);

/* How the region kernel would cut the rows x cols matrix m (row-major, host)
 * into dense blocks: stats_out[5] = {blocks, rows per block held in
 * registers (R), products per byte column (entries, zeros included), input
 * splits per byte column (sum of block input counts), non-zero
 * coefficients}. */
int pmrc_plan_stats(int rows, int cols, const uint8_t *m, int64_t *stats_out);

#ifdef __cplusplus
}
#endif
#endif /* PMRC_H */
