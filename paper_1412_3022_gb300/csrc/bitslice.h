// Bitsliced region kernels (bitslice.cu): encode schedules generated at
// build time, and schedules compiled at run time for other matrices.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "bs_emit.h"

namespace pmrc {

// Checksum of an encode matrix (row-major bytes), as stored with each
// generated kernel.
uint64_t bitslice_checksum(const uint8_t *m, size_t len);

// Kernel id for the code, or -1 if none was generated or its matrix differs.
int bitslice_find(int n, int k, int construction, int form, uint64_t checksum);

// XOR terms of the generated schedule per 32-byte column (for reporting).
long long bitslice_xors(int id);

// Encodes bytes [0, nbytes) of every block; nbytes must be a multiple of 32
// and every pointer 16-byte aligned.  in: k*alpha blocks, out: the encode
// matrix's output blocks (NULL not allowed).
cudaError_t bitslice_launch(int id, const uint8_t *const *in, uint8_t *const *out, size_t nbytes,
                            cudaStream_t stream);

int bitslice_max_pointers();

// Makes the shared-memory setting of built-in kernel `id` on the current
// device (once), so that later launches -- inside a stream capture too --
// need no attribute call.
cudaError_t bitslice_prepare(int id);


// A bitsliced kernel compiled at run time (NVRTC) for a matrix known only
// then: the rows of a reconstruction or a newcomer's apply (consecutive rows
// in blocks of at most 8 over the union of their inputs), or the encode
// matrix of a code without a built-in kernel (by_support: rows of identical
// support in blocks of at most 8, unless those do not fit the limits below,
// then consecutive rows); the same device code as the built-in kernels.
struct BsRuntimeKernel;

// kOk if M (rows x cols, row-major) fits one run-time launch: cols + rows
// <= bitslice_max_pointers() (512), at most 64 blocks, at most `max_inputs`
// inputs in a block; kEUnsupported with a message in err otherwise.  Host
// only.
int bitslice_check(const uint8_t *M, int rows, int cols, int max_inputs, bool by_support,
                   std::string &err);

// Kinds of run-time kernels: a matrix schedule (reconstruction rows,
// newcomer apply, encode), helper projections for one failed node, and the
// fused repair of one (failed node, helper set).
enum BsKind { kBsMatrix = 0, kBsProjection = 1, kBsFusedRepair = 2 };

// A compiled schedule not yet loaded: the cubin and what its launches need.
struct BsCompiled {
  std::string name;  // kernel name: bs_rt_<role>
  std::vector<char> cubin;
  int kind = kBsMatrix;
  int pairs = 0;  // warp pairs split each item's inputs (matrix kernels of consecutive rows)
  int nblocks = 0, ninputs = 0, noutputs = 0;
  int alpha = 0, d = 0;  // repair kernels: blocks per node, helpers
  std::vector<int> cost;
};

// Emits and compiles the schedule for M as kernel bs_rt_<role> (host only:
// NVRTC, no CUDA call, so it may run on any thread).  kEUnsupported when
// bitslice_check fails or NVRTC is missing or fails (message in err).
int bitslice_compile(const uint8_t *M, int rows, int cols, int max_inputs, bool by_support,
                     const char *role, BsCompiled &out, std::string &err);

// One launch of a two-launch product: the matrix schedule for M with the
// given blocks (each at most max_inputs inputs), over warp pairs, reading
// plane-layout inputs (in_planes) and/or storing plane-layout outputs
// (out_planes) -- see bs_emit_kernel.  Host only, like bitslice_compile.
int bitslice_compile_stage(const uint8_t *M, int rows, int cols, const std::vector<BsBlock> &blks,
                           int max_inputs, bool in_planes, bool out_planes, const char *role,
                           BsCompiled &out, std::string &err);

// Loads a compiled schedule as a CUDA library (the calling thread's device
// context must be usable).
int bitslice_load(const BsCompiled &c, std::shared_ptr<BsRuntimeKernel> &out, std::string &err);

// bitslice_compile, then bitslice_load.
int bitslice_build(const uint8_t *M, int rows, int cols, int max_inputs, bool by_support,
                   const char *role, std::shared_ptr<BsRuntimeKernel> &out, std::string &err);

// out[r] = sum_c M[r][c] in[c] over bytes [0, nbytes); nbytes a multiple of
// 32, every pointer 16-byte aligned; in[c] may be NULL for columns no row
// reads, out[r] may not be NULL.  dependent: a programmatic dependent launch
// after the stream's previous kernel (the second launch of a two-launch
// product, whose kernel waits for the first before reading it).
cudaError_t bitslice_launch_runtime(BsRuntimeKernel &k, const uint8_t *const *in,
                                    uint8_t *const *out, size_t nbytes, cudaStream_t stream,
                                    bool dependent = false);

// Repair schedules compiled at run time (host only, like bitslice_compile).
// Projection: phi (alpha entries, at least one non-zero), kernel
// bs_rt_<role>.  Fused repair: phi and the newcomer matrix D (alpha x d,
// row-major, alpha <= 8).  kEUnsupported when a limit is exceeded or NVRTC
// is missing or fails.
int bitslice_compile_projection(const uint8_t *phi, int alpha, const char *role, BsCompiled &out,
                                std::string &err);
int bitslice_compile_fused_repair(const uint8_t *phi, int alpha, const uint8_t *D, int d,
                                  const char *role, BsCompiled &out, std::string &err);

// Helper projections of nh helpers: in = nh*alpha blocks (helper h's at
// [h*alpha, h*alpha + alpha); blocks phi does not read may be NULL), out = nh
// blocks; nbytes a multiple of 32, pointers 16-byte aligned;
// nh*alpha + nh <= bitslice_max_pointers().
cudaError_t bitslice_launch_projection(BsRuntimeKernel &k, int nh, const uint8_t *const *in,
                                       uint8_t *const *out, size_t nbytes, cudaStream_t stream);

// Fused repair: in = d*alpha helper blocks (as above), out = alpha blocks.
cudaError_t bitslice_launch_fused_repair(BsRuntimeKernel &k, const uint8_t *const *in,
                                         uint8_t *const *out, size_t nbytes, cudaStream_t stream);

// The kind of a loaded run-time kernel (BsKind).
int bitslice_kind(const BsRuntimeKernel &k);

// Output blocks a run-time matrix kernel writes (its matrix's rows).
int bitslice_outputs(const BsRuntimeKernel &k);

}  // namespace pmrc
