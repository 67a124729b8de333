// Bitsliced region kernels: the encodes of the codes listed in
// gen_bitslice.cpp, and schedules compiled at run time (jit.cpp) for other
// matrices (reconstruction rows, newcomer applies, encodes of other codes).
//
// Same operation as region.cu (out[r] = sum_c M[r][c] * in[c], Sec. 2/3.1),
// for a matrix fixed when the schedule is generated, with a different inner
// loop:
//
//   * each thread owns 32 consecutive bytes of every block of a tile; it
//     streams its inputs through a 5-slot shared-memory ring with cp.async,
//     four inputs ahead of the one in use (the XOR work per input is short,
//     so the loads must be in flight well before they are needed), and
//     turns each into eight 32-bit bit planes (plane i = bit i of the 32
//     bytes) with a 3-stage transpose of the 8 words, each stage a pair of
//     bit-field selects (one 3-input logic op each) on shifted copies;
//   * from the planes it forms Q[s] (XOR of the subset s of planes 0-3) and
//     R[s] (subset of planes 4-7);
//   * output plane i of a row gains Q[a] ^ R[b] per input, where a and b are
//     the nibbles of row i of the coefficient's 8x8 bit matrix -- one 3-input
//     XOR per (row, plane, input), against three table lookups and two XORs
//     per 4 bytes in region.cu;
//   * accumulated planes go back to bytes with the same transpose (it is its
//     own inverse) and are stored with 16-byte streaming stores;
//   * the inputs of a block are walked by a loop whose body switches on the
//     input only for the accumulate XORs, halving the code of a block;
//   * the grid is persistent, one 512-thread CTA per SM: the sequence of
//     (block, 1 KiB column tile) items is cut into equal-cost contiguous
//     ranges, one per CTA, whose warps take the tiles in turn; so an SM holds
//     one block's straight-line code (tens of KiB; two blocks' at a range
//     boundary), fetched into its instruction caches once and re-executed,
//     and every SM gets the same work whatever the number of blocks.
//
// The built-in XOR schedules are generated at build time from the library's
// own construction (gen_bitslice.cpp); the launcher only uses a kernel whose
// matrix checksum equals the code's encode matrix.  Run-time schedules come
// from the same emitter (bs_emit.cpp).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "bitslice.h"
#include "bs_emit.h"
#include "code.h"
#include "device_info.h"
#include "jit.h"

namespace pmrc {
// a named namespace: the built-in kernels of the large codes are defined in
// translation units of their own (bitslice_k12.cu, bitslice_k16.cu) over the
// same launch-argument type
namespace bsk {

#include "bitslice_dev.cuh"

struct BsKernel {
  int n, k, construction, form;
  int nblocks, ninputs, noutputs;
  unsigned long long checksum;
  long long xors;
  void (*fn)(BsArgs);
  const int *cost;  // relative cost of each block per tile
};

#include "bitslice_gen.cuh"

}  // namespace bsk

using namespace bsk;

uint64_t bitslice_checksum(const uint8_t *m, size_t len) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < len; i++) {
    h ^= m[i];
    h *= 1099511628211ull;
  }
  return h;
}

int bitslice_find(int n, int k, int construction, int form, uint64_t checksum) {
  for (int i = 0; i < kBsNumKernels; i++) {
    const BsKernel &b = kBsKernels[i];
    if (b.n == n && b.k == k && b.construction == construction && b.form == form)
      return b.checksum == checksum ? i : -1;
  }
  return -1;
}

long long bitslice_xors(int id) { return id >= 0 && id < kBsNumKernels ? kBsKernels[id].xors : 0; }

namespace {

// One CTA per SM, each with an equal share of the schedule's cost.
cudaError_t bs_launch(const void *fn, int nblocks, const int *cost, int ninputs, int noutputs,
                      const uint8_t *const *in, uint8_t *const *out, size_t nbytes,
                      cudaStream_t stream, std::atomic<uint64_t> (&smem_set)[kMaxDevices],
                      int slot, size_t extra_smem = 0, bool dependent = false) {
  BsArgs a;
  a.nbytes = nbytes;
  a.hi28 = 1u << 28;
  a.hi30 = 1u << 30;
  a.hi31 = 1u << 31;
  a.x16 = 16;
  a.x4 = 4;
  a.x2 = 2;
  memset(a.ptr, 0, sizeof a.ptr);
  for (int i = 0; i < ninputs; i++) a.ptr[i] = const_cast<uint8_t *>(in[i]);
  for (int j = 0; j < noutputs; j++) a.ptr[ninputs + j] = out[j];
  const int sms = current_sm_count();
  const size_t smem = (size_t)kBsSlots * kBsThreads * kBsBytes + extra_smem;  // 80 KiB ring
  {
    const cudaError_t e = allow_max_smem(fn, smem_set, slot);
    if (e != cudaSuccess) return e;
  }
  // the work is the sequence of (block, tile) items g = b * ntiles + t; CTA
  // c takes a contiguous range of it holding 1/ncta of the total cost, so
  // every SM gets the same work whatever the block count, and a CTA runs one
  // block's code (two at a range boundary)
  const uint64_t ntiles = (nbytes + kBsUnit - 1) / kBsUnit;
  const uint64_t items = (uint64_t)nblocks * ntiles;
  const int ncta = (int)std::max<uint64_t>(1, std::min<uint64_t>(std::min(sms, kBsMaxCtas), items));
  a.ntiles = (uint32_t)ntiles;
  bs_cta_ranges(nblocks, cost, ntiles, ncta, a.cta_g);
  for (int c = ncta + 1; c <= kBsMaxCtas; c++) a.cta_g[c] = (uint32_t)items;
  void *args[] = {&a};
  if (!dependent) return cudaLaunchKernel(fn, dim3(ncta), dim3(kBsThreads), args, smem, stream);
  // programmatic dependent launch: the grid may be placed while the previous
  // kernel of the stream (which signals it) still runs; its kernel waits for
  // that kernel's completion (griddepcontrol.wait) before reading
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ncta);
  cfg.blockDim = dim3(kBsThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr = {};
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

std::atomic<uint64_t> g_static_smem_set[kMaxDevices];

// the device code, as text, for run-time compilation (generated from
// bitslice_dev.cuh at build time)
#include "bitslice_dev_src.inc"

}  // namespace

cudaError_t bitslice_prepare(int id) {
  if (id < 0 || id >= kBsNumKernels) return cudaErrorInvalidValue;
  return allow_max_smem(reinterpret_cast<const void *>(kBsKernels[id].fn), g_static_smem_set, id);
}

cudaError_t bitslice_launch(int id, const uint8_t *const *in, uint8_t *const *out, size_t nbytes,
                            cudaStream_t stream) {
  const BsKernel &b = kBsKernels[id];
  return bs_launch(reinterpret_cast<const void *>(b.fn), b.nblocks, b.cost, b.ninputs, b.noutputs,
                   in, out, nbytes, stream, g_static_smem_set, id);
}

struct BsRuntimeKernel {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t fn = nullptr;
  int kind = kBsMatrix;
  int pairs = 0;  // warp pairs split each item's inputs (bs_emit_kernel)
  int nblocks = 0, ninputs = 0, noutputs = 0;
  int alpha = 0, d = 0;
  std::vector<int> cost;
  std::atomic<uint64_t> smem_set[kMaxDevices] = {};
  ~BsRuntimeKernel() {
    if (lib) cudaLibraryUnload(lib);
  }
};

namespace {

int check_blocks(const std::vector<BsBlock> &blks, int max_inputs, std::string &err) {
  if ((int)blks.size() > kBsMaxBlocks) {
    err = "too many blocks for one bitsliced launch";
    return kEUnsupported;
  }
  for (const BsBlock &b : blks)
    if ((int)b.inputs.size() > max_inputs) {
      err = "a block reads more inputs than the run-time kernels take";
      return kEUnsupported;
    }
  return kOk;
}

// The blocks of a run-time schedule: rows of identical support when asked
// (encode matrices), unless that gives too many blocks or too wide ones;
// consecutive rows over the union of their inputs otherwise.
int runtime_blocks(const uint8_t *M, int rows, int cols, int max_inputs, bool by_support,
                   std::vector<BsBlock> &blks, std::string &err) {
  if (rows <= 0 || cols <= 0 || rows + cols > kBsMaxPtr) {
    err = "matrix too large for one bitsliced launch";
    return kEUnsupported;
  }
  if (by_support) {
    blks = bs_blocks_by_support(M, rows, cols);
    if (!check_blocks(blks, max_inputs, err)) return kOk;
  }
  blks = bs_blocks_chunked(M, rows, cols);
  return check_blocks(blks, max_inputs, err);
}

}  // namespace

int bitslice_check(const uint8_t *M, int rows, int cols, int max_inputs, bool by_support,
                   std::string &err) {
  std::vector<BsBlock> blks;
  return runtime_blocks(M, rows, cols, max_inputs, by_support, blks, err);
}

int bitslice_compile(const uint8_t *M, int rows, int cols, int max_inputs, bool by_support,
                     const char *role, BsCompiled &out, std::string &err) {
  std::vector<BsBlock> blks;
  int rc = runtime_blocks(M, rows, cols, max_inputs, by_support, blks, err);
  if (rc) return rc;
  out.name = std::string("bs_rt_") + role;
  const char *kname = out.name.c_str();
  // matrices cut into consecutive rows (reconstruction rows, newcomer
  // applies) are few blocks over many inputs: their launches have about one
  // tile per warp, so warp pairs split each item's inputs
  const bool pairs = !by_support;
  const BsEmitted em = bs_emit_kernel(M, rows, cols, blks, kname, true, pairs);
  const std::string src =
      "typedef unsigned char uint8_t;\ntypedef unsigned short uint16_t;\n"
      "typedef unsigned int uint32_t;\ntypedef unsigned long long uint64_t;\n" +
      std::string(kBsDevSrc) + "\n" + em.code;
  rc = jit_compile(src, kname, out.cubin, err);
  if (rc) return rc;
  out.kind = kBsMatrix;
  out.pairs = pairs ? 1 : 0;
  out.nblocks = (int)blks.size();
  out.ninputs = cols;
  out.noutputs = rows;
  out.cost = em.cost;
  return kOk;
}

int bitslice_load(const BsCompiled &c, std::shared_ptr<BsRuntimeKernel> &out, std::string &err) {
  auto k = std::make_shared<BsRuntimeKernel>();
  const int rc = jit_load(c.cubin, c.name.c_str(), &k->lib, &k->fn, err);
  if (rc) return rc;
  k->kind = c.kind;
  k->pairs = c.pairs;
  k->nblocks = c.nblocks;
  k->ninputs = c.ninputs;
  k->noutputs = c.noutputs;
  k->alpha = c.alpha;
  k->d = c.d;
  k->cost = c.cost;
  out = k;
  return kOk;
}

int bitslice_build(const uint8_t *M, int rows, int cols, int max_inputs, bool by_support,
                   const char *role, std::shared_ptr<BsRuntimeKernel> &out, std::string &err) {
  BsCompiled c;
  const int rc = bitslice_compile(M, rows, cols, max_inputs, by_support, role, c, err);
  return rc ? rc : bitslice_load(c, out, err);
}

cudaError_t bitslice_launch_runtime(BsRuntimeKernel &k, const uint8_t *const *in,
                                    uint8_t *const *out, size_t nbytes, cudaStream_t stream,
                                    bool dependent) {
  return bs_launch(reinterpret_cast<const void *>(k.fn), k.nblocks, k.cost.data(), k.ninputs,
                   k.noutputs, in, out, nbytes, stream, k.smem_set, 0,
                   k.pairs ? (size_t)kBsPairExchangeBytes : 0, dependent);
}

int bitslice_max_pointers() { return kBsMaxPtr; }

namespace {

std::string runtime_source(const std::string &code) {
  return "typedef unsigned char uint8_t;\ntypedef unsigned short uint16_t;\n"
         "typedef unsigned int uint32_t;\ntypedef unsigned long long uint64_t;\n" +
         std::string(kBsDevSrc) + "\n" + code;
}

bool any_nonzero(const uint8_t *v, int n) {
  for (int i = 0; i < n; i++)
    if (v[i]) return true;
  return false;
}

// Arguments common to the repair launches; in and out as for the matrix
// kernels (slot nin + r is output r).
void repair_args(BsArgs &a, size_t nbytes, int nin, const uint8_t *const *in, int nout,
                 uint8_t *const *out) {
  memset(&a, 0, sizeof a);
  a.nbytes = nbytes;
  a.hi28 = 1u << 28;
  a.hi30 = 1u << 30;
  a.hi31 = 1u << 31;
  a.x16 = 16;
  a.x4 = 4;
  a.x2 = 2;
  a.ntiles = (uint32_t)((nbytes + kBsUnit - 1) / kBsUnit);
  for (int i = 0; i < nin; i++) a.ptr[i] = const_cast<uint8_t *>(in[i]);
  for (int j = 0; j < nout; j++) a.ptr[nin + j] = out[j];
}

}  // namespace

int bitslice_compile_stage(const uint8_t *M, int rows, int cols, const std::vector<BsBlock> &blks,
                           int max_inputs, bool in_planes, bool out_planes, const char *role,
                           BsCompiled &out, std::string &err) {
  if (rows <= 0 || cols <= 0 || rows + cols > kBsMaxPtr) {
    err = "matrix too large for one bitsliced launch";
    return kEUnsupported;
  }
  int rc = check_blocks(blks, max_inputs, err);
  if (rc) return rc;
  out.name = std::string("bs_rt_") + role;
  const char *kname = out.name.c_str();
  const BsEmitted em = bs_emit_kernel(M, rows, cols, blks, kname, true, true, in_planes, out_planes);
  rc = jit_compile(runtime_source(em.code), kname, out.cubin, err);
  if (rc) return rc;
  out.kind = kBsMatrix;
  out.pairs = 1;
  out.nblocks = (int)blks.size();
  out.ninputs = cols;
  out.noutputs = rows;
  out.cost = em.cost;
  return kOk;
}


int bitslice_compile_projection(const uint8_t *phi, int alpha, const char *role, BsCompiled &out,
                                std::string &err) {
  if (alpha <= 0 || alpha + 1 > kBsMaxPtr || !any_nonzero(phi, alpha)) {
    err = "helper coefficients do not fit a bitsliced projection";
    return kEUnsupported;
  }
  out.name = std::string("bs_rt_") + role;
  const BsEmitted em = bs_emit_projection(phi, alpha, out.name);
  const int rc = jit_compile(runtime_source(em.code), out.name.c_str(), out.cubin, err);
  if (rc) return rc;
  out.kind = kBsProjection;
  out.alpha = alpha;
  out.d = 0;
  return kOk;
}

int bitslice_compile_fused_repair(const uint8_t *phi, int alpha, const uint8_t *D, int d,
                                  const char *role, BsCompiled &out, std::string &err) {
  if (alpha <= 0 || alpha > kBsFusedMaxAlpha || d < 2 || d * alpha + alpha > kBsMaxPtr ||
      !any_nonzero(phi, alpha)) {
    err = "repair does not fit the bitsliced fused kernel (alpha <= 8, d*alpha + alpha <= 512)";
    return kEUnsupported;
  }
  out.name = std::string("bs_rt_") + role;
  const BsEmitted em = bs_emit_fused_repair(phi, alpha, D, d, out.name);
  const int rc = jit_compile(runtime_source(em.code), out.name.c_str(), out.cubin, err);
  if (rc) return rc;
  out.kind = kBsFusedRepair;
  out.alpha = alpha;
  out.d = d;
  return kOk;
}

int bitslice_kind(const BsRuntimeKernel &k) { return k.kind; }

int bitslice_outputs(const BsRuntimeKernel &k) { return k.noutputs; }

cudaError_t bitslice_launch_projection(BsRuntimeKernel &k, int nh, const uint8_t *const *in,
                                       uint8_t *const *out, size_t nbytes, cudaStream_t stream) {
  if (k.kind != kBsProjection || nh <= 0 || nh * k.alpha + nh > kBsMaxPtr || nbytes % kBsBytes)
    return cudaErrorInvalidValue;
  BsArgs a;
  repair_args(a, nbytes, nh * k.alpha, in, nh, out);
  a.nh = (uint32_t)nh;
  a.ngroups = (uint32_t)((nh + kBsHelpersPerTask - 1) / kBsHelpersPerTask);
  a.ntasks = a.ntiles * a.ngroups;
  const void *fn = reinterpret_cast<const void *>(k.fn);
  const size_t smem = (size_t)kBsSlots * kBsThreads * kBsBytes;
  cudaError_t e = allow_max_smem(fn, k.smem_set, 0);
  if (e != cudaSuccess) return e;
  // two CTAs per SM (the projection kernel needs few registers): more loads
  // in flight for this memory-bound kernel
  const uint64_t warps = kBsThreads / 32;
  const int ncta = (int)std::max<uint64_t>(
      1, std::min<uint64_t>(2 * (uint64_t)current_sm_count(), (a.ntasks + warps - 1) / warps));
  void *args[] = {&a};
  return cudaLaunchKernel(fn, dim3(ncta), dim3(kBsThreads), args, smem, stream);
}

cudaError_t bitslice_launch_fused_repair(BsRuntimeKernel &k, const uint8_t *const *in,
                                         uint8_t *const *out, size_t nbytes, cudaStream_t stream) {
  if (k.kind != kBsFusedRepair || nbytes % kBsBytes) return cudaErrorInvalidValue;
  BsArgs a;
  repair_args(a, nbytes, k.d * k.alpha, in, k.alpha, out);
  a.nh = (uint32_t)k.d;
  const void *fn = reinterpret_cast<const void *>(k.fn);
  // the staging ring, then one exchange area (alpha x 8 planes x 32 lanes) per warp pair
  const size_t smem = (size_t)kBsSlots * kBsThreads * kBsBytes +
                      (size_t)(kBsThreads / 64) * k.alpha * 8 * 32 * 4;
  cudaError_t e = allow_max_smem(fn, k.smem_set, 0);
  if (e != cudaSuccess) return e;
  const int ncta = (int)std::max<uint64_t>(1, std::min<uint64_t>(current_sm_count(), a.ntiles));
  void *args[] = {&a};
  return cudaLaunchKernel(fn, dim3(ncta), dim3(kBsThreads), args, smem, stream);
}

}  // namespace pmrc
