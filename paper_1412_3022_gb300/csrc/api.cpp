// C ABI of libpmrc (include/pmrc.h): argument checks, plan cache, launches.
#include "../../include/pmrc.h"

#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "api_internal.h"
#include "bitslice.h"
#include "code.h"
#include "device_info.h"
#include "jit.h"
#include "plan.h"
#include "region.h"
#include "trace.h"

using namespace pmrc;

namespace {
thread_local std::string g_last_error;

int fail(int rc, const std::string &msg) {
  g_last_error = msg;
  return rc;
}
}  // namespace

namespace pmrc {

void set_last_error(const std::string &msg) { g_last_error = msg; }

std::shared_ptr<Plan> cached_plan(const pmrc_code *c, const std::string &key,
                                  const std::function<std::shared_ptr<Plan>()> &make) {
  std::lock_guard<std::mutex> g(c->mu);
  auto it = c->cache.find(key);
  if (it != c->cache.end()) return it->second;
  auto p = make();
  if (!p) return p;
  if (c->cache.size() >= kPlanCacheCap) c->cache.erase(c->cache.begin());
  c->cache[key] = p;
  return p;
}

int helper_plan(const pmrc_code *c, int f, int nh, std::shared_ptr<Plan> &out,
                std::string &err) {
  if (f < 0 || f >= c->m.n) {
    err = "failed node out of range";
    return kEInval;
  }
  const std::string key = "h:" + std::to_string(f) + ":" + std::to_string(nh);
  out = cached_plan(c, key, [&]() {
    Mat P;  // beta x alpha: the projection one helper applies to its blocks
    helper_matrix(c->m, f, P);
    const int a = c->m.alpha, b = c->m.beta;
    Mat M(nh * b, nh * a);  // block diagonal: helper h reads its own alpha blocks
    std::vector<int> slot(nh * b);
    for (int h = 0; h < nh; h++)
      for (int t = 0; t < b; t++) {
        for (int j = 0; j < a; j++) M.at(h * b + t, h * a + j) = P.at(t, j);
        slot[h * b + t] = h * b + t;
      }
    return make_plan(M, slot, nh * b);
  });
  return kOk;
}

int newcomer_plan(const pmrc_code *c, int f, const int *helpers, std::shared_ptr<Plan> &out,
                  std::string &err) {
  std::string key = "n:" + std::to_string(f);
  for (int i = 0; i < c->m.d; i++) key += "," + std::to_string(helpers[i]);
  {
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->cache.find(key);
    if (it != c->cache.end()) {
      out = it->second;
      return kOk;
    }
  }
  Mat D;
  int rc = newcomer_matrix(c->m, f, helpers, D, err);
  if (rc) return rc;
  out = cached_plan(c, key, [&]() {
    std::vector<int> slot(c->m.alpha);
    for (int j = 0; j < c->m.alpha; j++) slot[j] = j;
    return make_plan(D, slot, c->m.alpha);
  });
  return kOk;
}

int decode_plan(const pmrc_code *c, const int *nodes, const std::vector<char> &want,
                std::shared_ptr<Plan> &out, std::string &err) {
  const int K = c->m.K;
  std::string key = "d:";
  for (int i = 0; i < c->m.k; i++) key += std::to_string(nodes[i]) + ",";
  key += ":";
  for (int r = 0; r < K; r++) key += want[r] ? '1' : '0';
  {
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->cache.find(key);
    if (it != c->cache.end()) {
      out = it->second;
      return kOk;
    }
  }
  Mat Rinv;
  int rc = decode_matrix(c->m, nodes, Rinv, err);
  if (rc) return rc;
  out = cached_plan(c, key, [&]() {
    std::vector<int> slot(K);
    for (int r = 0; r < K; r++) slot[r] = want[r] ? r : -1;
    return make_plan(Rinv, slot, K);
  });
  return kOk;
}

int fused_repair_plan(const pmrc_code *c, int f, const int *helpers,
                      std::shared_ptr<FusedRepairPlan> &out, std::string &err) {
  std::string key = "r:" + std::to_string(f);
  for (int i = 0; i < c->m.d; i++) key += "," + std::to_string(helpers[i]);
  {
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->fused.find(key);
    if (it != c->fused.end()) {
      out = it->second;
      return kOk;
    }
  }
  Mat D;
  int rc = newcomer_matrix(c->m, f, helpers, D, err);
  if (rc) return rc;
  std::vector<uint8_t> phi;
  helper_coefficients(c->m, f, phi);
  auto p = make_fused_repair_plan(phi, D);
  std::lock_guard<std::mutex> g(c->mu);
  if (c->fused.size() >= kPlanCacheCap) c->fused.erase(c->fused.begin());
  c->fused[key] = p;
  out = p;
  return kOk;
}

// Which data rows a decode call must produce: non-NULL outputs, except a
// data block whose output pointer is a listed node block that holds it
// verbatim (a unit row of the code's generator: systematic MSR, MBR).
int decode_wanted(const pmrc_code *c, const int *nodes, const uint8_t *const *node_blocks,
                  uint8_t *const *data_out, std::vector<char> &want) {
  const int a = c->m.alpha, K = c->m.K;
  want.assign(K, 0);
  for (int r = 0; r < K; r++) want[r] = data_out[r] != nullptr;
  for (int i = 0; i < c->m.k; i++)
    for (int j = 0; j < a; j++) {
      const int s = c->m.unit_col[a * nodes[i] + j];  // data block this node block copies
      if (s >= 0 && data_out[s] == node_blocks[a * i + j]) want[s] = 0;
    }
  return kOk;
}

}  // namespace pmrc

namespace {

// reconstruction through run-time bitsliced kernels: AUTO uses them for
// blocks of at least this many bytes (the compilation, about a second per
// node set, is paid once per handle), and for reconstructions whose blocks
// read at most this many inputs
constexpr size_t kRuntimeMinBytes = 256 << 10;
constexpr size_t kRuntimeNewcomerMinBytes = 1 << 20;
// helper projections and the fused repair through run-time bitsliced
// kernels (compiled per failed node, resp. per failed node and helper set)
constexpr size_t kRuntimeHelperMinBytes = 256 << 10;
constexpr size_t kRuntimeRepairMinBytes = 256 << 10;
constexpr int kRuntimeMaxInputs = 64;
// AUTO compiles an encode schedule at run time only for encode matrices of
// at most this many non-zero coefficients: NVRTC's time grows faster than
// the schedule (GB300 host: a few seconds at 2048, tens of seconds at
// k = 16, n = 32); larger codes take it with PMRC_KERNEL_BITSLICED
constexpr int64_t kRuntimeAutoMaxNnz = 2048;

// GF(2^16) codes: user block i (B bytes, two byte planes) is the pair of
// GF(2^8) sub-blocks 2i (low plane) and 2i + 1 (high plane) of B/2 bytes.
std::vector<const uint8_t *> split_in(const uint8_t *const *p, int n, size_t half) {
  std::vector<const uint8_t *> v(2 * (size_t)n);
  for (int i = 0; i < n; i++) {
    v[2 * i] = p[i];
    v[2 * i + 1] = p[i] ? p[i] + half : nullptr;
  }
  return v;
}

std::vector<uint8_t *> split_out(uint8_t *const *p, int n, size_t half) {
  std::vector<uint8_t *> v(2 * (size_t)n);
  for (int i = 0; i < n; i++) {
    v[2 * i] = p[i];
    v[2 * i + 1] = p[i] ? p[i] + half : nullptr;
  }
  return v;
}

bool is16(const pmrc_code *c) { return c && c->m.w == 16; }

int not_for16(const char *what) {
  return fail(PMRC_EUNSUPPORTED, std::string(what) + " is not available for GF(2^16) codes");
}

int encode_body(const pmrc_code *c, const uint8_t *const *data, uint8_t *const *out,
                size_t nbytes, pmrc_stream_t stream);
int repair_helpers_body(const pmrc_code *c, int f, int nh, const int *helpers,
                        const uint8_t *const *blocks, uint8_t *const *out, size_t nbytes,
                        pmrc_stream_t stream);
int repair_newcomer_body(const pmrc_code *c, int f, const int *helpers,
                         const uint8_t *const *received, uint8_t *const *out, size_t nbytes,
                         pmrc_stream_t stream);
int decode_body(const pmrc_code *c, const int *nodes, const uint8_t *const *node_blocks,
                uint8_t *const *data_out, size_t nbytes, pmrc_stream_t stream);
std::shared_ptr<BsRuntimeKernel> runtime_kernel(const pmrc_code *c, const std::string &key,
                                                const char *role,
                                                const std::function<int(Mat &, std::string &)> &make,
                                                std::string &err, bool by_support, bool background);
void encode_matrix(const pmrc_code *c, Mat &M);
bool want_runtime(const pmrc_code *c, int policy, size_t nbytes, size_t auto_min);
std::shared_ptr<BsRuntimeKernel> projection_runtime(const pmrc_code *c, int f, bool background,
                                                    std::string &err);
std::shared_ptr<BsRuntimeKernel> fused_runtime(const pmrc_code *c, int f, const int *helpers,
                                               bool background, std::string &err);

}  // namespace

extern "C" {

const char *pmrc_last_error(void) { return g_last_error.c_str(); }

int pmrc_create(int n, int k, int d, int construction, int form, pmrc_code **out) {
  return pmrc_create_field(n, k, d, construction, form, 8, out);
}

int pmrc_create_field(int n, int k, int d, int construction, int form, int field_bits,
                      pmrc_code **out) {
  PMRC_TRACE("pmrc_create_field");
  if (!out) return fail(PMRC_EINVAL, "out is NULL");
  *out = nullptr;
  if (field_bits != 8 && field_bits != 16) return fail(PMRC_EINVAL, "field_bits must be 8 or 16");
  std::unique_ptr<pmrc_code> c(new (std::nothrow) pmrc_code());
  if (!c) return fail(PMRC_ENOMEM, "out of host memory");
  std::string err;
  int rc = field_bits == 16 ? build_code16(n, k, d, construction, form, c->m, err)
                            : build_code(n, k, d, construction, form, c->m, err);
  if (rc) return fail(rc, err);
  // encode plan: all rows (non-systematic) or the parity nodes' rows
  // (systematic: the first k nodes hold the data)
  Mat M;
  encode_matrix(c.get(), M);
  std::vector<int> slot(M.rows);
  for (int r = 0; r < M.rows; r++) slot[r] = r;
  c->encode = make_plan(M, slot, M.rows);
  c->bs_id = bitslice_find(n, k, construction, form, bitslice_checksum(M.v.data(), M.v.size()));
  *out = c.release();
  g_last_error.clear();
  return PMRC_OK;
}

void pmrc_destroy(pmrc_code *code) { delete code; }

int pmrc_code_params(const pmrc_code *c, int *p) {
  if (!c || !p) return fail(PMRC_EINVAL, "NULL argument");
  p[0] = c->m.n;
  p[1] = c->m.k;
  p[2] = c->m.d;
  p[3] = is16(c) ? c->m.f16.alpha : c->m.alpha;
  p[4] = c->m.construction;
  p[5] = c->m.systematic;
  return PMRC_OK;
}

int pmrc_code_blocks(const pmrc_code *c, int *data_blocks, int *coded_blocks) {
  if (!c || !data_blocks || !coded_blocks) return fail(PMRC_EINVAL, "NULL argument");
  *data_blocks = is16(c) ? c->m.f16.K : c->m.K;
  *coded_blocks = is16(c) ? c->m.f16.N : c->m.N;
  return PMRC_OK;
}

int pmrc_code_field_bits(const pmrc_code *c) { return c ? c->m.w : 0; }

int pmrc_code_generator16(const pmrc_code *c, uint16_t *g) {
  if (!c || !g) return fail(PMRC_EINVAL, "NULL argument");
  if (!is16(c)) return fail(PMRC_EINVAL, "not a GF(2^16) code");
  memcpy(g, c->m.f16.Gcode.data(), c->m.f16.Gcode.size() * sizeof(uint16_t));
  return PMRC_OK;
}

int pmrc_code_generator(const pmrc_code *c, uint8_t *g) {
  if (!c || !g) return fail(PMRC_EINVAL, "NULL argument");
  if (is16(c)) return not_for16("pmrc_code_generator (use pmrc_code_generator16)");
  memcpy(g, c->m.Gcode.v.data(), c->m.Gcode.v.size());
  return PMRC_OK;
}

int pmrc_helper_coefficients(const pmrc_code *c, int f, uint8_t *coef) {
  if (!c || !coef) return fail(PMRC_EINVAL, "NULL argument");
  if (is16(c)) return not_for16("pmrc_helper_coefficients");
  if (f < 0 || f >= c->m.n) return fail(PMRC_EINVAL, "failed node out of range");
  std::vector<uint8_t> v;
  helper_coefficients(c->m, f, v);
  memcpy(coef, v.data(), v.size());
  return PMRC_OK;
}

int pmrc_newcomer_matrix(const pmrc_code *c, int f, const int *helpers, uint8_t *d_out) {
  if (!c || !helpers || !d_out) return fail(PMRC_EINVAL, "NULL argument");
  if (is16(c)) return not_for16("pmrc_newcomer_matrix");
  Mat D;
  std::string err;
  int rc = newcomer_matrix(c->m, f, helpers, D, err);
  if (rc) return fail(rc, err);
  memcpy(d_out, D.v.data(), D.v.size());
  return PMRC_OK;
}

int pmrc_decode_matrix(const pmrc_code *c, const int *nodes, uint8_t *r_out) {
  if (!c || !nodes || !r_out) return fail(PMRC_EINVAL, "NULL argument");
  if (is16(c)) return not_for16("pmrc_decode_matrix");
  Mat R;
  std::string err;
  int rc = decode_matrix(c->m, nodes, R, err);
  if (rc) return fail(rc, err);
  memcpy(r_out, R.v.data(), R.v.size());
  return PMRC_OK;
}

int pmrc_plan_stats(int rows, int cols, const uint8_t *m, int64_t *st) {
  if (rows <= 0 || cols <= 0 || !m || !st) return fail(PMRC_EINVAL, "bad matrix");
  Mat M(rows, cols);
  memcpy(M.v.data(), m, (size_t)rows * cols);
  std::vector<int> slot(rows);
  for (int r = 0; r < rows; r++) slot[r] = r;
  auto p = make_plan(M, slot, rows);
  int64_t nb = 0, R = 0, ent = 0, ins = 0;
  auto add = [&](const Plan &q) {  // the plan itself, or each of its parts
    nb += (int64_t)q.blocks.size();
    if (!q.blocks.empty()) R = std::max<int64_t>(R, q.R);
    for (auto &b : q.blocks) {
      ent += (int64_t)b.inputs.size() * b.rows.size();
      ins += (int64_t)b.inputs.size();
    }
  };
  add(*p);
  for (auto &pt : p->parts) add(*pt.plan);
  st[0] = nb;
  st[1] = R;
  st[2] = ent;
  st[3] = ins;
  st[4] = p->nnz;
  return PMRC_OK;
}

int pmrc_default_helpers(const pmrc_code *c, int f, int *helpers_out) {
  if (!c || !helpers_out) return fail(PMRC_EINVAL, "NULL argument");
  std::string err;
  int rc = default_helpers(c->m, f, helpers_out, err);
  return rc ? fail(rc, err) : PMRC_OK;
}

int pmrc_wait_kernels(const pmrc_code *c, int timeout_ms) {
  if (!c) return fail(PMRC_EINVAL, "NULL argument");
  std::vector<std::shared_ptr<BsJob>> jobs;
  {
    std::lock_guard<std::mutex> g(c->mu);
    for (auto &kv : c->rt_jobs) jobs.push_back(kv.second);
  }
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  for (auto &j : jobs) {
    std::unique_lock<std::mutex> lk(j->mu);
    if (timeout_ms < 0)
      j->cv.wait(lk, [&] { return j->done; });
    else if (!j->cv.wait_until(lk, deadline, [&] { return j->done; }))
      return fail(PMRC_ETIMEOUT, "run-time kernels are still compiling");
  }
  return PMRC_OK;
}

int pmrc_runtime_kernels(const pmrc_code *c, int *ready, int *pending) {
  if (!c || !ready || !pending) return fail(PMRC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(c->mu);
  *ready = *pending = 0;
  for (auto &kv : c->rt) *ready += kv.second != nullptr;
  for (auto &kv : c->rt_jobs) {
    std::lock_guard<std::mutex> g2(kv.second->mu);
    if (!kv.second->done)
      ++*pending;
    else
      *ready += kv.second->rc == 0;
  }
  return PMRC_OK;
}

int pmrc_set_decode_kernel(pmrc_code *c, int which) {
  if (!c) return fail(PMRC_EINVAL, "NULL argument");
  if (which != PMRC_KERNEL_AUTO && which != PMRC_KERNEL_GENERIC && which != PMRC_KERNEL_BITSLICED)
    return fail(PMRC_EINVAL, "unknown kernel choice");
  c->decode_kernel = which;
  return PMRC_OK;
}

int pmrc_set_encode_kernel(pmrc_code *c, int which) {
  if (!c || which < PMRC_KERNEL_AUTO || which > PMRC_KERNEL_BITSLICED)
    return fail(PMRC_EINVAL, "bad handle or kernel choice");
  if (which == PMRC_KERNEL_BITSLICED && c->bs_id < 0) {
    // no built-in schedule: the encode matrix must fit a run-time kernel
    if (!jit_available())
      return fail(PMRC_EUNSUPPORTED, "no built-in bitsliced kernel for this code, and NVRTC is missing");
    Mat M;
    encode_matrix(c, M);
    std::string err;
    if (bitslice_check(M.v.data(), M.rows, M.cols, kRuntimeMaxInputs, true, err))
      return fail(PMRC_EUNSUPPORTED, "no bitsliced kernel for this code: " + err);
  }
  c->encode_kernel = which;
  return PMRC_OK;
}

int pmrc_encode(const pmrc_code *c, const uint8_t *const *data, uint8_t *const *out,
                size_t nbytes, pmrc_stream_t stream) {
  PMRC_TRACE("pmrc_encode");
  if (!c || !data || !out) return fail(PMRC_EINVAL, "NULL argument");
  if (is16(c)) {
    if (nbytes % 2) return fail(PMRC_EINVAL, "GF(2^16) blocks hold whole 2-byte symbols");
    const auto &f = c->m.f16;
    const int nout = c->m.systematic ? f.N - c->m.k * f.alpha : f.N;
    auto in8 = split_in(data, f.K, nbytes / 2);
    auto out8 = split_out(out, nout, nbytes / 2);
    return encode_body(c, in8.data(), out8.data(), nbytes / 2, stream);
  }
  return encode_body(c, data, out, nbytes, stream);
}

}  // extern "C"

namespace {

int encode_body(const pmrc_code *c, const uint8_t *const *data, uint8_t *const *out,
                size_t nbytes, pmrc_stream_t stream) {
  std::string err;
  const Plan &P = *c->encode;
  size_t done = 0;
  const int policy = c->encode_kernel;
  if (policy != PMRC_KERNEL_GENERIC && nbytes >= 32) {
    bool ok = true;
    for (int i = 0; i < P.nin && ok; i++) ok = data[i] && ((uintptr_t)data[i] % 16 == 0);
    for (int j = 0; j < P.nout && ok; j++) ok = out[j] && ((uintptr_t)out[j] % 16 == 0);
    if (ok && c->bs_id >= 0) {
      done = nbytes & ~(size_t)31;
      cudaError_t e = bitslice_launch(c->bs_id, data, out, done, (cudaStream_t)stream);
      if (e != cudaSuccess)
        return fail(PMRC_ECUDA, std::string("bitsliced encode launch: ") + cudaGetErrorString(e));
    } else if (ok && (policy == PMRC_KERNEL_BITSLICED ||
                      (nbytes >= kRuntimeMinBytes && P.nnz <= kRuntimeAutoMaxNnz))) {
      // no built-in schedule for this code: its encode matrix compiled at
      // run time (rows of identical support in blocks, as the built-in ones)
      std::string rerr;
      std::shared_ptr<BsRuntimeKernel> k = runtime_kernel(c, "e", "encode", [&](Mat &M, std::string &) {
        encode_matrix(c, M);
        return (int)kOk;
      }, rerr, true, policy != PMRC_KERNEL_BITSLICED);
      if (k) {
        done = nbytes & ~(size_t)31;
        const cudaError_t e = bitslice_launch_runtime(*k, data, out, done, (cudaStream_t)stream);
        if (e != cudaSuccess)
          return fail(PMRC_ECUDA, std::string("bitsliced encode launch: ") + cudaGetErrorString(e));
      } else if (policy == PMRC_KERNEL_BITSLICED) {
        return fail(PMRC_EUNSUPPORTED, "bitsliced encode: " + rerr);
      }
    }
  }
  if (done == nbytes) return PMRC_OK;
  int rc;
  if (done == 0) {
    rc = launch_region(*c->encode, data, out, nbytes, (cudaStream_t)stream, err);
  } else {  // ragged tail of the blocks
    std::vector<const uint8_t *> in2(P.nin);
    std::vector<uint8_t *> out2(P.nout);
    for (int i = 0; i < P.nin; i++) in2[i] = data[i] + done;
    for (int j = 0; j < P.nout; j++) out2[j] = out[j] + done;
    rc = launch_region(*c->encode, in2.data(), out2.data(), nbytes - done, (cudaStream_t)stream,
                       err);
  }
  return rc ? fail(rc, err) : PMRC_OK;
}

int repair_helpers_body(const pmrc_code *c, int f, int nh, const int *helpers,
                        const uint8_t *const *blocks, uint8_t *const *out, size_t nbytes,
                        pmrc_stream_t stream) {
  if (f < 0 || f >= c->m.n) return fail(PMRC_EINVAL, "failed node out of range");
  if (helpers)
    for (int h = 0; h < nh; h++)
      if (helpers[h] < 0 || helpers[h] >= c->m.n || helpers[h] == f)
        return fail(PMRC_EINVAL, "helper id out of range or equal to the failed node");
  for (int h = 0; h < nh * c->m.beta; h++)
    if (!out[h]) return fail(PMRC_EINVAL, "output block is NULL");
  std::shared_ptr<Plan> p;
  std::string err;
  int rc = helper_plan(c, f, nh, p, err);
  if (rc) return fail(rc, err);
  const cudaStream_t st = (cudaStream_t)stream;
  const int a = c->m.alpha;
  size_t done = 0;
  // bitsliced projections, compiled at run time per failed node: each block
  // phi_f reads is turned into bit planes once and multiplied by its
  // constant as XORs of planes
  if (c->m.beta == 1 && nh * a + nh <= bitslice_max_pointers() &&
      want_runtime(c, c->decode_kernel, nbytes, kRuntimeHelperMinBytes)) {
    std::vector<uint8_t> phi;
    helper_coefficients(c->m, f, phi);
    bool aligned = true;
    for (int h = 0; h < nh && aligned; h++) {
      for (int j = 0; j < a; j++)
        if (phi[j]) aligned = aligned && blocks[h * a + j] && (uintptr_t)blocks[h * a + j] % 16 == 0;
      aligned = aligned && (uintptr_t)out[h] % 16 == 0;
    }
    std::string rerr;
    std::shared_ptr<BsRuntimeKernel> k;
    if (aligned) k = projection_runtime(c, f, c->decode_kernel != PMRC_KERNEL_BITSLICED, rerr);
    if (k) {
      done = nbytes & ~(size_t)31;
      const cudaError_t e = bitslice_launch_projection(*k, nh, blocks, out, done, st);
      if (e != cudaSuccess)
        return fail(PMRC_ECUDA, std::string("bitsliced projection launch: ") + cudaGetErrorString(e));
    }
  }
  if (done == nbytes) return PMRC_OK;
  if (done == 0) {
    rc = launch_region(*p, blocks, out, nbytes, st, err);
  } else {  // ragged tail of the blocks
    std::vector<const uint8_t *> in2(nh * a);
    std::vector<uint8_t *> out2(nh);
    for (int i = 0; i < nh * a; i++) in2[i] = blocks[i] ? blocks[i] + done : nullptr;
    for (int h = 0; h < nh; h++) out2[h] = out[h] + done;
    rc = launch_region(*p, in2.data(), out2.data(), nbytes - done, st, err);
  }
  return rc ? fail(rc, err) : PMRC_OK;
}

int repair_newcomer_body(const pmrc_code *c, int f, const int *helpers,
                         const uint8_t *const *received, uint8_t *const *out, size_t nbytes,
                         pmrc_stream_t stream) {
  for (int j = 0; j < c->m.alpha; j++)
    if (!out[j]) return fail(PMRC_EINVAL, "output block is NULL");
  std::shared_ptr<Plan> p;
  std::string err;
  int rc = newcomer_plan(c, f, helpers, p, err);
  if (rc) return fail(rc, err);
  const cudaStream_t st = (cudaStream_t)stream;
  const int d = c->m.d * c->m.beta, a = c->m.alpha;
  size_t done = 0;
  // bitsliced newcomer, compiled at run time per (failed node, helpers)
  // like the reconstruction rows; a single 8-row block gives one 1 KiB tile
  // per warp, which beats the split-table kernel from 1 MiB blocks (at 1 MiB
  // 15 against 19 us), so AUTO takes it from there
  if (want_runtime(c, c->decode_kernel, nbytes, kRuntimeNewcomerMinBytes)) {
    bool aligned = true;
    for (int i = 0; i < d && aligned; i++) aligned = received[i] && (uintptr_t)received[i] % 16 == 0;
    for (int j = 0; j < a && aligned; j++) aligned = (uintptr_t)out[j] % 16 == 0;
    std::string key = "n:" + std::to_string(f);
    for (int i = 0; i < c->m.d; i++) key += "," + std::to_string(helpers[i]);
    std::string rerr;
    std::shared_ptr<BsRuntimeKernel> k;
    if (aligned)
      k = runtime_kernel(c, key, "newcomer", [&](Mat &M, std::string &e) {
        return newcomer_matrix(c->m, f, helpers, M, e);
      }, rerr, false, c->decode_kernel != PMRC_KERNEL_BITSLICED);
    if (k) {
      done = nbytes & ~(size_t)31;
      const cudaError_t e = bitslice_launch_runtime(*k, received, out, done, st);
      if (e != cudaSuccess)
        return fail(PMRC_ECUDA, std::string("bitsliced newcomer launch: ") + cudaGetErrorString(e));
    }
  }
  if (done == nbytes) return PMRC_OK;
  if (done == 0) {
    rc = launch_region(*p, received, out, nbytes, st, err);
  } else {  // ragged tail of the blocks
    std::vector<const uint8_t *> in2(d);
    std::vector<uint8_t *> out2(a);
    for (int i = 0; i < d; i++) in2[i] = received[i] + done;
    for (int j = 0; j < a; j++) out2[j] = out[j] + done;
    rc = launch_region(*p, in2.data(), out2.data(), nbytes - done, st, err);
  }
  return rc ? fail(rc, err) : PMRC_OK;
}

}  // namespace

extern "C" {

int pmrc_repair_helpers(const pmrc_code *c, int f, int nh, const int *helpers,
                        const uint8_t *const *blocks, uint8_t *const *out, size_t nbytes,
                        pmrc_stream_t stream) {
  PMRC_TRACE("pmrc_repair_helpers");
  if (!c || !blocks || !out || nh <= 0 || (nh > 1 && !helpers))
    return fail(PMRC_EINVAL, "NULL argument or nhelpers <= 0");
  if (f < 0 || f >= c->m.n) return fail(PMRC_EINVAL, "failed node out of range");
  if (helpers)
    for (int h = 0; h < nh; h++)
      if (helpers[h] < 0 || helpers[h] >= c->m.n || helpers[h] == f)
        return fail(PMRC_EINVAL, "helper id out of range or equal to the failed node");
  for (int h = 0; h < nh; h++)
    if (!out[h]) return fail(PMRC_EINVAL, "output block is NULL");
  if (is16(c)) {
    if (nbytes % 2) return fail(PMRC_EINVAL, "GF(2^16) blocks hold whole 2-byte symbols");
    auto in8 = split_in(blocks, nh * c->m.f16.alpha, nbytes / 2);
    auto out8 = split_out(out, nh, nbytes / 2);
    return repair_helpers_body(c, f, nh, helpers, in8.data(), out8.data(), nbytes / 2, stream);
  }
  return repair_helpers_body(c, f, nh, helpers, blocks, out, nbytes, stream);
}

int pmrc_repair_helper(const pmrc_code *c, int f, int helper, const uint8_t *const *blocks,
                       uint8_t *out, size_t nbytes, pmrc_stream_t stream) {
  if (!out) return fail(PMRC_EINVAL, "output block is NULL");
  return pmrc_repair_helpers(c, f, 1, &helper, blocks, &out, nbytes, stream);
}

int pmrc_repair_newcomer(const pmrc_code *c, int f, const int *helpers,
                         const uint8_t *const *received, uint8_t *const *out, size_t nbytes,
                         pmrc_stream_t stream) {
  PMRC_TRACE("pmrc_repair_newcomer");
  if (!c || !helpers || !received || !out) return fail(PMRC_EINVAL, "NULL argument");
  if (is16(c)) {
    if (nbytes % 2) return fail(PMRC_EINVAL, "GF(2^16) blocks hold whole 2-byte symbols");
    for (int j = 0; j < c->m.f16.alpha; j++)
      if (!out[j]) return fail(PMRC_EINVAL, "output block is NULL");
    auto in8 = split_in(received, c->m.d, nbytes / 2);
    auto out8 = split_out(out, c->m.f16.alpha, nbytes / 2);
    return repair_newcomer_body(c, f, helpers, in8.data(), out8.data(), nbytes / 2, stream);
  }
  return repair_newcomer_body(c, f, helpers, received, out, nbytes, stream);
}

int pmrc_repair(const pmrc_code *c, int f, const int *helpers, const uint8_t *const *blocks,
                uint8_t *const *out, size_t nbytes, pmrc_stream_t stream) {
  PMRC_TRACE("pmrc_repair");
  if (!c || !helpers || !blocks || !out) return fail(PMRC_EINVAL, "NULL argument");
  if (is16(c)) return not_for16("pmrc_repair (fused)");
  if (c->m.alpha > 16) return fail(PMRC_EUNSUPPORTED, "pmrc_repair needs alpha <= 16");
  std::string err;
  if (c->m.construction == kConsRs) {
    // one block per node and helper coefficient 1: the projections are the
    // helpers' blocks themselves, so the repair is the newcomer's 1 x k row
    // applied to them
    if (!out[0]) return fail(PMRC_EINVAL, "output block is NULL");
    std::shared_ptr<Plan> np;
    int rc = newcomer_plan(c, f, helpers, np, err);
    if (!rc) rc = launch_region(*np, blocks, out, nbytes, (cudaStream_t)stream, err);
    return rc ? fail(rc, err) : PMRC_OK;
  }
  std::shared_ptr<FusedRepairPlan> p;
  int rc = fused_repair_plan(c, f, helpers, p, err);
  if (rc) return fail(rc, err);
  const cudaStream_t st = (cudaStream_t)stream;
  const int a = c->m.alpha, d = c->m.d;
  size_t done = 0;
  // bitsliced fused repair, compiled at run time per (failed node, helpers):
  // projections as XORs of bit planes kept in registers, applied straight
  // to the newcomer matrix
  if (a <= 8 && want_runtime(c, c->decode_kernel, nbytes, kRuntimeRepairMinBytes)) {
    std::vector<uint8_t> phi;
    helper_coefficients(c->m, f, phi);
    bool aligned = true;
    for (int q = 0; q < d && aligned; q++)
      for (int j = 0; j < a; j++)
        if (phi[j]) aligned = aligned && blocks[q * a + j] && (uintptr_t)blocks[q * a + j] % 16 == 0;
    for (int r = 0; r < a && aligned; r++) aligned = out[r] && (uintptr_t)out[r] % 16 == 0;
    std::string rerr;
    std::shared_ptr<BsRuntimeKernel> k;
    if (aligned) k = fused_runtime(c, f, helpers, c->decode_kernel != PMRC_KERNEL_BITSLICED, rerr);
    if (k) {
      done = nbytes & ~(size_t)31;
      const cudaError_t e = bitslice_launch_fused_repair(*k, blocks, out, done, st);
      if (e != cudaSuccess)
        return fail(PMRC_ECUDA, std::string("bitsliced repair launch: ") + cudaGetErrorString(e));
    }
  }
  if (done == nbytes) return PMRC_OK;
  if (done == 0) {
    rc = launch_fused_repair(*p, blocks, out, nbytes, st, err);
  } else {  // ragged tail of the blocks
    std::vector<const uint8_t *> in2(d * a);
    std::vector<uint8_t *> out2(a);
    for (int i = 0; i < d * a; i++) in2[i] = blocks[i] ? blocks[i] + done : nullptr;
    for (int r = 0; r < a; r++) out2[r] = out[r] + done;
    rc = launch_fused_repair(*p, in2.data(), out2.data(), nbytes - done, st, err);
  }
  return rc ? fail(rc, err) : PMRC_OK;
}

int pmrc_read_degraded(const pmrc_code *c, int node, const int *helpers,
                       const uint8_t *const *blocks, uint8_t *const *out, size_t offset,
                       size_t length, pmrc_stream_t stream) {
  PMRC_TRACE("pmrc_read_degraded");
  if (!c || !helpers || !blocks || !out) return fail(PMRC_EINVAL, "NULL argument");
  if (!c->m.systematic) return fail(PMRC_EINVAL, "degraded reads need a systematic handle");
  if (node < 0 || node >= c->m.k) return fail(PMRC_EINVAL, "node is not a systematic node");
  const int nb = c->m.d * (is16(c) ? c->m.f16.alpha : c->m.alpha);
  std::vector<const uint8_t *> shifted(nb);
  for (int i = 0; i < nb; i++) shifted[i] = blocks[i] ? blocks[i] + offset : nullptr;
  return pmrc_repair(c, node, helpers, shifted.data(), out, length, stream);
}

int pmrc_repair_noalloc(const pmrc_code *c, int f, const int *helpers,
                        const uint8_t *const *blocks, uint8_t *const *out, size_t nbytes,
                        pmrc_stream_t stream) {
  if (!c || !helpers || !blocks || !out) return fail(PMRC_EINVAL, "NULL argument");
  if (is16(c)) return not_for16("pmrc_repair_noalloc");
  if (c->m.alpha > 16) return fail(PMRC_EUNSUPPORTED, "pmrc_repair_noalloc needs alpha <= 16");
  std::shared_ptr<FusedRepairPlan> p;
  std::string err;
  int rc = fused_repair_plan(c, f, helpers, p, err);
  if (rc) return fail(rc, err);
  rc = launch_fused_repair_noalloc(*p, blocks, out, nbytes, (cudaStream_t)stream, err);
  return rc ? fail(rc, err) : PMRC_OK;
}

int pmrc_decode(const pmrc_code *c, const int *nodes, const uint8_t *const *node_blocks,
                uint8_t *const *data_out, size_t nbytes, pmrc_stream_t stream) {
  PMRC_TRACE("pmrc_decode");
  if (!c || !nodes || !node_blocks || !data_out) return fail(PMRC_EINVAL, "NULL argument");
  {
    std::vector<char> seen(c->m.n, 0);
    for (int i = 0; i < c->m.k; i++) {
      if (nodes[i] < 0 || nodes[i] >= c->m.n || seen[nodes[i]])
        return fail(PMRC_EINVAL, "nodes: out of range or repeated node id");
      seen[nodes[i]] = 1;
    }
  }
  if (is16(c)) {
    if (nbytes % 2) return fail(PMRC_EINVAL, "GF(2^16) blocks hold whole 2-byte symbols");
    auto in8 = split_in(node_blocks, c->m.k * c->m.f16.alpha, nbytes / 2);
    auto out8 = split_out(data_out, c->m.f16.K, nbytes / 2);
    return decode_body(c, nodes, in8.data(), out8.data(), nbytes / 2, stream);
  }
  return decode_body(c, nodes, node_blocks, data_out, nbytes, stream);
}

}  // extern "C"

namespace {

// The rows pmrc_encode writes: every row of the code's generator
// (non-systematic form) or the parity nodes' rows of G' (systematic form).
void encode_matrix(const pmrc_code *c, Mat &M) {
  const int K = c->m.K, N = c->m.N, first = c->m.systematic ? c->m.k * c->m.alpha : 0;
  M = Mat(N - first, K);
  std::copy(c->m.Gcode.v.begin() + (size_t)first * K, c->m.Gcode.v.end(), M.v.begin());
}

// Moves a finished compilation into the handle's kernel cache (loading its
// cubin on the calling thread) and returns the kernel, or null with the
// reason in err.  Caller holds c->mu.
std::shared_ptr<BsRuntimeKernel> finish_job(const pmrc_code *c, const std::string &key,
                                            BsJob &job, std::string &err) {
  auto it = c->rt.find(key);
  if (it == c->rt.end()) {  // not yet moved by another thread
    std::shared_ptr<BsRuntimeKernel> k;
    std::string e = job.err;
    if (!job.rc) bitslice_load(job.out, k, e);
    if (c->rt.size() >= kPlanCacheCap) {
      if (c->rt.begin()->second) c->rt_retired.push_back(c->rt.begin()->second);
      c->rt_err.erase(c->rt.begin()->first);
      c->rt.erase(c->rt.begin());
    }
    it = c->rt.emplace(key, k).first;
    if (!k) c->rt_err[key] = e;
  }
  c->rt_jobs.erase(key);
  if (!it->second) err = c->rt_err[key];
  return it->second;
}

using BsCompileFn = std::function<int(BsCompiled &, std::string &)>;

// A bitsliced kernel compiled at run time, cached in the handle under `key`;
// null when it cannot be built (the reason in err, also cached).  `prepare`
// runs on the calling thread: it checks the request and returns the
// compilation to run (or an error code, cached as a failed key).  In the
// background (AUTO policies) the first call only starts the compilation and
// returns null with an empty err, as do later calls until it has finished:
// the caller runs the split-table kernel meanwhile.
std::shared_ptr<BsRuntimeKernel> runtime_kernel_job(
    const pmrc_code *c, const std::string &key,
    const std::function<int(BsCompileFn &, std::string &)> &prepare, std::string &err,
    bool background) {
  std::shared_ptr<BsJob> job;
  {
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->rt.find(key);
    if (it != c->rt.end()) {
      if (!it->second) err = c->rt_err[key];
      return it->second;
    }
    auto jt = c->rt_jobs.find(key);
    if (jt != c->rt_jobs.end()) job = jt->second;
  }
  if (!job) {
    BsCompileFn compile;
    const int rc = prepare(compile, err);
    if (rc) {
      std::lock_guard<std::mutex> g(c->mu);
      c->rt[key] = nullptr;
      c->rt_err[key] = err;
      return nullptr;
    }
    auto fresh = std::make_shared<BsJob>();
    {
      std::lock_guard<std::mutex> g(c->mu);
      auto jt = c->rt_jobs.find(key);
      if (jt != c->rt_jobs.end()) {  // another thread started it meanwhile
        job = jt->second;
      } else {
        job = fresh;
        c->rt_jobs[key] = job;
      }
    }
    if (job == fresh) {
      auto work = [job, compile]() {
        BsCompiled out;
        std::string e;
        const int rc = compile(out, e);
        {
          std::lock_guard<std::mutex> g(job->mu);
          job->rc = rc;
          job->err = e;
          job->out = std::move(out);
          job->done = true;
        }
        job->cv.notify_all();
      };
      if (background)
        jit_background(work);
      else
        work();
    }
  }
  {
    std::unique_lock<std::mutex> lk(job->mu);
    if (background && !job->done) {
      err.clear();
      return nullptr;
    }
    job->cv.wait(lk, [&] { return job->done; });
  }
  std::lock_guard<std::mutex> g(c->mu);
  return finish_job(c, key, *job, err);
}

// A bitsliced kernel compiled at run time for matrix M (blocks of rows of
// identical support when by_support, else consecutive rows); see
// runtime_kernel_job.
std::shared_ptr<BsRuntimeKernel> runtime_kernel(const pmrc_code *c, const std::string &key,
                                                const char *role,
                                                const std::function<int(Mat &, std::string &)> &make,
                                                std::string &err, bool by_support, bool background) {
  return runtime_kernel_job(c, key, [&](BsCompileFn &compile, std::string &e) {
    Mat M;
    int rc = make(M, e);
    if (!rc && M.rows == 0) {
      e = "no rows to compute";
      rc = kEUnsupported;
    }
    if (rc) return rc;
    compile = [M, by_support, role](BsCompiled &out, std::string &e2) {
      return bitslice_compile(M.v.data(), M.rows, M.cols, kRuntimeMaxInputs, by_support, role, out,
                              e2);
    };
    return (int)kOk;
  }, err, background);
}

// Bitsliced helper projections for failed node f (one kernel serves any
// number of helpers: phi_f is the same for all of them).
std::shared_ptr<BsRuntimeKernel> projection_runtime(const pmrc_code *c, int f, bool background,
                                                    std::string &err) {
  return runtime_kernel_job(c, "p:" + std::to_string(f), [&](BsCompileFn &compile, std::string &) {
    std::vector<uint8_t> phi;
    helper_coefficients(c->m, f, phi);
    const int alpha = c->m.alpha;
    compile = [phi, alpha](BsCompiled &out, std::string &e2) {
      return bitslice_compile_projection(phi.data(), alpha, "project", out, e2);
    };
    return (int)kOk;
  }, err, background);
}

// Bitsliced fused repair of failed node f from `helpers` (alpha <= 8).
std::shared_ptr<BsRuntimeKernel> fused_runtime(const pmrc_code *c, int f, const int *helpers,
                                               bool background, std::string &err) {
  std::string key = "r:" + std::to_string(f);
  for (int i = 0; i < c->m.d; i++) key += "," + std::to_string(helpers[i]);
  return runtime_kernel_job(c, key, [&](BsCompileFn &compile, std::string &e) {
    Mat D;
    const int rc = newcomer_matrix(c->m, f, helpers, D, e);
    if (rc) return rc;
    std::vector<uint8_t> phi;
    helper_coefficients(c->m, f, phi);
    const int alpha = c->m.alpha, d = c->m.d;
    compile = [phi, alpha, D, d](BsCompiled &out, std::string &e2) {
      return bitslice_compile_fused_repair(phi.data(), alpha, D.v.data(), d, "repair", out, e2);
    };
    return (int)kOk;
  }, err, background);
}

// Bitsliced reconstruction rows for this (nodes, wanted rows).
std::shared_ptr<BsRuntimeKernel> decode_runtime(const pmrc_code *c, const int *nodes,
                                                const std::vector<char> &want, bool background,
                                                std::string &err) {
  std::string key = "d:";
  for (int i = 0; i < c->m.k; i++) key += std::to_string(nodes[i]) + ",";
  key += ":";
  for (char w : want) key += w ? '1' : '0';
  return runtime_kernel(c, key, "decode", [&](Mat &M, std::string &e) {
    Mat R;
    int rc = decode_matrix(c->m, nodes, R, e);
    if (rc) return rc;
    std::vector<int> rows;
    for (int r = 0; r < c->m.K; r++)
      if (want[r]) rows.push_back(r);
    M = Mat((int)rows.size(), R.cols);
    for (size_t q = 0; q < rows.size(); q++)
      for (int col = 0; col < R.cols; col++) M.at((int)q, col) = R.at(rows[q], col);
    return (int)kOk;
  }, err, false, background);
}

// ALU lane-ops per 32-byte column of a bitsliced schedule (the kernels'
// instruction model: per block, 44 per input -- 24 transpose + 20 subset
// tables -- or 20 for a plane-layout input, 24 per output row unless it is
// stored in plane layout; 8 per non-zero coefficient).
long long schedule_cost(const Mat &M, const std::vector<BsBlock> &blks, bool in_planes,
                        bool out_planes) {
  long long c = 0;
  for (const BsBlock &B : blks)
    c += (long long)B.inputs.size() * (in_planes ? 20 : 44) + (out_planes ? 0 : 24 * (long long)B.rows.size());
  for (uint8_t v : M.v) c += v ? 8 : 0;
  return c;
}

bool blocks_fit(const std::vector<BsBlock> &blks, int rows, int cols) {
  if (rows <= 0 || cols <= 0 || rows + cols > bitslice_max_pointers()) return false;
  for (const BsBlock &B : blks)
    if ((int)B.inputs.size() > kRuntimeMaxInputs) return false;
  return true;
}

// The factored reconstruction of a systematic GF(2^8) code for these nodes
// and wanted rows: Z (all of z), W restricted to the wanted rows, their
// blocks, and the wanted data rows in W's order.  False when the code has no
// such form, no data row is missing, or a wanted row is a present data row
// (a copy the factored kernels do not make).
struct Factored {
  Mat Z, W;
  std::vector<int> own, rows;
  std::vector<BsBlock> zb, wb;
};

bool factored_form(const pmrc_code *c, const int *nodes, const std::vector<char> &want, Factored &F) {
  if (c->m.w != 8 || !c->m.systematic || c->m.construction == kConsMbr) return false;
  Mat Wall;
  std::vector<int> mcols;
  std::string e;
  if (decode_factors(c->m, nodes, F.Z, Wall, mcols, F.own, e) || mcols.empty()) return false;
  std::vector<int> at(c->m.K, -1);
  for (size_t i = 0; i < mcols.size(); i++) at[mcols[i]] = (int)i;
  std::vector<int> wi;
  for (int r = 0; r < c->m.K; r++)
    if (want[r]) {
      if (at[r] < 0) return false;
      wi.push_back(at[r]);
      F.rows.push_back(r);
    }
  if (wi.empty()) return false;
  const int m = (int)mcols.size();
  F.W = Mat((int)wi.size(), m);
  for (size_t q = 0; q < wi.size(); q++)
    for (int s2 = 0; s2 < m; s2++) F.W.at((int)q, s2) = Wall.at(wi[q], s2);
  F.zb = bs_blocks_grouped(F.Z.v.data(), m, F.Z.cols, F.own, kRuntimeMaxInputs);
  F.wb = bs_blocks_chunked(F.W.v.data(), F.W.rows, m);
  return true;
}

std::string nodes_key(const pmrc_code *c, const char *tag, const int *nodes) {
  std::string key = tag;
  for (int i = 0; i < c->m.k; i++) key += std::to_string(nodes[i]) + ",";
  return key;
}

std::string want_key(const std::vector<char> &want) {
  std::string key = ":";
  for (char w : want) key += w ? '1' : '0';
  return key;
}

// Whether a reconstruction of nbytes-byte blocks takes the factored
// two-launch kernels: their estimated work plus the second launch's cost
// (about 2 us of the GPU's ALU issue, 1227 lane-ops per column at 1 MiB)
// below the one-launch schedule's, or the one-launch schedule does not fit
// a launch.  The estimates are kept per (nodes, wanted rows).
bool prefer_factored(const pmrc_code *c, const int *nodes, const std::vector<char> &want,
                     size_t nbytes) {
  const std::string key = nodes_key(c, "", nodes) + want_key(want);
  std::pair<long long, long long> cost;
  bool known;
  {
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->decode_costs.find(key);
    known = it != c->decode_costs.end();
    if (known) cost = it->second;
  }
  if (!known) {
    cost = {-1, -1};
    Factored F;
    if (factored_form(c, nodes, want, F) && blocks_fit(F.zb, F.Z.rows, F.Z.cols) &&
        blocks_fit(F.wb, F.W.rows, F.W.cols))
      cost.second = schedule_cost(F.Z, F.zb, false, true) + schedule_cost(F.W, F.wb, true, false);
    Mat R;
    std::string e;
    if (cost.second >= 0 && !decode_matrix(c->m, nodes, R, e)) {
      std::vector<int> rows;
      for (int r = 0; r < c->m.K; r++)
        if (want[r]) rows.push_back(r);
      Mat M((int)rows.size(), R.cols);
      for (size_t q = 0; q < rows.size(); q++)
        for (int col = 0; col < R.cols; col++) M.at((int)q, col) = R.at(rows[q], col);
      const auto blks = bs_blocks_chunked(M.v.data(), M.rows, M.cols);
      if (blocks_fit(blks, M.rows, M.cols)) cost.first = schedule_cost(M, blks, false, false);
    }
    std::lock_guard<std::mutex> g(c->mu);
    if (c->decode_costs.size() >= kPlanCacheCap) c->decode_costs.erase(c->decode_costs.begin());
    c->decode_costs[key] = cost;
  }
  if (cost.second < 0) return false;
  if (cost.first < 0) return true;
  const double launch = 1227.0 * (double)(1u << 20) / (double)std::max<size_t>(nbytes, 1);
  return (double)cost.second + launch < (double)cost.first;
}

// The two run-time kernels of the factored reconstruction (stage 1 "fz":
// z = Z y stored in plane layout; stage 2 "fw": the wanted rows of W z), or
// false while either is compiling (background) or when one cannot be built.
bool factored_runtime(const pmrc_code *c, const int *nodes, const std::vector<char> &want,
                      bool background, std::shared_ptr<BsRuntimeKernel> &kz,
                      std::shared_ptr<BsRuntimeKernel> &kw, std::vector<int> &rows, int &m,
                      std::string &err) {
  const std::string zkey = nodes_key(c, "fz:", nodes), wkey = nodes_key(c, "fw:", nodes) + want_key(want);
  rows.clear();
  for (int r = 0; r < c->m.K; r++)  // the second launch writes the wanted rows in this order
    if (want[r]) rows.push_back(r);
  {  // both kernels loaded: no host work beyond the lookups
    std::lock_guard<std::mutex> g(c->mu);
    auto iz = c->rt.find(zkey), iw = c->rt.find(wkey);
    if (iz != c->rt.end() && iw != c->rt.end() && iz->second && iw->second) {
      kz = iz->second;
      kw = iw->second;
      m = bitslice_outputs(*kz);
      return true;
    }
  }
  Factored F;
  if (!factored_form(c, nodes, want, F)) {
    err = "no factored form";
    return false;
  }
  m = F.Z.rows;
  kz = runtime_kernel_job(c, zkey, [&](BsCompileFn &compile, std::string &) {
    const Mat Z = F.Z;
    const std::vector<BsBlock> zb = F.zb;
    compile = [Z, zb](BsCompiled &out, std::string &e2) {
      return bitslice_compile_stage(Z.v.data(), Z.rows, Z.cols, zb, kRuntimeMaxInputs, false, true,
                                    "dstage1", out, e2);
    };
    return (int)kOk;
  }, err, background);
  kw = runtime_kernel_job(c, wkey, [&](BsCompileFn &compile, std::string &) {
    const Mat W = F.W;
    const std::vector<BsBlock> wb = F.wb;
    compile = [W, wb](BsCompiled &out, std::string &e2) {
      return bitslice_compile_stage(W.v.data(), W.rows, W.cols, wb, kRuntimeMaxInputs, true, false,
                                    "dstage2", out, e2);
    };
    return (int)kOk;
  }, err, background);
  return kz && kw;
}

// Stream-ordered device scratch of the library's own (one pool per device,
// nothing released between calls): the intermediate of a two-launch
// product, allocated and freed in the order of the call's stream.
cudaError_t scratch_alloc(void **p, size_t n, cudaStream_t st) {
  static std::mutex mu;
  static cudaMemPool_t pools[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> g(mu);
    if (!pools[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pools[dev], &props);
      if (e != cudaSuccess) {
        pools[dev] = nullptr;
        return e;
      }
      uint64_t keep = UINT64_MAX;
      e = cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) return e;
    }
    pool = pools[dev];
  }
  return cudaMallocFromPoolAsync(p, n, pool, st);
}

// Whether a call of nbytes takes a run-time bitsliced kernel under the
// handle's policy (GF(2^8) codes only; AUTO from auto_min bytes per block).
bool want_runtime(const pmrc_code *c, int policy, size_t nbytes, size_t auto_min) {
  return c->m.w == 8 && nbytes >= 32 &&
         (policy == PMRC_KERNEL_BITSLICED || (policy == PMRC_KERNEL_AUTO && nbytes >= auto_min));
}

int decode_body(const pmrc_code *c, const int *nodes, const uint8_t *const *node_blocks,
                uint8_t *const *data_out, size_t nbytes, pmrc_stream_t stream) {
  std::vector<char> want;
  decode_wanted(c, nodes, node_blocks, data_out, want);
  std::shared_ptr<Plan> p;
  std::string err;
  int rc = decode_plan(c, nodes, want, p, err);
  if (rc) return fail(rc, err);
  for (int in : plan_reads(*p))
    if (!node_blocks[in]) return fail(PMRC_EINVAL, "a node block the reconstruction reads is NULL");
  const cudaStream_t st = (cudaStream_t)stream;
  size_t done = 0;
  // bitsliced path: reconstruction rows compiled at run time (GF(2^8)
  // codes; AUTO for blocks of at least kRuntimeMinBytes)
  const bool forced = c->decode_kernel == PMRC_KERNEL_BITSLICED;
  if (want_runtime(c, c->decode_kernel, nbytes, kRuntimeMinBytes)) {
    std::vector<int> rows;
    for (int r = 0; r < c->m.K; r++)
      if (want[r]) rows.push_back(r);
    const int KA = c->m.k * c->m.alpha;
    bool aligned = !rows.empty();
    for (int i = 0; i < KA && aligned; i++)
      aligned = !node_blocks[i] || (uintptr_t)node_blocks[i] % 16 == 0;
    for (int r : rows) aligned = aligned && (uintptr_t)data_out[r] % 16 == 0;
    std::string rerr;
    if (aligned && prefer_factored(c, nodes, want, nbytes)) {
      // x_M = W (Z y): the received parity blocks plus their present-data
      // terms, then B^-1, as two launches through a plane-layout
      // intermediate in stream-ordered scratch
      std::shared_ptr<BsRuntimeKernel> kz, kw;
      std::vector<int> frows;
      int m = 0;
      if (factored_runtime(c, nodes, want, !forced, kz, kw, frows, m, rerr)) {
        const size_t cut = nbytes & ~(size_t)31;
        void *zbuf = nullptr;
        cudaError_t e = scratch_alloc(&zbuf, (size_t)m * cut, st);
        if (e != cudaSuccess)
          return fail(PMRC_ENOMEM, std::string("reconstruction scratch: ") + cudaGetErrorString(e));
        std::vector<uint8_t *> z(m);
        for (int i = 0; i < m; i++) z[i] = static_cast<uint8_t *>(zbuf) + (size_t)i * cut;
        std::vector<const uint8_t *> zin(z.begin(), z.end());
        std::vector<uint8_t *> outs;
        for (int r : frows) outs.push_back(data_out[r]);
        e = bitslice_launch_runtime(*kz, node_blocks, z.data(), cut, st);
        if (e == cudaSuccess) e = bitslice_launch_runtime(*kw, zin.data(), outs.data(), cut, st, true);
        const cudaError_t fe = cudaFreeAsync(zbuf, st);
        if (e == cudaSuccess) e = fe;
        if (e != cudaSuccess)
          return fail(PMRC_ECUDA, std::string("bitsliced reconstruction launch: ") + cudaGetErrorString(e));
        done = cut;
      } else if (forced) {
        return fail(PMRC_EUNSUPPORTED, "bitsliced reconstruction: " + rerr);
      }
      aligned = false;  // not the one-launch schedule: done, or the split-table kernel meanwhile
    }
    std::shared_ptr<BsRuntimeKernel> k =
        aligned ? decode_runtime(c, nodes, want, !forced, rerr) : nullptr;
    if (!k && forced && done == 0)
      return fail(PMRC_EUNSUPPORTED, aligned ? "bitsliced reconstruction: " + rerr
                                             : "bitsliced reconstruction needs 16-byte aligned blocks");
    if (k) {
      std::vector<uint8_t *> outs;
      for (int r : rows) outs.push_back(data_out[r]);
      done = nbytes & ~(size_t)31;
      const cudaError_t e = bitslice_launch_runtime(*k, node_blocks, outs.data(), done, st);
      if (e != cudaSuccess)
        return fail(PMRC_ECUDA, std::string("bitsliced reconstruction launch: ") + cudaGetErrorString(e));
    }
  }
  if (done == nbytes) return PMRC_OK;
  if (done == 0) {
    rc = launch_region(*p, node_blocks, data_out, nbytes, st, err);
  } else {  // ragged tail of the blocks
    const int KA = c->m.k * c->m.alpha;
    std::vector<const uint8_t *> in2(KA);
    std::vector<uint8_t *> out2(c->m.K);
    for (int i = 0; i < KA; i++) in2[i] = node_blocks[i] ? node_blocks[i] + done : nullptr;
    for (int r = 0; r < c->m.K; r++) out2[r] = data_out[r] ? data_out[r] + done : nullptr;
    rc = launch_region(*p, in2.data(), out2.data(), nbytes - done, st, err);
  }
  return rc ? fail(rc, err) : PMRC_OK;
}

}  // namespace

extern "C" {

size_t pmrc_specific_workspace_bytes(const pmrc_code *c, size_t block_bytes) {
  if (!c || c->m.construction > 1 || is16(c)) return 0;  // PM-MSR over GF(2^8) only
  return specific_workspace_blocks(c->m) * specific_pitch(block_bytes);
}

}  // extern "C"

namespace {

int specific_plan(const pmrc_code *c, const int *nodes, bool precode, const std::vector<char> &want,
                  std::shared_ptr<SpecificPlan> &out, std::string &err) {
  std::string key = precode ? "P:" : "D:";
  for (int i = 0; i < c->m.k; i++) key += std::to_string(nodes[i]) + ",";
  key += ":";
  for (char w : want) key += w ? '1' : '0';
  {
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->specific.find(key);
    if (it != c->specific.end()) {
      out = it->second;
      return kOk;
    }
  }
  auto sp = std::make_shared<SpecificPlan>();
  int rc = build_specific(c->m, nodes, precode, want, *sp, err);
  if (rc) return rc;
  std::lock_guard<std::mutex> g(c->mu);
  if (c->specific.size() >= kPlanCacheCap) c->specific.erase(c->specific.begin());
  c->specific[key] = sp;
  out = sp;
  return kOk;
}

// The stage launches, in stream order, over the workspace (see specific.h).
int run_specific(const pmrc_code *c, SpecificPlan &sp, const uint8_t *const *in_blocks,
                 uint8_t *const *final_out, size_t nbytes, uint8_t *ws, cudaStream_t s,
                 std::string &err) {
  const size_t pitch = specific_pitch(nbytes);
  auto blocks = [&](uint8_t *base, int count) {
    std::vector<uint8_t *> v(count);
    for (int i = 0; i < count; i++) v[i] = base + (size_t)i * pitch;
    return v;
  };
  std::vector<uint8_t *> w0 = blocks(ws, sp.w0);
  std::vector<uint8_t *> w1 = blocks(ws + (size_t)sp.w0 * pitch, sp.w1);
  std::vector<uint8_t *> w2 = blocks(ws + (size_t)(sp.w0 + sp.w1) * pitch, sp.w2);
  auto cin = [](const std::vector<uint8_t *> &v) {
    return std::vector<const uint8_t *>(v.begin(), v.end());
  };
  int rc = launch_region(*sp.A, in_blocks, w0.data(), nbytes, s, err);
  if (!rc) rc = launch_region(*sp.PQ, cin(w0).data(), w1.data(), nbytes, s, err);
  if (!rc) rc = launch_region(*sp.UV, cin(w1).data(), w0.data(), nbytes, s, err);
  if (!rc) rc = launch_region(*sp.S, cin(w0).data(), sp.X || c->m.systematic ? w2.data() : final_out,
                              nbytes, s, err);
  if (!rc && sp.X) rc = launch_region(*sp.X, cin(w2).data(), final_out, nbytes, s, err);
  return rc;
}

}  // namespace

extern "C" {

int pmrc_decode_specific(const pmrc_code *c, const int *nodes, const uint8_t *const *node_blocks,
                         uint8_t *const *data_out, size_t nbytes, void *workspace,
                         size_t workspace_bytes, pmrc_stream_t stream) {
  PMRC_TRACE("pmrc_decode_specific");
  if (!c || !nodes || !node_blocks || !data_out) return fail(PMRC_EINVAL, "NULL argument");
  if (c->m.construction > 1)
    return fail(PMRC_EUNSUPPORTED, "the data collector of this library is the PM-MSR one");
  if (is16(c)) return not_for16("pmrc_decode_specific");
  {
    std::vector<char> seen(c->m.n, 0);
    for (int i = 0; i < c->m.k; i++) {
      if (nodes[i] < 0 || nodes[i] >= c->m.n || seen[nodes[i]])
        return fail(PMRC_EINVAL, "nodes: out of range or repeated node id");
      seen[nodes[i]] = 1;
    }
  }
  if (nbytes == 0) return PMRC_OK;
  if (!workspace || workspace_bytes < pmrc_specific_workspace_bytes(c, nbytes))
    return fail(PMRC_EINVAL, "workspace is NULL or smaller than pmrc_specific_workspace_bytes");
  std::vector<char> want;
  decode_wanted(c, nodes, node_blocks, data_out, want);
  std::shared_ptr<SpecificPlan> sp;
  std::string err;
  int rc = specific_plan(c, nodes, false, want, sp, err);
  if (rc) return fail(rc, err);
  const cudaStream_t s = (cudaStream_t)stream;
  rc = run_specific(c, *sp, node_blocks, data_out, nbytes, (uint8_t *)workspace, s, err);
  if (rc) return fail(rc, err);
  const int a = c->m.alpha;
  for (int r : sp->copy_rows) {  // data rows held by a listed node, not aliased
    int pos = 0;
    while (nodes[pos] != r / a) pos++;
    const cudaError_t e = cudaMemcpyAsync(data_out[r], node_blocks[a * pos + r % a], nbytes,
                                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(PMRC_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
  }
  return PMRC_OK;
}

int pmrc_encode_precode(const pmrc_code *c, const uint8_t *const *data, uint8_t *const *parity,
                        size_t nbytes, void *workspace, size_t workspace_bytes,
                        pmrc_stream_t stream) {
  PMRC_TRACE("pmrc_encode_precode");
  if (!c || !data || !parity) return fail(PMRC_EINVAL, "NULL argument");
  if (c->m.construction > 1)
    return fail(PMRC_EUNSUPPORTED, "precode encode is the PM-MSR systematic construction");
  if (is16(c)) return not_for16("pmrc_encode_precode");
  if (!c->m.systematic)
    return fail(PMRC_EINVAL, "precode encode produces a systematic code's parity");
  const int K = c->m.k * c->m.alpha, NP = (c->m.n - c->m.k) * c->m.alpha;
  for (int i = 0; i < K; i++)
    if (!data[i]) return fail(PMRC_EINVAL, "data block is NULL");
  for (int j = 0; j < NP; j++)
    if (!parity[j]) return fail(PMRC_EINVAL, "parity block is NULL");
  if (nbytes == 0) return PMRC_OK;
  if (!workspace || workspace_bytes < pmrc_specific_workspace_bytes(c, nbytes))
    return fail(PMRC_EINVAL, "workspace is NULL or smaller than pmrc_specific_workspace_bytes");
  std::vector<int> nodes(c->m.k);
  for (int i = 0; i < c->m.k; i++) nodes[i] = i;
  std::shared_ptr<SpecificPlan> sp;
  std::string err;
  int rc = specific_plan(c, nodes.data(), true, std::vector<char>(K, 1), sp, err);
  if (rc) return fail(rc, err);
  rc = run_specific(c, *sp, data, parity, nbytes, (uint8_t *)workspace, (cudaStream_t)stream, err);
  return rc ? fail(rc, err) : PMRC_OK;
}

}  // extern "C"
