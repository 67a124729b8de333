// Serving loop: continuous batching of encode, repair and reconstruction
// requests on one GPU.
//
// A scheduler thread owns a compute stream, kCopyLanes streams for each copy
// direction and a device arena whose size is the HBM budget.  Each pass of
// its loop:
//   1. admits queued requests in arrival order while a slot is free and the
//      arena has room for the request's inputs and outputs (first fit);
//      their input copies start at once, each on the host-to-device stream
//      with the fewest bytes queued;
//   2. marks requests whose inputs have landed as ready;
//   3. when fewer than two iterations are in flight, launches one iteration:
//      the work items of every ready request (batch.cu's persistent kernel)
//      in one launch, plus one built-in bitsliced launch per large encode,
//      followed by the output copies of those requests, each on the
//      device-to-host stream with the fewest bytes queued;
//   4. retires requests whose outputs are back: frees their arena range and
//      records submit-to-completion latency.
// Requests that arrive while an iteration runs are admitted and copied in
// meanwhile and join the next iteration, so transfers overlap compute and
// the work of many requests overlaps in one launch.  Coefficient plans are
// built at submission, on the caller's thread, and stay on the device in the
// code handles.  All waits on the device are event queries polled by the
// host: no device-side wait exists.
#include <cuda_runtime.h>

#include "trace.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pmrc.h"
#include "api_internal.h"
#include "batch_internal.h"
#include "bitslice.h"

using namespace pmrc;

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kAlign = 256;
constexpr int kCopyLanes = 4;  // copy streams per direction

// The copy stream with the fewest bytes queued.
int least_queued(const size_t *queued) {
  int best = 0;
  for (int l = 1; l < kCopyLanes; l++)
    if (queued[l] < queued[best]) best = l;
  return best;
}

// First-fit allocator over [0, size) with coalescing free list.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size) { free_[0] = size; }
  bool alloc(size_t n, size_t &off) {
    n = (n + kAlign - 1) & ~(kAlign - 1);
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= n) {
        off = it->first;
        const size_t rest = it->second - n;
        free_.erase(it);
        if (rest) free_[off + n] = rest;
        used_ += n;
        peak_ = std::max(peak_, used_);
        return true;
      }
    return false;
  }
  void release(size_t off, size_t n) {
    n = (n + kAlign - 1) & ~(kAlign - 1);
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }
  size_t peak() const { return peak_; }

 private:
  size_t size_, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;
};

enum State { kQueued, kCopyIn, kReady, kRunning, kDone, kFailed, kCancelled };

struct Req {
  uint64_t id = 0;
  int op = 0;
  const pmrc_code *code = nullptr;
  size_t B = 0;
  const uint8_t *in = nullptr;
  uint8_t *out = nullptr;
  bool device = false;  // in/out are the caller's device blocks (no arena, no copies)
  int failed = -1;
  std::vector<int> helpers, nodes;
  size_t in_bytes = 0, out_bytes = 0, nin = 0, nout = 0;
  size_t in_span = 0;  // in_bytes rounded up: outputs start 256-byte aligned
  size_t off = 0;
  int in_lane = -1, out_lane = -1;  // copy streams carrying the input / output copy
  int64_t user_bytes = 0;
  State state = kQueued;
  int status = PMRC_OK;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  Clock::time_point t_submit, t_done;
};

struct Iteration {
  cudaEvent_t done = nullptr;  // kernel finished
  std::vector<Req *> reqs;
  std::vector<WorkStripe> stripes;  // keeps the plans the kernel reads alive
  int buf = 0;
};

}  // namespace

struct pmrc_server {
  int device = 0;
  int max_slots = 0;
  uint8_t *arena_base = nullptr;
  std::unique_ptr<Arena> arena;
  // copies run on several streams per direction: one copy's fixed latency
  // overlaps the others', and a small request's copy need not queue behind
  // a large one; each copy goes to the stream with the fewest bytes queued
  cudaStream_t s_in[kCopyLanes] = {}, s_out[kCopyLanes] = {}, s_comp = nullptr;
  size_t in_queued[kCopyLanes] = {}, out_queued[kCopyLanes] = {};
  // double-buffered work lists in mapped pinned host memory: the kernel
  // reads them in place, so launching an iteration queues no copy behind
  // the requests' input copies on the copy engines
  unsigned *d_counter[2] = {nullptr, nullptr};
  WorkItem *h_items[2] = {nullptr, nullptr};
  uint8_t **h_ptrs[2] = {nullptr, nullptr};
  const WorkItem *m_items[2] = {nullptr, nullptr};  // device addresses of h_items, h_ptrs
  uint8_t *const *m_ptrs[2] = {nullptr, nullptr};
  cudaEvent_t buf_free[2] = {nullptr, nullptr};
  size_t item_cap = 0, ptr_cap = 0;
  int sms = 1;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req *> queue;
  std::vector<Req *> active;
  std::map<uint64_t, std::unique_ptr<Req>> reqs;
  std::deque<Iteration> inflight;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  int next_buf = 0;

  // statistics
  std::vector<double> lat_ms;
  int64_t done_bytes = 0, done_count = 0, failed_count = 0, iterations = 0;
  Clock::time_point t_first, t_last;
  bool any_done = false;

  void run();
  bool launch_iteration(std::vector<Req *> &ready, std::string &err);
};

namespace {

int sfail(int rc, const std::string &msg) {
  set_last_error(msg);
  return rc;
}

// Drops the record of a finished request once its result was collected.
void forget(pmrc_server *s, std::map<uint64_t, std::unique_ptr<Req>>::iterator it) {
  cudaEventDestroy(it->second->ev_in);
  cudaEventDestroy(it->second->ev_out);
  s->reqs.erase(it);
}

// Device pointers of a request's blocks: inside the arena, or the caller's
// device blocks for a device-resident request.
void block_ptrs(pmrc_server *s, Req *r, std::vector<const uint8_t *> &in,
                std::vector<uint8_t *> &out) {
  const uint8_t *ib = r->device ? r->in : s->arena_base + r->off;
  uint8_t *ob = r->device ? r->out : s->arena_base + r->off + r->in_span;
  in.resize(r->nin);
  out.resize(r->nout);
  for (size_t i = 0; i < r->nin; i++) in[i] = ib + i * r->B;
  for (size_t j = 0; j < r->nout; j++) out[j] = ob + j * r->B;
}

}  // namespace

bool pmrc_server::launch_iteration(std::vector<Req *> &ready, std::string &err) {
  // the work-list buffer must be free of the kernel that read it last
  const int b = next_buf;
  if (cudaEventQuery(buf_free[b]) == cudaErrorNotReady) return false;
  std::vector<WorkStripe> stripes(ready.size());
  std::vector<const WorkStripe *> sp;
  std::vector<Req *> ok;
  std::vector<BitslicedEncode> bitsliced;  // large encodes: own launches after the kernel
  for (size_t i = 0; i < ready.size(); i++) {
    Req *r = ready[i];
    std::vector<const uint8_t *> in;
    std::vector<uint8_t *> out;
    block_ptrs(this, r, in, out);
    std::string e2;
    int rc;
    BitslicedEncode be;
    if (r->op == PMRC_OP_ENCODE && bitsliced_encode_split(r->code, in.data(), out.data(), r->B, be)) {
      rc = kOk;
      if (be.nbytes < r->B) {  // the ragged tail goes with the batched kernel
        for (auto &p : in) p += be.nbytes;
        for (auto &p : out) p += be.nbytes;
        rc = stripe_encode(r->code, in.data(), out.data(), r->B - be.nbytes, stripes[i], e2);
        if (!rc) sp.push_back(&stripes[i]);
      }
      if (rc) {
        r->status = rc;
        r->state = kFailed;
        continue;
      }
      bitsliced.push_back(std::move(be));
      ok.push_back(r);
      continue;
    }
    if (r->op == PMRC_OP_ENCODE)
      rc = stripe_encode(r->code, in.data(), out.data(), r->B, stripes[i], e2);
    else if (r->op == PMRC_OP_REPAIR)
      rc = stripe_repair(r->code, r->failed, r->helpers.data(), in.data(), out.data(), r->B,
                         stripes[i], e2);
    else
      rc = stripe_decode(r->code, r->nodes.data(), in.data(), out.data(), r->B, stripes[i], e2);
    if (rc) {
      r->status = rc;
      r->state = kFailed;
      continue;
    }
    sp.push_back(&stripes[i]);
    ok.push_back(r);
  }
  WorkList wl;
  if (!sp.empty()) {
    int rc = worklist_build(sp, 64 << 10, kItemsPerCta * sms * 2, wl, err);
    if (rc) {
      for (Req *r : ok) {
        r->status = rc;
        r->state = kFailed;
      }
      ok.clear();
    }
  }
  if (wl.items.size() > item_cap || wl.ptrs.size() > ptr_cap) {
    err = "iteration larger than the server's work-list capacity";
    for (Req *r : ok) {
      r->status = PMRC_EUNSUPPORTED;
      r->state = kFailed;
    }
    ok.clear();
  }
  Iteration it;
  it.buf = b;
  cudaEventCreateWithFlags(&it.done, cudaEventDisableTiming);
  for (const auto &be : bitsliced) {  // attribute set outside the launch sequence
    const cudaError_t pe = bitslice_prepare(be.id);
    if (pe != cudaSuccess) {
      err = std::string("serving bitsliced setup: ") + cudaGetErrorString(pe);
      for (Req *r : ok) {
        r->status = PMRC_ECUDA;
        r->state = kFailed;
      }
      ok.clear();
      bitsliced.clear();
    }
  }
  if (!ok.empty() && !wl.items.empty()) {
    memcpy(h_items[b], wl.items.data(), wl.items.size() * sizeof(WorkItem));
    memcpy(h_ptrs[b], wl.ptrs.data(), wl.ptrs.size() * sizeof(uint8_t *));
    const int per_sm = std::min(2, worklist_ctas_per_sm(wl.smem));
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)sms * per_sm, (int64_t)wl.items.size()));
    cudaError_t e = worklist_launch(m_items[b], (int)wl.items.size(), m_ptrs[b], d_counter[b],
                                    grid, wl.smem, wl.ptr_area, s_comp);
    cudaEventRecord(buf_free[b], s_comp);
    if (e != cudaSuccess) {
      err = std::string("serving launch: ") + cudaGetErrorString(e);
      for (Req *r : ok) {
        r->status = PMRC_ECUDA;
        r->state = kFailed;
      }
      ok.clear();
    }
  }
  if (!ok.empty())
    for (const auto &be : bitsliced) {
      const cudaError_t e = bitslice_launch(be.id, be.in.data(), be.out.data(), be.nbytes, s_comp);
      if (e != cudaSuccess) {
        err = std::string("serving bitsliced launch: ") + cudaGetErrorString(e);
        for (Req *r : ok) {
          r->status = PMRC_ECUDA;
          r->state = kFailed;
        }
        ok.clear();
        break;
      }
    }
  cudaEventRecord(it.done, s_comp);
  // outputs go back as soon as the iteration's kernels are done
  bool waited[kCopyLanes] = {};
  for (Req *r : ok) {
    const int l = least_queued(out_queued);
    if (!waited[l]) cudaStreamWaitEvent(s_out[l], it.done, 0);
    waited[l] = true;
    if (!r->device) {
      cudaMemcpyAsync(r->out, arena_base + r->off + r->in_span, r->out_bytes,
                      cudaMemcpyDeviceToHost, s_out[l]);
      out_queued[l] += r->out_bytes;
      r->out_lane = l;
    }
    cudaEventRecord(r->ev_out, s_out[l]);
    r->state = kRunning;
  }
  it.reqs = ok;
  it.stripes = std::move(stripes);
  inflight.push_back(std::move(it));
  next_buf ^= 1;
  iterations++;
  return true;
}

void pmrc_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    bool progress = false;
    // 1. admit
    while (!queue.empty() && (int)active.size() < max_slots) {
      Req *r = queue.front();
      if (r->device) {  // its blocks are already on the device: ready at once
        queue.pop_front();
        r->state = kReady;
        active.push_back(r);
        progress = true;
        continue;
      }
      size_t off;
      if (!arena->alloc(r->in_span + r->out_bytes, off)) break;
      queue.pop_front();
      r->off = off;
      const int l = least_queued(in_queued);
      cudaMemcpyAsync(arena_base + off, r->in, r->in_bytes, cudaMemcpyHostToDevice, s_in[l]);
      cudaEventRecord(r->ev_in, s_in[l]);
      in_queued[l] += r->in_bytes;
      r->in_lane = l;
      r->state = kCopyIn;
      active.push_back(r);
      progress = true;
    }
    // 2. inputs landed
    std::vector<Req *> ready;
    for (Req *r : active) {
      if (r->state == kCopyIn && cudaEventQuery(r->ev_in) == cudaSuccess) {
        r->state = kReady;
        in_queued[r->in_lane] -= r->in_bytes;
      }
      if (r->state == kReady) ready.push_back(r);
    }
    // 3. launch an iteration over every ready request
    if (!ready.empty() && inflight.size() < 2) {
      std::string err;
      if (launch_iteration(ready, err)) progress = true;
      if (!err.empty()) set_last_error(err);
    }
    // 4. retire requests whose outputs are back
    while (!inflight.empty() && cudaEventQuery(inflight.front().done) == cudaSuccess) {
      cudaEventDestroy(inflight.front().done);
      inflight.pop_front();
      progress = true;
    }
    for (size_t i = 0; i < active.size();) {
      Req *r = active[i];
      // finished: outputs copied back (the copy follows the iteration's
      // kernel on the copy-back stream), or refused while building the
      // iteration (then it was never part of one)
      const bool fin = (r->state == kRunning && cudaEventQuery(r->ev_out) == cudaSuccess) ||
                       r->state == kFailed;
      if (fin) {
        if (r->state == kRunning) r->state = kDone;
        if (r->out_lane >= 0) out_queued[r->out_lane] -= r->out_bytes;
        if (!r->device) arena->release(r->off, r->in_span + r->out_bytes);
        r->t_done = Clock::now();
        if (r->state == kDone) {
          lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit)
                               .count());
          done_bytes += r->user_bytes;
          done_count++;
          if (!any_done) t_first = r->t_submit;
          any_done = true;
          t_last = r->t_done;
        } else {
          failed_count++;
        }
        active.erase(active.begin() + i);
        progress = true;
        cv_done.notify_all();
      } else {
        i++;
      }
    }
    if (stop && queue.empty() && active.empty() && inflight.empty()) break;
    if (!progress) {
      if (queue.empty() && active.empty() && inflight.empty())
        cv_work.wait(lk, [&] { return stop || !queue.empty(); });
      else
        cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

extern "C" {

int pmrc_server_create(size_t budget_bytes, int max_slots, pmrc_server **out) {
  if (!out || budget_bytes < kAlign || max_slots < 1)
    return sfail(PMRC_EINVAL, "server needs out, a budget and at least one slot");
  *out = nullptr;
  std::unique_ptr<pmrc_server> s(new (std::nothrow) pmrc_server());
  if (!s) return sfail(PMRC_ENOMEM, "out of host memory");
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
  if (e == cudaSuccess) e = cudaMalloc(&s->arena_base, budget_bytes);
  if (e != cudaSuccess)
    return sfail(e == cudaErrorMemoryAllocation ? PMRC_ENOMEM : PMRC_ECUDA,
                 std::string("server arena: ") + cudaGetErrorString(e));
  s->arena.reset(new Arena(budget_bytes));
  s->max_slots = max_slots;
  // generous work-list capacity: items are 4 KiB x 16 tiles per block
  s->item_cap = 1 << 20;
  s->ptr_cap = 1 << 20;
  for (int b = 0; b < 2 && e == cudaSuccess; b++) {
    e = cudaMalloc(&s->d_counter[b], sizeof(unsigned));
    if (e == cudaSuccess)
      e = cudaHostAlloc(&s->h_items[b], s->item_cap * sizeof(WorkItem), cudaHostAllocMapped);
    if (e == cudaSuccess)
      e = cudaHostAlloc(&s->h_ptrs[b], s->ptr_cap * sizeof(uint8_t *), cudaHostAllocMapped);
    void *mi = nullptr, *mp = nullptr;
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&mi, s->h_items[b], 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&mp, s->h_ptrs[b], 0);
    s->m_items[b] = static_cast<const WorkItem *>(mi);
    s->m_ptrs[b] = static_cast<uint8_t *const *>(mp);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->buf_free[b], cudaEventDisableTiming);
  }
  for (int l = 0; l < kCopyLanes && e == cudaSuccess; l++) {
    e = cudaStreamCreateWithFlags(&s->s_in[l], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_out[l], cudaStreamNonBlocking);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    pmrc_server_destroy(s.release());
    return sfail(PMRC_ECUDA, std::string("server setup: ") + cudaGetErrorString(e));
  }
  pmrc_server *raw = s.get();
  raw->worker = std::thread([raw] { raw->run(); });
  *out = s.release();
  return PMRC_OK;
}

void pmrc_server_destroy(pmrc_server *s) {
  if (!s) return;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
  }
  for (auto &kv : s->reqs) {
    if (kv.second->ev_in) cudaEventDestroy(kv.second->ev_in);
    if (kv.second->ev_out) cudaEventDestroy(kv.second->ev_out);
  }
  for (int b = 0; b < 2; b++) {
    cudaFree(s->d_counter[b]);
    cudaFreeHost(s->h_items[b]);
    cudaFreeHost(s->h_ptrs[b]);
    if (s->buf_free[b]) cudaEventDestroy(s->buf_free[b]);
  }
  for (int l = 0; l < kCopyLanes; l++) {
    if (s->s_in[l]) cudaStreamDestroy(s->s_in[l]);
    if (s->s_out[l]) cudaStreamDestroy(s->s_out[l]);
  }
  if (s->s_comp) cudaStreamDestroy(s->s_comp);
  cudaFree(s->arena_base);
  delete s;
}

int pmrc_server_submit(pmrc_server *s, const pmrc_request *q, uint64_t *id_out) {
  PMRC_TRACE("pmrc_server_submit");
  const Clock::time_point t_submit = Clock::now();
  if (!s || !q || !q->code || !q->in || !q->out || q->block_bytes == 0)
    return sfail(PMRC_EINVAL, "NULL argument or empty block");
  const pmrc_code *c = q->code;
  if (c->m.w != 8) return sfail(PMRC_EUNSUPPORTED, "the server takes GF(2^8) codes");
  std::unique_ptr<Req> r(new (std::nothrow) Req());
  if (!r) return sfail(PMRC_ENOMEM, "out of host memory");
  r->op = q->op & ~PMRC_REQ_DEVICE;
  r->device = (q->op & PMRC_REQ_DEVICE) != 0;
  r->code = c;
  r->B = q->block_bytes;
  r->in = q->in;
  r->out = q->out;
  // K data blocks, KA = k alpha blocks on the first k (or any k) nodes, N coded
  const size_t a = c->m.alpha, K = c->m.K, KA = (size_t)c->m.k * a, N = c->m.N;
  // Build (or find) the request's coefficient plan here, on the caller's
  // thread, and upload it to the server's device: the scheduler then only
  // assembles work items.  Plan time counts in the request's latency.
  std::string err;
  int rc = kOk;
  const void *image = nullptr;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != s->device) cudaSetDevice(s->device);
  switch (r->op) {
    case PMRC_OP_ENCODE:
      r->nin = K;
      r->nout = c->m.systematic ? N - KA : N;
      r->user_bytes = (int64_t)K * r->B;
      rc = c->encode->device_image(&image, err);
      break;
    case PMRC_OP_REPAIR: {
      if (!q->helpers) {
        rc = kEInval;
        err = "repair needs helpers";
        break;
      }
      if (a > 16) {
        rc = kEUnsupported;
        err = "served repair needs alpha <= 16";
        break;
      }
      r->failed = q->failed;
      r->helpers.assign(q->helpers, q->helpers + c->m.d);
      std::shared_ptr<FusedRepairPlan> fp;
      rc = fused_repair_plan(c, q->failed, q->helpers, fp, err);
      if (!rc) rc = fp->device_image(&image, err);
      r->nin = (size_t)c->m.d * a;
      r->nout = a;
      r->user_bytes = (int64_t)a * r->B;
      break;
    }
    case PMRC_OP_DECODE: {
      if (!q->nodes) {
        rc = kEInval;
        err = "decode needs nodes";
        break;
      }
      r->nodes.assign(q->nodes, q->nodes + c->m.k);
      std::vector<char> seen(c->m.n, 0);
      for (int i = 0; i < c->m.k && !rc; i++) {
        if (q->nodes[i] < 0 || q->nodes[i] >= c->m.n || seen[q->nodes[i]]) {
          rc = kEInval;
          err = "nodes: out of range or repeated node id";
        } else {
          seen[q->nodes[i]] = 1;
        }
      }
      if (!rc) {
        std::shared_ptr<Plan> dp;
        rc = decode_plan(c, q->nodes, std::vector<char>(K, 1), dp, err);
        if (!rc) rc = dp->device_image(&image, err);
      }
      r->nin = KA;
      r->nout = K;
      r->user_bytes = (int64_t)K * r->B;
      break;
    }
    default:
      rc = kEInval;
      err = "unknown operation";
  }
  if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
  if (rc) return sfail(rc, err);
  r->in_bytes = r->nin * r->B;
  r->out_bytes = r->nout * r->B;
  r->in_span = (r->in_bytes + kAlign - 1) & ~(kAlign - 1);
  if (!r->device && r->in_span + r->out_bytes > s->arena->size())
    return sfail(PMRC_ENOMEM, "request larger than the server's HBM budget");
  if (r->device) {  // the kernel reads and writes the caller's blocks in place
    bool aligned = ((uintptr_t)r->in % 16 == 0) && ((uintptr_t)r->out % 16 == 0) && r->B % 16 == 0;
    if (!aligned) return sfail(PMRC_EINVAL, "device-resident blocks must be 16-byte aligned");
  }
  if (cudaEventCreateWithFlags(&r->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return sfail(PMRC_ECUDA, "cudaEventCreate");
  r->t_submit = t_submit;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return sfail(PMRC_EBUSY, "server is stopping");
    r->id = s->next_id++;
    if (id_out) *id_out = r->id;
    s->queue.push_back(r.get());
    s->reqs[r->id] = std::move(r);
  }
  s->cv_work.notify_one();
  return PMRC_OK;
}

int pmrc_server_poll(pmrc_server *s, uint64_t id, int *status, double *latency_ms) {
  if (!s) return sfail(PMRC_EINVAL, "NULL server");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(PMRC_EINVAL, "unknown request id");
  Req *r = it->second.get();
  const bool fin = r->state == kDone || r->state == kFailed || r->state == kCancelled;
  if (status) *status = r->state == kDone ? PMRC_OK : r->status;
  if (latency_ms)
    *latency_ms = fin ? std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count()
                      : -1.0;
  if (fin) forget(s, it);
  return fin ? 1 : 0;
}

int pmrc_server_wait(pmrc_server *s, uint64_t id, int timeout_ms, int *status,
                     double *latency_ms) {
  if (!s) return sfail(PMRC_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(PMRC_EINVAL, "unknown request id");
  Req *r = it->second.get();
  auto fin = [&] { return r->state == kDone || r->state == kFailed || r->state == kCancelled; };
  if (timeout_ms < 0)
    s->cv_done.wait(lk, fin);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), fin))
    return sfail(PMRC_ETIMEOUT, "request not finished within the timeout");
  if (status) *status = r->state == kDone ? PMRC_OK : r->status;
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  forget(s, it);
  return PMRC_OK;
}

int pmrc_server_cancel(pmrc_server *s, uint64_t id) {
  if (!s) return sfail(PMRC_EINVAL, "NULL server");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(PMRC_EINVAL, "unknown request id");
  Req *r = it->second.get();
  if (r->state != kQueued) return sfail(PMRC_EBUSY, "request already admitted");
  s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
  r->state = kCancelled;
  r->status = PMRC_EBUSY;
  r->t_done = Clock::now();
  s->cv_done.notify_all();
  return PMRC_OK;
}

int pmrc_server_stats(pmrc_server *s, double *out) {
  if (!s || !out) return sfail(PMRC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(s->mu);
  std::vector<double> v = s->lat_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) {
    if (v.empty()) return 0.0;
    size_t i = (size_t)std::min<double>(v.size() - 1, std::max(0.0, p * v.size() - 1e-9));
    return v[i];
  };
  const double span =
      s->any_done ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
  out[0] = (double)s->done_count;
  out[1] = (double)s->failed_count;
  out[2] = pct(0.50);
  out[3] = pct(0.99);
  out[4] = v.empty() ? 0.0 : v.back();
  out[5] = (double)s->done_bytes;
  out[6] = span > 0 ? s->done_bytes / span / 1e9 : 0.0;
  out[7] = (double)s->arena->peak();
  out[8] = (double)s->iterations;
  out[9] = (double)s->arena->size();
  return PMRC_OK;
}

int pmrc_server_reset_stats(pmrc_server *s) {
  if (!s) return sfail(PMRC_EINVAL, "NULL server");
  std::lock_guard<std::mutex> g(s->mu);
  s->lat_ms.clear();
  s->done_bytes = s->done_count = s->failed_count = s->iterations = 0;
  s->any_done = false;
  return PMRC_OK;
}

}  // extern "C"
