// Run-time compilation of generated kernels (NVRTC) for sm_103a.
//
// NVRTC is loaded with dlopen on first use, so the library has no link-time
// dependency on it: without it, jit_available() is false and callers keep
// their region-kernel path.  The compiled cubin is loaded as a CUDA library
// (cudaLibraryLoadData) and the kernel looked up by its C name.
#include "jit.h"

#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <thread>
#include <cstring>
#include <mutex>
#include <vector>

namespace pmrc {

namespace {

struct Nvrtc {
  bool ok = false;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  int major = 0, minor = 0;  // NVRTC version (part of the cache key)
};

const Nvrtc &nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    void *h = nullptr;
    for (const char *name : {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so"})
      if (!h) h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
    if (!h) return;
    n.create = reinterpret_cast<decltype(n.create)>(dlsym(h, "nvrtcCreateProgram"));
    n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(h, "nvrtcCompileProgram"));
    n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
    n.log = reinterpret_cast<decltype(n.log)>(dlsym(h, "nvrtcGetProgramLog"));
    n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
    n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
    n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
    n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
    auto version = reinterpret_cast<decltype(&nvrtcVersion)>(dlsym(h, "nvrtcVersion"));
    if (version) version(&n.major, &n.minor);
  });
  return n;
}

constexpr int kNumOpts = 3;
const char *const kOpts[kNumOpts] = {"--gpu-architecture=sm_103a", "-std=c++17", "-w"};

// Directory of the on-disk cubin cache, read at each compilation (they are
// rare): $PMRC_KERNEL_CACHE when set (empty, "0" or "off" turns the cache
// off), else $XDG_CACHE_HOME/pmrc, else $HOME/.cache/pmrc, created (mode
// 0700) when missing; "" when no writable directory results.
std::string cache_dir() {
  const char *env = getenv("PMRC_KERNEL_CACHE");
  if (env) return (*env && strcmp(env, "0") != 0 && strcmp(env, "off") != 0) ? env : "";
  const char *xdg = getenv("XDG_CACHE_HOME"), *home = getenv("HOME");
  std::string base;
  if (xdg && *xdg)
    base = xdg;
  else if (home && *home)
    base = std::string(home) + "/.cache";
  if (base.empty()) return "";
  mkdir(base.c_str(), 0700);  // EEXIST is fine
  const std::string d = base + "/pmrc";
  mkdir(d.c_str(), 0700);
  return access(d.c_str(), W_OK | X_OK) == 0 ? d : "";
}

// Path of the cached cubin for this source, or "" without a cache directory.
std::string cache_path(const std::string &src, const Nvrtc &n) {
  const std::string d = cache_dir();
  if (d.empty()) return "";
  const char *dir = d.c_str();
  uint64_t h = 1469598103934665603ull;  // FNV-1a over source, options, version
  auto mix = [&](const char *p, size_t len) {
    for (size_t i = 0; i < len; i++) {
      h ^= (uint8_t)p[i];
      h *= 1099511628211ull;
    }
  };
  mix(src.data(), src.size());
  for (const char *o : kOpts) mix(o, strlen(o) + 1);
  const int ver[2] = {n.major, n.minor};
  mix(reinterpret_cast<const char *>(ver), sizeof ver);
  char name[64];
  snprintf(name, sizeof name, "/pmrc-%016llx.cubin", (unsigned long long)h);
  return std::string(dir) + name;
}

bool read_cached(const std::string &path, std::vector<char> &cubin) {
  FILE *f = fopen(path.c_str(), "rb");
  if (!f) return false;
  std::vector<char> buf;
  char chunk[65536];
  size_t got;
  while ((got = fread(chunk, 1, sizeof chunk, f)) > 0) buf.insert(buf.end(), chunk, chunk + got);
  fclose(f);
  if (buf.size() < 4 || memcmp(buf.data(), "\x7f" "ELF", 4) != 0) return false;  // not a cubin
  cubin.swap(buf);
  return true;
}

// Written to a temporary name and renamed, so readers never see a partial file.
void write_cached(const std::string &path, const std::vector<char> &cubin) {
  const std::string tmp = path + "." + std::to_string((long long)getpid()) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "wb");
  if (!f) return;
  const bool ok = fwrite(cubin.data(), 1, cubin.size(), f) == cubin.size();
  if (fclose(f) != 0 || !ok || rename(tmp.c_str(), path.c_str()) != 0) remove(tmp.c_str());
}

// A small pool of compile threads, started on first use and joined when
// the process exits (a function-local static whose destructor is registered
// after NVRTC's, see jit_background, and so runs before them).
class JitPool {
 public:
  void submit(std::function<void()> fn) {
    std::lock_guard<std::mutex> g(mu_);
    if (stop_) return;
    q_.push_back(std::move(fn));
    if (workers_.size() < kWorkers) workers_.emplace_back([this] { run(); });
    cv_.notify_one();
  }
  ~JitPool() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
      q_.clear();
    }
    cv_.notify_all();
    for (auto &t : workers_) t.join();
  }

 private:
  static constexpr size_t kWorkers = 2;
  void run() {
    for (;;) {
      std::function<void()> job;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [this] { return stop_ || !q_.empty(); });
        if (stop_) return;
        job = std::move(q_.front());
        q_.pop_front();
      }
      job();
    }
  }
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<std::function<void()>> q_;
  std::vector<std::thread> workers_;
  bool stop_ = false;
};

JitPool &pool() {
  static JitPool p;
  return p;
}

}  // namespace

bool jit_available() { return nvrtc().ok; }

void jit_background(std::function<void()> fn) {
  // NVRTC is loaded before the pool exists, so its exit-time destructors,
  // registered at load, run after the pool's, which waits for the workers
  nvrtc();
  pool().submit(std::move(fn));
}

int jit_compile(const std::string &src, const char *kernel_name, std::vector<char> &cubin,
                std::string &err) {
  const Nvrtc &n = nvrtc();
  if (!n.ok) {
    err = "NVRTC (libnvrtc) could not be loaded";
    return kEUnsupported;
  }
  const std::string cached = cache_path(src, n);
  if (!cached.empty() && read_cached(cached, cubin)) return kOk;
  nvrtcProgram prog;
  if (n.create(&prog, src.c_str(), kernel_name, 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    err = "nvrtcCreateProgram failed";
    return kEUnsupported;
  }
  const nvrtcResult rc = n.compile(prog, kNumOpts, kOpts);
  if (rc != NVRTC_SUCCESS) {
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) n.log(prog, &log[0]);
    err = "run-time compilation failed: " + log.substr(0, 400);
    n.destroy(&prog);
    return kEUnsupported;
  }
  size_t cs = 0;
  n.cubin_size(prog, &cs);
  cubin.assign(cs, 0);
  n.cubin(prog, cubin.data());
  n.destroy(&prog);
  if (!cached.empty()) write_cached(cached, cubin);
  return kOk;
}

int jit_load(const std::vector<char> &cubin, const char *kernel_name, cudaLibrary_t *lib,
             cudaKernel_t *fn, std::string &err) {
  cudaError_t e = cudaLibraryLoadData(lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) {
    err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
    return kECuda;
  }
  e = cudaLibraryGetKernel(fn, *lib, kernel_name);
  if (e != cudaSuccess) {
    cudaLibraryUnload(*lib);
    *lib = nullptr;
    err = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e);
    return kECuda;
  }
  return kOk;
}

}  // namespace pmrc
