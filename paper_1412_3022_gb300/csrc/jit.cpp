// Run-time compilation of generated kernels (NVRTC) for sm_103a.
//
// NVRTC is loaded with dlopen on first use, so the library has no link-time
// dependency on it: without it, jit_available() is false and callers keep
// their region-kernel path.  The compiled cubin is loaded as a CUDA library
// (cudaLibraryLoadData) and the kernel looked up by its C name.
#include "jit.h"

#include <dlfcn.h>
#include <nvrtc.h>

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
  });
  return n;
}

}  // namespace

bool jit_available() { return nvrtc().ok; }

int jit_compile(const std::string &src, const char *kernel_name, std::vector<char> &cubin,
                std::string &err) {
  const Nvrtc &n = nvrtc();
  if (!n.ok) {
    err = "NVRTC (libnvrtc) could not be loaded";
    return kEUnsupported;
  }
  nvrtcProgram prog;
  if (n.create(&prog, src.c_str(), kernel_name, 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    err = "nvrtcCreateProgram failed";
    return kEUnsupported;
  }
  const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-w"};
  const nvrtcResult rc = n.compile(prog, 3, opts);
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
