// Exercises jit_compile's on-disk cubin cache on the CPU (NVRTC only, no
// GPU): argv[1] is the cache directory (PMRC_KERNEL_CACHE is set by the
// caller).  Prints "ok <size>" after two compilations of one source, or
// "nonvrtc" when NVRTC cannot be loaded.
#include <cstdio>
#include <string>
#include <vector>

#include "jit.h"

int main() {
  if (!pmrc::jit_available()) {
    printf("nonvrtc\n");
    return 0;
  }
  const std::string src =
      "extern \"C\" __global__ void probe_kernel(int *p) { p[threadIdx.x] = 3 * threadIdx.x; }\n";
  std::vector<char> a, b;
  std::string err;
  if (pmrc::jit_compile(src, "probe_kernel", a, err)) {
    printf("compile failed: %s\n", err.c_str());
    return 1;
  }
  if (pmrc::jit_compile(src, "probe_kernel", b, err)) {
    printf("second compile failed: %s\n", err.c_str());
    return 1;
  }
  if (a != b || a.size() < 4) {
    printf("cubins differ\n");
    return 1;
  }
  printf("ok %zu\n", a.size());
  return 0;
}
