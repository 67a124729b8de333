// Integer pipe rates on this GPU, behind bench.py's ALU roofline: each
// variant runs 8 independent dependency chains per thread of one PTX
// instruction (or a 1:1 mix of two) for 4000 iterations on 4 CTAs of 256
// threads per SM, and prints lane-ops per clock per SM from CUDA-event time
// (at 2.0 GHz).  Run it under ncu with the pipe counters
// (sm__inst_executed_pipe_alu / _fma / _fmaheavy / _fmalite) to see which
// pipe each instruction issues to.  Build and run:
//   nvcc -std=c++17 -gencode arch=compute_103a,code=sm_103a -O3 -o bench_alu_pipes bench_alu_pipes.cu
//   ./bench_alu_pipes
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define ASM3(op, d, a, b, c) asm volatile(op " %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c))
#define ASM2(op, d, a, b) asm volatile(op " %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b))

template <int V>
__device__ __forceinline__ void step(uint32_t (&a)[8], uint32_t k) {
#pragma unroll
  for (int j = 0; j < 8; j++) {
    uint32_t n = a[(j + 1) & 7], d;
    if constexpr (V == 0) ASM3("prmt.b32", d, a[j], n, k ^ j);                 // prmt
    if constexpr (V == 2) ASM2("xor.b32", d, a[j], n);                          // xor2
    if constexpr (V == 3) ASM2("add.u32", d, a[j], n);                          // iadd
    if constexpr (V == 4) ASM3("shf.l.wrap.b32", d, a[j], n, k);               // shf
    if constexpr (V == 5) ASM3("mad.lo.u32", d, a[j], n, k);                   // imad
    if constexpr (V == 6) { if (j & 1) ASM2("xor.b32", d, a[j], n); else ASM3("prmt.b32", d, a[j], n, k ^ j); }  // prmt+xor
    if constexpr (V == 7) { if (j & 1) ASM2("add.u32", d, a[j], n); else ASM2("xor.b32", d, a[j], n); }          // xor+add
    if constexpr (V == 8) { if (j & 1) ASM2("add.u32", d, a[j], n); else ASM3("prmt.b32", d, a[j], n, k ^ j); }  // prmt+add
    if constexpr (V == 9) { if (j & 1) ASM3("mad.lo.u32", d, a[j], n, k); else ASM2("xor.b32", d, a[j], n); }    // xor+imad
    a[j] = d;
  }
}

template <>
__device__ __forceinline__ void step<1>(uint32_t (&a)[8], uint32_t k) {
#pragma unroll
  for (int j = 0; j < 8; j++) {
    uint32_t n = a[(j + 1) & 7], d;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x6A;" : "=r"(d) : "r"(a[j]), "r"(n), "r"(k));  // (a&b)^c
    a[j] = d;
  }
}

template <int V>
__global__ void kern(uint32_t *out, uint32_t seed, int iters) {
  uint32_t t = threadIdx.x + blockIdx.x * blockDim.x;
  uint32_t a[8];
#pragma unroll
  for (int j = 0; j < 8; j++) a[j] = seed * (t + 3 * j + 1) + j;
  uint32_t k = seed ^ (t * 0x9E3779B9u);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 8; u++) step<V>(a, k);
  }
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) r += a[j];
  out[t] = r;
}

int main() {
  int sms;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int threads = 256, blocks = sms * 4;
  uint32_t *out;
  cudaMalloc(&out, sizeof(uint32_t) * threads * blocks);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const char *names[] = {"prmt", "lop3", "xor2", "iadd", "shf", "imad", "prmt+xor", "xor+add", "prmt+add", "xor+imad"};
  int iters = 4000;
  for (int v = 0; v < 10; v++) {
    float ms = 0;
    for (int rep = 0; rep < 2; rep++) {
      cudaEventRecord(e0);
      switch (v) {
        case 0: kern<0><<<blocks, threads>>>(out, 7, iters); break;
        case 1: kern<1><<<blocks, threads>>>(out, 7, iters); break;
        case 2: kern<2><<<blocks, threads>>>(out, 7, iters); break;
        case 3: kern<3><<<blocks, threads>>>(out, 7, iters); break;
        case 4: kern<4><<<blocks, threads>>>(out, 7, iters); break;
        case 5: kern<5><<<blocks, threads>>>(out, 7, iters); break;
        case 6: kern<6><<<blocks, threads>>>(out, 7, iters); break;
        case 7: kern<7><<<blocks, threads>>>(out, 7, iters); break;
        case 8: kern<8><<<blocks, threads>>>(out, 7, iters); break;
        case 9: kern<9><<<blocks, threads>>>(out, 7, iters); break;
      }
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    double ops = (double)threads * blocks * iters * 64;
    printf("%-9s ms=%.3f  ops/clk/SM@2.0GHz=%.1f  err=%s\n", names[v], ms,
           ops / (ms * 1e-3) / sms / 2.0e9, cudaGetErrorString(cudaGetLastError()));
  }
  return 0;
}
