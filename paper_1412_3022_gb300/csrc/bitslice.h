// Bitsliced encode kernels generated at build time (bitslice.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

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

}  // namespace pmrc
