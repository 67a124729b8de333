// Launch of the GF(2^8) region multiply-XOR kernel over a plan.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "plan.h"

namespace pmrc {

// out[j] = sum_c M[row j][c] * in[c] over `nbytes` bytes, for the matrix the
// plan was built from.  in[] has plan.nin device pointers, out[] plan.nout
// (NULL entries of out[] are not written; NULL entries of in[] are allowed
// for columns the plan never reads).  Asynchronous on `stream`.
int launch_region(Plan &plan, const uint8_t *const *in, uint8_t *const *out, size_t nbytes,
                  cudaStream_t stream, std::string &err);

}  // namespace pmrc
