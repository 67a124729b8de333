// Built-in bitsliced encode kernel of the n=32, k=16 sparse systematic code (the
// schedule gen_bitslice.cpp writes from the library's construction, as for
// the codes in bitslice.cu), in a translation unit of its own: its few
// thousand coefficients take most of the library's compile time, and
// compiling it apart lets the build run it in parallel with the rest.
#include <cuda_runtime.h>

#include <cstdint>

namespace pmrc {
namespace bsk {

#include "bitslice_dev.cuh"
#include "bitslice_gen_k16.cuh"

}  // namespace bsk
}  // namespace pmrc
