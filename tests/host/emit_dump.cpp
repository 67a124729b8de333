// Prints a random matrix and the bitsliced schedule the emitter writes for
// it (both block rules, optionally split over warp pairs), for
// tests/test_host_units.py to evaluate.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "bs_emit.h"

int main(int argc, char **argv) {
  const int rows = argc > 1 ? atoi(argv[1]) : 13, cols = argc > 2 ? atoi(argv[2]) : 9;
  const bool by_support = argc > 3 && atoi(argv[3]) != 0;
  std::mt19937 rng(argc > 4 ? atoi(argv[4]) : 1);
  std::vector<uint8_t> M((size_t)rows * cols);
  for (auto &v : M) v = (rng() % 4 == 0) ? 0 : (uint8_t)(rng() & 0xFF);
  const auto blks = by_support ? pmrc::bs_blocks_by_support(M.data(), rows, cols)
                               : pmrc::bs_blocks_chunked(M.data(), rows, cols);
  const bool pairs = argc > 5 && atoi(argv[5]) != 0;
  const pmrc::BsEmitted e = pmrc::bs_emit_kernel(M.data(), rows, cols, blks, "k", true, pairs);
  printf("MATRIX %d %d\n", rows, cols);
  for (int r = 0; r < rows; r++) {
    for (int c = 0; c < cols; c++) printf("%d ", M[(size_t)r * cols + c]);
    printf("\n");
  }
  printf("CODE\n%s", e.code.c_str());
  return 0;
}
