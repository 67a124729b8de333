// Prints a random factored product -- Z (m x cols: row i starts from its own
// column own[i] with coefficient 1, plus random terms on shared columns) and
// W (r x m) -- and the two launch schedules the emitter writes for it:
// stage 1 (Z, rows grouped by their shared columns, plane-layout outputs)
// and stage 2 (W, consecutive rows, plane-layout inputs), for
// tests/test_host_units.py to evaluate one after the other.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "bs_emit.h"

int main(int argc, char **argv) {
  const int m = argc > 1 ? atoi(argv[1]) : 21, shared = argc > 2 ? atoi(argv[2]) : 35;
  const int r = argc > 3 ? atoi(argv[3]) : m, groups = argc > 4 ? atoi(argv[4]) : 7;
  std::mt19937 rng(argc > 5 ? atoi(argv[5]) : 1);
  const int cols = shared + m;
  std::vector<uint8_t> Z((size_t)m * cols, 0), W((size_t)r * m);
  std::vector<int> own(m);
  // rows of one group share their columns (a support), as the sparse
  // code's parity rows of one slot do
  std::vector<std::vector<int>> sup(groups);
  for (auto &s : sup)
    for (int q = 0; q < shared; q++)
      if (rng() % 3 == 0) s.push_back(q);
  for (int i = 0; i < m; i++) {
    own[i] = shared + i;
    Z[(size_t)i * cols + own[i]] = 1;
    for (int q : sup[i % groups]) Z[(size_t)i * cols + q] = (uint8_t)(1 + rng() % 255);
  }
  for (auto &v : W) v = (rng() % 6 == 0) ? 0 : (uint8_t)(rng() & 0xFF);
  const int max_inputs = argc > 6 ? atoi(argv[6]) : 64;
  const auto zb = pmrc::bs_blocks_grouped(Z.data(), m, cols, own, max_inputs);
  const auto wb = pmrc::bs_blocks_chunked(W.data(), r, m);
  printf("Z %d %d\n", m, cols);
  for (int i = 0; i < m; i++) {
    for (int q = 0; q < cols; q++) printf("%d ", Z[(size_t)i * cols + q]);
    printf("\n");
  }
  printf("W %d %d\n", r, m);
  for (int i = 0; i < r; i++) {
    for (int q = 0; q < m; q++) printf("%d ", W[(size_t)i * m + q]);
    printf("\n");
  }
  printf("BLOCKS");
  for (const auto &B : zb) {
    printf(" ");
    for (size_t q = 0; q < B.rows.size(); q++) printf("%s%d", q ? "," : "", B.rows[q]);
    printf("/%zu", B.inputs.size());
  }
  printf("\nSTAGE1\n%s", pmrc::bs_emit_kernel(Z.data(), m, cols, zb, "k", true, true, false, true).code.c_str());
  printf("STAGE2\n%s", pmrc::bs_emit_kernel(W.data(), r, m, wb, "k", true, true, true, false).code.c_str());
  return 0;
}
