// Checks bs_cta_ranges (the bitsliced launcher's split of (block, tile) work
// items into per-CTA ranges) on many shapes; prints "ok" or the first
// violated property.
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "bs_emit.h"

int main() {
  std::mt19937 rng(7);
  int cases = 0;
  for (int trial = 0; trial < 20000; trial++) {
    const int nblocks = 1 + (int)(rng() % 64);
    const uint64_t ntiles = 1 + rng() % (trial % 3 == 0 ? 8 : 5000);
    const int ncta = 1 + (int)(rng() % 256);
    std::vector<int> cost(nblocks);
    for (int &c : cost) c = 100 + (int)(rng() % 2000);
    std::vector<uint32_t> g(ncta + 1, 0xFFFFFFFFu);
    pmrc::bs_cta_ranges(nblocks, cost.data(), ntiles, ncta, g.data());
    const uint64_t items = (uint64_t)nblocks * ntiles;
    if (g[0] != 0 || g[ncta] != items) {
      printf("endpoints: trial %d\n", trial);
      return 1;
    }
    double total = 0, maxc = 0;
    for (int c : cost) total += (double)c * ntiles, maxc = maxc > c ? maxc : c;
    for (int c = 0; c < ncta; c++) {
      if (g[c] > g[c + 1]) {
        printf("not monotone: trial %d cta %d\n", trial, c);
        return 1;
      }
      double w = 0;  // this CTA's cost
      for (uint64_t x = g[c]; x < g[c + 1]; x++) w += cost[x / ntiles];
      // within one tile's cost of an equal share (when every CTA can get one)
      if (items >= (uint64_t)ncta && (w > total / ncta + maxc + 1e-6 || w < total / ncta - maxc - 1e-6)) {
        printf("unbalanced: trial %d cta %d cost %.0f share %.0f\n", trial, c, w, total / ncta);
        return 1;
      }
    }
    cases++;
  }
  printf("ok %d\n", cases);
  return 0;
}
