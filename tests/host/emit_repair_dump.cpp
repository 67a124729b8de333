// Prints random helper coefficients phi (alpha entries, some zero), a random
// newcomer matrix D (alpha x d) and the projection and fused repair schedules
// the emitter writes for them, for tests/test_host_units.py to evaluate.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "bs_emit.h"

int main(int argc, char **argv) {
  const int alpha = argc > 1 ? atoi(argv[1]) : 7, d = argc > 2 ? atoi(argv[2]) : 14;
  std::mt19937 rng(argc > 3 ? atoi(argv[3]) : 1);
  const int zeros = argc > 4 ? atoi(argv[4]) : 1;
  std::vector<uint8_t> phi(alpha), D((size_t)alpha * d);
  for (auto &v : phi) v = (zeros && rng() % 3 == 0) ? 0 : (uint8_t)(1 + rng() % 255);
  if (argc > 5) {  // a single coefficient 1 (the sparse code's failed node among the first alpha)
    for (auto &v : phi) v = 0;
    phi[atoi(argv[5]) % alpha] = 1;
  }
  bool any = false;
  for (auto v : phi) any = any || v;
  if (!any) phi[0] = 1;
  for (auto &v : D) v = (rng() % 5 == 0) ? 0 : (uint8_t)(rng() & 0xFF);
  printf("PHI");
  for (auto v : phi) printf(" %d", v);
  printf("\nD %d %d\n", alpha, d);
  for (int r = 0; r < alpha; r++) {
    for (int q = 0; q < d; q++) printf("%d ", D[(size_t)r * d + q]);
    printf("\n");
  }
  printf("PROJ\n%s", pmrc::bs_emit_projection(phi.data(), alpha, "kp").code.c_str());
  printf("FUSED\n%s", pmrc::bs_emit_fused_repair(phi.data(), alpha, D.data(), d, "kf").code.c_str());
  return 0;
}
