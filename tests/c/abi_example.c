/* A caller of libqs in plain C: a 20-qubit GHZ state through the C ABI,
 * its norm, a TFIM-style expectation and a few samples.  Compiled and
 * linked by the CPU test suite; running it needs a GPU. */
#include <stdio.h>

#include "include/qs.h"

int main(void) {
  qs_state* s = NULL;
  const int n = 20;
  const double h[8] = {0.7071067811865476, 0, 0.7071067811865476, 0, 0.7071067811865476, 0, -0.7071067811865476, 0};
  const double x[8] = {0, 0, 1, 0, 1, 0, 0, 0};
  if (qs_alloc(n, QS_C128, &s) != QS_OK) {
    fprintf(stderr, "qs_alloc: %s\n", qs_last_error());
    return 1;
  }
  qs_apply_1q(s, 0, h);
  for (int q = 0; q + 1 < n; ++q) {
    const int c = q;
    qs_apply_controlled(s, &c, 1, q + 1, x);
  }
  double norm = 0.0, e = 0.0;
  const uint64_t xm[2] = {0, 1}, zm[2] = {3, 0};
  const double cf[2] = {1.0, 1.0};
  qs_norm2(s, &norm);
  qs_expect_pauli(s, 2, xm, zm, cf, &e); /* Z0 Z1 + X0 */
  const double u[4] = {0.1, 0.4, 0.6, 0.9};
  uint64_t out[4];
  qs_sample(s, 4, u, out);
  const qs_status st = qs_sync(s);
  printf("status %d norm %.15f energy %.15f samples %llu %llu %llu %llu\n", (int)st, norm, e,
         (unsigned long long)out[0], (unsigned long long)out[1], (unsigned long long)out[2],
         (unsigned long long)out[3]);
  qs_free(s);
  return st == QS_OK ? 0 : 1;
}
