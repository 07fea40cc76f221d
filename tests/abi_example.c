/* A propagation through the C ABI alone, in plain C99: the ring circuit on
 * n = 8 qubits (RZZ(0.4) on every bond, then RX(0.6) and RZ(0.3) on every
 * qubit) applied three times in the Heisenberg picture, observable
 * (1/n) sum_i Z_i merged by translations (Z_n) after every layer, and <O>
 * for the state |0...0>.
 *
 * Exit status: 0 on success, 2 when no CUDA device can be used (pp_create
 * reports PP_ERR_CUDA), 1 on any other failure.  Every failure prints the
 * call, its status and pp_last_error(). */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "pp.h"

#define N 8

static int failed(pp_status st, const char* what) {
  if (st == PP_OK) return 0;
  fprintf(stderr, "%s failed: status %d: %s\n", what, (int)st, pp_last_error());
  return 1;
}

int main(void) {
  pp_config cfg;
  if (failed(pp_config_default(&cfg), "pp_config_default")) return 1;
  cfg.n_qubits = N;
  cfg.symmetry = PP_SYM_ZN;
  cfg.coeff_eps = 1e-6;

  /* O = (1/n) sum_q Z_q: x words zero, z word with bit q */
  uint64_t x[N], z[N];
  double coef[N];
  for (int q = 0; q < N; ++q) {
    x[q] = 0;
    z[q] = (uint64_t)1 << q;
    coef[q] = 1.0 / N;
  }
  pp_ctx* ctx = NULL;
  pp_status st = pp_create(&cfg, N, x, z, coef, &ctx);
  if (failed(st, "pp_create")) return st == PP_ERR_CUDA ? 2 : 1;

  /* one layer in time order: RZZ on the n bonds, RX, RZ on every qubit */
  pp_pauli gates[3 * N];
  double theta[3 * N];
  memset(gates, 0, sizeof gates);
  for (int q = 0; q < N; ++q) {
    gates[q].z[0] = ((uint64_t)1 << q) | ((uint64_t)1 << ((q + 1) % N));
    theta[q] = 0.4;
    gates[N + q].x[0] = (uint64_t)1 << q;
    theta[N + q] = 0.6;
    gates[2 * N + q].z[0] = (uint64_t)1 << q;
    theta[2 * N + q] = 0.3;
  }
  for (int layer = 0; layer < 3; ++layer) {
    if (failed(pp_apply_layer(ctx, 3 * N, gates, theta, 1), "pp_apply_layer")) {
      pp_destroy(ctx);
      return 1;
    }
  }

  /* |0...0>: Bloch vector (0, 0, 1) on every qubit */
  double bloch[3 * N];
  for (int q = 0; q < N; ++q) {
    bloch[3 * q] = 0.0;
    bloch[3 * q + 1] = 0.0;
    bloch[3 * q + 2] = 1.0;
  }
  double value = 0.0;
  int64_t live = 0, stored = 0;
  if (failed(pp_expect(ctx, bloch, &value), "pp_expect") ||
      failed(pp_num_terms(ctx, &live, &stored), "pp_num_terms")) {
    pp_destroy(ctx);
    return 1;
  }
  printf("<O> = %.15f with %lld representatives\n", value, (long long)live);
  return failed(pp_destroy(ctx), "pp_destroy");
}
