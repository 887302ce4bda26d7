/* A plain C client of libpf.so (no Python, no torch, no CUDA runtime of its own): builds the
 * two-bus case (slack at bus 0 with V = 1, theta = 0; a lossless line r = 0, x = 0.1; a PQ
 * load 0.5 + j0.2 at bus 1), evaluates F and J at one state through the host-buffer entry
 * point and prints them with the pattern, for tests/test_gpu_c_client.py to check. */
#include <stdio.h>
#include <string.h>

#include "pf.h"

int main(void) {
  const int32_t from[1] = {0}, to[1] = {1}, load_bus[1] = {1};
  const double r[1] = {0.0}, x[1] = {0.1}, load_p[1] = {0.5}, load_q[1] = {0.2};
  pf_system s;
  memset(&s, 0, sizeof s);
  s.n_bus = 2;
  s.n_branch = 1;
  s.br_from = from;
  s.br_to = to;
  s.br_r = r;
  s.br_x = x;
  s.n_load = 1;
  s.load_bus = load_bus;
  s.load_p = load_p;
  s.load_q = load_q;
  s.slack_bus = 0;
  s.slack_vset = 1.0;
  s.slack_theta = 0.0;
  pf_ctx *ctx = NULL;
  if (pf_build(&s, PF_REDUCED, NULL, &ctx) != PF_OK) {
    fprintf(stderr, "pf_build: %s\n", pf_last_error());
    return 1;
  }
  pf_dims d;
  if (pf_get_dims(ctx, &d) != PF_OK || d.n_x != 4 || d.n_f != 2 || d.nnz != 4) {
    fprintf(stderr, "unexpected sizes\n");
    return 1;
  }
  const double state[4] = {0.0, -0.05, 1.0, 0.97};      /* theta_0, theta_1, V_0, V_1 */
  double F[2], J[4];
  int32_t rowptr[3], colind[4];
  if (pf_residual_jacobian_host(ctx, state, F, J, NULL) != PF_OK || pf_pattern(ctx, 0, rowptr, colind) != PF_OK ||
      pf_check_device(ctx, NULL) != PF_OK) {
    fprintf(stderr, "evaluation: %s\n", pf_last_error());
    return 1;
  }
  printf("F %.17g %.17g\n", F[0], F[1]);
  printf("J %.17g %.17g %.17g %.17g\n", J[0], J[1], J[2], J[3]);
  printf("rowptr %d %d %d\n", rowptr[0], rowptr[1], rowptr[2]);
  printf("colind %d %d %d %d\n", colind[0], colind[1], colind[2], colind[3]);
  pf_destroy(ctx);
  return 0;
}
