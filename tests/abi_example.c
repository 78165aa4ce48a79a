/* C usage example of the libparo ABI: create a handle, set the potential,
 * iterate, destroy.  tests/test_library_abi.py compiles it with -Wall -Werror
 * and links it against the library. */
#include <math.h>
#include <stdio.h>
#include "paro.h"

/* d_Vq: 8*nx*ny*nz potential values at the Gauss points (device);
 * d_U: (n_interior x N) initial orbitals (device), overwritten by the Ritz vectors. */
int lowest_states(const double* d_Vq, double* d_U, int N, double* lambda /* host[N] */) {
  const double lo[3] = {-8, -8, -8}, hi[3] = {8, 8, 8};
  paro_mesh m;
  if (paro_mesh_create(&m, 64, 64, 64, lo, hi, PARO_MIXED, NULL) != PARO_OK) {
    fprintf(stderr, "%s\n", paro_last_error(NULL));
    return -1;
  }
  paro_params p;
  paro_default_params(&p);
  p.tol = 1e-8;     /* stop on max |delta lambda| < 1e-8 */
  lambda[0] = NAN;  /* start with a Rayleigh-Ritz step on span(U) */
  paro_stats s = {0};
  int rc = paro_set_potential(m, d_Vq, 0.0 /* sigma */);
  if (rc == PARO_OK) rc = paro_iterate(m, N, d_U, lambda, &p, &s);
  if (rc != PARO_OK) fprintf(stderr, "%s\n", paro_last_error(m));
  else printf("%d outer iterations, lambda_1 = %.10f\n", s.outer_iters, lambda[0]);
  paro_mesh_destroy(m);
  return rc;
}
