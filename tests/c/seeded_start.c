/* A C caller of the library, with no Python and no host-side generator:
 * creates a complex-double context, draws the seeded initial state of
 * Eq. fun through rotgp_init_analytic(seed) and writes the (N+1)^d points
 * (interleaved re, im doubles, x fastest) to a file.
 *
 * usage: seeded_start OUT SEED FUNCTION NX NY [NZ]   (spacings 0.2, 0.25, 0.3)
 */
#include <stdio.h>
#include <stdlib.h>

#include "rotgp.h"

int main(int argc, char** argv) {
  if (argc < 6) {
    fprintf(stderr, "usage: %s OUT SEED FUNCTION NX NY [NZ]\n", argv[0]);
    return 2;
  }
  rotgp_grid grid = {argc > 6 ? 3 : 2, {atoi(argv[4]), atoi(argv[5]), argc > 6 ? atoi(argv[6]) : 0},
                     {0.2, 0.25, 0.3}};
  rotgp_phys phys = {1.0, 1.1, 1.2, 10.0, 0.5, 1e-3};
  rotgp_ctx* ctx = NULL;
  int rc = rotgp_create(&grid, &phys, ROTGP_FP64, NULL, &ctx);
  if (rc) {
    fprintf(stderr, "create: %s\n", rotgp_last_error(NULL));
    return 1;
  }
  rc = rotgp_init_analytic(ctx, atoi(argv[3]), 1, strtoull(argv[2], NULL, 10), 1.0, 0.8);
  size_t pts = (size_t)(grid.n[0] + 1) * (grid.n[1] + 1) * (grid.dim == 3 ? grid.n[2] + 1 : 1);
  double* psi = (double*)malloc(pts * 2 * sizeof(double));
  if (!rc) rc = rotgp_get_psi(ctx, psi, 0, 1);
  if (rc) {
    fprintf(stderr, "rotgp: %s\n", rotgp_last_error(ctx));
    return 1;
  }
  FILE* f = fopen(argv[1], "wb");
  if (!f || fwrite(psi, sizeof(double), 2 * pts, f) != 2 * pts) return 1;
  fclose(f);
  free(psi);
  rotgp_destroy(ctx);
  return 0;
}
