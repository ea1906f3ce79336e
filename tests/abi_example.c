/* A plain C99 client of the library's C ABI (no PyTorch, no C++): the host-only entry points, then
 * one context with the library's own allocator on the default stream.  Prints one line per call.
 * Built and run by tests/test_c_client.py. */
#include <stdio.h>
#include <stdlib.h>

#include "mhd.h"

int main(void) {
  printf("footprint %zu\n", mhd_footprint_bytes(64, MHD_FP64, 2));
  printf("footprint_bad %zu\n", mhd_footprint_bytes(48, MHD_FP64, 1));
  printf("shells %d\n", (int)mhd_num_shells(64));
  mhd_params p = {0};
  p.n = 16;
  p.batch = 1;
  p.precision = MHD_FP64;
  p.integrator = MHD_AB2;
  mhd_phys phys = {1e-2, 1e-2, 1.0};
  mhd_ctx *ctx = NULL;
  p.n = 48;
  printf("init_bad %d\n", (int)mhd_init(&p, &phys, &ctx));
  p.n = 16;
  mhd_status st = mhd_init(&p, &phys, &ctx);
  printf("init %d\n", (int)st);
  if (st == MHD_OK) {
    const size_t n3 = 16 * 16 * 16;
    double *rho = malloc(n3 * sizeof(double)), *u = calloc(3 * n3, sizeof(double)),
           *b = calloc(3 * n3, sizeof(double));
    for (size_t i = 0; i < n3; ++i) rho[i] = 1.0;
    printf("set %d\n", (int)mhd_set_state(ctx, 0, rho, u, b, 0));
    printf("step %d\n", (int)mhd_step(ctx, 3));
    printf("sync %d\n", (int)mhd_synchronize(ctx));
    mhd_diag d;
    printf("diag %d %lld\n", (int)mhd_diagnostics(ctx, 0, &d), (long long)d.step);
    free(rho);
    free(u);
    free(b);
    mhd_destroy(ctx);
  }
  return 0;
}
