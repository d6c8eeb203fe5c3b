/* A C program that drives the library through include/snap.h alone: a dry isothermal column
 * in the x-z plane (discretely hydrostatic reference built here), a seeded horizontal wind
 * and a warm anomaly; 20 CFL steps in FP64; the domain mass and the total of
 * rho e + rho g z must be conserved (closed box of free-slip walls), and the state must stay
 * finite. Prints "ok" and exits 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "snap.h"

#define NX 96
#define NZ 40

static int check(int rc, const char *what, snap_ctx *ctx) {
  if (rc != SNAP_OK) {
    fprintf(stderr, "%s failed: %s (%s)\n", what, snap_status_string(rc), snap_last_error(ctx));
    return 1;
  }
  return 0;
}

int main(void) {
  const double R = 287.0, g = 9.81, gam = 1.4, T0 = 300.0, dx = 50.0, dz = 50.0;
  double rho_bar[NZ], pf[NZ + 1];
  pf[0] = 1e5;
  for (int k = 0; k < NZ; ++k) { /* rho_k from the mean of its face pressures */
    double r = pf[k] / (R * T0);
    for (int it = 0; it < 100; ++it) r = (pf[k] - 0.5 * g * r * dz) / (R * T0);
    rho_bar[k] = r;
    pf[k + 1] = pf[k] - g * r * dz;
  }
  snap_grid_desc d = {0};
  d.nx = NX;
  d.ny = 1;
  d.nz = NZ;
  d.dx = dx;
  d.dy = dx;
  d.dz = dz;
  for (int s = 0; s < 6; ++s) d.bc[s] = SNAP_REFLECT;
  d.grav = g;
  d.gamma_d = gam;
  d.R_d = R;
  d.rho_bar = rho_bar;
  d.p_bar_face = pf;
  d.dtype = SNAP_F64;
  d.cfl = 0.8;
  d.satadj_max_iter = 20;
  d.satadj_tol = 1e-12;
  d.weno_eps = 1e-6;
  snap_ctx *ctx = NULL;
  if (check(snap_init_grid(&ctx, &d, 1), "snap_init_grid", NULL)) return 1;

  /* fields: rho, rho u, rho w, rho e (full energy) */
  const long n = (long)NX * NZ;
  double *Y = malloc(sizeof(double) * 4 * n);
  unsigned long long state = 1901029550ull;
  for (int k = 0; k < NZ; ++k)
    for (int i = 0; i < NX; ++i) {
      const long c = (long)k * NX + i;
      state = state * 6364136223846793005ull + 1442695040888963407ull;
      const double noise = (double)(state >> 11) / 9007199254740992.0 - 0.5;
      const double x = (i + 0.5) * dx, z = (k + 0.5) * dz;
      const double warm = exp(-((x - 2400.0) * (x - 2400.0) + (z - 600.0) * (z - 600.0)) / 1.6e5);
      const double p = 0.5 * (pf[k] + pf[k + 1]);
      const double rho = rho_bar[k] / (1.0 + 0.01 * warm); /* warmer at the same pressure */
      const double u = 2.0 * sin(6.283185307179586 * x / (NX * dx)) + 0.1 * noise;
      Y[c] = rho;
      Y[n + c] = rho * u;
      Y[2 * n + c] = 0.0;
      Y[3 * n + c] = p / (gam - 1.0) + 0.5 * rho * u * u;
    }
  if (check(snap_set_state(ctx, 0, Y, SNAP_F64, 0, NULL), "snap_set_state", ctx)) return 1;
  snap_budget b0, b1;
  if (check(snap_budget_compute(ctx, 0, &b0), "snap_budget_compute", ctx)) return 1;
  double dt = 0.0;
  if (check(snap_step(ctx, 20, 0.0, &dt, &b1), "snap_step", ctx)) return 1;
  if (check(snap_get_state(ctx, 0, Y, SNAP_F64, 0, NULL), "snap_get_state", ctx)) return 1;
  for (long c = 0; c < 4 * n; ++c)
    if (!isfinite(Y[c])) {
      fprintf(stderr, "non-finite state\n");
      return 1;
    }
  const double dm = fabs(b1.total[0] / b0.total[0] - 1.0);
  const double de = fabs(b1.energy_with_potential / b0.energy_with_potential - 1.0);
  /* five more steps from Y in one call, against set_state, the same steps and get_state */
  double *A = (double *)malloc(sizeof(double) * 4 * n), *B = (double *)malloc(sizeof(double) * 4 * n);
  if (!A || !B) return 1;
  if (check(snap_step_io(ctx, 0, Y, A, SNAP_F64, 5, 0.0), "snap_step_io", ctx)) return 1;
  if (check(snap_set_state(ctx, 0, Y, SNAP_F64, 0, NULL), "snap_set_state", ctx)) return 1;
  if (check(snap_step(ctx, 5, 0.0, NULL, NULL), "snap_step", ctx)) return 1;
  if (check(snap_get_state(ctx, 0, B, SNAP_F64, 0, NULL), "snap_get_state", ctx)) return 1;
  for (long c = 0; c < 4 * n; ++c)
    if (A[c] != B[c]) {
      fprintf(stderr, "snap_step_io differs at %ld\n", c);
      return 1;
    }
  free(A);
  free(B);
  snap_free(ctx);
  free(Y);
  if (!(dt > 0.0) || dm > 1e-12 || de > 1e-12) {
    fprintf(stderr, "dt %g mass drift %g energy drift %g\n", dt, dm, de);
    return 1;
  }
  printf("ok dt %.6g mass %.3g energy %.3g\n", dt, dm, de);
  return 0;
}
