/* snap_oracle.c -- plain FP64 CPU reference of one SNAP finite-volume step.
 *
 * TEST INFRASTRUCTURE: called only by the tests, the smoke check and the CPU-baseline leg
 * of the benchmark. Nothing in the product library links, loads or calls it, and it
 * shares no code with the CUDA path. Whole-array loops in the order the paper states the
 * method; no blocking, fusion or reordering.
 *
 * Paper: C. Li and X. Chen, ApJS 2019 (arXiv 1901.02955). Each function names the
 * passage it follows; readings of passages the paper leaves open are marked READING.
 */
#include "snap_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------------------
 * layout helpers
 * ------------------------------------------------------------------------------------- */
static int nmom_of(const orc_grid *g) { return g->ny > 1 ? 3 : 2; }
static int im0_of(const orc_grid *g) { return 1 + g->nvap + g->nvap * g->ncond; }
int orc_nvar(const orc_grid *g) { return im0_of(g) + nmom_of(g) + 1; }
static int icond(const orc_grid *g, int i, int j) { return 1 + g->nvap + i * g->ncond + j; }
/* momentum slot of spatial direction d (0 x, 1 y, 2 z) */
static int mom_slot(const orc_grid *g, int d) {
  if (g->ny > 1) return im0_of(g) + d;
  return im0_of(g) + (d == 2 ? 1 : 0);
}

/* Thermodynamic constants per unit mass (Sec. 2 and App. A):
 *   c_vd = R_d/(gamma_d-1), R_i = R_d/eps_i, c_vi = sigma_vi c_vd, c_pi = c_vi + R_i,
 *   c_ij = sigma_ij c_vd, dc_ij = c_ij - c_pi (Eq. latent),
 *   mu_ij = mu_i - (L^r_ij + dc_ij T^r) with mu_i = 0 (Eq. muij). */
static double c_vd(const orc_grid *g) { return g->Rd / (g->gamma_d - 1.0); }
static double R_vap(const orc_grid *g, int i) { return g->Rd / g->eps[i]; }
static double c_pv(const orc_grid *g, int i) { return g->sig_v[i] * c_vd(g) + R_vap(g, i); }
static double dc_of(const orc_grid *g, int i, int j) {
  return g->sig_c[i][j] * c_vd(g) - c_pv(g, i);
}
static double mu_of(const orc_grid *g, int i, int j) {
  return -(g->Lref[i][j] + dc_of(g, i, j) * g->Tref[i]);
}

/* ---------------------------------------------------------------------------------------
 * Sec. 4.2, Eq. weno5: fifth-order WENO interpolant to the face i-1/2 from the left,
 * q = (Q_{i-3}, Q_{i-2}, Q_{i-1}, Q_i, Q_{i+1}).
 * READING: the nonlinear weights are those of Jiang & Shu (1996), which the paper cites
 * without printing: smoothness indicators beta_k of the three 3-cell stencils,
 * alpha_k = d_k / (eps + beta_k)^2 with d = (0.1, 0.6, 0.3), normalised to sum 1.
 * ------------------------------------------------------------------------------------- */
static void weno5_betas(const double q[5], double b[3]) {
  double t;
  t = q[0] - 2.0 * q[1] + q[2];
  b[0] = 13.0 / 12.0 * t * t;
  t = q[0] - 4.0 * q[1] + 3.0 * q[2];
  b[0] += 0.25 * t * t;
  t = q[1] - 2.0 * q[2] + q[3];
  b[1] = 13.0 / 12.0 * t * t;
  t = q[1] - q[3];
  b[1] += 0.25 * t * t;
  t = q[2] - 2.0 * q[3] + q[4];
  b[2] = 13.0 / 12.0 * t * t;
  t = 3.0 * q[2] - 4.0 * q[3] + q[4];
  b[2] += 0.25 * t * t;
}

void orc_weno5_weights(const double q[5], double eps, double w[3]) {
  static const double d[3] = {0.1, 0.6, 0.3};
  double b[3], a[3], s = 0.0;
  weno5_betas(q, b);
  for (int k = 0; k < 3; ++k) {
    a[k] = d[k] / ((eps + b[k]) * (eps + b[k]));
    s += a[k];
  }
  for (int k = 0; k < 3; ++k) w[k] = a[k] / s;
}

double orc_weno5(const double q[5], double eps) {
  double w[3];
  orc_weno5_weights(q, eps, w);
  /* the three third-order candidate interpolants of Eq. weno5 */
  double v0 = q[0] / 3.0 - 7.0 / 6.0 * q[1] + 11.0 / 6.0 * q[2];
  double v1 = -q[1] / 6.0 + 5.0 / 6.0 * q[2] + q[3] / 3.0;
  double v2 = q[2] / 3.0 + 5.0 / 6.0 * q[3] - q[4] / 6.0;
  return w[0] * v0 + w[1] * v1 + w[2] * v2;
}

/* Sec. 4.2: the fifth-order polynomial interpolant I_poly. */
double orc_weno5_poly(const double q[5]) {
  return q[0] / 30.0 - 13.0 / 60.0 * q[1] + 47.0 / 60.0 * q[2] + 9.0 / 20.0 * q[3] -
         q[4] / 20.0;
}

/* ---------------------------------------------------------------------------------------
 * App. B: conserved Y -> primitive X = (rho, q_i, q_ij, u, [v], w, p), plus T (Eq. eos)
 * and the effective adiabatic index gamma.
 * ------------------------------------------------------------------------------------- */
static void mix_factors(const orc_grid *g, const double *X, double *num, double *den) {
  /* num = 1 + sum q_i (sigma_vi - 1) + sum q_ij (sigma_ij - 1)
   * den = 1 + sum q_i (1/eps_i - 1) - sum q_ij                       (App. B, Eq. p2) */
  double n = 1.0, d = 1.0;
  for (int i = 0; i < g->nvap; ++i) {
    n += X[1 + i] * (g->sig_v[i] - 1.0);
    d += X[1 + i] * (1.0 / g->eps[i] - 1.0);
    for (int j = 0; j < g->ncond; ++j) {
      double qij = X[icond(g, i, j)];
      n += qij * (g->sig_c[i][j] - 1.0);
      d -= qij;
    }
  }
  *num = n;
  *den = d;
}

void orc_cons_to_prim(const orc_grid *g, const double *Y, double *X, double *T, double *gamma) {
  const int im0 = im0_of(g), nm = nmom_of(g), nv = orc_nvar(g);
  double rho = 0.0;
  for (int s = 0; s < im0; ++s) rho += Y[s];
  X[0] = rho;
  for (int s = 1; s < im0; ++s) X[s] = Y[s] / rho;
  double K = 0.0;
  for (int m = 0; m < nm; ++m) {
    X[im0 + m] = Y[im0 + m] / rho;
    K += 0.5 * rho * X[im0 + m] * X[im0 + m];
  }
  double A = 0.0;
  for (int i = 0; i < g->nvap; ++i)
    for (int j = 0; j < g->ncond; ++j) A += mu_of(g, i, j) * Y[icond(g, i, j)];
  double U = Y[nv - 1] - K - A;
  double num, den;
  mix_factors(g, X, &num, &den);
  double p = (g->gamma_d - 1.0) * den / num * U;
  X[nv - 1] = p;
  if (T) *T = p / (rho * g->Rd * den);
  if (gamma) *gamma = 1.0 + (g->gamma_d - 1.0) * den / num;
}

void orc_prim_to_cons(const orc_grid *g, const double *X, double *Y) {
  const int im0 = im0_of(g), nm = nmom_of(g), nv = orc_nvar(g);
  double rho = X[0], rd = rho;
  for (int s = 1; s < im0; ++s) {
    Y[s] = rho * X[s];
    rd -= Y[s];
  }
  Y[0] = rd;
  double K = 0.0;
  for (int m = 0; m < nm; ++m) {
    Y[im0 + m] = rho * X[im0 + m];
    K += 0.5 * rho * X[im0 + m] * X[im0 + m];
  }
  double A = 0.0;
  for (int i = 0; i < g->nvap; ++i)
    for (int j = 0; j < g->ncond; ++j) A += mu_of(g, i, j) * Y[icond(g, i, j)];
  double num, den;
  mix_factors(g, X, &num, &den);
  Y[nv - 1] = num / den * X[nv - 1] / (g->gamma_d - 1.0) + K + A;
}

/* App. D: integrated Clausius-Clapeyron relation over condensate (i,1):
 * p* = p^r exp[beta (1 - 1/t) - delta ln t], t = T/T^r, beta = (L^r + dc T^r)/(R_i T^r),
 * delta = dc/R_i. */
double orc_sat_pressure(const orc_grid *g, int i, double T) {
  double Ri = R_vap(g, i), dc = dc_of(g, i, 0);
  double beta = (g->Lref[i][0] + dc * g->Tref[i]) / (Ri * g->Tref[i]);
  double delta = dc / Ri;
  double t = T / g->Tref[i];
  return g->pref[i] * exp(beta * (1.0 - 1.0 / t) - delta * log(t));
}

/* ---------------------------------------------------------------------------------------
 * Sec. 4.1, Eqs. rp and ru: LMARS.
 * READINGS (the paper defers details to Chen et al. 2013):
 *  - rho c = (rho_L + rho_R)/2 * (c_L + c_R)/2 with c^2 = gamma p / rho (gamma of App. B).
 *  - Eqs. rp/ru use the pressure perturbation p' = p - pref ("perturbation pressure in the
 *    vertical"); a constant pref cancels from both, so the same form serves every face.
 *  - Flux = u* Phi_S + p'* n, with S the upwind side (left if u* > 0, else right) and
 *    Phi = (rho_d, rho_i, rho_ij, rho u, [rho v], rho w, rho e + p) built from the
 *    reconstructed primitives of side S; p in rho e + p is the total pressure pref + p'_S.
 *    The reference pressure's own momentum flux is accounted for in the gravity source.
 * ------------------------------------------------------------------------------------- */
void orc_lmars(const orc_grid *g, const double *XL, const double *XR, int dir, double pref,
               double *F, double *ustar, double *pstar) {
  const int im0 = im0_of(g), nm = nmom_of(g), nv = orc_nvar(g);
  const int mn = mom_slot(g, dir);
  double numL, denL, numR, denR;
  mix_factors(g, XL, &numL, &denL);
  mix_factors(g, XR, &numR, &denR);
  double pL = pref + XL[nv - 1], pR = pref + XR[nv - 1];
  double gamL = 1.0 + (g->gamma_d - 1.0) * denL / numL;
  double gamR = 1.0 + (g->gamma_d - 1.0) * denR / numR;
  double cL = sqrt(gamL * pL / XL[0]), cR = sqrt(gamR * pR / XR[0]);
  double rhoc = 0.5 * (XL[0] + XR[0]) * 0.5 * (cL + cR);
  double uL = XL[mn], uR = XR[mn];
  double ps = 0.5 * (XL[nv - 1] + XR[nv - 1]) - 0.5 * rhoc * (uR - uL); /* Eq. rp */
  double us = 0.5 * (uL + uR) - (XR[nv - 1] - XL[nv - 1]) / (2.0 * rhoc); /* Eq. ru */
  const double *XS = us > 0.0 ? XL : XR;
  double numS = us > 0.0 ? numL : numR, denS = us > 0.0 ? denL : denR;
  double pS = us > 0.0 ? pL : pR;
  double rhoS = XS[0];
  double mflux = us * rhoS;
  double qsum = 0.0;
  for (int s = 1; s < im0; ++s) {
    F[s] = mflux * XS[s];
    qsum += XS[s];
  }
  F[0] = mflux * (1.0 - qsum);
  double K = 0.0;
  for (int m = 0; m < nm; ++m) {
    F[im0 + m] = mflux * XS[im0 + m];
    K += 0.5 * rhoS * XS[im0 + m] * XS[im0 + m];
  }
  F[mn] += ps;
  double A = 0.0;
  for (int i = 0; i < g->nvap; ++i)
    for (int j = 0; j < g->ncond; ++j) A += mu_of(g, i, j) * rhoS * XS[icond(g, i, j)];
  double rhoe = numS / denS * pS / (g->gamma_d - 1.0) + K + A; /* App. B */
  F[nv - 1] = us * (rhoe + pS);
  if (ustar) *ustar = us;
  if (pstar) *pstar = ps;
}

/* ---------------------------------------------------------------------------------------
 * App. D: isochoric saturation adjustment of one cell.
 * READINGS:
 *  - Each vapour i exchanges mass only with its first condensate (cloud, j = 1); further
 *    condensates (precipitation) are left unchanged.
 *  - One sweep visits the vapours in table order; each computes the projected molar
 *    transfer dq of Eq. dxf with the isochoric alpha (App. D, second form, which carries
 *    the 1/T the first form omits), limits it to [-q_cloud, q_vapour], and moves the mass.
 *    Temperature and pressure are then recomputed exactly from the conserved total energy
 *    (Eq. energy) and the equation of state (Eq. eos); rho_d, rho e and the momenta never
 *    change. If p* >= p (s >= 1, boiling) the cloud evaporates entirely.
 *  - Stop when every |dq| <= tol (q_vapour + q_cloud) in a sweep, or report -1 after
 *    max_iter sweeps.
 * Molar fractions count condensates among the moles (App. D): with
 * N = rho_d + sum_k (rho_k + sum_j rho_kj)/eps_k, q^_i = rho_i/(eps_i N).
 * ------------------------------------------------------------------------------------- */
int orc_satadj_cell(const orc_grid *g, double *Y, int max_iter, double tol) {
  const int nv = orc_nvar(g);
  double X[64], T;
  if (g->nvap == 0 || g->ncond == 0) return 0;
  for (int sweep = 1; sweep <= max_iter; ++sweep) {
    int converged = 1;
    for (int i = 0; i < g->nvap; ++i) {
      orc_cons_to_prim(g, Y, X, &T, NULL);
      double p = X[nv - 1];
      double N = Y[0], gas = Y[0], heat = 0.0;
      for (int k = 0; k < g->nvap; ++k) {
        double tot = Y[1 + k];
        for (int j = 0; j < g->ncond; ++j) tot += Y[icond(g, k, j)];
        N += tot / g->eps[k];
        gas += Y[1 + k] / g->eps[k];
      }
      for (int k = 0; k < g->nvap; ++k) {
        double tot = Y[1 + k];
        for (int j = 0; j < g->ncond; ++j) tot += Y[icond(g, k, j)];
        /* (q^_k + sum_j q^_kj)(sigma^_vk - 1), sigma^_vk = c^_vk / c^_vd = sigma_vk eps_k */
        heat += tot / (g->eps[k] * N) * (g->sig_v[k] * g->eps[k] - 1.0);
      }
      double qv = Y[1 + i] / (g->eps[i] * N);
      double qc = Y[icond(g, i, 0)] / (g->eps[i] * N);
      double gsum = gas / N - qv; /* other gases */
      double s = orc_sat_pressure(g, i, T) / p;
      double dq;
      if (s >= 1.0) {
        dq = -qc;
      } else {
        double Ri = R_vap(g, i), dc = dc_of(g, i, 0);
        double beta = (g->Lref[i][0] + dc * g->Tref[i]) / (Ri * g->Tref[i]);
        double delta = dc / Ri;
        double t = T / g->Tref[i];
        double alpha = (g->gamma_d - 1.0) * (beta / t - delta - 1.0) / (1.0 + heat);
        double r = s / (1.0 - s);
        dq = (qv - r * gsum) /
             (1.0 + s / ((1.0 - s) * (1.0 - s)) * (beta / t - delta) * alpha * gsum);
      }
      /* positivity limit; at a limit the whole phase moves, exactly */
      double drho;
      if (dq >= qv) {
        dq = qv;
        drho = Y[1 + i];
      } else if (dq <= -qc) {
        dq = -qc;
        drho = -Y[icond(g, i, 0)];
      } else {
        drho = dq * g->eps[i] * N;
      }
      Y[1 + i] -= drho;
      Y[icond(g, i, 0)] += drho;
      if (fabs(dq) > tol * (qv + qc)) converged = 0;
    }
    if (converged) return sweep;
  }
  return -1;
}

/* ---------------------------------------------------------------------------------------
 * Sec. 3: the Kessler scheme, integrated by backward Euler (Eq. x_n+1). For vapour i with
 * cloud c = (i,1) and precipitation r = (i,2), in mass mixing ratios of the total density
 * (fixed by the reactions, like rho_d and rho e):
 *   Phi_v = -k1 (q_v - q*)^+ + k4 q_r (q* - q_v)^+
 *   Phi_c =  k1 (q_v - q*)^+ - k3 q_c q_r - k2 q_c
 *   Phi_r = -k4 q_r (q* - q_v)^+ + k3 q_c q_r + k2 q_c
 * with q* = p*_i(T) / (R_i T rho) the saturation mixing ratio over the cloud.
 * READINGS: Newton iterations X^m = X^{m-1} + (I/dt - J)^-1 [Phi(X^{m-1}) - (X^{m-1} -
 * X^n)/dt], with T (hence q*) recomputed from the conserved energy at every iteration, on
 * one form of the rates at a time (see orc_kessler_cell). The
 * printed Jacobians hold q* fixed and leave out the derivatives of the evaporation term with
 * respect to q_r. Here J is the full Jacobian: those derivatives, and q* varying through T,
 * which the reactions change at fixed rho e and rho (dT/dq_k = -rho (mu_k + c_k T) / C_v with
 * mu_k, c_k of vapour, cloud or rain, and d(q*)/dT = q* ((beta/t - delta) - 1)/T from App. D).
 * With q* held, fast condensation (k1 dt >> 1) makes the iteration diverge: the latent heat
 * of the condensed vapour raises q* by a few times the condensed amount (about 4x for water
 * near 300 K). The fixed point, the backward Euler solution, is the same. Vapours are treated
 * one after the other; the iteration stops when |dX| <= tol (q_v + q_c + q_r).
 * ------------------------------------------------------------------------------------- */
/* Kessler rates Phi of vapour i at mixing ratios x (density rho fixed), the backward Euler
 * residual G = Phi - (x - xn)/dt, and (with J != NULL) its Jacobian dG/dx = J - I/dt with J
 * the full Jacobian of Phi (see the readings above). Y holds the cell and is updated to x. */
static void kessler_residual(const orc_grid *g, double *Y, int i, double rho, const double x[3],
                             const double xn[3], double dt, int saturated, double G[3],
                             double J[3][3], double *sup_out) {
  const int vi = 1 + i, ci = icond(g, i, 0), ri = icond(g, i, 1);
  const double k1 = g->kessler_k[0], k2 = g->kessler_k[1], k3 = g->kessler_k[2],
               k4 = g->kessler_k[3];
  double X[64], T;
  Y[vi] = rho * x[0];
  Y[ci] = rho * x[1];
  Y[ri] = rho * x[2];
  orc_cons_to_prim(g, Y, X, &T, NULL);
  const double qs = orc_sat_pressure(g, i, T) / (R_vap(g, i) * T * rho);
  const double sup = x[0] - qs;
  if (sup_out) *sup_out = sup;
  double phi[3];
  if (saturated) {
    phi[0] = -k1 * sup;
    phi[1] = k1 * sup - k3 * x[1] * x[2] - k2 * x[1];
    phi[2] = k3 * x[1] * x[2] + k2 * x[1];
  } else {
    phi[0] = -k4 * x[2] * sup;
    phi[1] = -k3 * x[1] * x[2] - k2 * x[1];
    phi[2] = k4 * x[2] * sup + k3 * x[1] * x[2] + k2 * x[1];
  }
  for (int r = 0; r < 3; ++r) G[r] = phi[r] - (x[r] - xn[r]) / dt;
  if (!J) return;
  /* d(q*)/dX_k through T at fixed energy */
  double Cv = c_vd(g) * Y[0];
  for (int a = 0; a < g->nvap; ++a) {
    Cv += g->sig_v[a] * c_vd(g) * Y[1 + a];
    for (int b = 0; b < g->ncond; ++b) Cv += g->sig_c[a][b] * c_vd(g) * Y[icond(g, a, b)];
  }
  const double Ri = R_vap(g, i), dc = dc_of(g, i, 0);
  const double beta = (g->Lref[i][0] + dc * g->Tref[i]) / (Ri * g->Tref[i]);
  const double delta = dc / Ri, tt = T / g->Tref[i];
  const double dqs = qs * ((beta / tt - delta) - 1.0) / T;
  const double dTdq[3] = {-rho * (g->sig_v[i] * c_vd(g) * T) / Cv,
                          -rho * (mu_of(g, i, 0) + g->sig_c[i][0] * c_vd(g) * T) / Cv,
                          -rho * (mu_of(g, i, 1) + g->sig_c[i][1] * c_vd(g) * T) / Cv};
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) J[r][q] = 0.0;
  /* d sup / dx_q = delta_q0 - dqs dTdq[q] */
  double dsup[3];
  for (int q = 0; q < 3; ++q) dsup[q] = (q == 0 ? 1.0 : 0.0) - dqs * dTdq[q];
  if (saturated) {
    for (int q = 0; q < 3; ++q) {
      J[0][q] += -k1 * dsup[q];
      J[1][q] += k1 * dsup[q];
    }
  } else {
    for (int q = 0; q < 3; ++q) {
      J[0][q] += -k4 * x[2] * dsup[q];
      J[2][q] += k4 * x[2] * dsup[q];
    }
    J[0][2] += -k4 * sup;
    J[2][2] += k4 * sup;
  }
  J[1][1] += -k2 - k3 * x[2];
  J[1][2] += -k3 * x[1];
  J[2][1] += k2 + k3 * x[2];
  J[2][2] += k3 * x[1];
  for (int r = 0; r < 3; ++r) J[r][r] -= 1.0 / dt;
}

/* Newton iterations on one form of the rates (saturated or not), each smooth in X; the
 * unknowns are (q_v, q_c) with q_r = tot - q_v - q_c. Returns the iteration count (x
 * converged), or -1; *sup receives q_v - q* at the result. */
static int kessler_branch(const orc_grid *g, double *Y, int i, double rho, const double xn[3],
                          double dt, int saturated, double x[3], double *sup) {
  const double tot = xn[0] + xn[1] + xn[2];
  x[0] = xn[0];
  x[1] = xn[1];
  x[2] = xn[2];
  for (int m = 1; m <= g->kessler_max_iter; ++m) {
    double G[3], J[3][3], dx[3];
    kessler_residual(g, Y, i, rho, x, xn, dt, saturated, G, J, sup);
    /* Newton step on the first two equations: (dG_r/dq_q - dG_r/dq_r) d = -G_r, r, q < 2 */
    const double a00 = J[0][0] - J[0][2], a01 = J[0][1] - J[0][2];
    const double a10 = J[1][0] - J[1][2], a11 = J[1][1] - J[1][2];
    const double det = a00 * a11 - a01 * a10;
    dx[0] = (-G[0] * a11 + G[1] * a01) / det;
    dx[1] = (-G[1] * a00 + G[0] * a10) / det;
    x[0] += dx[0];
    x[1] += dx[1];
    x[2] = tot - x[0] - x[1];
    if (fabs(dx[0]) + fabs(dx[1]) <= g->kessler_tol * (fabs(x[0]) + fabs(x[1]) + fabs(x[2]))) {
      kessler_residual(g, Y, i, rho, x, xn, dt, saturated, G, NULL, sup);
      return m;
    }
  }
  return -1;
}

int orc_kessler_cell(const orc_grid *g, double *Y, double dt) {
  const int im0 = im0_of(g);
  if (!g->kessler || g->nvap == 0 || g->ncond < 2) return 0;
  double rho = 0.0;
  for (int s = 0; s < im0; ++s) rho += Y[s];
  int worst = 0;
  for (int i = 0; i < g->nvap; ++i) {
    const int vi = 1 + i, ci = icond(g, i, 0), ri = icond(g, i, 1);
    const double xn[3] = {Y[vi] / rho, Y[ci] / rho, Y[ri] / rho};
    /* the rates change form where the vapour crosses saturation: solve with the form of the
     * initial state, and with the other form if the result lies on the wrong side (the rates
     * are continuous there, so the backward Euler solution lies on one side or on the edge) */
    double x[3], sup, sup_n;
    kessler_residual(g, Y, i, rho, xn, xn, dt, 1, x, NULL, &sup_n);
    int first = sup_n > 0.0, it = -1, accepted = 0;
    for (int attempt = 0; attempt < 2 && !accepted; ++attempt) {
      const int sat = attempt == 0 ? first : !first;
      it = kessler_branch(g, Y, i, rho, xn, dt, sat, x, &sup);
      if (it > 0 && (sat ? sup > 0.0 : sup <= 0.0)) accepted = 1;
    }
    if (!accepted) {
      /* the solution sits on the edge: vapour at saturation, the saturated form's result */
      it = kessler_branch(g, Y, i, rho, xn, dt, 1, x, &sup);
    }
    Y[vi] = rho * x[0];
    Y[ci] = rho * x[1];
    Y[ri] = rho * x[2];
    if (it < 0) worst = -1;
    else if (worst >= 0 && it > worst) worst = it;
  }
  return worst;
}

/* App. A, Eq. theta_e: theta_e = T (p0/p_d)^(R_d q_d / c) exp(L q_v / (c T)), c = c_pd q_d +
 * c_l q_t, with the mass fractions q of the total density, q_t = q_v + q_cloud, p_d the
 * partial pressure of dry air, L = L^r - (c_l - c_pv)(T - T^r) the latent heat at T (Eq.
 * latent) and c_l the cloud's heat capacity. */
int orc_theta_e(const orc_grid *g, const double *Y, double *theta_e) {
  if (g->nvap != 1 || g->ncond < 1) return -3;
  const int nv = orc_nvar(g), im0 = im0_of(g);
  const long ncell = (long)g->nx * g->ny * g->nz;
  const double cpd = g->gamma_d * c_vd(g), cl = g->sig_c[0][0] * c_vd(g);
  const double dc = dc_of(g, 0, 0);
  double Yc[64], X[64], T;
  for (long c = 0; c < ncell; ++c) {
    for (int v = 0; v < nv; ++v) Yc[v] = Y[v * ncell + c];
    orc_cons_to_prim(g, Yc, X, &T, NULL);
    double rho = 0.0;
    for (int s = 0; s < im0; ++s) rho += Yc[s];
    const double qd = Yc[0] / rho, qv = Yc[1] / rho, qt = (Yc[1] + Yc[icond(g, 0, 0)]) / rho;
    const double pd = Yc[0] * g->Rd * T;
    const double L = g->Lref[0][0] - dc * (T - g->Tref[0]);
    const double cc = cpd * qd + cl * qt;
    theta_e[c] = T * pow(1e5 / pd, g->Rd * qd / cc) * exp(L * qv / (cc * T));
  }
  return 0;
}

/* Exact equilibrium of the same cell (test pin): the internal energy U = rho e - K is fixed;
 * at trial temperature T each vapour holds min(total_i, p*_i(T)/(R_i T)) and its cloud the
 * rest; F(T) = C_v(T) T + A(T) - U is strictly increasing, so bisection finds the root. */
static double satadj_residual(const orc_grid *g, const double *Y0, double U, double T,
                              double *Yout) {
  const int nv = orc_nvar(g);
  memcpy(Yout, Y0, sizeof(double) * (size_t)nv);
  for (int i = 0; i < g->nvap; ++i) {
    double tot = Y0[1 + i] + Y0[icond(g, i, 0)];
    double v = orc_sat_pressure(g, i, T) / (R_vap(g, i) * T);
    if (v > tot) v = tot;
    Yout[1 + i] = v;
    Yout[icond(g, i, 0)] = tot - v;
  }
  double Cv = Yout[0];
  double A = 0.0;
  for (int i = 0; i < g->nvap; ++i) {
    Cv += g->sig_v[i] * Yout[1 + i];
    for (int j = 0; j < g->ncond; ++j) {
      Cv += g->sig_c[i][j] * Yout[icond(g, i, j)];
      A += mu_of(g, i, j) * Yout[icond(g, i, j)];
    }
  }
  Cv *= c_vd(g);
  return Cv * T + A - U;
}

int orc_satadj_bisect(const orc_grid *g, double *Y) {
  const int im0 = im0_of(g), nm = nmom_of(g), nv = orc_nvar(g);
  double rho = 0.0, K = 0.0, Yt[64];
  for (int s = 0; s < im0; ++s) rho += Y[s];
  for (int m = 0; m < nm; ++m) K += 0.5 * Y[im0 + m] * Y[im0 + m] / rho;
  double U = Y[nv - 1] - K;
  double lo = 10.0, hi = 5000.0;
  if (satadj_residual(g, Y, U, lo, Yt) > 0.0 || satadj_residual(g, Y, U, hi, Yt) < 0.0)
    return -1;
  for (int it = 0; it < 400 && hi - lo > 1e-15 * hi; ++it) {
    double mid = 0.5 * (lo + hi);
    if (satadj_residual(g, Y, U, mid, Yt) > 0.0)
      hi = mid;
    else
      lo = mid;
  }
  satadj_residual(g, Y, U, 0.5 * (lo + hi), Yt);
  memcpy(Y, Yt, sizeof(double) * (size_t)nv);
  return 0;
}

/* ---------------------------------------------------------------------------------------
 * Whole-grid right-hand side L(Y) of Eq. forward.
 * Primitive cell values are held with three ghost cells per side in each active direction.
 * READINGS:
 *  - Boundaries: a reflecting side mirrors every primitive and negates the normal velocity;
 *    a periodic side wraps. The vertical direction must be reflecting.
 *  - The pressure carried in the primitive vector is the perturbation p' = p - pbar_k about
 *    the fixed reference state (cell value pbar_k = (pbar_{k-1/2} + pbar_{k+1/2})/2), in all
 *    directions; ghosts mirror p'. Faces of level k use pbar_k as reference in x and y and
 *    pbar_{k-1/2} on the lower z face.
 *  - Vertical momentum source: -(rho_k - rho_bar_k) g, the gravity term of Eq. mom3 once
 *    the reference profile's discrete hydrostatic balance
 *    (pbar_{k+1/2} - pbar_{k-1/2})/dz = -g rho_bar_k is taken out of the pressure flux.
 *  - Energy source -rho g w (Sec. 2) is discretised as -g (F_rho,k-1/2 + F_rho,k+1/2)/2 from
 *    the vertical total-mass fluxes, so the sum of rho e + rho g z is conserved in a closed
 *    box; the pointwise -g (rho w)_k form is available as an option.
 *  - Constant viscosity (used by the density-current workload; Sec. 5.1 applies it to
 *    momentum and to the thermodynamic equation): at each face, from the two adjacent cell
 *    values, the momentum flux -rho_f nu du/dn and the energy flux
 *    -rho_f nu u_f . du/dn - rho_f c_pd nu Pi_f dtheta/dn, where theta = T / Pi and
 *    Pi = (p / 1e5 Pa)^(R_d/c_pd) (App. C, Eq. theta, dry); the subscript f is the mean of
 *    the two cells. Ghost cells mirror theta, so no heat crosses a wall, except below a
 *    fixed bottom temperature (Sec. 6), whose ghosts hold theta = T_bottom / Pi; a no-slip
 *    wall's ghosts carry the reversed tangential velocity, so the wall exerts a stress.
 *  - Lower boundary of the Jovian simulation (Sec. 6; READING): a no-slip wall and a fixed
 *    temperature are set in the ghost cells below z = 0, which mirror pressure, composition
 *    and (negated) velocity and hold T_bottom, their density scaled by T / T_bottom at that
 *    pressure. The mirrored pressure and normal velocity keep u* = 0 at the wall, so no mass
 *    or energy is advected through it; in an inviscid run the fixed temperature only enters
 *    the reconstruction next to the wall, with viscosity it drives the heat flux above.
 * ------------------------------------------------------------------------------------- */
typedef struct {
  int nxe, nye, nze, ox, oy, oz;
} ext_dims;

static long ext_index(const ext_dims *e, int k, int j, int i) {
  return ((long)(k + e->oz) * e->nye + (j + e->oy)) * e->nxe + (i + e->ox);
}

static int wrap_or_mirror(int idx, int n, int bc_lo, int bc_hi, int *flip) {
  *flip = 0;
  if (idx < 0) {
    if (bc_lo == ORC_PERIODIC) return ((idx % n) + n) % n;
    *flip = 1;
    return -1 - idx;
  }
  if (idx >= n) {
    if (bc_hi == ORC_PERIODIC) return idx % n;
    *flip = 1;
    return 2 * n - 1 - idx;
  }
  return idx;
}

static double pbar_cell(const orc_grid *g, int k) {
  return 0.5 * (g->p_bar_face[k] + g->p_bar_face[k + 1]);
}

/* Velocities of a ghost cell that mirrors a cell across a wall normal to direction d: a
 * free-slip wall negates the normal velocity only, a no-slip wall every component (Sec. 6,
 * the no-slip lower boundary of the Jovian simulation). */
static void wall_ghost(const orc_grid *g, double *X, long next, long dst, int d, int bc) {
  if (bc == ORC_NOSLIP) {
    for (int m = 0; m < nmom_of(g); ++m) X[(long)(im0_of(g) + m) * next + dst] *= -1.0;
  } else {
    X[(long)mom_slot(g, d) * next + dst] *= -1.0;
  }
}

/* Sec. 2, Eq. d3 and the momentum and energy equations with sedimentation: a condensate
 * (i,j) with terminal velocity w^t_j carries through a z face the extra fluxes
 *   mass w^t rho_ij, momentum w^t rho_ij u_m, energy w^t rho_ij e_ij,
 *   e_ij = c_ij T + |u|^2/2 + mu_ij (Sec. 2).
 * READINGS: the face values come from the reconstructed state on the side the condensate
 * comes from (above when w^t < 0); no condensate passes a wall (free-slip or no-slip), so
 * precipitation collects in the lowest layer; the frictional heating -sum rho_ij g w^t of the
 * energy equation is the sedimentation part of -g F_rho in the gravity source of orc_rhs,
 * whose total-mass flux includes these mass fluxes. */
static void sedimentation_flux(const orc_grid *g, const double *XL, const double *XR,
                               double pref, int k, double *F) {
  const int im0 = im0_of(g), nm = nmom_of(g), nv = orc_nvar(g);
  if ((k == 0 && g->bc[4] != ORC_PERIODIC) || (k == g->nz && g->bc[5] != ORC_PERIODIC)) return;
  for (int j = 0; j < g->ncond; ++j) {
    const double wt = g->w_term[j];
    if (wt == 0.0) continue;
    const double *XS = wt < 0.0 ? XR : XL;
    double num, den, u2 = 0.0;
    mix_factors(g, XS, &num, &den);
    const double T = (pref + XS[nv - 1]) / (XS[0] * g->Rd * den);
    for (int m = 0; m < nm; ++m) u2 += XS[im0 + m] * XS[im0 + m];
    for (int i = 0; i < g->nvap; ++i) {
      const int c = icond(g, i, j);
      const double ms = wt * XS[0] * XS[c];
      F[c] += ms;
      for (int m = 0; m < nm; ++m) F[im0 + m] += ms * XS[im0 + m];
      F[nv - 1] += ms * (g->sig_c[i][j] * c_vd(g) * T + 0.5 * u2 + mu_of(g, i, j));
    }
  }
}

int orc_rhs(const orc_grid *g, const double *Y, double *dYdt) {
  const int nx = g->nx, ny = g->ny, nz = g->nz, nv = orc_nvar(g), im0 = im0_of(g);
  const int three_d = ny > 1;
  if (nx < 1 || ny < 1 || nz < 3) return -1;
  if (g->bc[4] == ORC_PERIODIC || g->bc[5] == ORC_PERIODIC) return -1; /* z: walls */
  if ((g->bc[0] != ORC_PERIODIC || g->bc[1] != ORC_PERIODIC) && nx < 3) return -1;
  if (three_d && (g->bc[2] != ORC_PERIODIC || g->bc[3] != ORC_PERIODIC) && ny < 3) return -1;
  if (!(g->T_bottom >= 0.0)) return -1;
  ext_dims e = {nx + 6, three_d ? ny + 6 : 1, nz + 6, 3, three_d ? 3 : 0, 3};
  const long next = (long)e.nxe * e.nye * e.nze;
  const long ncell = (long)nx * ny * nz;
  double *X = calloc((size_t)(nv * next), sizeof(double));
  double *Tx = calloc((size_t)next, sizeof(double));  /* theta */
  double *Px = calloc((size_t)next, sizeof(double));  /* Pi */
  double *F = malloc(sizeof(double) * (size_t)nv * (size_t)(nx + 1) * (ny + 1) * (nz + 1));
  double *Frho_z = malloc(sizeof(double) * (size_t)nx * ny * (nz + 1));
  if (!X || !Tx || !Px || !F || !Frho_z) {
    free(X); free(Tx); free(Px); free(F); free(Frho_z);
    return -2;
  }
  double Yc[64], Xc[64];
  const double cpd = g->gamma_d * c_vd(g);

  /* 1. primitives of interior cells (App. B), pressure stored as p' = p - pbar_k */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long c = ((long)k * ny + j) * nx + i;
        for (int v = 0; v < nv; ++v) Yc[v] = Y[v * ncell + c];
        double T;
        orc_cons_to_prim(g, Yc, Xc, &T, NULL);
        double Pi = pow(Xc[nv - 1] / 1e5, (g->gamma_d - 1.0) / g->gamma_d);
        Xc[nv - 1] -= pbar_cell(g, k);
        long x = ext_index(&e, k, j, i);
        for (int v = 0; v < nv; ++v) X[v * next + x] = Xc[v];
        Tx[x] = T / Pi;
        Px[x] = Pi;
      }

  /* 2. ghost cells */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int gi = -3; gi < nx + 3; ++gi) {
        if (gi >= 0 && gi < nx) continue;
        int flip, si = wrap_or_mirror(gi, nx, g->bc[0], g->bc[1], &flip);
        long dst = ext_index(&e, k, j, gi), src = ext_index(&e, k, j, si);
        for (int v = 0; v < nv; ++v) X[v * next + dst] = X[v * next + src];
        Tx[dst] = Tx[src];
        Px[dst] = Px[src];
        if (flip) wall_ghost(g, X, next, dst, 0, g->bc[gi < 0 ? 0 : 1]);
      }
  if (three_d)
    for (int k = 0; k < nz; ++k)
      for (int gj = -3; gj < ny + 3; ++gj)
        for (int i = 0; i < nx; ++i) {
          if (gj >= 0 && gj < ny) continue;
          int flip, sj = wrap_or_mirror(gj, ny, g->bc[2], g->bc[3], &flip);
          long dst = ext_index(&e, k, gj, i), src = ext_index(&e, k, sj, i);
          for (int v = 0; v < nv; ++v) X[v * next + dst] = X[v * next + src];
          Tx[dst] = Tx[src];
          Px[dst] = Px[src];
          if (flip) wall_ghost(g, X, next, dst, 1, g->bc[gj < 0 ? 2 : 3]);
        }
  for (int gk = -3; gk < nz + 3; ++gk)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        if (gk >= 0 && gk < nz) continue;
        int flip, sk = wrap_or_mirror(gk, nz, g->bc[4], g->bc[5], &flip);
        long dst = ext_index(&e, gk, j, i), src = ext_index(&e, sk, j, i);
        for (int v = 0; v < nv; ++v) X[v * next + dst] = X[v * next + src];
        Tx[dst] = Tx[src];
        Px[dst] = Px[src];
        if (flip) wall_ghost(g, X, next, dst, 2, g->bc[gk < 0 ? 4 : 5]);
        if (gk < 0 && g->T_bottom > 0.0) {
          /* Sec. 6 lower boundary: the ghost holds T_bottom at the mirrored pressure and
           * composition, so its density is the mirrored one times T / T_bottom */
          const double T = Tx[src] * Px[src];
          X[dst] *= T / g->T_bottom;
          Tx[dst] = g->T_bottom / Px[src];
        }
      }

  for (long v = 0; v < nv * ncell; ++v) dYdt[v] = 0.0;

  /* 3. per direction: reconstruct both face states (Eq. q+ with m = 3), Riemann flux
   *    (Eq. riemann via LMARS), then the flux difference of Eq. forward. */
  for (int d = 0; d < 3; ++d) {
    if (d == 1 && !three_d) continue;
    const int fx = (d == 0), fy = (d == 1), fz = (d == 2);
    const int nfx = nx + fx, nfy = ny + fy, nfz = nz + fz;
    const double h = d == 0 ? g->dx : (d == 1 ? g->dy : g->dz);
    for (int k = 0; k < nfz; ++k)
      for (int j = 0; j < nfy; ++j)
        for (int i = 0; i < nfx; ++i) {
          double XL[64], XR[64], Ff[64], st[5];
          /* stencil cell s (s = -3..+2) lies s cells along d from the face's right cell */
          for (int v = 0; v < nv; ++v) {
            double col[6];
            for (int s = -3; s <= 2; ++s)
              col[s + 3] = X[v * next + ext_index(&e, k + s * fz, j + s * fy, i + s * fx)];
            for (int s = 0; s < 5; ++s) st[s] = col[s]; /* Q_{i-3} .. Q_{i+1} */
            XL[v] = orc_weno5(st, g->weno_eps);
            for (int s = 0; s < 5; ++s) st[s] = col[5 - s]; /* Q_{i+2} .. Q_{i-2} */
            XR[v] = orc_weno5(st, g->weno_eps);
          }
          double pref = fz ? g->p_bar_face[k] : pbar_cell(g, k);
          orc_lmars(g, XL, XR, d, pref, Ff, NULL, NULL);
          if (g->nu > 0.0) {
            long cl = ext_index(&e, k - fz, j - fy, i - fx), cr = ext_index(&e, k, j, i);
            double rl = X[cl], rr = X[cr];
            double rf = 0.5 * (rl + rr), work = 0.0;
            for (int m = 0; m < nmom_of(g); ++m) {
              double ul = X[(long)(im0 + m) * next + cl], ur = X[(long)(im0 + m) * next + cr];
              double grad = (ur - ul) / h;
              Ff[im0 + m] -= rf * g->nu * grad;
              work += 0.5 * (ul + ur) * grad;
            }
            double heat = 0.5 * (Px[cl] + Px[cr]) * (Tx[cr] - Tx[cl]) / h;
            Ff[nv - 1] -= rf * g->nu * work + rf * cpd * g->nu * heat;
          }
          if (fz) sedimentation_flux(g, XL, XR, pref, k, Ff);
          long fidx = ((long)k * nfy + j) * nfx + i;
          long nf = (long)nfx * nfy * nfz;
          for (int v = 0; v < nv; ++v) F[v * nf + fidx] = Ff[v];
          if (fz) {
            double m = 0.0;
            for (int s = 0; s < im0; ++s) m += Ff[s];
            Frho_z[((long)k * ny + j) * nx + i] = m;
          }
        }
    long nf = (long)nfx * nfy * nfz;
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          long c = ((long)k * ny + j) * nx + i;
          long f0 = ((long)k * nfy + j) * nfx + i;
          long f1 = ((long)(k + fz) * nfy + (j + fy)) * nfx + (i + fx);
          for (int v = 0; v < nv; ++v) dYdt[v * ncell + c] -= (F[v * nf + f1] - F[v * nf + f0]) / h;
        }
  }

  /* 4. gravity sources (Eq. mom3 and the energy equation of Sec. 2), and the forcing of the
   *    Jovian simulation (Sec. 6):
   *    cooling: d(rho e)/dt -= C_v Q, C_v = sum_k c_k rho_k, in the levels whose reference
   *      pressure pbar_k lies in [cool_p_lo, cool_p_hi];
   *    sponge: d(rho u_h)/dt -= rho u_h / (tau0 (pbar_k/p0)^2) for the horizontal momenta
   *      where pbar_k < p0; rho e is left unchanged, so the damped kinetic energy turns into
   *      heat.
   *    READING: the bands and the sponge time use the fixed reference pressure of the level. */
  const int mw = mom_slot(g, 2);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long c = ((long)k * ny + j) * nx + i;
        const double pk = pbar_cell(g, k);
        if (g->cool_rate != 0.0 && pk >= g->cool_p_lo && pk <= g->cool_p_hi) {
          double Cv = c_vd(g) * Y[c];
          for (int a = 0; a < g->nvap; ++a) {
            Cv += g->sig_v[a] * c_vd(g) * Y[(long)(1 + a) * ncell + c];
            for (int b = 0; b < g->ncond; ++b)
              Cv += g->sig_c[a][b] * c_vd(g) * Y[(long)icond(g, a, b) * ncell + c];
          }
          dYdt[(long)(nv - 1) * ncell + c] -= Cv * g->cool_rate;
        }
        if (g->sponge_tau0 > 0.0 && pk < g->sponge_p0) {
          const double r = pk / g->sponge_p0, tau = g->sponge_tau0 * r * r;
          for (int d = 0; d < 2; ++d) {
            if (d == 1 && !three_d) continue;
            const long m = (long)mom_slot(g, d) * ncell + c;
            dYdt[m] -= Y[m] / tau;
          }
        }
        double rho = X[ext_index(&e, k, j, i)];
        dYdt[(long)mw * ncell + c] -= (rho - g->rho_bar[k]) * g->grav;
        if (g->gravity_energy_pointwise) {
          dYdt[(long)(nv - 1) * ncell + c] -= g->grav * Y[(long)mw * ncell + c];
        } else {
          double fb = Frho_z[((long)k * ny + j) * nx + i];
          double ft = Frho_z[((long)(k + 1) * ny + j) * nx + i];
          dYdt[(long)(nv - 1) * ncell + c] -= g->grav * 0.5 * (fb + ft);
        }
      }
  free(X);
  free(Tx);
  free(Px);
  free(F);
  free(Frho_z);
  return 0;
}

/* Sec. 4.3: third-order TVD (SSP) Runge-Kutta of Shu & Osher:
 *   stage 0: Y1 = Yn + dt L(Yn)
 *   stage 1: Y2 = 3/4 Yn + 1/4 (Y1 + dt L(Y1))
 *   stage 2: Yn+1 = 1/3 Yn + 2/3 (Y2 + dt L(Y2)) */
void orc_rk3_combine(int stage, long n, const double *Yn, const double *Ys, const double *L,
                     double dt, double *Yout) {
  for (long c = 0; c < n; ++c) {
    double ys = Ys[c] + dt * L[c];
    if (stage == 0)
      Yout[c] = ys;
    else if (stage == 1)
      Yout[c] = 0.75 * Yn[c] + 0.25 * ys;
    else
      Yout[c] = Yn[c] / 3.0 + 2.0 / 3.0 * ys;
  }
}

int orc_stage(const orc_grid *g, int stage, const double *Yn, const double *Ys, double dt,
              double *Yout) {
  const int nv = orc_nvar(g);
  const long ncell = (long)g->nx * g->ny * g->nz;
  double *L = malloc(sizeof(double) * (size_t)(nv * ncell));
  if (!L) return -2;
  int rc = orc_rhs(g, Ys, L);
  if (rc) {
    free(L);
    return rc;
  }
  orc_rk3_combine(stage, nv * ncell, Yn, Ys, L, dt, Yout);
  free(L);
  int worst = 0;
  if (g->satadj && g->nvap > 0 && g->ncond > 0) {
    double Yc[64];
    for (long c = 0; c < ncell; ++c) {
      for (int v = 0; v < nv; ++v) Yc[v] = Yout[v * ncell + c];
      int it = orc_satadj_cell(g, Yc, g->satadj_max_iter, g->satadj_tol);
      if (it < 0) worst = -1;
      else if (worst >= 0 && it > worst) worst = it;
      for (int v = 0; v < nv; ++v) Yout[v * ncell + c] = Yc[v];
    }
  }
  return worst;
}

/* READING: the paper gives no time-step rule. For the unsplit update of Eq. forward,
 * dt = cfl / max over cells of sum_d (|u_d| + c) / dx_d, from the state at the start of the
 * step, held for all three stages. */
double orc_dt_cfl(const orc_grid *g, const double *Y, double cfl) {
  const int nv = orc_nvar(g);
  const long ncell = (long)g->nx * g->ny * g->nz;
  double Yc[64], Xc[64], rate = 0.0;
  for (long c = 0; c < ncell; ++c) {
    for (int v = 0; v < nv; ++v) Yc[v] = Y[v * ncell + c];
    double gam;
    orc_cons_to_prim(g, Yc, Xc, NULL, &gam);
    double cs = sqrt(gam * Xc[nv - 1] / Xc[0]);
    double r = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (d == 1 && g->ny == 1) continue;
      double h = d == 0 ? g->dx : (d == 1 ? g->dy : g->dz);
      r += (fabs(Xc[mom_slot(g, d)]) + cs) / h;
    }
    if (r > rate) rate = r;
  }
  return cfl / rate;
}

int orc_step(const orc_grid *g, double *Y, int nsteps, double dt, double cfl, double *dt_last) {
  const int nv = orc_nvar(g);
  const long n = (long)nv * g->nx * g->ny * g->nz;
  double *Y1 = malloc(sizeof(double) * (size_t)n), *Y2 = malloc(sizeof(double) * (size_t)n);
  if (!Y1 || !Y2) {
    free(Y1); free(Y2);
    return -2;
  }
  int worst = 0;
  for (int s = 0; s < nsteps; ++s) {
    double h = dt > 0.0 ? dt : orc_dt_cfl(g, Y, cfl);
    if (dt_last) *dt_last = h;
    int r0 = orc_stage(g, 0, Y, Y, h, Y1);
    int r1 = orc_stage(g, 1, Y, Y1, h, Y2);
    int r2 = orc_stage(g, 2, Y, Y2, h, Y1);
    if (r0 < -1 || r1 < -1 || r2 < -1) {
      free(Y1); free(Y2);
      return -2;
    }
    if (r0 < 0 || r1 < 0 || r2 < 0) worst = -1;
    memcpy(Y, Y1, sizeof(double) * (size_t)n);
    if (g->kessler && g->nvap > 0 && g->ncond >= 2) {
      double Yc[64];
      const long ncell = (long)g->nx * g->ny * g->nz;
      for (long c = 0; c < ncell; ++c) {
        for (int v = 0; v < nv; ++v) Yc[v] = Y[v * ncell + c];
        if (orc_kessler_cell(g, Yc, h) < 0) worst = -1;
        for (int v = 0; v < nv; ++v) Y[v * ncell + c] = Yc[v];
      }
    }
  }
  free(Y1);
  free(Y2);
  return worst;
}

void orc_budget(const orc_grid *g, const double *Y, double *out) {
  const int nv = orc_nvar(g), im0 = im0_of(g);
  const long ncell = (long)g->nx * g->ny * g->nz;
  const double vol = g->dx * (g->ny > 1 ? g->dy : 1.0) * g->dz;
  for (int v = 0; v <= nv; ++v) out[v] = 0.0;
  for (int k = 0; k < g->nz; ++k) {
    double z = (k + 0.5) * g->dz;
    for (long c = (long)k * g->nx * g->ny; c < (long)(k + 1) * g->nx * g->ny; ++c) {
      double rho = 0.0;
      for (int v = 0; v < nv; ++v) out[v] += Y[v * ncell + c] * vol;
      for (int s = 0; s < im0; ++s) rho += Y[s * ncell + c];
      out[nv] += (Y[(long)(nv - 1) * ncell + c] + rho * g->grav * z) * vol;
    }
  }
}

/* =======================================================================================
 * Discrete adjoint of the inviscid stage (reverse of Eq. forward with WENO5 and LMARS, the
 * gravity source, the SSP-RK3 combine and the saturation adjustment), written by hand as
 * the transpose of the forward routines above, step by step in reverse order. Not part of
 * the paper: it differentiates the paper's discrete scheme. Branches are held fixed (upwind
 * side of LMARS, which vapours keep cloud), and the time step is a given constant.
 * ======================================================================================= */

/* I = orc_weno5(q) and its gradient dI/dq_j. With w_k = a_k / S, a_k = d_k (eps + b_k)^-2:
 * dI/dq_j = sum_k w_k dv_k/dq_j + sum_m (v_m - I)/S * (-2 a_m / (eps + b_m)) db_m/dq_j. */
static double weno5_grad(const double q[5], double eps, double grad[5]) {
  static const double d[3] = {0.1, 0.6, 0.3};
  static const double dv[3][5] = {{1.0 / 3.0, -7.0 / 6.0, 11.0 / 6.0, 0.0, 0.0},
                                  {0.0, -1.0 / 6.0, 5.0 / 6.0, 1.0 / 3.0, 0.0},
                                  {0.0, 0.0, 1.0 / 3.0, 5.0 / 6.0, -1.0 / 6.0}};
  double b[3], a[3], v[3], db[3][5], S = 0.0, I = 0.0;
  double t1, t2;
  t1 = q[0] - 2.0 * q[1] + q[2];
  t2 = q[0] - 4.0 * q[1] + 3.0 * q[2];
  b[0] = 13.0 / 12.0 * t1 * t1 + 0.25 * t2 * t2;
  {
    const double e1[5] = {1, -2, 1, 0, 0}, e2[5] = {1, -4, 3, 0, 0};
    for (int j = 0; j < 5; ++j) db[0][j] = 13.0 / 6.0 * t1 * e1[j] + 0.5 * t2 * e2[j];
  }
  t1 = q[1] - 2.0 * q[2] + q[3];
  t2 = q[1] - q[3];
  b[1] = 13.0 / 12.0 * t1 * t1 + 0.25 * t2 * t2;
  {
    const double e1[5] = {0, 1, -2, 1, 0}, e2[5] = {0, 1, 0, -1, 0};
    for (int j = 0; j < 5; ++j) db[1][j] = 13.0 / 6.0 * t1 * e1[j] + 0.5 * t2 * e2[j];
  }
  t1 = q[2] - 2.0 * q[3] + q[4];
  t2 = 3.0 * q[2] - 4.0 * q[3] + q[4];
  b[2] = 13.0 / 12.0 * t1 * t1 + 0.25 * t2 * t2;
  {
    const double e1[5] = {0, 0, 1, -2, 1}, e2[5] = {0, 0, 3, -4, 1};
    for (int j = 0; j < 5; ++j) db[2][j] = 13.0 / 6.0 * t1 * e1[j] + 0.5 * t2 * e2[j];
  }
  for (int k = 0; k < 3; ++k) {
    a[k] = d[k] / ((eps + b[k]) * (eps + b[k]));
    S += a[k];
    v[k] = 0.0;
    for (int j = 0; j < 5; ++j) v[k] += dv[k][j] * q[j];
  }
  for (int k = 0; k < 3; ++k) I += a[k] / S * v[k];
  for (int j = 0; j < 5; ++j) {
    double gj = 0.0;
    for (int k = 0; k < 3; ++k) {
      gj += a[k] / S * dv[k][j];
      gj += (v[k] - I) / S * (-2.0 * a[k] / (eps + b[k])) * db[k][j];
    }
    grad[j] = gj;
  }
  return I;
}

double orc_weno5_gradient(const double q[5], double eps, double grad[5]) {
  return weno5_grad(q, eps, grad);
}

/* Transpose of mix_factors: accumulate into Xb the adjoint of (num, den). */
static void mix_factors_adjoint(const orc_grid *g, double numb, double denb, double *Xb) {
  for (int i = 0; i < g->nvap; ++i) {
    Xb[1 + i] += numb * (g->sig_v[i] - 1.0) + denb * (1.0 / g->eps[i] - 1.0);
    for (int j = 0; j < g->ncond; ++j) Xb[icond(g, i, j)] += numb * (g->sig_c[i][j] - 1.0) - denb;
  }
}

/* Transpose of orc_lmars: given Fbar (nvar), accumulate XLbar, XRbar. The forward quantities
 * are recomputed first, then each assignment of orc_lmars is reversed in the opposite order. */
static void lmars_adjoint(const orc_grid *g, const double *XL, const double *XR, int dir,
                          double pref, const double *Fbar, double *XLb, double *XRb) {
  const int im0 = im0_of(g), nm = nmom_of(g), nv = orc_nvar(g), mn = mom_slot(g, dir);
  const double gm1 = g->gamma_d - 1.0;
  /* forward recomputation */
  double numL, denL, numR, denR;
  mix_factors(g, XL, &numL, &denL);
  mix_factors(g, XR, &numR, &denR);
  double pL = pref + XL[nv - 1], pR = pref + XR[nv - 1];
  double gamL = 1.0 + gm1 * denL / numL, gamR = 1.0 + gm1 * denR / numR;
  double cL = sqrt(gamL * pL / XL[0]), cR = sqrt(gamR * pR / XR[0]);
  double rhoc = 0.5 * (XL[0] + XR[0]) * 0.5 * (cL + cR);
  double uL = XL[mn], uR = XR[mn];
  double us = 0.5 * (uL + uR) - (XR[nv - 1] - XL[nv - 1]) / (2.0 * rhoc);
  /* reverse of the upwind part; at u* = 0 the flux has a kink between the two sides and
   * the average of both one-sided derivatives is taken (what a central difference sees) */
  double usb = 0.0;
  const double psb = Fbar[mn];
  double numLb = 0.0, denLb = 0.0, numRb = 0.0, denRb = 0.0;
  for (int side = 0; side < 2; ++side) {
    const int use_left = side == 0;
    double wgt = us > 0.0 ? (use_left ? 1.0 : 0.0) : (us < 0.0 ? (use_left ? 0.0 : 1.0) : 0.5);
    if (wgt == 0.0) continue;
    const double *XS = use_left ? XL : XR;
    double *XSb = use_left ? XLb : XRb;
    double numS = use_left ? numL : numR, denS = use_left ? denL : denR;
    double pS = use_left ? pL : pR, rhoS = XS[0], mf = us * rhoS;
    double qsum = 0.0, u2 = 0.0, muq = 0.0;
    for (int t = 1; t < im0; ++t) qsum += XS[t];
    for (int m = 0; m < nm; ++m) u2 += XS[im0 + m] * XS[im0 + m];
    for (int i = 0; i < g->nvap; ++i)
      for (int j = 0; j < g->ncond; ++j) muq += mu_of(g, i, j) * XS[icond(g, i, j)];
    double K = 0.5 * rhoS * u2, A = rhoS * muq;
    double rhoe = numS / denS * pS / gm1 + K + A;
    /* F[E] = u* (rho e + p_S) */
    usb += wgt * Fbar[nv - 1] * (rhoe + pS);
    double rhoeb = wgt * Fbar[nv - 1] * us;
    double pSb = wgt * Fbar[nv - 1] * us;
    /* rho e = (num/den) p_S/(gamma_d - 1) + K + A */
    pSb += rhoeb * numS / denS / gm1;
    double rb = rhoeb * pS / gm1;
    if (use_left) {
      numLb += rb / denS;
      denLb += -rb * numS / (denS * denS);
    } else {
      numRb += rb / denS;
      denRb += -rb * numS / (denS * denS);
    }
    double rhoSb = rhoeb * (0.5 * u2 + muq);
    for (int i = 0; i < g->nvap; ++i)
      for (int j = 0; j < g->ncond; ++j) XSb[icond(g, i, j)] += rhoeb * rhoS * mu_of(g, i, j);
    for (int m = 0; m < nm; ++m) XSb[im0 + m] += rhoeb * rhoS * XS[im0 + m];
    /* mass, tracer and momentum fluxes: F[t] = mf q_t, F[0] = mf (1 - sum q), F[m] = mf u_m */
    double mfb = Fbar[0] * (1.0 - qsum);
    for (int t = 1; t < im0; ++t) {
      mfb += Fbar[t] * XS[t];
      XSb[t] += wgt * (Fbar[t] - Fbar[0]) * mf;
    }
    for (int m = 0; m < nm; ++m) {
      mfb += Fbar[im0 + m] * XS[im0 + m];
      XSb[im0 + m] += wgt * Fbar[im0 + m] * mf;
    }
    /* mf = u* rho_S */
    usb += wgt * mfb * rhoS;
    rhoSb += wgt * mfb * us;
    XSb[0] += rhoSb;
    XSb[nv - 1] += pSb;
  }
  double rhocb = 0.0;
  /* us = (uL + uR)/2 - (p'R - p'L)/(2 rho c) */
  XLb[mn] += 0.5 * usb;
  XRb[mn] += 0.5 * usb;
  XRb[nv - 1] += -usb / (2.0 * rhoc);
  XLb[nv - 1] += usb / (2.0 * rhoc);
  rhocb += usb * (XR[nv - 1] - XL[nv - 1]) / (2.0 * rhoc * rhoc);
  /* ps = (p'L + p'R)/2 - rho c (uR - uL)/2 */
  XLb[nv - 1] += 0.5 * psb;
  XRb[nv - 1] += 0.5 * psb;
  rhocb += -0.5 * (uR - uL) * psb;
  XRb[mn] += -0.5 * rhoc * psb;
  XLb[mn] += 0.5 * rhoc * psb;
  /* rho c = (rhoL + rhoR)/2 (cL + cR)/2 */
  XLb[0] += 0.25 * (cL + cR) * rhocb;
  XRb[0] += 0.25 * (cL + cR) * rhocb;
  double cLb = 0.25 * (XL[0] + XR[0]) * rhocb, cRb = cLb;
  /* c = sqrt(gamma p / rho), gamma = 1 + (gamma_d - 1) den / num */
  XLb[nv - 1] += cLb * cL / (2.0 * pL);
  XLb[0] += -cLb * cL / (2.0 * XL[0]);
  XRb[nv - 1] += cRb * cR / (2.0 * pR);
  XRb[0] += -cRb * cR / (2.0 * XR[0]);
  double gLb = cLb * cL / (2.0 * gamL), gRb = cRb * cR / (2.0 * gamR);
  denLb += gLb * gm1 / numL;
  numLb += -gLb * gm1 * denL / (numL * numL);
  denRb += gRb * gm1 / numR;
  numRb += -gRb * gm1 * denR / (numR * numR);
  mix_factors_adjoint(g, numLb, denLb, XLb);
  mix_factors_adjoint(g, numRb, denRb, XRb);
}

/* Transpose of orc_cons_to_prim at the cell state Y (the pressure entry of Xb is the adjoint
 * of p; subtracting the constant p_bar_k has unit derivative). Adds into Yb. */
static void cons_to_prim_adjoint(const orc_grid *g, const double *Y, const double *Xb,
                                 double *Yb) {
  const int im0 = im0_of(g), nm = nmom_of(g), nv = orc_nvar(g);
  const double gm1 = g->gamma_d - 1.0;
  double X[64];
  orc_cons_to_prim(g, Y, X, NULL, NULL);
  double rho = X[0], K = 0.0, A = 0.0, u2 = 0.0;
  for (int m = 0; m < nm; ++m) u2 += X[im0 + m] * X[im0 + m];
  K = 0.5 * rho * u2;
  for (int i = 0; i < g->nvap; ++i)
    for (int j = 0; j < g->ncond; ++j) A += mu_of(g, i, j) * Y[icond(g, i, j)];
  double U = Y[nv - 1] - K - A, num, den;
  mix_factors(g, X, &num, &den);
  /* p = (gamma_d - 1) (den / num) U */
  const double pb = Xb[nv - 1];
  double Ub = pb * gm1 * den / num, rb = pb * gm1 * U;
  double Qb[64];
  for (int t = 0; t < nv; ++t) Qb[t] = 0.0;
  for (int t = 1; t < im0; ++t) Qb[t] = Xb[t];
  mix_factors_adjoint(g, -rb * den / (num * num), rb / num, Qb);
  /* U = Y_E - K - A */
  Yb[nv - 1] += Ub;
  double Kb = -Ub;
  for (int i = 0; i < g->nvap; ++i)
    for (int j = 0; j < g->ncond; ++j) Yb[icond(g, i, j)] += -Ub * mu_of(g, i, j);
  /* K = |m|^2 / (2 rho), u = m / rho, q_t = Y_t / rho, rho = sum of the densities */
  double rhob = Xb[0] - Kb * 0.5 * u2;
  for (int m = 0; m < nm; ++m) {
    Yb[im0 + m] += Kb * X[im0 + m] + Xb[im0 + m] / rho;
    rhob += -Xb[im0 + m] * X[im0 + m] / rho;
  }
  for (int t = 1; t < im0; ++t) {
    Yb[t] += Qb[t] / rho;
    rhob += -Qb[t] * X[t] / rho;
  }
  for (int t = 0; t < im0; ++t) Yb[t] += rhob;
}

int orc_rhs_adjoint(const orc_grid *g, const double *Y, const double *mu, double *Ybar) {
  const int nx = g->nx, ny = g->ny, nz = g->nz, nv = orc_nvar(g), im0 = im0_of(g);
  const int three_d = ny > 1;
  if (g->nu > 0.0) return -3; /* inviscid only */
  for (int j = 0; j < g->ncond; ++j)
    if (g->w_term[j] != 0.0) return -3; /* no sedimentation */
  if (g->cool_rate != 0.0 || g->sponge_tau0 > 0.0) return -3; /* no forcing */
  for (int s = 0; s < 6; ++s)
    if (g->bc[s] == ORC_NOSLIP) return -3; /* free-slip or periodic sides only */
  if (g->T_bottom > 0.0) return -3;       /* no fixed bottom temperature */
  if (nx < 1 || ny < 1 || nz < 3) return -1;
  ext_dims e = {nx + 6, three_d ? ny + 6 : 1, nz + 6, 3, three_d ? 3 : 0, 3};
  const long next = (long)e.nxe * e.nye * e.nze;
  const long ncell = (long)nx * ny * nz;
  double *X = calloc((size_t)(nv * next), sizeof(double));
  double *Xb = calloc((size_t)(nv * next), sizeof(double));
  double *Fbz = calloc((size_t)nx * ny * (nz + 1), sizeof(double));
  if (!X || !Xb || !Fbz) {
    free(X); free(Xb); free(Fbz);
    return -2;
  }
  double Yc[64], Xc[64];
  /* forward: primitives and ghosts, as in orc_rhs */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long c = ((long)k * ny + j) * nx + i;
        for (int v = 0; v < nv; ++v) Yc[v] = Y[v * ncell + c];
        orc_cons_to_prim(g, Yc, Xc, NULL, NULL);
        Xc[nv - 1] -= pbar_cell(g, k);
        long x = ext_index(&e, k, j, i);
        for (int v = 0; v < nv; ++v) X[v * next + x] = Xc[v];
      }
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int gi = -3; gi < nx + 3; ++gi) {
        if (gi >= 0 && gi < nx) continue;
        int flip, si = wrap_or_mirror(gi, nx, g->bc[0], g->bc[1], &flip);
        long dst = ext_index(&e, k, j, gi), src = ext_index(&e, k, j, si);
        for (int v = 0; v < nv; ++v) X[v * next + dst] = X[v * next + src];
        if (flip) X[(long)mom_slot(g, 0) * next + dst] *= -1.0;
      }
  if (three_d)
    for (int k = 0; k < nz; ++k)
      for (int gj = -3; gj < ny + 3; ++gj)
        for (int i = 0; i < nx; ++i) {
          if (gj >= 0 && gj < ny) continue;
          int flip, sj = wrap_or_mirror(gj, ny, g->bc[2], g->bc[3], &flip);
          long dst = ext_index(&e, k, gj, i), src = ext_index(&e, k, sj, i);
          for (int v = 0; v < nv; ++v) X[v * next + dst] = X[v * next + src];
          if (flip) X[(long)mom_slot(g, 1) * next + dst] *= -1.0;
        }
  for (int gk = -3; gk < nz + 3; ++gk)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        if (gk >= 0 && gk < nz) continue;
        int flip, sk = wrap_or_mirror(gk, nz, g->bc[4], g->bc[5], &flip);
        long dst = ext_index(&e, gk, j, i), src = ext_index(&e, sk, j, i);
        for (int v = 0; v < nv; ++v) X[v * next + dst] = X[v * next + src];
        if (flip) X[(long)mom_slot(g, 2) * next + dst] *= -1.0;
      }
  for (long v = 0; v < nv * ncell; ++v) Ybar[v] = 0.0;

  /* reverse of the gravity sources: -(rho - rho_bar) g on rho w, -g (F_rho,b + F_rho,t)/2
   * on rho e */
  const int mw = mom_slot(g, 2);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long c = ((long)k * ny + j) * nx + i;
        for (int s = 0; s < im0; ++s) Ybar[(long)s * ncell + c] += -g->grav * mu[(long)mw * ncell + c];
        double me = mu[(long)(nv - 1) * ncell + c];
        Fbz[((long)k * ny + j) * nx + i] += -0.5 * g->grav * me;
        Fbz[((long)(k + 1) * ny + j) * nx + i] += -0.5 * g->grav * me;
      }

  /* reverse of the flux divergence, LMARS and WENO5 per face */
  for (int d = 0; d < 3; ++d) {
    if (d == 1 && !three_d) continue;
    const int fx = (d == 0), fy = (d == 1), fz = (d == 2);
    const int nfx = nx + fx, nfy = ny + fy, nfz = nz + fz;
    const double h = d == 0 ? g->dx : (d == 1 ? g->dy : g->dz);
    for (int k = 0; k < nfz; ++k)
      for (int j = 0; j < nfy; ++j)
        for (int i = 0; i < nfx; ++i) {
          double XL[64], XR[64], Fb[64], XLb[64], XRb[64], colq[64][6];
          /* Fbar = (mu_right - mu_left) / h over the interior cells next to the face */
          for (int v = 0; v < nv; ++v) Fb[v] = 0.0;
          const int il = i - fx, jl = j - fy, kl = k - fz;
          if (il >= 0 && jl >= 0 && kl >= 0) {
            long c = ((long)kl * ny + jl) * nx + il;
            for (int v = 0; v < nv; ++v) Fb[v] -= mu[v * ncell + c] / h;
          }
          if (i < nx && j < ny && k < nz) {
            long c = ((long)k * ny + j) * nx + i;
            for (int v = 0; v < nv; ++v) Fb[v] += mu[v * ncell + c] / h;
          }
          if (fz) {
            double fr = Fbz[((long)k * ny + j) * nx + i];
            for (int s = 0; s < im0; ++s) Fb[s] += fr;
          }
          /* forward face states */
          for (int v = 0; v < nv; ++v) {
            double st[5];
            for (int s = -3; s <= 2; ++s)
              colq[v][s + 3] = X[v * next + ext_index(&e, k + s * fz, j + s * fy, i + s * fx)];
            for (int s = 0; s < 5; ++s) st[s] = colq[v][s];
            XL[v] = orc_weno5(st, g->weno_eps);
            for (int s = 0; s < 5; ++s) st[s] = colq[v][5 - s];
            XR[v] = orc_weno5(st, g->weno_eps);
            XLb[v] = XRb[v] = 0.0;
          }
          double pref = fz ? g->p_bar_face[k] : pbar_cell(g, k);
          lmars_adjoint(g, XL, XR, d, pref, Fb, XLb, XRb);
          /* WENO5 transposes onto the stencil cells s = -3..2 */
          for (int v = 0; v < nv; ++v) {
            double st[5], gr[5];
            for (int s = 0; s < 5; ++s) st[s] = colq[v][s];
            weno5_grad(st, g->weno_eps, gr);
            for (int s = 0; s < 5; ++s)
              Xb[v * next + ext_index(&e, k + (s - 3) * fz, j + (s - 3) * fy, i + (s - 3) * fx)] +=
                  XLb[v] * gr[s];
            for (int s = 0; s < 5; ++s) st[s] = colq[v][5 - s];
            weno5_grad(st, g->weno_eps, gr);
            for (int s = 0; s < 5; ++s)
              Xb[v * next + ext_index(&e, k + (2 - s) * fz, j + (2 - s) * fy, i + (2 - s) * fx)] +=
                  XRb[v] * gr[s];
          }
        }
  }

  /* reverse of the ghost fill: fold ghost adjoints onto their source cells */
  for (int gk = -3; gk < nz + 3; ++gk)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        if (gk >= 0 && gk < nz) continue;
        int flip, sk = wrap_or_mirror(gk, nz, g->bc[4], g->bc[5], &flip);
        long dst = ext_index(&e, gk, j, i), src = ext_index(&e, sk, j, i);
        for (int v = 0; v < nv; ++v) {
          double b = Xb[v * next + dst];
          if (flip && v == mom_slot(g, 2)) b = -b;
          Xb[v * next + src] += b;
        }
      }
  if (three_d)
    for (int k = 0; k < nz; ++k)
      for (int gj = -3; gj < ny + 3; ++gj)
        for (int i = 0; i < nx; ++i) {
          if (gj >= 0 && gj < ny) continue;
          int flip, sj = wrap_or_mirror(gj, ny, g->bc[2], g->bc[3], &flip);
          long dst = ext_index(&e, k, gj, i), src = ext_index(&e, k, sj, i);
          for (int v = 0; v < nv; ++v) {
            double b = Xb[v * next + dst];
            if (flip && v == mom_slot(g, 1)) b = -b;
            Xb[v * next + src] += b;
          }
        }
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int gi = -3; gi < nx + 3; ++gi) {
        if (gi >= 0 && gi < nx) continue;
        int flip, si = wrap_or_mirror(gi, nx, g->bc[0], g->bc[1], &flip);
        long dst = ext_index(&e, k, j, gi), src = ext_index(&e, k, j, si);
        for (int v = 0; v < nv; ++v) {
          double b = Xb[v * next + dst];
          if (flip && v == mom_slot(g, 0)) b = -b;
          Xb[v * next + src] += b;
        }
      }

  /* reverse of the primitive map (App. B) */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long c = ((long)k * ny + j) * nx + i;
        long x = ext_index(&e, k, j, i);
        double Xbc[64], Ybc[64];
        for (int v = 0; v < nv; ++v) {
          Yc[v] = Y[v * ncell + c];
          Xbc[v] = Xb[v * next + x];
          Ybc[v] = 0.0;
        }
        cons_to_prim_adjoint(g, Yc, Xbc, Ybc);
        for (int v = 0; v < nv; ++v) Ybar[v * ncell + c] += Ybc[v];
      }
  free(X);
  free(Xb);
  free(Fbz);
  return 0;
}

/* Transpose of the saturation adjustment of one cell at its converged result Yout (App. D).
 * The iteration converges to the equilibrium in which every vapour i that keeps cloud holds
 * the saturation density rho*_i(T) = p*_i(T)/(R_i T), its cloud the rest of the species
 * total, while a vapour without cloud holds the whole total. T follows from the conserved
 * energy: F(T) = T C_v(T) + A(T) - (rho e - K) = 0 with C_v = sum of c_k rho_k and
 * A = sum mu_ij rho_ij over the adjusted composition. The derivative of the map
 * Yin -> Yout is therefore that of the equilibrium (implicit function theorem on F):
 *   dT/dy = -(dF/dy)/(dF/dT),  dF/dT = C_v + sum_{saturated i} rho*_i' (T (c_vi - c_i1) - mu_i1),
 *   rho*_i' = rho*_i ((beta_i/t - delta_i)/T - 1/T), t = T/T^r_i,
 * and dF/dy at fixed T: -1 for rho e, u_m for the momenta, T c_vd - |u|^2/2 for rho_d,
 * T c_i1 + mu_i1 - |u|^2/2 for the total of a saturated species, T c_vi - |u|^2/2 for the
 * total of an unsaturated one, T c_ij + mu_ij - |u|^2/2 for the other condensates.
 * lam_in = (dYout/dYin)^T lam_out. The saturated set is read from Yout (cloud > 0); at its
 * edge (cloud appearing or vanishing) the map has a kink, not differentiated here. */
int orc_satadj_adjoint_cell(const orc_grid *g, const double *Yout, const double *lam_out,
                            double *lam_in) {
  const int im0 = im0_of(g), nm = nmom_of(g), nv = orc_nvar(g);
  for (int v = 0; v < nv; ++v) lam_in[v] = lam_out[v];
  if (g->nvap == 0 || g->ncond == 0) return 0;
  double X[64], T;
  orc_cons_to_prim(g, Yout, X, &T, NULL);
  const double cvd = c_vd(g);
  double u2 = 0.0, Cv = cvd * Yout[0];
  for (int m = 0; m < nm; ++m) u2 += X[im0 + m] * X[im0 + m];
  for (int i = 0; i < g->nvap; ++i) {
    Cv += g->sig_v[i] * cvd * Yout[1 + i];
    for (int j = 0; j < g->ncond; ++j) Cv += g->sig_c[i][j] * cvd * Yout[icond(g, i, j)];
  }
  double dFdT = Cv, gT = 0.0, dF[64];
  dF[0] = T * cvd - 0.5 * u2;
  for (int m = 0; m < nm; ++m) dF[im0 + m] = X[im0 + m];
  dF[nv - 1] = -1.0;
  for (int i = 0; i < g->nvap; ++i) {
    const int vi = 1 + i, ci = icond(g, i, 0);
    const int sat = Yout[ci] > 0.0;
    const double c_v = g->sig_v[i] * cvd, c_c = g->sig_c[i][0] * cvd, mu_c = mu_of(g, i, 0);
    for (int j = 1; j < g->ncond; ++j)
      dF[icond(g, i, j)] = T * g->sig_c[i][j] * cvd + mu_of(g, i, j) - 0.5 * u2;
    if (sat) {
      double Ri = R_vap(g, i), dc = dc_of(g, i, 0);
      double beta = (g->Lref[i][0] + dc * g->Tref[i]) / (Ri * g->Tref[i]);
      double delta = dc / Ri, t = T / g->Tref[i];
      double rs = orc_sat_pressure(g, i, T) / (Ri * T);
      double drs = rs * ((beta / t - delta) / T - 1.0 / T);
      dFdT += drs * (T * (c_v - c_c) - mu_c);
      gT += drs * (lam_out[vi] - lam_out[ci]);
      dF[vi] = dF[ci] = T * c_c + mu_c - 0.5 * u2;
      lam_in[vi] = lam_in[ci] = lam_out[ci];
    } else {
      dF[vi] = dF[ci] = T * c_v - 0.5 * u2;
      lam_in[vi] = lam_in[ci] = lam_out[vi];
    }
  }
  const double coef = -gT / dFdT;
  for (int v = 0; v < nv; ++v) lam_in[v] += coef * dF[v];
  return 0;
}

static void satadj_adjoint_grid(const orc_grid *g, const double *Yout, double *lam) {
  const int nv = orc_nvar(g);
  const long ncell = (long)g->nx * g->ny * g->nz;
  double Yc[64] = {0}, lo[64] = {0}, li[64];
  for (long c = 0; c < ncell; ++c) {
    for (int v = 0; v < nv; ++v) {
      Yc[v] = Yout[v * ncell + c];
      lo[v] = lam[v * ncell + c];
    }
    orc_satadj_adjoint_cell(g, Yc, lo, li);
    for (int v = 0; v < nv; ++v) lam[v * ncell + c] = li[v];
  }
}

/* Adjoint of one SSP-RK3 step with time step dt (Sec. 4.3 in reverse): given lam_out =
 * dJ/dY^{n+1}, returns lam_in = dJ/dY^n. The intermediate stages are recomputed from Yn. */
int orc_step_adjoint(const orc_grid *g, const double *Yn, double dt, const double *lam_out,
                     double *lam_in) {
  const int nv = orc_nvar(g);
  const long n = (long)nv * g->nx * g->ny * g->nz;
  double *Y1 = malloc(sizeof(double) * (size_t)n), *Y2 = malloc(sizeof(double) * (size_t)n);
  double *mu = calloc((size_t)n, sizeof(double)), *Yb = malloc(sizeof(double) * (size_t)n);
  double *l2 = malloc(sizeof(double) * (size_t)n), *l1 = malloc(sizeof(double) * (size_t)n);
  double *Y3 = malloc(sizeof(double) * (size_t)n), *l3 = malloc(sizeof(double) * (size_t)n);
  const int sa = g->satadj && g->nvap > 0 && g->ncond > 0;
  int rc = -2;
  if (g->kessler) {
    rc = -3; /* the microphysics is not differentiated */
    goto done;
  }
  if (!Y1 || !Y2 || !mu || !Yb || !l2 || !l1 || !Y3 || !l3) goto done;
  if ((rc = orc_stage(g, 0, Yn, Yn, dt, Y1)) < 0) goto done;
  if ((rc = orc_stage(g, 1, Yn, Y1, dt, Y2)) < 0) goto done;
  if (sa && (rc = orc_stage(g, 2, Yn, Y2, dt, Y3)) < 0) goto done;
  /* each stage ends with the saturation adjustment: its transpose comes first */
  for (long c = 0; c < n; ++c) l3[c] = lam_out[c];
  if (sa) satadj_adjoint_grid(g, Y3, l3);
  /* stage 2: Y3 = Yn/3 + 2/3 (Y2 + dt L(Y2)) */
  for (long c = 0; c < n; ++c) mu[c] = 2.0 / 3.0 * dt * l3[c];
  if ((rc = orc_rhs_adjoint(g, Y2, mu, Yb))) goto done;
  for (long c = 0; c < n; ++c) {
    l2[c] = 2.0 / 3.0 * l3[c] + Yb[c];
    lam_in[c] = l3[c] / 3.0;
  }
  if (sa) satadj_adjoint_grid(g, Y2, l2);
  /* stage 1: Y2 = 3/4 Yn + 1/4 (Y1 + dt L(Y1)) */
  for (long c = 0; c < n; ++c) mu[c] = 0.25 * dt * l2[c];
  if ((rc = orc_rhs_adjoint(g, Y1, mu, Yb))) goto done;
  for (long c = 0; c < n; ++c) {
    l1[c] = 0.25 * l2[c] + Yb[c];
    lam_in[c] += 0.75 * l2[c];
  }
  if (sa) satadj_adjoint_grid(g, Y1, l1);
  /* stage 0: Y1 = Yn + dt L(Yn) */
  for (long c = 0; c < n; ++c) mu[c] = dt * l1[c];
  if ((rc = orc_rhs_adjoint(g, Yn, mu, Yb))) goto done;
  for (long c = 0; c < n; ++c) lam_in[c] += l1[c] + Yb[c];
  rc = 0;
done:
  free(Y1); free(Y2); free(mu); free(Yb); free(l2); free(l1); free(Y3); free(l3);
  return rc;
}
