/* snap_oracle.h -- plain FP64 CPU reference of one SNAP finite-volume step.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may call this code. The product library never links or loads it, and this
 * oracle shares no code, header, table or helper with the CUDA path.
 *
 * Sources (Li & Chen 2019, "Simulating Non-hydrostatic atmospheres on Planets"):
 *   conserved / primitive vectors and their conversion ............ App. B
 *   equation of state, total energy, latent heat, chem. potential . Sec. 2
 *   finite-volume update, Riemann problem, reconstruction ........ Sec. 4, Eqs. forward, riemann, q+
 *   LMARS face pressure and velocity ............................. Sec. 4.1, Eqs. rp, ru
 *   fifth-order WENO and the linear interpolant ................... Sec. 4.2, Eq. weno5
 *   SSP (TVD) Runge-Kutta 3 ........................................ Sec. 4.3
 *   saturation adjustment (isochoric) .............................. App. D, Eqs. dx, dxf, u
 * Readings of passages the paper leaves open are stated at each function in snap_oracle.c.
 *
 * Every array is FP64, structure-of-arrays Y[field][k][j][i] with i fastest, interior cells
 * only. Field order (App. B): rho_d, rho_i (nvap), rho_ij (nvap x ncond grouped by vapour),
 * rho u, [rho v when ny > 1], rho w, rho e.
 */
#ifndef SNAP_ORACLE_H
#define SNAP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXV 4
#define ORC_MAXC 2

/* Boundary of one side: a free-slip wall (ghosts mirror the state, normal velocity negated),
 * periodic, or a no-slip wall (ghosts mirror the state with every velocity component
 * negated). */
enum { ORC_REFLECT = 0, ORC_PERIODIC = 1, ORC_NOSLIP = 2 };

typedef struct {
  int nx, ny, nz;               /* ny == 1: x-z plane with no y direction */
  double dx, dy, dz;
  int bc[6];                    /* x-, x+, y-, y+, z-, z+ */
  double grav, gamma_d, Rd;
  int nvap, ncond;              /* vapours; condensates per vapour */
  double eps[ORC_MAXV];         /* m_i / m_d */
  double sig_v[ORC_MAXV];       /* c_v,i / c_vd */
  double Tref[ORC_MAXV];        /* reference temperature of vapour i */
  double pref[ORC_MAXV];        /* saturation pressure over condensate (i,1) at Tref */
  double sig_c[ORC_MAXV][ORC_MAXC]; /* c_ij / c_vd */
  double Lref[ORC_MAXV][ORC_MAXC];  /* latent heat of condensate (i,j) at Tref */
  const double *rho_bar;        /* [nz] reference density */
  const double *p_bar_face;     /* [nz+1] reference pressure at level faces */
  double nu;                    /* constant kinematic viscosity (0: inviscid) */
  int satadj;                   /* apply saturation adjustment after each stage */
  int satadj_max_iter;
  double satadj_tol;
  double weno_eps;
  int gravity_energy_pointwise; /* 0: -g (F_rho,k-1/2 + F_rho,k+1/2)/2 ; 1: -g (rho w)_k */
  /* Sec. 2, Eq. d3: terminal velocity of condensate phase j of every vapour (m/s, < 0 falls);
   * nonzero values add the sedimentation fluxes of mass, momentum and energy in z */
  double w_term[ORC_MAXC];
  /* Sec. 3: Kessler microphysics after every step, backward Euler with Newton iterations:
   * k1 condensation, k2 autoconversion, k3 accretion, k4 evaporation of precipitation */
  int kessler;
  double kessler_k[4];
  int kessler_max_iter;
  double kessler_tol;
  /* Sec. 6 forcing of the Jovian simulation (0 disables each): a body cooling of cool_rate
   * K/s at constant volume in levels whose reference pressure lies in [cool_p_lo, cool_p_hi];
   * a sponge relaxing the horizontal momenta at 1/(tau0 (p/p0)^2) where p < p0 */
  double cool_rate, cool_p_lo, cool_p_hi;
  double sponge_tau0, sponge_p0;
  /* Sec. 6 lower boundary: > 0 holds the ghost cells below z = 0 at this temperature (K),
   * with the pressure, composition and velocities of the cells they mirror (0: off) */
  double T_bottom;
} orc_grid;

int orc_nvar(const orc_grid *g);

/* ---- pointwise pieces (exposed for the pins) ---- */
double orc_weno5(const double q[5], double eps);          /* I_weno(q_{i-3..i+1}) */
double orc_weno5_poly(const double q[5]);                 /* I_poly */
void orc_weno5_weights(const double q[5], double eps, double w[3]);

/* App. B: X = (rho, q_i, q_ij, u, [v], w, p) with the TOTAL pressure p. Also returns T and
 * the effective adiabatic index gamma (may be NULL). */
void orc_cons_to_prim(const orc_grid *g, const double *Y, double *X, double *T, double *gamma);
void orc_prim_to_cons(const orc_grid *g, const double *X, double *Y);
double orc_sat_pressure(const orc_grid *g, int i, double T);

/* LMARS flux through a face with unit normal along momentum component `dir` (0 x, 1 y, 2 z
 * in the 3-D numbering; in the x-z plane use 0 for x and 2 for z). XL/XR are primitive
 * states whose last entry is the pressure perturbation p' = p - pref; pref is the reference
 * pressure at this face. F receives nvar fluxes; ustar / pstar (may be NULL) receive the
 * face velocity u* and the face pressure perturbation p'*. */
void orc_lmars(const orc_grid *g, const double *XL, const double *XR, int dir, double pref,
               double *F, double *ustar, double *pstar);

/* App. D saturation adjustment of one cell, in place; returns the number of sweeps used or
 * -1 when it did not converge within max_iter. */
int orc_satadj_cell(const orc_grid *g, double *Ycell, int max_iter, double tol);
/* Exact equilibrium by bisection on temperature (test pin for orc_satadj_cell). */
int orc_satadj_bisect(const orc_grid *g, double *Ycell);

/* Sec. 3 Kessler scheme on one cell, in place: each vapour i with its cloud (i,1) and
 * precipitation (i,2) advances its mass mixing ratios by one backward Euler step of length
 * dt (Newton iterations of Eq. x_n+1). Returns the largest iteration count, or -1 when an
 * iteration did not converge. */
int orc_kessler_cell(const orc_grid *g, double *Ycell, double dt);

/* App. A, Eq. theta_e (Emanuel's 4.5.11): equivalent potential temperature of each cell of a
 * state with one vapour, whose first condensate is the cloud (precipitation is not part of
 * q_t), p0 = 1e5 Pa. Returns -3 unless the grid has exactly one vapour. */
int orc_theta_e(const orc_grid *g, const double *Y, double *theta_e);

/* ---- whole-grid pieces ---- */
/* dYdt = L(Y): minus the flux divergence plus the gravity source (and viscous fluxes). */
int orc_rhs(const orc_grid *g, const double *Y, double *dYdt);
/* One SSP-RK3 stage combine (Sec. 4.3) on n values: stage 0, 1, 2. */
void orc_rk3_combine(int stage, long n, const double *Yn, const double *Ys, const double *L,
                     double dt, double *Yout);
/* One Runge-Kutta stage: Yout = combine(Yn, Ys + dt L(Ys)), then saturation adjustment.
 * Returns the largest sweep count, or -1 if a cell did not converge. */
int orc_stage(const orc_grid *g, int stage, const double *Yn, const double *Ys, double dt,
              double *Yout);
/* nsteps full steps in place; dt <= 0 means recompute dt = cfl * min dx/(|u|+c) per step.
 * With g->kessler set, the Kessler scheme follows each step (time splitting). */
int orc_step(const orc_grid *g, double *Y, int nsteps, double dt, double cfl, double *dt_last);
double orc_dt_cfl(const orc_grid *g, const double *Y, double cfl);
/* out[f] = sum of field f times the cell volume (nvar values), out[nvar] = sum of
 * (rho e + rho g z) times the cell volume. */
void orc_budget(const orc_grid *g, const double *Y, double *out);

/* ---- discrete adjoint (inviscid): transposes of the routines above ---- */
double orc_weno5_gradient(const double q[5], double eps, double grad[5]);
/* Ybar = (dL/dY)^T mu at state Y (returns -3 for viscous grids, with sedimentation, forcing,
 * a no-slip wall or a fixed bottom temperature). */
int orc_rhs_adjoint(const orc_grid *g, const double *Y, const double *mu, double *Ybar);
/* lam_in = (dYout/dYin)^T lam_out for the saturation adjustment of one cell, evaluated at its
 * converged result Yout (App. D equilibrium; see the definition for the derivation). */
int orc_satadj_adjoint_cell(const orc_grid *g, const double *Yout, const double *lam_out,
                            double *lam_in);
/* lam_in = (dY^{n+1}/dY^n)^T lam_out for one step of time step dt from Yn (with the
 * saturation adjustment after every stage when g->satadj is set; -3 with the Kessler
 * scheme, which is not differentiated). */
int orc_step_adjoint(const orc_grid *g, const double *Yn, double dt, const double *lam_out,
                     double *lam_in);

#ifdef __cplusplus
}
#endif
#endif
