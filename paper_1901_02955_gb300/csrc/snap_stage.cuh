// snap_stage.cuh -- device code of one explicit Runge-Kutta stage of the SNAP finite-volume
// scheme (Li & Chen 2019), templated on arithmetic type and field layout. Included by the
// per-configuration translation units kern_*.cu.
//
// One CTA owns a tile of TX x TY x TZ interior cells. It builds the primitives of the tile and
// of a 3-cell halo in each direction in shared memory (ghost cells of the domain boundary are
// synthesised here: mirrored with the normal velocity negated, or wrapped), then for each
// direction reconstructs both face states with WENO5 (Sec. 4.2), solves the LMARS Riemann
// problem (Sec. 4.1) and keeps the face fluxes in shared memory; the owned cells accumulate
// the flux divergence (Eq. forward), add the gravity source, combine the Runge-Kutta stage
// (Sec. 4.3), apply the saturation adjustment (App. D) and store. Face states and fluxes never
// leave the SM.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "snap_internal.h"

namespace snap {

// ------------------------------------------------------------------------------------------
// arithmetic helpers per type
// ------------------------------------------------------------------------------------------
template <class R>
struct Ar;
template <>
struct Ar<float> {
  // approximate reciprocal (hardware rcp, ~1 ulp) -- FP32 path only
  static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float exp_(float x) { return expf(x); }
  static __device__ __forceinline__ float log_(float x) { return logf(x); }
  static __device__ __forceinline__ float pow_(float x, float y) { return powf(x, y); }
  static constexpr double eps = 1.1920928955078125e-07;
};
template <>
struct Ar<double> {
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
  static __device__ __forceinline__ double log_(double x) { return log(x); }
  static __device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }
  static constexpr double eps = 2.220446049250313e-16;
};

// Field layout of the conserved / primitive vectors (App. B):
// 0 rho_d | 1.. vapours | condensates grouped by vapour | momenta | energy.
template <int NVAP_, int NCOND_, bool D3_>
struct Lay {
  static constexpr int NVAP = NVAP_, NCOND = NCOND_;
  static constexpr bool D3 = D3_;
  static constexpr int NMOM = D3 ? 3 : 2;
  static constexpr int IM0 = 1 + NVAP + NVAP * NCOND;
  static constexpr int NV = IM0 + NMOM + 1;
  static constexpr int IE = NV - 1;
  static __host__ __device__ constexpr int cond(int i, int j) { return 1 + NVAP + i * NCOND + j; }
  // momentum slot of spatial direction d (0 x, 1 y, 2 z)
  static __host__ __device__ constexpr int mom(int d) {
    return D3 ? IM0 + d : IM0 + (d == 2 ? 1 : 0);
  }
  static constexpr bool MOIST = NVAP > 0 && NCOND > 0;
};

template <bool D3>
struct Tile;
template <>
struct Tile<false> {  // x-z plane
  static constexpr int TX = 32, TY = 1, TZ = 16, NT = 256;
};
template <>
struct Tile<true> {
  static constexpr int TX = 8, TY = 8, TZ = 4, NT = 256;
};

template <bool D3>
struct Box {
  using T = Tile<D3>;
  static constexpr int HX = 3, HY = D3 ? 3 : 0, HZ = 3;
  static constexpr int BX = T::TX + 6, BY = T::TY + 2 * HY, BZ = T::TZ + 6;
  static constexpr int NBOX = BX * BY * BZ;
  static constexpr int NFX = (T::TX + 1) * T::TY * T::TZ;
  static constexpr int NFY = D3 ? T::TX * (T::TY + 1) * T::TZ : 0;
  static constexpr int NFZ = T::TX * T::TY * (T::TZ + 1);
  static constexpr int NF = NFX > NFZ ? (NFX > NFY ? NFX : NFY) : (NFZ > NFY ? NFZ : NFY);
  static constexpr int NCELL = T::TX * T::TY * T::TZ;
  static constexpr int CPT = NCELL / T::NT;  // owned cells per thread
  static __device__ __forceinline__ int at(int bx, int by, int bz) {
    return (bz * BY + by) * BX + bx;
  }
};

// ------------------------------------------------------------------------------------------
// thermodynamics (Sec. 2, App. B)
// ------------------------------------------------------------------------------------------
// Conserved -> primitive. y holds the stored state, whose energy entry is rho e - eref with
// eref = pbar / (gamma_d - 1). x receives (rho, q_i, q_ij, u, [v], w, p - pbar), the total
// pressure is returned in p_tot and T in T_out. Dry: p - pbar = (gamma_d - 1)(y_E - K) is
// formed from small numbers. Moist: the inversion U = rho e - K - A, T = U / C_v, p = R_m T
// runs in FP64.
template <class R, class L>
__device__ __forceinline__ void cons_to_prim(const Phys &ph, const R *y, R *x, double pbar,
                                             double eref, R &p_tot, R &T_out) {
  R rho = y[0];
#pragma unroll
  for (int s = 1; s < L::IM0; ++s) rho += y[s];
  const R ir = Ar<R>::rcp(rho);
  x[0] = rho;
#pragma unroll
  for (int s = 1; s < L::IM0; ++s) x[s] = y[s] * ir;
  R K = R(0);
#pragma unroll
  for (int m = 0; m < L::NMOM; ++m) {
    x[L::IM0 + m] = y[L::IM0 + m] * ir;
    K += y[L::IM0 + m] * x[L::IM0 + m];
  }
  K *= R(0.5);
  if constexpr (L::NVAP == 0) {
    // dry: p = (gamma_d - 1) (rho e - K), so p - pbar = (gamma_d - 1) (y_E - K)
    const R pp = R(ph.gamma_d - 1.0) * (y[L::IE] - K);
    x[L::IE] = pp;
    const R p = pp + R(pbar);
    p_tot = p;
    T_out = p * Ar<R>::rcp(rho * R(ph.R_d));
    (void)eref;
  } else {
    double A = 0.0, Cv = y[0], Rm = y[0];
#pragma unroll
    for (int i = 0; i < L::NVAP; ++i) {
      Cv += ph.sig_v[i] * double(y[1 + i]);
      Rm += ph.inv_eps[i] * double(y[1 + i]);
#pragma unroll
      for (int j = 0; j < L::NCOND; ++j) {
        Cv += ph.sig_c[i][j] * double(y[L::cond(i, j)]);
        A += ph.mu[i][j] * double(y[L::cond(i, j)]);
      }
    }
    Cv *= ph.c_vd;
    Rm *= ph.R_d;
    double U = (double(y[L::IE]) + eref) - double(K) - A;
    double T = U / Cv;
    double p = Rm * T;
    p_tot = R(p);
    T_out = R(T);
    x[L::IE] = R(p - pbar);
  }
}

// mixing factors of App. B: num = 1 + sum q_i (sigma_vi - 1) + sum q_ij (sigma_ij - 1),
// den = 1 + sum q_i (1/eps_i - 1) - sum q_ij
template <class R, class L>
__device__ __forceinline__ void mix_factors(const Phys &ph, const R *x, R &num, R &den) {
  num = R(1);
  den = R(1);
#pragma unroll
  for (int i = 0; i < L::NVAP; ++i) {
    num += x[1 + i] * R(ph.sig_v[i] - 1.0);
    den += x[1 + i] * R(ph.inv_eps[i] - 1.0);
#pragma unroll
    for (int j = 0; j < L::NCOND; ++j) {
      num += x[L::cond(i, j)] * R(ph.sig_c[i][j] - 1.0);
      den -= x[L::cond(i, j)];
    }
  }
}

// ------------------------------------------------------------------------------------------
// WENO5 (Sec. 4.2, Eq. weno5) with Jiang-Shu weights: value at face i-1/2 from the left,
// (a..e) = Q_{i-3} .. Q_{i+1}.
// ------------------------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R weno5(R a, R b, R c, R d, R e, R eps) {
  R t, b0, b1, b2;
  t = a - R(2) * b + c;
  b0 = R(13.0 / 12.0) * t * t;
  t = a - R(4) * b + R(3) * c;
  b0 += R(0.25) * t * t;
  t = b - R(2) * c + d;
  b1 = R(13.0 / 12.0) * t * t;
  t = b - d;
  b1 += R(0.25) * t * t;
  t = c - R(2) * d + e;
  b2 = R(13.0 / 12.0) * t * t;
  t = R(3) * c - R(4) * d + e;
  b2 += R(0.25) * t * t;
  R s0 = eps + b0, s1 = eps + b1, s2 = eps + b2;
  R a0 = R(0.1) * Ar<R>::rcp(s0 * s0);
  R a1 = R(0.6) * Ar<R>::rcp(s1 * s1);
  R a2 = R(0.3) * Ar<R>::rcp(s2 * s2);
  R v0 = a * R(1.0 / 3.0) - R(7.0 / 6.0) * b + R(11.0 / 6.0) * c;
  R v1 = -b * R(1.0 / 6.0) + R(5.0 / 6.0) * c + d * R(1.0 / 3.0);
  R v2 = c * R(1.0 / 3.0) + R(5.0 / 6.0) * d - e * R(1.0 / 6.0);
  return Ar<R>::div(a0 * v0 + a1 * v1 + a2 * v2, a0 + a1 + a2);
}

// ------------------------------------------------------------------------------------------
// LMARS (Sec. 4.1, Eqs. rp, ru) on primitive face states carrying p' = p - pref.
// rho c from the side averages; upwind side by the sign of u*; flux u* Phi_S + p'* n with
// Phi = (rho_d, rho_i, rho_ij, rho u, [rho v], rho w, rho e + p) of side S.
// ------------------------------------------------------------------------------------------
template <class R, class L>
__device__ __forceinline__ void lmars(const Phys &ph, const R *XL, const R *XR, int dir,
                                      R pref, R *F) {
  const int mn = L::mom(dir);
  R numL, denL, numR, denR;
  mix_factors<R, L>(ph, XL, numL, denL);
  mix_factors<R, L>(ph, XR, numR, denR);
  const R gm1 = R(ph.gamma_d - 1.0);
  R pL = pref + XL[L::IE], pR = pref + XR[L::IE];
  R gamL, gamR;
  if constexpr (L::NVAP == 0) {
    gamL = gamR = R(ph.gamma_d);
  } else {
    gamL = R(1) + gm1 * Ar<R>::div(denL, numL);
    gamR = R(1) + gm1 * Ar<R>::div(denR, numR);
  }
  R cL = Ar<R>::sqrt_(gamL * pL * Ar<R>::rcp(XL[0]));
  R cR = Ar<R>::sqrt_(gamR * pR * Ar<R>::rcp(XR[0]));
  R rhoc = R(0.5) * (XL[0] + XR[0]) * R(0.5) * (cL + cR);
  R uL = XL[mn], uR = XR[mn];
  R ps = R(0.5) * (XL[L::IE] + XR[L::IE]) - R(0.5) * rhoc * (uR - uL);
  R us = R(0.5) * (uL + uR) - Ar<R>::div(XR[L::IE] - XL[L::IE], R(2) * rhoc);
  const bool left = us > R(0);
  const R *XS = left ? XL : XR;
  R numS = left ? numL : numR, denS = left ? denL : denR, pS = left ? pL : pR;
  R rhoS = XS[0];
  R mf = us * rhoS;
  R qsum = R(0);
#pragma unroll
  for (int s = 1; s < L::IM0; ++s) {
    F[s] = mf * XS[s];
    qsum += XS[s];
  }
  F[0] = mf * (R(1) - qsum);
  R K = R(0);
#pragma unroll
  for (int m = 0; m < L::NMOM; ++m) {
    F[L::IM0 + m] = mf * XS[L::IM0 + m];
    K += XS[L::IM0 + m] * XS[L::IM0 + m];
  }
  K *= R(0.5) * rhoS;
  F[mn] += ps;
  R A = R(0);
#pragma unroll
  for (int i = 0; i < L::NVAP; ++i)
#pragma unroll
    for (int j = 0; j < L::NCOND; ++j) A += R(ph.mu[i][j]) * XS[L::cond(i, j)];
  A *= rhoS;
  R rhoe;
  if constexpr (L::NVAP == 0)
    rhoe = pS * Ar<R>::rcp(gm1) + K;
  else
    rhoe = Ar<R>::div(numS, denS) * pS * Ar<R>::rcp(gm1) + K + A;
  F[L::IE] = us * (rhoe + pS);
}

// ------------------------------------------------------------------------------------------
// App. D saturation adjustment of one cell (isochoric). Each sweep visits the vapours in
// order: projected molar transfer of Eq. dxf with the isochoric alpha, limited to keep both
// phases non-negative, then T and p follow from the conserved energy and the equation of
// state. Returns the sweep count, or -1 without convergence.
// ------------------------------------------------------------------------------------------
template <class R, class L>
__device__ __forceinline__ void cell_Tp(const Phys &ph, const R *y, double eref, double &T,
                                        double &p) {
  double rho = 0.0, K2 = 0.0, A = 0.0, Cv = y[0], Rm = y[0];
#pragma unroll
  for (int s = 0; s < L::IM0; ++s) rho += double(y[s]);
#pragma unroll
  for (int m = 0; m < L::NMOM; ++m) K2 += double(y[L::IM0 + m]) * double(y[L::IM0 + m]);
#pragma unroll
  for (int i = 0; i < L::NVAP; ++i) {
    Cv += ph.sig_v[i] * double(y[1 + i]);
    Rm += ph.inv_eps[i] * double(y[1 + i]);
#pragma unroll
    for (int j = 0; j < L::NCOND; ++j) {
      Cv += ph.sig_c[i][j] * double(y[L::cond(i, j)]);
      A += ph.mu[i][j] * double(y[L::cond(i, j)]);
    }
  }
  double U = (double(y[L::IE]) + eref) - 0.5 * K2 / rho - A;
  T = U / (Cv * ph.c_vd);
  p = Rm * ph.R_d * T;
}

template <class R, class L>
__device__ int satadj_cell(const Phys &ph, R *y, double eref, int max_iter, double tol) {
  if constexpr (!L::MOIST) {
    return 0;
  } else {
    for (int sweep = 1; sweep <= max_iter; ++sweep) {
      bool conv = true;
#pragma unroll
      for (int i = 0; i < L::NVAP; ++i) {
        double Td, pd;
        cell_Tp<R, L>(ph, y, eref, Td, pd);
        R T = R(Td), p = R(pd);
        const R dTr = R(Td - ph.Tref[i]);  // T - T^r kept accurate: s(T) is steep
        R N = y[0], gas = y[0], heat = R(0);
#pragma unroll
        for (int k = 0; k < L::NVAP; ++k) {
          R tot = y[1 + k];
#pragma unroll
          for (int j = 0; j < L::NCOND; ++j) tot += y[L::cond(k, j)];
          N += tot * R(ph.inv_eps[k]);
          gas += y[1 + k] * R(ph.inv_eps[k]);
          heat += tot * R(ph.inv_eps[k]) * R(ph.sig_hat[k] - 1.0);
        }
        const R iN = Ar<R>::rcp(N);
        heat *= iN;
        R qv = y[1 + i] * R(ph.inv_eps[i]) * iN;
        R qc = y[L::cond(i, 0)] * R(ph.inv_eps[i]) * iN;
        R gsum = gas * iN - qv;
        R t = T * R(1.0 / ph.Tref[i]);
        // p* = p^r exp[beta (1 - 1/t) - delta ln t] with 1 - 1/t = (T - T^r) / T
        R ps = R(ph.pref[i]) *
               Ar<R>::exp_(R(ph.beta[i]) * dTr * Ar<R>::rcp(T) - R(ph.delta[i]) * Ar<R>::log_(t));
        R s = Ar<R>::div(ps, p);
        R dq;
        if (s >= R(1)) {
          dq = -qc;
        } else {
          R bt = R(ph.beta[i]) * Ar<R>::rcp(t) - R(ph.delta[i]);
          R alpha = R(ph.gamma_d - 1.0) * (bt - R(1)) * Ar<R>::rcp(R(1) + heat);
          R om = R(1) - s;
          R r = Ar<R>::div(s, om);
          dq = Ar<R>::div(qv - r * gsum, R(1) + Ar<R>::div(s, om * om) * bt * alpha * gsum);
        }
        R drho;
        if (dq >= qv) {
          dq = qv;
          drho = y[1 + i];
        } else if (dq <= -qc) {
          dq = -qc;
          drho = -y[L::cond(i, 0)];
        } else {
          drho = dq * R(ph.eps[i]) * N;
        }
        y[1 + i] -= drho;
        y[L::cond(i, 0)] += drho;
        if (fabs(double(dq)) > tol * double(qv + qc)) conv = false;
      }
      if (conv) return sweep;
    }
    return -1;
  }
}

// CFL rate sum_d (|u_d| + c) / dx_d of one cell (the time-step rule of the library).
template <class R, class L>
__device__ __forceinline__ double cell_rate(const Phys &ph, const R *y, double eref, double idx,
                                            double idy, double idz) {
  double T, p;
  double rho = 0.0;
#pragma unroll
  for (int s = 0; s < L::IM0; ++s) rho += double(y[s]);
  if constexpr (L::NVAP == 0) {
    double K2 = 0.0;
#pragma unroll
    for (int m = 0; m < L::NMOM; ++m) K2 += double(y[L::IM0 + m]) * double(y[L::IM0 + m]);
    p = (ph.gamma_d - 1.0) * ((double(y[L::IE]) + eref) - 0.5 * K2 / rho);
    T = 0.0;
  } else {
    cell_Tp<R, L>(ph, y, eref, T, p);
  }
  // gamma of App. B from the mass fractions
  double num = 1.0, den = 1.0;
#pragma unroll
  for (int i = 0; i < L::NVAP; ++i) {
    num += double(y[1 + i]) / rho * (ph.sig_v[i] - 1.0);
    den += double(y[1 + i]) / rho * (ph.inv_eps[i] - 1.0);
#pragma unroll
    for (int j = 0; j < L::NCOND; ++j) {
      num += double(y[L::cond(i, j)]) / rho * (ph.sig_c[i][j] - 1.0);
      den -= double(y[L::cond(i, j)]) / rho;
    }
  }
  double gam = 1.0 + (ph.gamma_d - 1.0) * den / num;
  double c = sqrt(gam * p / rho);
  double r = (fabs(double(y[L::mom(0)])) / rho + c) * idx + (fabs(double(y[L::mom(2)])) / rho + c) * idz;
  if constexpr (L::D3) r += (fabs(double(y[L::mom(1)])) / rho + c) * idy;
  (void)T;
  return r;
}

__device__ __forceinline__ int map_index(int g, int n, int bc_lo, int bc_hi, bool &flip) {
  flip = false;
  if (g < 0) {
    if (bc_lo == 1) return ((g % n) + n) % n;
    flip = true;
    return -1 - g;
  }
  if (g >= n) {
    if (bc_hi == 1) return g % n;
    flip = true;
    return 2 * n - 1 - g;
  }
  return g;
}

__device__ __forceinline__ int find_domain(const int *prefix, int ndom, int tile) {
  int lo = 0, hi = ndom - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(prefix + mid) <= tile)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ double block_max(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < int(blockDim.x >> 5)) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

// ------------------------------------------------------------------------------------------
// the fused stage kernel
// ------------------------------------------------------------------------------------------
template <class R, class L, bool VISC>
struct StageSmem {
  using B = Box<L::D3>;
  static constexpr size_t prim = sizeof(R) * L::NV * B::NBOX;
  static constexpr size_t visc = VISC ? sizeof(R) * 2 * B::NBOX : 0;
  static constexpr size_t flux = sizeof(R) * L::NV * B::NF;
  static constexpr size_t red = 32 * sizeof(double);
  static constexpr size_t total = prim + visc + flux + red;
};

template <class R, class L, bool VISC>
__global__ void __launch_bounds__(Tile<L::D3>::NT)
    stage_kernel(const StageArgs a) {
  using T = Tile<L::D3>;
  using B = Box<L::D3>;
  using S = StageSmem<R, L, VISC>;
  constexpr int NV = L::NV;
  extern __shared__ __align__(16) unsigned char smem[];
  R *s_prim = reinterpret_cast<R *>(smem);
  R *s_th = reinterpret_cast<R *>(smem + S::prim);
  R *s_pi = s_th + (VISC ? B::NBOX : 0);
  R *s_flux = reinterpret_cast<R *>(smem + S::prim + S::visc);
  double *s_red = reinterpret_cast<double *>(smem + S::prim + S::visc + S::flux);
  const Phys &ph = a.ph;
  const R weps = R(ph.weno_eps);

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int dm = find_domain(a.tile_domain, a.ndom, tile);
    const DomDev &D = a.doms[dm];
    const int nx = D.nx, ny = D.ny, nz = D.nz;
    const long long ncell = D.ncell;
    const int lt = tile - D.tile_begin;
    const int x0 = (lt % D.tx) * T::TX;
    const int y0 = ((lt / D.tx) % D.ty) * T::TY;
    const int z0 = (lt / (D.tx * D.ty)) * T::TZ;
    const int ex = min(T::TX, nx - x0), ey = min(T::TY, ny - y0), ez = min(T::TZ, nz - z0);
    const R *Ys = reinterpret_cast<const R *>(D.buf[a.stage == 0 ? 0 : a.stage]);
    const R *Yn = reinterpret_cast<const R *>(D.buf[0]);
    R *Yo = reinterpret_cast<R *>(D.buf[a.stage == 0 ? 1 : (a.stage == 1 ? 2 : 0)]);
    double dt;
    if (a.stage == 0) {
      dt = D.dt_fixed > 0.0 ? D.dt_fixed : D.cfl / __longlong_as_double((long long)*D.rate);
      if (lt == 0 && threadIdx.x == 0) *D.dt_step = dt;
    } else {
      dt = *D.dt_step;
      if (a.stage == 1 && lt == 0 && threadIdx.x == 0) *D.rate = 0ull;
    }

    // ---- 1. owned cells: load, keep the conserved values, store primitives -------------
    R ys[B::CPT][NV];
#pragma unroll
    for (int m = 0; m < B::CPT; ++m) {
      const int c = threadIdx.x + m * T::NT;
      const int lx = c % T::TX, ly = (c / T::TX) % T::TY, lz = c / (T::TX * T::TY);
      if (lx < ex && ly < ey && lz < ez) {
        const long long g = ((long long)(z0 + lz) * ny + (y0 + ly)) * nx + (x0 + lx);
#pragma unroll
        for (int v = 0; v < NV; ++v) ys[m][v] = Ys[v * ncell + g];
        R x[NV], pt, Tt;
        cons_to_prim<R, L>(ph, ys[m], x, D.p_cell[z0 + lz], D.e_ref[z0 + lz], pt, Tt);
        const int bi = B::at(lx + 3, ly + B::HY, lz + 3);
#pragma unroll
        for (int v = 0; v < NV; ++v) s_prim[v * B::NBOX + bi] = x[v];
        if constexpr (VISC) {
          const R Pi = Ar<R>::pow_(pt * R(1e-5), R(ph.kappa));
          s_th[bi] = Tt * Ar<R>::rcp(Pi);
          s_pi[bi] = Pi;
        }
      }
    }
    // ---- 2. halo cells of the cross (x, y, z), ghosts synthesised from the boundary rule --
    {
      const int nhx = 6 * ey * ez, nhy = L::D3 ? 6 * ex * ez : 0, nhz = 6 * ex * ey;
      for (int h = threadIdx.x; h < nhx + nhy + nhz; h += T::NT) {
        int bx, by, bz, dirn;
        if (h < nhx) {
          int r = h % 6, q = h / 6;
          bx = r < 3 ? r : ex + r;
          by = q % ey + B::HY;
          bz = q / ey + 3;
          dirn = 0;
        } else if (h < nhx + nhy) {
          int hh = h - nhx;
          int r = (hh / ex) % 6, q = hh / (6 * ex);
          bx = hh % ex + 3;
          by = r < 3 ? r : ey + r;
          bz = q + 3;
          dirn = 1;
        } else {
          int hh = h - nhx - nhy;
          int r = (hh / (ex * ey)) % 6;
          bx = hh % ex + 3;
          by = (hh / ex) % ey + B::HY;
          bz = r < 3 ? r : ez + r;
          dirn = 2;
        }
        int gx = x0 + bx - 3, gy = y0 + by - B::HY, gz = z0 + bz - 3;
        bool flip = false;
        if (dirn == 0) gx = map_index(gx, nx, D.bc[0], D.bc[1], flip);
        if (dirn == 1) gy = map_index(gy, ny, D.bc[2], D.bc[3], flip);
        if (dirn == 2) gz = map_index(gz, nz, D.bc[4], D.bc[5], flip);
        const long long g = ((long long)gz * ny + gy) * nx + gx;
        R y[NV], x[NV], pt, Tt;
#pragma unroll
        for (int v = 0; v < NV; ++v) y[v] = Ys[v * ncell + g];
        cons_to_prim<R, L>(ph, y, x, D.p_cell[gz], D.e_ref[gz], pt, Tt);
        if (flip) x[L::mom(dirn)] = -x[L::mom(dirn)];
        const int bi = B::at(bx, by, bz);
#pragma unroll
        for (int v = 0; v < NV; ++v) s_prim[v * B::NBOX + bi] = x[v];
        if constexpr (VISC) {
          const R Pi = Ar<R>::pow_(pt * R(1e-5), R(ph.kappa));
          s_th[bi] = Tt * Ar<R>::rcp(Pi);
          s_pi[bi] = Pi;
        }
      }
    }
    __syncthreads();

    R acc[B::CPT][NV];
#pragma unroll
    for (int m = 0; m < B::CPT; ++m)
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[m][v] = R(0);

    // ---- 3. per direction: WENO5 both sides, LMARS, flux divergence ---------------------
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d == 1 && !L::D3) continue;
      const int fx = d == 0, fy = d == 1, fz = d == 2;
      const int nfx = ex + fx, nfy = ey + fy, nfz = ez + fz;
      const int sx = T::TX + fx, sy = T::TY + fy;  // flux array strides
      const int stride = d == 0 ? 1 : (d == 1 ? B::BX : B::BX * B::BY);
      const double hd = d == 0 ? D.dx : (d == 1 ? D.dy : D.dz);
      for (int f = threadIdx.x; f < nfx * nfy * nfz; f += T::NT) {
        const int ix = f % nfx, iy = (f / nfx) % nfy, iz = f / (nfx * nfy);
        const int bi = B::at(ix + 3, iy + B::HY, iz + 3);  // right cell of the face
        R QL[NV], QR[NV], F[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const R *q = s_prim + v * B::NBOX + bi;
          R q0 = q[-3 * stride], q1 = q[-2 * stride], q2 = q[-stride], q3 = q[0],
            q4 = q[stride], q5 = q[2 * stride];
          QL[v] = weno5<R>(q0, q1, q2, q3, q4, weps);
          QR[v] = weno5<R>(q5, q4, q3, q2, q1, weps);
        }
        const R pref = R(fz ? D.p_face[z0 + iz] : D.p_cell[z0 + iz]);
        lmars<R, L>(ph, QL, QR, d, pref, F);
        if constexpr (VISC) {
          const int bl = bi - stride;
          const R rl = s_prim[bl], rr = s_prim[bi];
          const R rf = R(0.5) * (rl + rr);
          const R ih = R(1.0 / hd), nu = R(ph.nu);
          R work = R(0);
#pragma unroll
          for (int mm = 0; mm < L::NMOM; ++mm) {
            const R ul = s_prim[(L::IM0 + mm) * B::NBOX + bl];
            const R ur = s_prim[(L::IM0 + mm) * B::NBOX + bi];
            const R grad = (ur - ul) * ih;
            F[L::IM0 + mm] -= rf * nu * grad;
            work += R(0.5) * (ul + ur) * grad;
          }
          const R heat = R(0.5) * (s_pi[bl] + s_pi[bi]) * (s_th[bi] - s_th[bl]) * ih;
          F[L::IE] -= rf * nu * work + rf * R(ph.c_pd) * nu * heat;
        }
        const int fi = (iz * sy + iy) * sx + ix;
#pragma unroll
        for (int v = 0; v < NV; ++v) s_flux[v * B::NF + fi] = F[v];
      }
      __syncthreads();
      const R ih = R(1.0 / hd);
#pragma unroll
      for (int m = 0; m < B::CPT; ++m) {
        const int c = threadIdx.x + m * T::NT;
        const int lx = c % T::TX, ly = (c / T::TX) % T::TY, lz = c / (T::TX * T::TY);
        if (lx < ex && ly < ey && lz < ez) {
          const int f0 = (lz * sy + ly) * sx + lx;
          const int f1 = ((lz + fz) * sy + (ly + fy)) * sx + (lx + fx);
#pragma unroll
          for (int v = 0; v < NV; ++v)
            acc[m][v] -= (s_flux[v * B::NF + f1] - s_flux[v * B::NF + f0]) * ih;
        }
      }
      if (d != 2) __syncthreads();
    }

    // ---- 4. sources, stage combine, saturation adjustment, store ------------------------
    double rate_max = 0.0;
    const double tol = fmax(ph.satadj_tol, 32.0 * Ar<R>::eps);
#pragma unroll
    for (int m = 0; m < B::CPT; ++m) {
      const int c = threadIdx.x + m * T::NT;
      const int lx = c % T::TX, ly = (c / T::TX) % T::TY, lz = c / (T::TX * T::TY);
      if (lx < ex && ly < ey && lz < ez) {
        const int k = z0 + lz;
        const int bi = B::at(lx + 3, ly + B::HY, lz + 3);
        const R rho = s_prim[bi];
        acc[m][L::mom(2)] -= (rho - R(D.rho_bar[k])) * R(D.grav);
        const int f0 = (lz * T::TY + ly) * T::TX + lx;
        const int f1 = ((lz + 1) * T::TY + ly) * T::TX + lx;
        R mb = R(0), mt = R(0);
#pragma unroll
        for (int s = 0; s < L::IM0; ++s) {
          mb += s_flux[s * B::NF + f0];
          mt += s_flux[s * B::NF + f1];
        }
        acc[m][L::IE] -= R(D.grav) * R(0.5) * (mb + mt);
        const long long g = ((long long)k * ny + (y0 + ly)) * nx + (x0 + lx);
        R yo[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const R s1 = ys[m][v] + R(dt) * acc[m][v];
          if (a.stage == 0) {
            yo[v] = s1;
          } else {
            const R yn = Yn[v * ncell + g];
            yo[v] = a.stage == 1 ? R(0.75) * yn + R(0.25) * s1
                                 : yn * R(1.0 / 3.0) + R(2.0 / 3.0) * s1;
          }
        }
        if constexpr (L::MOIST) {
          if (ph.satadj) {
            const int it = satadj_cell<R, L>(ph, yo, D.e_ref[k], ph.satadj_max_iter, tol);
            if (it < 0)
              atomicOr(a.flags, (unsigned)kFlagNoConv);
            else
              atomicMax(a.max_sweeps, it);
          }
        }
        R rs = R(0);
#pragma unroll
        for (int s = 0; s < L::IM0; ++s) rs += yo[s];
        if (!(rs > R(0)) || !isfinite(double(yo[L::IE]))) atomicOr(a.flags, (unsigned)kFlagNonFinite);
#pragma unroll
        for (int v = 0; v < NV; ++v) Yo[v * ncell + g] = yo[v];
        if (a.stage == 2)
          rate_max = fmax(rate_max,
                          cell_rate<R, L>(ph, yo, D.e_ref[k], 1.0 / D.dx, 1.0 / D.dy, 1.0 / D.dz));
      }
    }
    if (a.stage == 2) {
      double bm = block_max(rate_max, s_red);
      if (threadIdx.x == 0) atomicMax(D.rate, (unsigned long long)__double_as_longlong(bm));
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// auxiliary kernels: CFL rate, budget, saturation adjustment over a domain
// ------------------------------------------------------------------------------------------
template <class R, class L>
__global__ void __launch_bounds__(256) rate_kernel(const StageArgs a, int dm, int buf) {
  __shared__ double red[32];
  const DomDev &D = a.doms[dm];
  const R *Y = reinterpret_cast<const R *>(D.buf[buf]);
  double r = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < D.ncell;
       c += (long long)gridDim.x * blockDim.x) {
    R y[L::NV];
#pragma unroll
    for (int v = 0; v < L::NV; ++v) y[v] = Y[v * D.ncell + c];
    const double er = D.e_ref[c / ((long long)D.nx * D.ny)];
    r = fmax(r, cell_rate<R, L>(a.ph, y, er, 1.0 / D.dx, 1.0 / D.dy, 1.0 / D.dz));
  }
  double bm = block_max(r, red);
  if (threadIdx.x == 0) atomicMax(D.rate, (unsigned long long)__double_as_longlong(bm));
}

// Per-block FP64 partial sums in a fixed order: nv field totals and sum(rho e + rho g z),
// all times the cell volume.
template <class R, class L>
__global__ void __launch_bounds__(256) budget_kernel(const StageArgs a, int dm, int buf,
                                                     double *partials) {
  constexpr int NO = L::NV + 1;
  __shared__ double red[NO][8];
  const DomDev &D = a.doms[dm];
  const R *Y = reinterpret_cast<const R *>(D.buf[buf]);
  const double vol = D.dx * (D.ny > 1 ? D.dy : 1.0) * D.dz;
  const long long plane = (long long)D.nx * D.ny;
  double s[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) s[o] = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < D.ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const long long k = c / plane;
    const double z = (double(k) + 0.5) * D.dz;
    const double er = D.e_ref[k];
    double rho = 0.0;
#pragma unroll
    for (int v = 0; v < L::NV; ++v) {
      double y = double(Y[v * D.ncell + c]);
      if (v == L::IE) y += er;
      s[v] += y;
      if (v < L::IM0) rho += y;
    }
    s[L::NV] += (double(Y[(long long)L::IE * D.ncell + c]) + er) + rho * D.grav * z;
  }
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    double v = s[o];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[o][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < NO) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    partials[(long long)blockIdx.x * NO + threadIdx.x] = t * vol;
  }
}

// Second pass of the budget: sums the per-block partials in block order (deterministic).
template <int Dummy = 0>
__global__ void budget_finish_kernel(const double *partials, int nblocks, int no, double *out) {
  for (int o = threadIdx.x; o < no; o += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[(long long)b * no + o];
    out[o] = t;
  }
}

template <class R, class L>
__global__ void __launch_bounds__(256) satadj_kernel(const StageArgs a, int dm, int buf) {
  const DomDev &D = a.doms[dm];
  R *Y = reinterpret_cast<R *>(D.buf[buf]);
  const double tol = fmax(a.ph.satadj_tol, 32.0 * Ar<R>::eps);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < D.ncell;
       c += (long long)gridDim.x * blockDim.x) {
    R y[L::NV];
#pragma unroll
    for (int v = 0; v < L::NV; ++v) y[v] = Y[v * D.ncell + c];
    const double er = D.e_ref[c / ((long long)D.nx * D.ny)];
    const int it = satadj_cell<R, L>(a.ph, y, er, a.ph.satadj_max_iter, tol);
    if (it < 0)
      atomicOr(a.flags, (unsigned)kFlagNoConv);
    else
      atomicMax(a.max_sweeps, it);
#pragma unroll
    for (int v = 0; v < L::NV; ++v) Y[v * D.ncell + c] = y[v];
  }
}

// ------------------------------------------------------------------------------------------
// host launchers of one configuration
// ------------------------------------------------------------------------------------------
template <class R, class L, bool VISC>
struct Family {
  using S = StageSmem<R, L, VISC>;
  static cudaError_t prepare() {
    return cudaFuncSetAttribute(stage_kernel<R, L, VISC>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::total));
  }
  static cudaError_t stage(const StageArgs &a, int grid, cudaStream_t s) {
    stage_kernel<R, L, VISC><<<grid, Tile<L::D3>::NT, S::total, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t rate(const StageArgs &a, int dm, int buf, cudaStream_t s) {
    rate_kernel<R, L><<<304, 256, 0, s>>>(a, dm, buf);
    return cudaGetLastError();
  }
  static cudaError_t budget(const StageArgs &a, int dm, int buf, double *partials, int nblocks,
                            double *out, cudaStream_t s) {
    budget_kernel<R, L><<<nblocks, 256, 0, s>>>(a, dm, buf, partials);
    budget_finish_kernel<><<<1, 32, 0, s>>>(partials, nblocks, L::NV + 1, out);
    return cudaGetLastError();
  }
  static cudaError_t satadj(const StageArgs &a, int dm, int buf, cudaStream_t s) {
    satadj_kernel<R, L><<<608, 256, 0, s>>>(a, dm, buf);
    return cudaGetLastError();
  }
  static KernelSet set() {
    KernelSet k;
    k.tile[0] = Tile<L::D3>::TX;
    k.tile[1] = Tile<L::D3>::TY;
    k.tile[2] = Tile<L::D3>::TZ;
    k.threads = Tile<L::D3>::NT;
    k.smem_stage = S::total;
    k.stage = &stage;
    k.rate = &rate;
    k.budget = &budget;
    k.satadj = &satadj;
    k.prepare = &prepare;
    return k;
  }
};

}  // namespace snap
