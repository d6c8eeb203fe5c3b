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

#include <type_traits>

#include "snap_internal.h"

namespace snap {

// ------------------------------------------------------------------------------------------
// arithmetic helpers per type
// ------------------------------------------------------------------------------------------
template <class R>
struct Ar;
template <>
struct Ar<float> {
  // a b + c rounded once, whatever the compiler would contract: the same source then rounds
  // the same way in every kernel it is inlined into
  static __device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  // approximate reciprocal: the special-function unit's rcp.approx.ftz.f32 alone (~1 ulp; a
  // subnormal argument or result flushes to zero, which no reciprocal of the scheme meets:
  // densities, eps + beta >= 1e-6 and the weight sums are normal numbers)
  static __device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  // a / b as a times the approximate reciprocal (~2 ulp; b a normal number, as every divisor
  // of the scheme is: densities, heat capacities, mixing factors, sound-speed sums)
  static __device__ __forceinline__ float div(float a, float b) { return a * rcp(b); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float exp_(float x) { return expf(x); }
  static __device__ __forceinline__ float log_(float x) { return logf(x); }
  static __device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
  static __device__ __forceinline__ float pow_(float x, float y) { return powf(x, y); }
  // exp2(y log2 x) on the special-function unit: a few ulp when |y log2 x| is small, as for
  // the Exner function (p / 1e5)^(R/c_p) near 1 bar
  static __device__ __forceinline__ float pow_small(float x, float y) { return __powf(x, y); }
  // sqrt of a positive argument as x * rsqrt(x) (~2 ulp): sound speeds
  static __device__ __forceinline__ float sqrt_pos(float x) { return x * rsqrtf(x); }
  // sound speed sqrt(gp / rho) as gp / sqrt(gp rho): one reciprocal square root, no division
  static __device__ __forceinline__ float sound_speed(float gp, float rho) {
    return gp * rsqrtf(gp * rho);
  }
  static constexpr double eps = 1.1920928955078125e-07;
};
template <>
struct Ar<double> {
  static __device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
  // Reciprocal by Newton-Raphson iteration y <- y + y (1 - x y), which squares the relative
  // error at each step, from the hardware's approximate FP64 reciprocal (rcp.approx.ftz.f64,
  // about 1e-6): two steps reach the last bit (equal to the IEEE quotient on a million random
  // normal arguments across the exponent range). Zero, infinite, NaN and subnormal x give NaN.
  static __device__ __forceinline__ double rcp(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
  }
  // a / b within about an ulp (the product rounds once more than the quotient)
  static __device__ __forceinline__ double div(double a, double b) { return a * rcp(b); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
  static __device__ __forceinline__ double log_(double x) { return log(x); }
  static __device__ __forceinline__ double log1p_(double x) { return log1p(x); }
  static __device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }
  // exp(y log x): the error of the product y log x, |y log x| eps, adds to exp's and log's own
  // few ulp, far below 1e-15 for the Exner function between 0.1 and 10 bar; pow's extended-
  // precision logarithm costs about twice as many FP64 operations
  static __device__ __forceinline__ double pow_small(double x, double y) { return exp(y * log(x)); }
  static __device__ __forceinline__ double sqrt_pos(double x) { return sqrt(x); }
  static __device__ __forceinline__ double sound_speed(double gp, double rho) {
    return gp * rsqrt(gp * rho);
  }
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

template <class R>
__device__ __forceinline__ const CstT<R> &cst(const StageArgs &a);
template <>
__device__ __forceinline__ const CstT<float> &cst<float>(const StageArgs &a) { return a.cf; }
template <>
__device__ __forceinline__ const CstT<double> &cst<double>(const StageArgs &a) { return a.cd; }

// Tile shape: TX x TY x TZ owned cells per CTA of NT threads (TY = 1 in the x-z plane).
// MINB: CTAs per SM the kernel is compiled for (second __launch_bounds__ argument), which caps
// its registers; 0 leaves the register count to the compiler.
template <int TX_, int TY_, int TZ_, int NT_ = 256, int MINB_ = 0>
struct TileT {
  static constexpr int TX = TX_, TY = TY_, TZ = TZ_, NT = NT_, MINB = MINB_;
};

template <class T, bool D3>
struct Box {
  static constexpr int HX = 3, HY = D3 ? 3 : 0, HZ = 3;
  static constexpr int BX = T::TX + 6, BY = T::TY + 2 * HY, BZ = T::TZ + 6;
  static constexpr int NBOX = BX * BY * BZ;
  static constexpr int NFX = (T::TX + 1) * T::TY * T::TZ;
  static constexpr int NFY = D3 ? T::TX * (T::TY + 1) * T::TZ : 0;
  static constexpr int NFZ = T::TX * T::TY * (T::TZ + 1);
  static constexpr int NF = NFX > NFZ ? (NFX > NFY ? NFX : NFY) : (NFZ > NFY ? NFZ : NFY);
  static constexpr int NCELL = T::TX * T::TY * T::TZ;
  static constexpr int CPT = (NCELL + T::NT - 1) / T::NT;  // owned cells per thread
  static __host__ __device__ __forceinline__ int at(int bx, int by, int bz) {
    return (bz * BY + by) * BX + bx;
  }
  // Storage of the primitives in shared memory. x-z: the whole box. 3-D: only the cross the
  // stencils use -- x-lines through the owned y, z range with both x halos (contiguous, so
  // x stencils have unit stride), then the y halos of the owned x, z range, then the z halos
  // of the owned x, y range -- about half the box, which lets a third CTA fit on an SM.
  // Ragged tiles put their far halos inside the owned index range; the fill and the reads use
  // the same map, so a location is never claimed twice.
  static constexpr int NXB = BX * T::TY * T::TZ;
  static constexpr int NYH = D3 ? T::TX * 6 * T::TZ : 0;
  static constexpr int NZH = T::TX * T::TY * 6;
  static constexpr int NSTORE = D3 ? NXB + NYH + NZH : NBOX;
  static __host__ __device__ __forceinline__ int idx(int bx, int by, int bz) {
    if constexpr (!D3) {
      return at(bx, by, bz);
    } else {
      const int oy = by - 3, oz = bz - 3;
      if ((unsigned)oy < (unsigned)T::TY && (unsigned)oz < (unsigned)T::TZ)
        return (oz * T::TY + oy) * BX + bx;
      if ((unsigned)oz < (unsigned)T::TZ)  // y halo: by in 0..2 or TY+3..TY+5
        return NXB + (oz * 6 + (by < 3 ? by : by - T::TY)) * T::TX + (bx - 3);
      return NXB + NYH + ((bz < 3 ? bz : bz - T::TZ) * T::TY + oy) * T::TX + (bx - 3);
    }
  }
  // idx for a location whose z (idx_y) or y (idx_z) lies in the owned range, as along a y or z
  // reconstruction window: one range test instead of two
  static __host__ __device__ __forceinline__ int idx_y(int bx, int by, int bz) {
    const int oy = by - 3, oz = bz - 3;
    if ((unsigned)oy < (unsigned)T::TY) return (oz * T::TY + oy) * BX + bx;
    return NXB + (oz * 6 + (by < 3 ? by : by - T::TY)) * T::TX + (bx - 3);
  }
  static __host__ __device__ __forceinline__ int idx_z(int bx, int by, int bz) {
    const int oy = by - 3, oz = bz - 3;
    if ((unsigned)oz < (unsigned)T::TZ) return (oz * T::TY + oy) * BX + bx;
    return NXB + NYH + ((bz < 3 ? bz : bz - T::TZ) * T::TY + oy) * T::TX + (bx - 3);
  }
};

// Shared-memory arrays of NV fields per location (primitives, face states, fluxes) keep the
// fields of one location together in 16-byte groups (4 floats or 2 doubles), then, for the
// fields left over, an 8-byte pair (floats) and a single field: 11 FP32 fields as 4 + 4 + 2
// + 1, 7 as 4 + 2 + 1, 4 as one group. Each group of an N-location array is a plane of
// N x (group width) values at element N x (its first field), so one vector access moves the
// group of a location: a window point, face state or flux of the four dry fields is one
// 16-byte access instead of four.
template <class R, int NV>
struct SV {
  static constexpr int W = sizeof(R) == 4 ? 4 : 2;       // fields of a 16-byte group
  static constexpr int NF = NV / W;                       // full groups
  static constexpr int T2 = (sizeof(R) == 4 && NV % W >= 2) ? 1 : 0;  // a pair after them
  static constexpr int T1 = (NV % W) % 2;                 // a single last field
  static constexpr int P2 = NF * W;                       // first field of the pair
  static constexpr int P1 = NF * W + 2 * T2;              // the single field
  static_assert(P2 * sizeof(R) % 16 == 0, "the pair's plane must start on a 16-byte boundary");
  static __host__ __device__ __forceinline__ int at(int v, int i, int N) {
    if (v < P2) return ((v / W) * N + i) * W + v % W;
    if (v < P1) return P2 * N + i * 2 + (v - P2);
    return P1 * N + i;
  }
  template <class Vec>
  static __device__ __forceinline__ void ld(const R *p, R *out) {
    const Vec t = *reinterpret_cast<const Vec *>(p);
    const R *e = reinterpret_cast<const R *>(&t);
#pragma unroll
    for (int j = 0; j < int(sizeof(Vec) / sizeof(R)); ++j) out[j] = e[j];
  }
  template <class Vec>
  static __device__ __forceinline__ void st(R *p, const R *in) {
    Vec t;
    R *e = reinterpret_cast<R *>(&t);
#pragma unroll
    for (int j = 0; j < int(sizeof(Vec) / sizeof(R)); ++j) e[j] = in[j];
    *reinterpret_cast<Vec *>(p) = t;
  }
  using V16 = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
  // the fields [first, first + width) of group g of location i (g < NF: a 16-byte group;
  // g == NF: the pair, or the single field)
  static __device__ __forceinline__ void load_group(const R *base, int g, int i, int N, R *out) {
    if (g < NF) {
      ld<V16>(base + (g * N + i) * W, out);
    } else if (T2 && g == NF) {
      ld<float2>(base + P2 * N + i * 2, out);
    } else {
      out[0] = base[P1 * N + i];
    }
  }
  static __device__ __forceinline__ void load(const R *base, int i, int N, R *out) {
#pragma unroll
    for (int g = 0; g < NF; ++g) ld<V16>(base + (g * N + i) * W, out + g * W);
    if constexpr (T2) ld<float2>(base + P2 * N + i * 2, out + P2);
    if constexpr (T1) out[P1] = base[P1 * N + i];
  }
  static __device__ __forceinline__ void store(R *base, int i, int N, const R *in) {
#pragma unroll
    for (int g = 0; g < NF; ++g) st<V16>(base + (g * N + i) * W, in + g * W);
    if constexpr (T2) st<float2>(base + P2 * N + i * 2, in + P2);
    if constexpr (T1) base[P1 * N + i] = in[P1];
  }
};

// Per-level reference values in the kernel's type: FP32 kernels read FP32 copies, FP64
// kernels the FP64 originals.
template <class R>
struct Prof;
template <>
struct Prof<float> {
  static __device__ __forceinline__ float pc(const DomDev &D, int k) { return D.pc_f[k]; }
  static __device__ __forceinline__ float pf(const DomDev &D, int k) { return D.pf_f[k]; }
  static __device__ __forceinline__ float er(const DomDev &D, int k) { return D.er_f[k]; }
  // rho - rho_bar_k from the conserved densities y: dry air minus the FP32 head of rho_bar is
  // exact (the two are within a factor of 2), the tracers are added to that small difference,
  // and the FP32 tail of rho_bar (rb_lo) last
  template <class L>
  static __device__ __forceinline__ float drho(const DomDev &D, int k, const float *y) {
    float r = y[0] - D.rb_hi[k];
#pragma unroll
    for (int s = 1; s < L::IM0; ++s) r += y[s];
    return r - D.rb_lo[k];
  }
  static __device__ __forceinline__ float grav(const DomDev &D) { return D.fgrav; }
  static __device__ __forceinline__ float ih(const DomDev &D, int d) {
    return d == 0 ? D.fidx : (d == 1 ? D.fidy : D.fidz);
  }
};
template <>
struct Prof<double> {
  static __device__ __forceinline__ double pc(const DomDev &D, int k) { return D.p_cell[k]; }
  static __device__ __forceinline__ double pf(const DomDev &D, int k) { return D.p_face[k]; }
  static __device__ __forceinline__ double er(const DomDev &D, int k) { return D.e_ref[k]; }
  template <class L>
  static __device__ __forceinline__ double drho(const DomDev &D, int k, const double *y) {
    double r = y[0];
#pragma unroll
    for (int s = 1; s < L::IM0; ++s) r += y[s];
    return r - D.rho_bar[k];
  }
  static __device__ __forceinline__ double grav(const DomDev &D) { return D.grav; }
  static __device__ __forceinline__ double ih(const DomDev &D, int d) {
    return d == 0 ? D.idx : (d == 1 ? D.idy : D.idz);
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
__device__ __forceinline__ void cons_to_prim(const Phys &ph, const CstT<R> &C, const DomDev &D,
                                             int k, const R *y, R *x, R &p_tot, R &T_out) {
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
    const R pp = C.gm1 * (y[L::IE] - K);
    x[L::IE] = pp;
    const R p = pp + Prof<R>::pc(D, k);
    p_tot = p;
    T_out = p * ir * C.iR_d;
  } else if constexpr (sizeof(R) == 8) {
    // FP64 kernels: U = rho e - K - A, T = U / C_v, p = R_m T directly
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
    double U = (double(y[L::IE]) + D.e_ref[k]) - double(K) - A;
    double T = Ar<double>::div(U, Cv);
    double p = Rm * T;
    p_tot = R(p);
    T_out = R(T);
    x[L::IE] = R(p - D.p_cell[k]);
  } else {
    // FP32 kernels: the same p, rewritten so that only small numbers cancel. With the sums
    // over densities C = rho_d + sum sigma_v,i rho_i + sum sigma_ij rho_ij and
    // G = rho_d + sum rho_i / eps_i, p = R_d G T = (gamma_d - 1) (1 + delta) U with
    // delta = (G - C) / C, a sum over tracers only. Since e_ref = pbar / (gamma_d - 1),
    //   p - pbar = (gamma_d - 1) [ (y_E - K - A) + delta (y_E + e_ref - K - A) ],
    // accurate to ~1e-3 Pa at 1e6..1e7 Pa without FP64 (y_E = rho e - e_ref is stored).
    R A = R(0), Cv = y[0], dG = R(0);
#pragma unroll
    for (int i = 0; i < L::NVAP; ++i) {
      Cv += C.sig_v[i] * y[1 + i];
      dG += (C.inv_eps[i] - C.sig_v[i]) * y[1 + i];
#pragma unroll
      for (int j = 0; j < L::NCOND; ++j) {
        Cv += C.sig_c[i][j] * y[L::cond(i, j)];
        dG -= C.sig_c[i][j] * y[L::cond(i, j)];
        A += C.mu[i][j] * y[L::cond(i, j)];
      }
    }
    const R delta = dG * Ar<R>::rcp(Cv);
    const R small = y[L::IE] - K - A;
    const R pp = C.gm1 * (small + delta * (small + Prof<R>::er(D, k)));
    x[L::IE] = pp;
    p_tot = pp + Prof<R>::pc(D, k);
    T_out = R(0);  // not needed by the moist kernels
  }
}

// mixing factors of App. B: num = 1 + sum q_i (sigma_vi - 1) + sum q_ij (sigma_ij - 1),
// den = 1 + sum q_i (1/eps_i - 1) - sum q_ij
template <class R, class L>
__device__ __forceinline__ void mix_factors(const CstT<R> &C, const R *x, R &num, R &den) {
  num = R(1);
  den = R(1);
#pragma unroll
  for (int i = 0; i < L::NVAP; ++i) {
    num += x[1 + i] * C.sigv_m1[i];
    den += x[1 + i] * C.ieps_m1[i];
#pragma unroll
    for (int j = 0; j < L::NCOND; ++j) {
      num += x[L::cond(i, j)] * C.sigc_m1[i][j];
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
__device__ __forceinline__ void lmars(const CstT<R> &C, const R *XL, const R *XR, int dir,
                                      R pref, R *F) {
  const int mn = L::mom(dir);
  R numL, denL, numR, denR;
  mix_factors<R, L>(C, XL, numL, denL);
  mix_factors<R, L>(C, XR, numR, denR);
  const R gm1 = C.gm1;
  R pL = pref + XL[L::IE], pR = pref + XR[L::IE];
  R gamL, gamR;
  if constexpr (L::NVAP == 0) {
    gamL = gamR = C.gamma_d;
  } else {
    gamL = R(1) + gm1 * Ar<R>::div(denL, numL);
    gamR = R(1) + gm1 * Ar<R>::div(denR, numR);
  }
  R cL = Ar<R>::sound_speed(gamL * pL, XL[0]);
  R cR = Ar<R>::sound_speed(gamR * pR, XR[0]);
  R rhoc = R(0.5) * (XL[0] + XR[0]) * R(0.5) * (cL + cR);
  R uL = XL[mn], uR = XR[mn];
  R ps = R(0.5) * (XL[L::IE] + XR[L::IE]) - R(0.5) * rhoc * (uR - uL);
  R us = R(0.5) * (uL + uR) - Ar<R>::div(XR[L::IE] - XL[L::IE], R(2) * rhoc);
  const bool left = us > R(0);
  R XS[L::NV];
#pragma unroll
  for (int v = 0; v < L::NV; ++v) XS[v] = left ? XL[v] : XR[v];
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
    for (int j = 0; j < L::NCOND; ++j) A += C.mu[i][j] * XS[L::cond(i, j)];
  A *= rhoS;
  R rhoe;
  if constexpr (L::NVAP == 0)
    rhoe = pS * C.igm1 + K;
  else
    rhoe = Ar<R>::div(numS, denS) * pS * C.igm1 + K + A;
  F[L::IE] = us * (rhoe + pS);
}

// ------------------------------------------------------------------------------------------
// App. D saturation adjustment of one cell (isochoric). Each sweep visits the vapours in
// order: projected molar transfer of Eq. dxf with the isochoric alpha, limited to keep both
// phases non-negative, then T and p follow from the conserved energy and the equation of
// state. Returns the sweep count, or -1 without convergence.
// ------------------------------------------------------------------------------------------
// An FP64 quotient a / b for the kernels of type R: FP64 kernels to about an ulp (two
// Newton-Raphson steps, Ar<double>::div); FP32 kernels, whose states hold 7 digits, to ~1e-12
// (one step from the approximate FP64 reciprocal)
template <class R>
__device__ __forceinline__ double quot64(double a, double b) {
  if constexpr (sizeof(R) == 8) {
    return Ar<double>::div(a, b);
  } else {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
    r = fma(r, fma(-b, r, 1.0), r);
    return a * r;
  }
}

template <class R, class L>
__device__ __forceinline__ void cell_Tp(const Phys &ph, const R *y, double eref, double &T,
                                        double &p, double *Cv_out = nullptr,
                                        double *Rm_out = nullptr) {
  double Cv = y[0], Rm = y[0];
#pragma unroll
  for (int i = 0; i < L::NVAP; ++i) {
    Cv += ph.sig_v[i] * double(y[1 + i]);
    Rm += ph.inv_eps[i] * double(y[1 + i]);
#pragma unroll
    for (int j = 0; j < L::NCOND; ++j) Cv += ph.sig_c[i][j] * double(y[L::cond(i, j)]);
  }
  double U;
  if constexpr (sizeof(R) == 4) {
    // FP32 states: the kinetic and latent energies (about 1e-4 of U) and the density they
    // need are summed in FP32 -- their rounding is ~1e-10 of U, far below what the state holds
    // -- and the inversion itself (U, the heat capacity, T, p) stays in FP64 with a quotient
    // good to ~1e-12 (one Newton-Raphson step from the approximate FP64 reciprocal); an FP64
    // instruction costs ~32 FP32 ones on this part
    float rho = y[0], K2 = 0.0f, A = 0.0f;
#pragma unroll
    for (int s = 1; s < L::IM0; ++s) rho += y[s];
#pragma unroll
    for (int m = 0; m < L::NMOM; ++m) K2 = fmaf(y[L::IM0 + m], y[L::IM0 + m], K2);
#pragma unroll
    for (int i = 0; i < L::NVAP; ++i)
#pragma unroll
      for (int j = 0; j < L::NCOND; ++j) A = fmaf(float(ph.mu[i][j]), y[L::cond(i, j)], A);
    U = (double(y[L::IE]) + eref) - double(0.5f * K2 * Ar<float>::rcp(rho) + A);
    T = quot64<R>(U, Cv * ph.c_vd);
  } else {
    double rho = 0.0, K2 = 0.0, A = 0.0;
#pragma unroll
    for (int s = 0; s < L::IM0; ++s) rho += double(y[s]);
#pragma unroll
    for (int m = 0; m < L::NMOM; ++m) K2 += double(y[L::IM0 + m]) * double(y[L::IM0 + m]);
#pragma unroll
    for (int i = 0; i < L::NVAP; ++i)
#pragma unroll
      for (int j = 0; j < L::NCOND; ++j) A += ph.mu[i][j] * double(y[L::cond(i, j)]);
    // quotients by the Newton-Raphson reciprocal of Ar<double> (within about an ulp of the
    // IEEE quotient, a third of its FP64 instructions)
    U = (double(y[L::IE]) + eref) - 0.5 * K2 * Ar<double>::rcp(rho) - A;
    T = Ar<double>::div(U, Cv * ph.c_vd);
  }
  p = Rm * ph.R_d * T;
  if (Cv_out) *Cv_out = Cv * ph.c_vd;  // heat capacity at constant volume, J/(m^3 K)
  if (Rm_out) *Rm_out = Rm;            // sum of the gas densities / molar-mass ratios
}

template <class R, class L>
__device__ int satadj_cell(const Phys &ph, const CstT<R> &C, R *y, double eref, R eref_r,
                           int max_iter) {
  if constexpr (!L::MOIST) {
    return 0;
  } else {
    if constexpr (sizeof(R) == 4) {
      // FP32 screen: App. D's projected transfer is negative exactly when the vapour's partial
      // pressure is below saturation, and is then limited to the cloud present. A cloud-free
      // vapour that is subsaturated by more than the FP32 error of this estimate (1e-3
      // relative margin) therefore needs no transfer; if all vapours qualify the cell is left
      // unchanged, as the FP64 iteration would leave it, after one sweep.
      R rho = y[0], K2 = R(0), A = R(0), Cv = y[0];
      bool clear = true;
#pragma unroll
      for (int s = 1; s < L::IM0; ++s) rho += y[s];
#pragma unroll
      for (int m = 0; m < L::NMOM; ++m) K2 += y[L::IM0 + m] * y[L::IM0 + m];
#pragma unroll
      for (int i = 0; i < L::NVAP; ++i) {
        Cv += C.sig_v[i] * y[1 + i];
        if (y[L::cond(i, 0)] != R(0)) clear = false;
#pragma unroll
        for (int j = 0; j < L::NCOND; ++j) {
          Cv += C.sig_c[i][j] * y[L::cond(i, j)];
          A += C.mu[i][j] * y[L::cond(i, j)];
        }
      }
      if (clear) {
        // T = U / (c_vd C) with c_vd = R_d / (gamma_d - 1)
        const R T = ((y[L::IE] + eref_r) - R(0.5) * K2 * Ar<R>::rcp(rho) - A) *
                    Ar<R>::rcp(Cv) * C.gm1 * C.iR_d;
#pragma unroll
        for (int i = 0; i < L::NVAP; ++i) {
          const R t = T * C.inv_Tref[i];
          const R ps = C.pref[i] * Ar<R>::exp_(C.beta[i] * (R(1) - Ar<R>::rcp(t)) -
                                               C.delta[i] * Ar<R>::log_(t));
          const R pv = y[1 + i] * C.R_d * C.inv_eps[i] * T;  // rho_i R_i T
          if (!(pv < R(0.999) * ps)) clear = false;
        }
        if (clear) return 1;
      }
    }
    // T and p from the conserved energy once, in FP64 (Eq. energy, App. B); after each
    // transfer they are carried forward in FP64 by the change of the two densities: rho e
    // and the momenta are fixed, so C_v T + A is, and T' = T - (dA + T dC) / (C_v + dC),
    // p' = R_d (R_m + dR_m) T' -- exact algebra, no inversion per sweep
    double Td = 0.0, pd = 0.0, Cvd = 0.0, Rmd = 0.0;
    cell_Tp<R, L>(ph, y, eref, Td, pd, &Cvd, &Rmd);
    for (int sweep = 1; sweep <= max_iter; ++sweep) {
      bool conv = true;
#pragma unroll
      for (int i = 0; i < L::NVAP; ++i) {
        R T = R(Td), p = R(pd);
        const R dTr = R(Td - ph.Tref[i]);  // T - T^r kept accurate: s(T) is steep
        R N = y[0], gas = y[0], heat = R(0);
#pragma unroll
        for (int k = 0; k < L::NVAP; ++k) {
          R tot = y[1 + k];
#pragma unroll
          for (int j = 0; j < L::NCOND; ++j) tot += y[L::cond(k, j)];
          N += tot * C.inv_eps[k];
          gas += y[1 + k] * C.inv_eps[k];
          heat += tot * C.inv_eps[k] * C.sighat_m1[k];
        }
        const R iN = Ar<R>::rcp(N);
        heat *= iN;
        R qv = y[1 + i] * C.inv_eps[i] * iN;
        R qc = y[L::cond(i, 0)] * C.inv_eps[i] * iN;
        R gsum = gas * iN - qv;
        R t = T * C.inv_Tref[i];
        // p* = p^r exp[beta (1 - 1/t) - delta ln t] with 1 - 1/t = (T - T^r) / T
        const R arg = C.beta[i] * dTr * Ar<R>::rcp(T) - C.delta[i] * Ar<R>::log_(t);
        R ps = C.pref[i] * Ar<R>::exp_(arg);
        // the arithmetic type holds p* only to ~(|arg| + 2) eps relative (the exponent's own
        // rounding), so the transfer cannot settle below that: the stop test allows 4 times it
        const R tol = fmax(C.satadj_tol, R(4) * (fabs(arg) + R(2)) * R(Ar<R>::eps));
        R s = Ar<R>::div(ps, p);
        R dq;
        if (s >= R(1)) {
          dq = -qc;
        } else {
          R bt = C.beta[i] * Ar<R>::rcp(t) - C.delta[i];
          R alpha = C.gm1 * (bt - R(1)) * Ar<R>::rcp(R(1) + heat);
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
          drho = dq * C.eps[i] * N;
        }
        if (drho != R(0)) {
          const R yv = y[1 + i], yc = y[L::cond(i, 0)];
          y[1 + i] -= drho;
          y[L::cond(i, 0)] += drho;
          // the changes as stored (after rounding to the state's type)
          if constexpr (sizeof(R) == 4) {
            // FP32 states: the increments in FP32 (good to ~1e-7 of themselves, ~1e-10 of T),
            // accumulated into the FP64 T, heat capacity and gas sum
            const R dv = y[1 + i] - yv, dc = y[L::cond(i, 0)] - yc;
            const R dC = (C.sig_v[i] * dv + C.sig_c[i][0] * dc) * C.c_vd;
            const R dT = (C.mu[i][0] * dc + R(Td) * dC) * Ar<R>::rcp(R(Cvd) + dC);
            Td -= double(dT);
            Cvd += double(dC);
            Rmd += double(C.inv_eps[i] * dv);
          } else {
            const double dv = double(y[1 + i]) - double(yv);
            const double dc = double(y[L::cond(i, 0)]) - double(yc);
            const double dC = (ph.sig_v[i] * dv + ph.sig_c[i][0] * dc) * ph.c_vd;
            Td -= quot64<R>(ph.mu[i][0] * dc + Td * dC, Cvd + dC);
            Cvd += dC;
            Rmd += ph.inv_eps[i] * dv;
          }
          pd = Rmd * ph.R_d * Td;
        }
        if (fabs(dq) > tol * (qv + qc)) conv = false;
      }
      if (conv) return sweep;
    }
    return -1;
  }
}

// The cell a ghost at index g (at most n beyond either edge of an axis of n >= 3 cells)
// copies: wrapped on a periodic side (one add or subtract, no integer division), mirrored at a
// wall (flip set).
__device__ __forceinline__ int map_index(int g, int n, int bc_lo, int bc_hi, bool &flip) {
  flip = false;
  if (g < 0) {
    if (bc_lo == 1) return g + n;
    flip = true;
    return -1 - g;
  }
  if (g >= n) {
    if (bc_hi == 1) return g - n;
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
// Sedimentation (Sec. 2, Eq. d3 and the momentum and energy equations with terminal
// velocities): condensate (i,j) falling at w^t_j carries through a z face the extra fluxes
// w^t rho_ij (mass), w^t rho_ij u_m (momentum) and w^t rho_ij e_ij with e_ij = c_ij T +
// |u|^2/2 + mu_ij (energy), from the reconstructed state on the side it comes from (above
// when w^t < 0). The frictional heating of the energy equation enters through the total
// mass flux of the gravity-energy source.
// ------------------------------------------------------------------------------------------
template <class R, class L>
__device__ __forceinline__ void sediment_flux(const CstT<R> &C, const R *XL, const R *XR,
                                              R pref, R *F) {
#pragma unroll
  for (int j = 0; j < L::NCOND; ++j) {
    const R wt = C.w_term[j];
    if (wt == R(0)) continue;
    const bool up = wt < R(0);  // falling: the state above the face
    R XS[L::NV];
#pragma unroll
    for (int v = 0; v < L::NV; ++v) XS[v] = up ? XR[v] : XL[v];
    R num, den, u2 = R(0);
    mix_factors<R, L>(C, XS, num, den);
    const R T = (pref + XS[L::IE]) * Ar<R>::rcp(XS[0] * C.R_d * den);
#pragma unroll
    for (int m = 0; m < L::NMOM; ++m) u2 += XS[L::IM0 + m] * XS[L::IM0 + m];
#pragma unroll
    for (int i = 0; i < L::NVAP; ++i) {
      const int c = L::cond(i, j);
      const R ms = wt * XS[0] * XS[c];
      F[c] += ms;
#pragma unroll
      for (int m = 0; m < L::NMOM; ++m) F[L::IM0 + m] += ms * XS[L::IM0 + m];
      F[L::IE] += ms * (C.sig_c[i][j] * C.c_vd * T + R(0.5) * u2 + C.mu[i][j]);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Kessler scheme (Sec. 3) on one cell, backward Euler over dt (Eq. x_n+1), in densities: for
// vapour i with cloud (i,0) and precipitation (i,1), s = rho_v - rho*(T), rho* = p*/(R_i T),
//   saturated (s > 0):  F_v = -k1 s, F_c = k1 s - k3 rho_c rho_r / rho - k2 rho_c,
//                       F_r = k3 rho_c rho_r / rho + k2 rho_c
//   otherwise:          F_v = -k4 rho_r s / rho, F_c = -k3 rho_c rho_r / rho - k2 rho_c,
//                       F_r = k4 rho_r s / rho + k3 rho_c rho_r / rho + k2 rho_c
// (the mass-mixing-ratio rates of Sec. 3 times the fixed total density rho). Newton on
// G = F(y) - (y - y_n)/dt in (rho_v, rho_c) with rho_r = total - rho_v - rho_c, the full
// Jacobian (rho* varies with T, which the reactions change at fixed rho e: dT/drho_k =
// -(mu_k + c_k T)/C_v), one form of the rates at a time: the form of the initial state, then
// the other if the result lies on the wrong side of saturation, else the saturated form.
// T is inverted from the energy in FP64. Returns the largest iteration count or -1.
// ------------------------------------------------------------------------------------------
template <class R, class L>
__device__ __forceinline__ void kessler_eval(const Phys &ph, const CstT<R> &C, const R *y,
                                             double T0, R Cv0, int i, R rho, const R *yn, R dt,
                                             bool sat, R G[2], R A[2][2], R &s_out,
                                             R &tol_out) {
  const int vi = 1 + i, ci = L::cond(i, 0), ri = L::cond(i, 1);
  // T from T0, the FP64 temperature of the densities yn this vapour started from, and the
  // phase changes since: rho e and the momenta are fixed, so C_v T + A is (Sec. 2), and
  // T = T0 - (sum_k mu_k d_k + T0 sum_k c_k d_k) / (C_v0 + sum_k c_k d_k) over the vapour,
  // cloud and precipitation changes d_k (the vapour's mu is zero) -- no FP64 inversion per
  // Newton iteration
  const R dv = y[vi] - yn[0], dc = y[ci] - yn[1], dr = y[ri] - yn[2];
  const R dC = (C.sig_v[i] * dv + C.sig_c[i][0] * dc + C.sig_c[i][1] * dr) * C.c_vd;
  const R dA = C.mu[i][0] * dc + C.mu[i][1] * dr;
  const R incr = -(dA + R(T0) * dC) * Ar<R>::rcp(Cv0 + dC);
  const R T = R(T0) + incr, iT = Ar<R>::rcp(T), t = T * C.inv_Tref[i], it = Ar<R>::rcp(t);
  // T - T^r kept accurate (T0 - T^r from the FP64 temperature): rho*(T) is steep,
  // d ln rho*/d ln T ~ beta / t ~ 20 near water's triple point, so T rounded to FP32 alone
  // would put ~1e-6 relative noise into s = rho_v - rho* -- the size of the FP32 Newton stop
  // tolerance
  const R dTr = R(T0 - ph.Tref[i]) + incr;
  const R arg = C.beta[i] * dTr * iT - C.delta[i] * Ar<R>::log1p_(dTr * C.inv_Tref[i]);
  const R rs = C.pref[i] * Ar<R>::exp_(arg) * C.eps[i] * C.iR_d * iT;  // p* / (R_i T)
  // rho* is held only to ~(|arg| + 2) eps relative: the Newton stop test allows 4 times it
  tol_out = fmax(C.kessler_tol, R(4) * (fabs(arg) + R(2)) * R(Ar<R>::eps));
  const R drs = rs * ((C.beta[i] * it - C.delta[i]) - R(1)) * iT;
  R Cv = y[0];
#pragma unroll
  for (int a = 0; a < L::NVAP; ++a) {
    Cv += C.sig_v[a] * y[1 + a];
#pragma unroll
    for (int b = 0; b < L::NCOND; ++b) Cv += C.sig_c[a][b] * y[L::cond(a, b)];
  }
  const R iCv = Ar<R>::rcp(Cv * C.c_vd);
  // d s / d rho_k for k = vapour, cloud, precipitation (dT/drho_k at fixed energy)
  const R ds[3] = {R(1) + drs * (C.sig_v[i] * C.c_vd * T) * iCv,
                   drs * (C.mu[i][0] + C.sig_c[i][0] * C.c_vd * T) * iCv,
                   drs * (C.mu[i][1] + C.sig_c[i][1] * C.c_vd * T) * iCv};
  const R k1 = C.kk[0], k2 = C.kk[1], k3 = C.kk[2], k4 = C.kk[3], ir = Ar<R>::rcp(rho);
  const R yv = y[vi], yc = y[ci], yr = y[ri], s = yv - rs;
  s_out = s;
  // Equations: the vapour rate G_v and the vapour-plus-cloud rate G_v + G_c, in which the
  // stiff condensation term k1 s cancels exactly (with G_v and G_c separately the 2 x 2
  // determinant would cancel two terms of order k1^2, fatal in FP32 for k1 = 1e9).
  const R acc = k3 * yc * yr * ir;
  R Fv, Fvc, Jv[3], Jvc[3];  // rates and their derivatives by (rho_v, rho_c, rho_r)
  if (sat) {
    Fv = -k1 * s;
    Fvc = -acc - k2 * yc;
#pragma unroll
    for (int q = 0; q < 3; ++q) Jv[q] = -k1 * ds[q];
    Jvc[0] = R(0);
  } else {
    const R e = k4 * yr * ir;
    Fv = -e * s;
    Fvc = -e * s - acc - k2 * yc;
#pragma unroll
    for (int q = 0; q < 3; ++q) Jv[q] = -e * ds[q];
    Jv[2] -= k4 * s * ir;
    Jvc[0] = Jv[0];
  }
  Jvc[1] = (sat ? R(0) : Jv[1]) - k3 * yr * ir - k2;
  Jvc[2] = (sat ? R(0) : Jv[2]) - k3 * yc * ir;
  const R idt = Ar<R>::rcp(dt);
  G[0] = Fv - (yv - yn[0]) * idt;
  G[1] = Fvc - ((yv - yn[0]) + (yc - yn[1])) * idt;
  // 2 x 2 Jacobian in (rho_v, rho_c) with rho_r = total - rho_v - rho_c
  A[0][0] = Jv[0] - Jv[2] - idt;
  A[0][1] = Jv[1] - Jv[2];
  A[1][0] = Jvc[0] - Jvc[2] - idt;
  A[1][1] = Jvc[1] - Jvc[2] - idt;
}

template <class R, class L>
__device__ __forceinline__ int kessler_branch(const Phys &ph, const CstT<R> &C, R *y,
                                              double T0, R Cv0, int i, R rho, const R *yn,
                                              R tot, R dt, bool sat, R &s) {
  const int vi = 1 + i, ci = L::cond(i, 0), ri = L::cond(i, 1);
  y[vi] = yn[0];
  y[ci] = yn[1];
  y[ri] = yn[2];
  for (int m = 1; m <= ph.kessler_max_iter; ++m) {
    R G[2], A[2][2], tol;
    kessler_eval<R, L>(ph, C, y, T0, Cv0, i, rho, yn, dt, sat, G, A, s, tol);
    const R idet = Ar<R>::rcp(A[0][0] * A[1][1] - A[0][1] * A[1][0]);
    const R dv = (-G[0] * A[1][1] + G[1] * A[0][1]) * idet;
    const R dc = (-G[1] * A[0][0] + G[0] * A[1][0]) * idet;
    y[vi] += dv;
    y[ci] += dc;
    y[ri] = tot - y[vi] - y[ci];
    if (fabs(dv) + fabs(dc) <= tol * (fabs(y[vi]) + fabs(y[ci]) + fabs(y[ri]))) {
      R Gt[2], At[2][2], tt;
      kessler_eval<R, L>(ph, C, y, T0, Cv0, i, rho, yn, dt, sat, Gt, At, s, tt);
      return m;
    }
  }
  return -1;
}

template <class R, class L>
__device__ int kessler_cell(const Phys &ph, const CstT<R> &C, R *y, double eref, R dt) {
  if constexpr (!(L::NVAP > 0 && L::NCOND >= 2)) {
    return 0;
  } else {
    R rho = R(0);
#pragma unroll
    for (int s = 0; s < L::IM0; ++s) rho += y[s];
    // the cell's temperature and heat capacity once in FP64; each vapour then updates them
    // by its own phase changes
    double T0, p0, Cv0;
    cell_Tp<R, L>(ph, y, eref, T0, p0, &Cv0);
    int worst = 0;
    for (int i = 0; i < L::NVAP; ++i) {
      const int vi = 1 + i, ci = L::cond(i, 0), ri = L::cond(i, 1);
      const R yn[3] = {y[vi], y[ci], y[ri]};
      const R tot = yn[0] + yn[1] + yn[2];
      R G[2], A[2][2], s0, s, tol0;
      const R cv0 = R(Cv0);
      kessler_eval<R, L>(ph, C, y, T0, cv0, i, rho, yn, dt, true, G, A, s0, tol0);
      const bool first = s0 > R(0);
      int it = kessler_branch<R, L>(ph, C, y, T0, cv0, i, rho, yn, tot, dt, first, s);
      if (!(it > 0 && (first ? s > R(0) : s <= R(0)))) {
        it = kessler_branch<R, L>(ph, C, y, T0, cv0, i, rho, yn, tot, dt, !first, s);
        if (!(it > 0 && (!first ? s > R(0) : s <= R(0))))
          it = kessler_branch<R, L>(ph, C, y, T0, cv0, i, rho, yn, tot, dt, true, s);
      }
      {  // this vapour's phase changes, in FP64, carried to the next vapour's T0 and C_v0
        const double dv = double(y[vi]) - double(yn[0]), dc = double(y[ci]) - double(yn[1]);
        const double dr = double(y[ri]) - double(yn[2]);
        const double dC = (ph.sig_v[i] * dv + ph.sig_c[i][0] * dc + ph.sig_c[i][1] * dr) * ph.c_vd;
        const double dA = ph.mu[i][0] * dc + ph.mu[i][1] * dr;
        T0 -= quot64<R>(dA + T0 * dC, Cv0 + dC);
        Cv0 += dC;
      }
      if (it < 0)
        worst = -1;
      else if (worst >= 0 && it > worst)
        worst = it;
    }
    return worst;
  }
}

__device__ __forceinline__ float block_max_f(float v, float *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < int(blockDim.x >> 5)) ? red[l] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

// Asynchronous global -> shared copy of one element (cp.async, completed by cp_async_wait):
// the stage input Y^n of the owned cells is fetched while the tile is being computed.
template <class R>
__device__ __forceinline__ void cp_async_elem(R *smem_dst, const R *gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  if constexpr (sizeof(R) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
// Flag accesses of the resident step: a load with acquire and a store with release
// semantics at device scope (the data written before the release is visible to a CTA whose
// acquire load saw the flag).
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ------------------------------------------------------------------------------------------
// the fused stage kernel
// ------------------------------------------------------------------------------------------
// WENO5 of Sec. 4.2 evaluated once per cell c for both of its faces from the five cells
// (a, b, c, d, e) = Q_{c-2} .. Q_{c+2}:
//   qm = left state at face c+1/2   = I_weno(Q_{c-2}, .., Q_{c+2})
//   qp = right state at face c-1/2  = I_weno(Q_{c+2}, .., Q_{c-2})  (Eq. q+, mirror stencil)
// The Jiang-Shu smoothness indicator of a 3-cell triple does not depend on the direction the
// triple is read in, so the three indicators (and their inverse squares) serve both faces; the
// mirror stencil takes them in reverse order. The linear weights are folded into the
// candidate coefficients, so each face needs one normalising reciprocal.
// Common factors cancel in a face's normalisation sum_k w_k q_k / sum_k w_k, so the kernel
// takes (a) every eps + beta_k times 12/13: beta_k = 13/12 s^2 + 1/4 r^2 becomes s^2 + 3/13 r^2
// (three operations instead of four) against eps 12/13; (b) the linear weights (0.1, 0.6, 0.3)
// times 10: each normalisation g0 + 6 g1 + 3 g2 is two fused multiply-adds. And since the
// weights sum to the normalisation, a face state is c + sum_k w_k (q_k - c) / sum_k w_k, where
// each offset q_k - c is a short combination of the neighbour differences u = c - b,
// v = d - c, w = b - a, z = e - d, which also give the indicators' stencils.
template <class R>
__device__ __forceinline__ void weno5_pair(R a, R b, R c, R d, R e, R eps, R &qm, R &qp) {
  // every multiply-add below is an explicit fused one (Ar::fma_), so that each kernel
  // instantiation rounds the same way whatever its register allocation
  using A = Ar<R>;
  constexpr R k3 = R(3.0 / 13.0);
  const R u = c - b, v = d - c, w = b - a, z = e - d;
  R t;
  t = u - w;  // a - 2b + c
  R b0 = t * t;
  t = A::fma_(R(3), u, -w);  // a - 4b + 3c
  b0 = A::fma_(k3 * t, t, b0);
  t = v - u;  // b - 2c + d
  R b1 = t * t;
  const R bd = b - d;
  b1 = A::fma_(k3 * bd, bd, b1);
  t = z - v;  // c - 2d + e
  R b2 = t * t;
  t = A::fma_(R(-3), v, z);  // 3c - 4d + e
  b2 = A::fma_(k3 * t, t, b2);
  eps *= R(12.0 / 13.0);
  // inverse squares 1 / (eps + beta_k)^2, shared by both faces. FP64 (whose reciprocal is a
  // multi-instruction sequence on a slow pipe) forms them up to the common factor
  // 1 / (e0 e1 e2)^2, which cancels in each face's normalisation: g_k = (product of the other
  // two e)^2 -- no reciprocal here, and the two normalisations below share one.
  R g0, g1, g2;
  if constexpr (sizeof(R) == 8) {
    const R e0 = eps + b0, e1 = eps + b1, e2 = eps + b2;
    g0 = e1 * e2;
    g1 = e0 * e2;
    g2 = e0 * e1;
  } else {
    g0 = A::rcp(eps + b0);
    g1 = A::rcp(eps + b1);
    g2 = A::rcp(eps + b2);
  }
  g0 *= g0;
  g1 *= g1;
  g2 *= g2;
  // ten times the linear weight, (1, 6, 3), times the candidate interpolant of Eq. weno5 less
  // c: (1/3, -7/6, 11/6) - c = 5/6 u - 1/3 w; (-1/6, 5/6, 1/3) - c = 1/6 u + 1/3 v;
  // (1/3, 5/6, -1/6) - c = 2/3 v - 1/6 z. The right state reads the window backwards (u, v, w,
  // z become -v, -u, -z, -w) and takes the weights in reverse order.
  const R m0 = A::fma_(R(5.0 / 6.0), u, R(-1.0 / 3.0) * w);
  const R m1 = A::fma_(R(2), v, u);
  const R m2 = A::fma_(R(2), v, R(-0.5) * z);
  const R p0 = A::fma_(R(-5.0 / 6.0), v, R(1.0 / 3.0) * z);
  const R p1 = bd - u;  // -v - 2u
  const R p2 = A::fma_(R(-2), u, R(0.5) * w);
  const R Sm = A::fma_(R(3), g2, A::fma_(R(6), g1, g0));
  const R Sp = A::fma_(R(3), g0, A::fma_(R(6), g1, g2));
  const R Nm = A::fma_(g0, m0, A::fma_(g1, m1, g2 * m2));
  const R Np = A::fma_(g2, p0, A::fma_(g1, p1, g0 * p2));
  if constexpr (sizeof(R) == 8) {
    // 1/Sm = Sp / (Sm Sp) and 1/Sp = Sm / (Sm Sp); one division each only if the product
    // leaves the exponent range (g ~ e^4, so Sm Sp ~ e^8: eps far below 1e-6 or huge beta)
    const R Z = A::rcp(Sm * Sp);  // NaN outside the normal range: the test below fails
    if (Z > R(0) && Z < R(INFINITY)) {
      qm = A::fma_(Nm, Sp * Z, c);
      qp = A::fma_(Np, Sm * Z, c);
    } else {
      qm = c + Nm / Sm;
      qp = c + Np / Sp;
    }
  } else {
    qm = A::fma_(Nm, A::rcp(Sm), c);
    qp = A::fma_(Np, A::rcp(Sp), c);
  }
}

// weno5_pair<float> for two variables at once on the packed FP32x2 pipe of sm_100-class SMs
// (one instruction per two lanes of arithmetic: the reconstruction is issue-bound); the
// reciprocals stay scalar on the special-function unit.
__device__ __forceinline__ float2 f2c(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 f2rcp(float2 x) {
  return make_float2(Ar<float>::rcp(x.x), Ar<float>::rcp(x.y));
}
__device__ __forceinline__ void weno5_pair2(float2 a, float2 b, float2 c, float2 d, float2 e,
                                            float eps, float2 &qm, float2 &qp) {
  // the scaled indicators and weights and the difference form of weno5_pair
  const float2 k3 = f2c(3.0f / 13.0f), m1f = f2c(-1.0f);
  const float2 u = __ffma2_rn(m1f, b, c), v = __ffma2_rn(m1f, c, d), w = __ffma2_rn(m1f, a, b),
               z = __ffma2_rn(m1f, d, e);
  float2 t = __ffma2_rn(m1f, w, u);  // a - 2b + c
  float2 b0 = __fmul2_rn(t, t);
  t = __ffma2_rn(f2c(3.0f), u, __fmul2_rn(m1f, w));  // a - 4b + 3c
  b0 = __ffma2_rn(__fmul2_rn(k3, t), t, b0);
  t = __ffma2_rn(m1f, u, v);  // b - 2c + d
  float2 b1 = __fmul2_rn(t, t);
  const float2 bd = __ffma2_rn(m1f, d, b);  // b - d
  b1 = __ffma2_rn(__fmul2_rn(k3, bd), bd, b1);
  t = __ffma2_rn(m1f, v, z);  // c - 2d + e
  float2 b2 = __fmul2_rn(t, t);
  t = __ffma2_rn(f2c(-3.0f), v, z);  // 3c - 4d + e
  b2 = __ffma2_rn(__fmul2_rn(k3, t), t, b2);
  const float2 ke = f2c(eps * (12.0f / 13.0f));
  float2 g0 = f2rcp(__fadd2_rn(ke, b0)), g1 = f2rcp(__fadd2_rn(ke, b1)),
         g2 = f2rcp(__fadd2_rn(ke, b2));
  g0 = __fmul2_rn(g0, g0);
  g1 = __fmul2_rn(g1, g1);
  g2 = __fmul2_rn(g2, g2);
  const float2 m0 = __ffma2_rn(f2c(5.0f / 6.0f), u, __fmul2_rn(f2c(-1.0f / 3.0f), w));
  const float2 m1 = __ffma2_rn(f2c(2.0f), v, u);
  const float2 m2 = __ffma2_rn(f2c(2.0f), v, __fmul2_rn(f2c(-0.5f), z));
  const float2 p0 = __ffma2_rn(f2c(-5.0f / 6.0f), v, __fmul2_rn(f2c(1.0f / 3.0f), z));
  const float2 p1 = __ffma2_rn(m1f, u, bd);  // -v - 2u = (b - d) - u
  const float2 p2 = __ffma2_rn(f2c(-2.0f), u, __fmul2_rn(f2c(0.5f), w));
  const float2 Sm = __ffma2_rn(f2c(3.0f), g2, __ffma2_rn(f2c(6.0f), g1, g0));
  const float2 Sp = __ffma2_rn(f2c(3.0f), g0, __ffma2_rn(f2c(6.0f), g1, g2));
  const float2 nm = __ffma2_rn(g0, m0, __ffma2_rn(g1, m1, __fmul2_rn(g2, m2)));
  const float2 np = __ffma2_rn(g2, p0, __ffma2_rn(g1, p1, __fmul2_rn(g0, p2)));
  qm = __ffma2_rn(nm, f2rcp(Sm), c);
  qp = __ffma2_rn(np, f2rcp(Sp), c);
}

// CFL rate sum_d (|u_d| + c) / dx_d in the kernel's type (FP32 kernels: FP32; the time step
// only needs a few digits). The energy entry is stored as rho e - eref.
template <class R, class L>
__device__ __forceinline__ R cell_rate_r(const CstT<R> &C, const R *y, R eref, R idx, R idy,
                                         R idz) {
  R rho = y[0];
#pragma unroll
  for (int s = 1; s < L::IM0; ++s) rho += y[s];
  const R ir = Ar<R>::rcp(rho);
  R K2 = R(0);
#pragma unroll
  for (int m = 0; m < L::NMOM; ++m) K2 += y[L::IM0 + m] * y[L::IM0 + m];
  R num = R(1), den = R(1), A = R(0), Cv = y[0], Rm = y[0];
#pragma unroll
  for (int i = 0; i < L::NVAP; ++i) {
    num += y[1 + i] * ir * C.sigv_m1[i];
    den += y[1 + i] * ir * C.ieps_m1[i];
    Cv += C.sig_v[i] * y[1 + i];
    Rm += C.inv_eps[i] * y[1 + i];
#pragma unroll
    for (int j = 0; j < L::NCOND; ++j) {
      num += y[L::cond(i, j)] * ir * C.sigc_m1[i][j];
      den -= y[L::cond(i, j)] * ir;
      Cv += C.sig_c[i][j] * y[L::cond(i, j)];
      A += C.mu[i][j] * y[L::cond(i, j)];
    }
  }
  const R U = (y[L::IE] + eref) - R(0.5) * K2 * ir - A;
  // p = R_d R_m T and T = U / (c_vd C_v), with R_m, C_v here the sums over densities
  const R p = C.gm1 * Rm * Ar<R>::div(U, Cv);
  const R gam = R(1) + C.gm1 * Ar<R>::div(den, num);
  const R c = Ar<R>::sqrt_pos(gam * p * ir);
  R r = (fabs(y[L::mom(0)]) * ir + c) * idx + (fabs(y[L::mom(2)]) * ir + c) * idz;
  if constexpr (L::D3) r += (fabs(y[L::mom(1)]) * ir + c) * idy;
  return r;
}

template <class R, class L, bool VISC, class T>
struct StageSmem {
  using B = Box<T, L::D3>;
  static constexpr size_t prim = (sizeof(R) * L::NV * B::NSTORE + 15) / 16 * 16;
  static constexpr size_t visc = VISC ? (sizeof(R) * 2 * B::NSTORE + 15) / 16 * 16 : 0;
  // left states (then fluxes) and right states, each array starting on a 16-byte boundary:
  // the grouped layout moves 16-byte vectors
  static constexpr size_t face_half = (sizeof(R) * L::NV * B::NF + 15) / 16 * 16;
  static constexpr size_t face = 2 * face_half;
  static constexpr size_t red = 32 * sizeof(double);
  static constexpr size_t base = prim + visc + face + red;
  static_assert(prim % 16 == 0 && visc % 16 == 0 && face_half % 16 == 0 && red % 16 == 0,
                "every shared-memory array of the stage starts on a 16-byte boundary");
  // Y^n of the owned cells, prefetched by cp.async, when it costs no resident CTA per SM
  // (228 KB of shared memory per SM, 1 KB reserved per CTA)
  static constexpr size_t yn_bytes = sizeof(R) * L::NV * B::NCELL;
  static constexpr bool PREFETCH = 233472 / (base + yn_bytes + 1024) >= 233472 / (base + 1024);
  static constexpr size_t yn = PREFETCH ? yn_bytes : 0;
  static constexpr size_t total = base + yn;
};

// Grid-wide barrier of the persistent step kernel (all CTAs co-resident by a cooperative
// launch). Every wait is bounded: after spin_limit clock cycles (about 2 s by default) the CTA
// records kFlagTimeout and proceeds, so a fault can corrupt results but never hang the device.
// The host clears the barrier state before every persistent launch, so a count left behind by
// a wait that gave up does not open a later barrier early. absent_cta (a test aid, -1 in
// normal use) names a CTA that neither arrives nor waits, which makes every other CTA's wait
// run out.
__device__ __forceinline__ void grid_barrier(GridSync *gs, unsigned int nblocks,
                                             unsigned int *flags, long long spin_limit,
                                             int absent_cta) {
  __syncthreads();
  if (threadIdx.x == 0 && int(blockIdx.x) != absent_cta) {
    volatile unsigned int *vgen = &gs->gen;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&gs->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&gs->count, 0u);
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (clock64() - t0 > spin_limit) {
          atomicOr(flags, (unsigned)kFlagTimeout);
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// One stage over the CTA's tiles. RES (the resident step, one tile per CTA for all three
// stages): for stages 1 and 2 ys holds the owned cells' stage input on entry (the previous
// stage's output, kept in registers) instead of being loaded; Y^n of the owned cells is kept
// in shared memory from stage 0 on; the time step of stage 0 stays in s_red[0]; ghost cells
// are read past L1 (other CTAs wrote them during this launch); the CFL maximum goes to
// D.rate_next (the step's own rate stays readable until every CTA has formed its time step);
// ys receives the stage output.
template <class R, class L, bool VISC, class T, bool MICRO, bool RES = false>
__device__ __forceinline__ void stage_tiles(const StageArgs &a, const int stage,
                                            unsigned char *smem,
                                            R (&ys)[Box<T, L::D3>::CPT][L::NV]) {
  using B = Box<T, L::D3>;
  using S = StageSmem<R, L, VISC, T>;
  using P = Prof<R>;
  constexpr int NV = L::NV;
  constexpr int TX = T::TX, TY = T::TY, TZ = T::TZ, NT = T::NT;
  R *s_prim = reinterpret_cast<R *>(smem);
  R *s_th = reinterpret_cast<R *>(smem + S::prim);
  R *s_pi = s_th + (VISC ? B::NSTORE : 0);
  R *s_fl = reinterpret_cast<R *>(smem + S::prim + S::visc);  // left states, then fluxes
  R *s_fr = s_fl + S::face_half / sizeof(R);                   // right states
  using V = SV<R, NV>;
  double *s_red = reinterpret_cast<double *>(smem + S::prim + S::visc + S::face);
  R *s_yn = reinterpret_cast<R *>(smem + S::base);  // used when S::PREFETCH
  const Phys &ph = a.ph;
  const CstT<R> &C = cst<R>(a);
  const R weps = C.weno_eps;
  const int tid = threadIdx.x;

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int dm = find_domain(a.tile_domain, a.ndom, tile);
    const DomDev &D = a.doms[dm];
    const int nx = D.nx, ny = D.ny, nz = D.nz;
    const long long ncell = D.ncell;
    const int lt = tile - D.tile_begin;
    const int x0 = (lt % D.tx) * TX;
    const int y0 = ((lt / D.tx) % D.ty) * TY;
    const int z0 = (lt / (D.tx * D.ty)) * TZ;
    const int ex = min(TX, nx - x0), ey = min(TY, ny - y0), ez = min(TZ, nz - z0);
    const R *Ys = reinterpret_cast<const R *>(a.buf_s ? a.buf_s : D.buf[stage]);
    const R *Yn = reinterpret_cast<const R *>(a.buf_n ? a.buf_n : D.buf[0]);
    R *Yo = reinterpret_cast<R *>(a.buf_o ? a.buf_o : D.buf[stage == 0 ? 1 : (stage == 1 ? 2 : 0)]);
    // the stage's time step, formed once per CTA
    if (tid == 0) {
      double dt;
      if (stage == 0) {
        dt = a.dt_override > 0.0 ? a.dt_override
             : (D.dt_fixed > 0.0 ? D.dt_fixed : D.cfl / __longlong_as_double((long long)*D.rate));
        if (lt == 0) *D.dt_step = dt;
      } else if (!RES) {
        dt = *(volatile double *)D.dt_step;
        if (stage == 1 && lt == 0) *D.rate = 0ull;
      } else {
        dt = s_red[0];  // this CTA's own stage-0 time step
      }
      s_red[0] = dt;
    }

    // ---- 1. owned cells: load, keep the conserved values, store primitives -------------
    if constexpr (S::PREFETCH && !RES) {
      if (stage != 0) {
#pragma unroll
        for (int m = 0; m < B::CPT; ++m) {
          const int c = tid + m * NT;
          const int lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
          if (c < B::NCELL && lx < ex && ly < ey && lz < ez) {
            const long long g = ((long long)(z0 + lz) * ny + (y0 + ly)) * nx + (x0 + lx);
#pragma unroll
            for (int v = 0; v < NV; ++v) cp_async_elem<R>(s_yn + v * B::NCELL + c, Yn + v * ncell + g);
          }
        }
        cp_async_commit();
      }
    }
#pragma unroll
    for (int m = 0; m < B::CPT; ++m) {
      const int c = tid + m * NT;
      const int lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
      if (c < B::NCELL && lx < ex && ly < ey && lz < ez) {
        const int k = z0 + lz;
        const long long g = ((long long)k * ny + (y0 + ly)) * nx + (x0 + lx);
        if (!RES || stage == 0) {
#pragma unroll
          for (int v = 0; v < NV; ++v) ys[m][v] = Ys[v * ncell + g];
          if constexpr (RES && S::PREFETCH) {
#pragma unroll
            for (int v = 0; v < NV; ++v) s_yn[v * B::NCELL + c] = ys[m][v];
          }
        }
        R x[NV], pt, Tt;
        cons_to_prim<R, L>(ph, C, D, k, ys[m], x, pt, Tt);
        const int bi = B::idx(lx + 3, ly + B::HY, lz + 3);
        V::store(s_prim, bi, B::NSTORE, x);
        if constexpr (VISC) {
          const R Pi = Ar<R>::pow_small(pt * R(1e-5), C.kappa);
          s_th[bi] = pt * Ar<R>::rcp(x[0] * Pi) * C.iR_d;
          s_pi[bi] = Pi;
        }
      }
    }
    // ---- 2. halo of the cross (x, y, z), boundary ghosts synthesised --------------------
    {
      constexpr int NHX = 6 * TY * TZ, NHY = L::D3 ? 6 * TX * TZ : 0, NHZ = 6 * TX * TY;
      for (int h = tid; h < NHX + NHY + NHZ; h += NT) {
        int bx, by, bz, dirn, layer;
        bool ok;
        if (h < NHX) {
          const int r = h % 6, q = h / 6, ly = q % TY, lz = q / TY;
          layer = r;
          ok = ly < ey && lz < ez;
          bx = r < 3 ? r : ex + r;
          by = ly + B::HY;
          bz = lz + 3;
          dirn = 0;
        } else if (h < NHX + NHY) {
          const int hh = h - NHX, lx = hh % TX, r = (hh / TX) % 6, lz = hh / (6 * TX);
          layer = r;
          ok = lx < ex && lz < ez;
          bx = lx + 3;
          by = r < 3 ? r : ey + r;
          bz = lz + 3;
          dirn = 1;
        } else {
          const int hh = h - NHX - NHY, lx = hh % TX, ly = (hh / TX) % TY, r = hh / (TX * TY);
          layer = r;
          ok = lx < ex && ly < ey;
          bx = lx + 3;
          by = ly + B::HY;
          bz = r < 3 ? r : ez + r;
          dirn = 2;
        }
        if (!ok) continue;
        int gx = x0 + bx - 3, gy = y0 + by - B::HY, gz = z0 + bz - 3;
        // the side this ghost lies beyond (x-, x+, y-, y+, z-, z+)
        const int side = 2 * dirn + ((dirn == 0 ? gx : (dirn == 1 ? gy : gz)) < 0 ? 0 : 1);
        bool flip = false;
        const R *src = Ys;
        long long g, nsrc = ncell;
        if (dirn == 0 && (gx < 0 || gx >= nx) && D.bc[side] == kBcHalo && !a.buf_s) {
          // a slab boundary: the neighbouring slab's cells (a linked domain's stage input,
          // or the ghost buffer the caller filled)
          const int h = side, hn = D.hnx[h];
          src = reinterpret_cast<const R *>(D.hsrc[h][stage]);
          nsrc = (long long)hn * ny * nz;
          g = ((long long)gz * ny + gy) * hn + D.hoff[h] + (h ? gx - nx : gx + 3);
        } else {
          if (dirn == 0) gx = map_index(gx, nx, D.bc[0], D.bc[1], flip);
          if (dirn == 1) gy = map_index(gy, ny, D.bc[2], D.bc[3], flip);
          if (dirn == 2) gz = map_index(gz, nz, D.bc[4], D.bc[5], flip);
          g = ((long long)gz * ny + gy) * nx + gx;
        }
        R y[NV], x[NV], pt, Tt;
        if constexpr (RES) {
#pragma unroll
          for (int v = 0; v < NV; ++v) y[v] = __ldcg(src + v * nsrc + g);
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) y[v] = src[v * nsrc + g];
        }
        cons_to_prim<R, L>(ph, C, D, gz, y, x, pt, Tt);
        if (flip) {
          // a wall: free-slip negates the normal velocity, no-slip every component
          if (D.bc[side] == kBcNoSlip) {
#pragma unroll
            for (int m = 0; m < L::NMOM; ++m) x[L::IM0 + m] = -x[L::IM0 + m];
          } else {
            x[L::mom(dirn)] = -x[L::mom(dirn)];
          }
          // Sec. 6 lower boundary: the ghost holds T_bot at the mirrored pressure and
          // composition, so its density is p / (R_d den T_bot) (App. B: p = rho R_d den T,
          // den the mixing factor), the mirrored density times T / T_bot
          if (side == 4 && D.T_bot > 0.0) {
            R num, den;
            mix_factors<R, L>(C, x, num, den);
            x[0] = pt * C.iR_d * Ar<R>::rcp(den * R(D.T_bot));
          }
        }
        const int bi = B::idx(bx, by, bz);
        V::store(s_prim, bi, B::NSTORE, x);
        // the viscous heat flux reads theta and the Exner function only on the two sides of
        // a face, so of the halo only the ring next to the tile (layers 2 and 3) needs them
        if constexpr (VISC) {
          if (layer == 2 || layer == 3) {
            const R Pi = Ar<R>::pow_small(pt * R(1e-5), C.kappa);
            s_th[bi] = pt * Ar<R>::rcp(x[0] * Pi) * C.iR_d;
            s_pi[bi] = Pi;
          }
        }
      }
    }
    __syncthreads();
    const R dt = R(s_red[0]);

    R acc[B::CPT][NV];
#pragma unroll
    for (int m = 0; m < B::CPT; ++m)
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[m][v] = R(0);

    // ---- 3. per direction: WENO5 per cell (both faces), LMARS per face, divergence -------
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d == 1 && !L::D3) continue;
      const int fx = d == 0, fy = d == 1, fz = d == 2;
      // face array strides: faces along d are numbered 0..T_d
      const int sx = TX + fx, sy = TY + fy;
      const int stride = d == 0 ? 1 : (d == 1 ? B::BX : B::BX * B::BY);
      const int ed = d == 0 ? ex : (d == 1 ? ey : ez);
      // 3a. reconstruction over the owned cells and one more on each side along d
      {
        const int rx = TX + 2 * fx, ry = TY + 2 * fy, rz = TZ + 2 * fz;
        const int nrec = rx * ry * rz;
        constexpr int MAXREC = (TX + 2) * (TY + (L::D3 ? 2 : 0)) * (TZ + 2);
#pragma unroll
        for (int r = 0; r < (MAXREC + NT - 1) / NT; ++r) {
          const int it = tid + r * NT;
          int lx = it % rx, ly = (it / rx) % ry, lz = it / (rx * ry);
          lx -= fx;
          ly -= fy;
          lz -= fz;
          const int ld = fx ? lx : (fy ? ly : lz);
          if (it < nrec && ld <= ed && lx < ex + fx && ly < ey + fy && lz < ez + fz) {
            // the five cells of the window along d: a fixed stride in the x-z box and along the
            // 3-D x-lines; mapped one by one where a 3-D y or z window leaves the x-lines
            int o[5];
            if (L::D3 && !fx) {
              // the window's fixed coordinate lies in the owned range
#pragma unroll
              for (int k = 0; k < 5; ++k)
                o[k] = fy ? B::idx_y(lx + 3, ly + B::HY + (k - 2), lz + 3)
                          : B::idx_z(lx + 3, ly + B::HY, lz + 3 + (k - 2));
            } else {
              const int bi = B::idx(lx + 3, ly + B::HY, lz + 3);
#pragma unroll
              for (int k = 0; k < 5; ++k) o[k] = bi + (k - 2) * stride;
            }
            const int fl = ((lz + fz) * sy + (ly + fy)) * sx + (lx + fx);  // face c+1/2
            const int fr = (lz * sy + ly) * sx + lx;                        // face c-1/2
            const bool has_l = ld < ed, has_r = ld >= 0;
            R QM[NV], QP[NV];
            // one group of fields at a time (the group's five window points, one vector access
            // each): FP32 pairs on the packed FP32x2 pipe, an odd field alone
#pragma unroll
            for (int g = 0; g < V::NF + V::T2 + V::T1; ++g) {
              const int f0 = g < V::NF ? g * V::W : (g == V::NF && V::T2 ? V::P2 : V::P1);
              const int n = g < V::NF ? V::W : (g == V::NF && V::T2 ? 2 : 1);
              R X[5][V::W];
#pragma unroll
              for (int k = 0; k < 5; ++k) V::load_group(s_prim, g, o[k], B::NSTORE, X[k]);
              if constexpr (sizeof(R) == 4) {
#pragma unroll
                for (int j = 0; j + 1 < V::W; j += 2) {
                  if (j + 1 < n) {
                    float2 qm, qp;
                    weno5_pair2(make_float2(X[0][j], X[0][j + 1]), make_float2(X[1][j], X[1][j + 1]),
                                make_float2(X[2][j], X[2][j + 1]), make_float2(X[3][j], X[3][j + 1]),
                                make_float2(X[4][j], X[4][j + 1]), weps, qm, qp);
                    QM[f0 + j] = qm.x, QM[f0 + j + 1] = qm.y, QP[f0 + j] = qp.x, QP[f0 + j + 1] = qp.y;
                  }
                }
                if (n == 1)
                  weno5_pair<R>(X[0][0], X[1][0], X[2][0], X[3][0], X[4][0], weps, QM[f0], QP[f0]);
              } else {
#pragma unroll
                for (int j = 0; j < V::W; ++j)
                  if (j < n)
                    weno5_pair<R>(X[0][j], X[1][j], X[2][j], X[3][j], X[4][j], weps, QM[f0 + j],
                                  QP[f0 + j]);
              }
            }
            if (has_l) V::store(s_fl, fl, B::NF, QM);
            if (has_r) V::store(s_fr, fr, B::NF, QP);
          }
        }
      }
      __syncthreads();
      // 3b. LMARS flux per face (and the viscous flux), written over the left state
      {
        const int nface = sx * sy * (TZ + fz);
#pragma unroll
        for (int r = 0; r < (B::NF + NT - 1) / NT; ++r) {
          const int f = tid + r * NT;
          const int ix = f % sx, iy = (f / sx) % sy, iz = f / (sx * sy);
          if (f >= nface || ix >= ex + fx || iy >= ey + fy || iz >= ez + fz) continue;
          R QL[NV], QR[NV], F[NV];
          V::load(s_fl, f, B::NF, QL);
          V::load(s_fr, f, B::NF, QR);
          const R pref = fz ? P::pf(D, z0 + iz) : P::pc(D, z0 + iz);
          lmars<R, L>(C, QL, QR, d, pref, F);
          if constexpr (L::MOIST && MICRO) {
            // no condensate passes a wall
            const int kf = z0 + iz;
            if (fz && ph.sediment && !(kf == 0 && D.bc[4] != kBcPeriodic) &&
                !(kf == nz && D.bc[5] != kBcPeriodic))
              sediment_flux<R, L>(C, QL, QR, pref, F);
          }
          if constexpr (VISC) {
            const int bi = B::idx(ix + 3, iy + B::HY, iz + 3);  // right cell of the face
            const int bl = B::idx(ix + 3 - fx, iy + B::HY - fy, iz + 3 - fz);
            R XLc[NV], XRc[NV];  // primitives of the two cells of the face
            V::load(s_prim, bl, B::NSTORE, XLc);
            V::load(s_prim, bi, B::NSTORE, XRc);
            const R rf = R(0.5) * (XLc[0] + XRc[0]);
            const R ih = P::ih(D, d), nu = C.nu;
            R work = R(0);
#pragma unroll
            for (int mm = 0; mm < L::NMOM; ++mm) {
              const R ul = XLc[L::IM0 + mm];
              const R ur = XRc[L::IM0 + mm];
              const R grad = (ur - ul) * ih;
              F[L::IM0 + mm] -= rf * nu * grad;
              work += R(0.5) * (ul + ur) * grad;
            }
            const R heat = R(0.5) * (s_pi[bl] + s_pi[bi]) * (s_th[bi] - s_th[bl]) * ih;
            F[L::IE] -= rf * nu * work + rf * C.c_pd * nu * heat;
          }
          V::store(s_fl, f, B::NF, F);
        }
      }
      __syncthreads();
      // 3c. flux divergence of the owned cells (Eq. forward)
      const R ih = P::ih(D, d);
#pragma unroll
      for (int m = 0; m < B::CPT; ++m) {
        const int c = tid + m * NT;
        const int lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
        if (c < B::NCELL && lx < ex && ly < ey && lz < ez) {
          const int f0 = (lz * sy + ly) * sx + lx;
          const int f1 = ((lz + fz) * sy + (ly + fy)) * sx + (lx + fx);
          R F1[NV], F0[NV];
          V::load(s_fl, f1, B::NF, F1);
          V::load(s_fl, f0, B::NF, F0);
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[m][v] -= (F1[v] - F0[v]) * ih;
        }
      }
      if (d != 2) __syncthreads();
    }

    // ---- 4. gravity source, stage combine, saturation adjustment, store ------------------
    if constexpr (S::PREFETCH && !RES) {
      if (stage != 0) cp_async_wait();  // this thread's own copies of Y^n
    }
    R rate_max = R(0);
#pragma unroll
    for (int m = 0; m < B::CPT; ++m) {
      const int c = tid + m * NT;
      const int lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
      if (c < B::NCELL && lx < ex && ly < ey && lz < ez) {
        const int k = z0 + lz;
        const R grav = P::grav(D);
        // vertical momentum: -(rho - rho_bar) g (Eq. mom3 with the reference balance removed)
        acc[m][L::mom(2)] -= P::template drho<L>(D, k, ys[m]) * grav;
        // energy: -g (F_rho,k-1/2 + F_rho,k+1/2) / 2 with the vertical total-mass fluxes
        const int f0 = (lz * TY + ly) * TX + lx;
        const int f1 = ((lz + 1) * TY + ly) * TX + lx;
        R mb = R(0), mt = R(0);
#pragma unroll
        for (int s = 0; s < L::IM0; ++s) {
          mb += s_fl[V::at(s, f0, B::NF)];
          mt += s_fl[V::at(s, f1, B::NF)];
        }
        acc[m][L::IE] -= grav * R(0.5) * (mb + mt);
        if constexpr (MICRO && L::MOIST) {
          // forcing of the Jovian simulation (Sec. 6) by the level's reference pressure
          const R pk = P::pc(D, k);
          if (C.cool_rate != R(0) && pk >= C.cool_p_lo && pk <= C.cool_p_hi) {
            R Cv = ys[m][0];  // heat capacity at constant volume / c_vd
#pragma unroll
            for (int i2 = 0; i2 < L::NVAP; ++i2) {
              Cv += C.sig_v[i2] * ys[m][1 + i2];
#pragma unroll
              for (int j2 = 0; j2 < L::NCOND; ++j2) Cv += C.sig_c[i2][j2] * ys[m][L::cond(i2, j2)];
            }
            acc[m][L::IE] -= Cv * C.c_vd * C.cool_rate;
          }
          if (C.sponge_itau0 != R(0) && pk * C.sponge_ip0 < R(1)) {
            const R r = pk * C.sponge_ip0, rate = C.sponge_itau0 * Ar<R>::rcp(r * r);
            acc[m][L::mom(0)] -= ys[m][L::mom(0)] * rate;
            if constexpr (L::D3) acc[m][L::mom(1)] -= ys[m][L::mom(1)] * rate;
          }
        }
        const long long g = ((long long)k * ny + (y0 + ly)) * nx + (x0 + lx);
        R yo[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const R s1 = ys[m][v] + dt * acc[m][v];
          if (stage == 0) {
            yo[v] = s1;
          } else {
            const R yn = S::PREFETCH ? s_yn[v * B::NCELL + c] : Yn[v * ncell + g];
            // (1 - w) Y^n + w s1 as Y^n + w (s1 - Y^n): the two weights sum to exactly one.
            // With 1/3 and 2/3 each rounded to FP32 they sum to 1 + 3e-8, which scales the
            // whole state by that much every step (a mass drift of 1e-3 over 30,000 steps)
            // (an explicit fused multiply-add, so that every kernel that inlines this rounds
            // it the same way)
            const R wgt = stage == 1 ? R(0.25) : R(2.0 / 3.0);
            yo[v] = fma(wgt, s1 - yn, yn);
          }
        }
        if constexpr (L::MOIST) {
          if (ph.satadj) {
            const int it =
                satadj_cell<R, L>(ph, C, yo, D.e_ref[k], P::er(D, k), ph.satadj_max_iter);
            if (it < 0)
              atomicOr(a.flags, (unsigned)kFlagNoConv);
            else if (it > 2)
              atomicMax(a.max_sweeps, it);
          }
          // the microphysics follows each step (time splitting), over the step's dt
          if (MICRO && stage == 2 && ph.kessler) {
            if (kessler_cell<R, L>(ph, C, yo, D.e_ref[k], dt) < 0)
              atomicOr(a.flags, (unsigned)kFlagNoConv);
          }
        }
        R rs = R(0);
#pragma unroll
        for (int s = 0; s < L::IM0; ++s) rs += yo[s];
        if (!(rs > R(0)) || !isfinite(yo[L::IE])) atomicOr(a.flags, (unsigned)kFlagNonFinite);
#pragma unroll
        for (int v = 0; v < NV; ++v) Yo[v * ncell + g] = yo[v];
        if constexpr (RES) {
#pragma unroll
          for (int v = 0; v < NV; ++v) ys[m][v] = yo[v];
        }
        if (stage == 2)
          rate_max = fmax(rate_max, cell_rate_r<R, L>(C, yo, P::er(D, k), P::ih(D, 0),
                                                      P::ih(D, 1), P::ih(D, 2)));
      }
    }
    if (stage == 2) {
      double bm;
      if constexpr (sizeof(R) == 4)
        bm = double(block_max_f(rate_max, reinterpret_cast<float *>(s_red + 1)));
      else
        bm = block_max(rate_max, s_red + 1);
      if (tid == 0)
        atomicMax(RES ? D.rate_next : D.rate, (unsigned long long)__double_as_longlong(bm));
    }
    __syncthreads();
  }
}

// One Runge-Kutta stage over all tiles of all domains.
template <class R, class L, bool VISC, class T, bool MICRO>
__global__ void __launch_bounds__(T::NT, T::MINB) stage_kernel(const StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  R ys[Box<T, L::D3>::CPT][L::NV];
  stage_tiles<R, L, VISC, T, MICRO>(a, a.stage, smem, ys);
}

// One whole step (three stages) in a single persistent cooperative launch: the CTAs walk the
// tile queue of every domain per stage and meet at a grid barrier between stages.
template <class R, class L, bool VISC, class T, bool MICRO>
__global__ void __launch_bounds__(T::NT, T::MINB) step_kernel(const StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  R ys[Box<T, L::D3>::CPT][L::NV];
#pragma unroll 1
  for (int st = 0; st < 3; ++st) {
    stage_tiles<R, L, VISC, T, MICRO>(a, st, smem, ys);
    if (st < 2) grid_barrier(a.gsync, gridDim.x, a.flags, a.spin_limit, a.absent_cta);
  }
}

// One whole step in a single cooperative launch with one tile per CTA (every tile of the
// launch co-resident): each CTA keeps its tile's state in registers through the three stages
// and, between stages, waits only for the tiles its ghost cells come from -- a flag per tile,
// set to 3 seq + s + 1 once the tile's stage-s output is in memory (seq counts the launches) --
// instead of a grid barrier or a new launch. Waits are bounded like the grid barrier's. The
// last CTA to finish moves each domain's next CFL rate into place and advances seq.
template <class R, class L, bool VISC, class T, bool MICRO>
__global__ void __launch_bounds__(T::NT, T::MINB) resident_step_kernel(const StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int s_seq;
  R ys[Box<T, L::D3>::CPT][L::NV];
  const int tile = blockIdx.x, tid = threadIdx.x;
  if (tid == 0) s_seq = ld_acquire_u32(&a.res->seq);
  __syncthreads();
  const unsigned int seq = s_seq;
  const int d0 = a.dep_begin[tile], nd = a.dep_begin[tile + 1] - d0;
#pragma unroll 1
  for (int st = 0; st < 3; ++st) {
    if (st > 0) {
      // the tiles this one's ghost cells come from have finished stage st - 1
      const unsigned int want = 3u * seq + unsigned(st);
      for (int i = tid; i < nd; i += blockDim.x) {
        const unsigned int *f = a.tile_flags + a.dep_list[d0 + i];
        const long long t0 = clock64();
        while (int(ld_acquire_u32(f) - want) < 0) {
          if (clock64() - t0 > a.spin_limit) {
            atomicOr(a.flags, (unsigned)kFlagTimeout);
            break;
          }
          __nanosleep(20);
        }
      }
      __syncthreads();
    }
    stage_tiles<R, L, VISC, T, MICRO, true>(a, st, smem, ys);  // ends with a CTA barrier
    if (st < 2 && tid == 0) {
      __threadfence();
      st_release_u32(a.tile_flags + tile, 3u * seq + unsigned(st) + 1u);
    }
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&a.res->done, 1u) == gridDim.x - 1) {
      __threadfence();
      for (int d = 0; d < a.ndom; ++d) {
        const DomDev &D = a.doms[d];
        *D.rate = atomicExch(D.rate_next, 0ull);
      }
      a.res->done = 0u;
      __threadfence();
      st_release_u32(&a.res->seq, seq + 1u);
    }
  }
}

// ------------------------------------------------------------------------------------------
// auxiliary kernels: CFL rate, budget, saturation adjustment over a domain
// ------------------------------------------------------------------------------------------
// The blocks take (level, chunk of blockDim.x cells of the level) items in turn, so the level
// of a cell comes from one division per item, not one per cell.
template <class R, class L>
__global__ void __launch_bounds__(256) rate_kernel(const StageArgs a, int dm, int buf) {
  __shared__ double red[32];
  const DomDev &D = a.doms[dm];
  const R *Y = reinterpret_cast<const R *>(D.buf[buf]);
  const long long plane = (long long)D.nx * D.ny;
  const long long chunks = (plane + blockDim.x - 1) / blockDim.x;
  const long long items = chunks * D.nz;
  double r = 0.0;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int k = int(it / chunks);
    const long long p = (it - k * chunks) * blockDim.x + threadIdx.x;
    if (p < plane) {
      const long long c = k * plane + p;
      R y[L::NV];
#pragma unroll
      for (int v = 0; v < L::NV; ++v) y[v] = Y[v * D.ncell + c];
      r = fmax(r, double(cell_rate_r<R, L>(cst<R>(a), y, Prof<R>::er(D, k), Prof<R>::ih(D, 0),
                                           Prof<R>::ih(D, 1), Prof<R>::ih(D, 2))));
    }
  }
  double bm = block_max(r, red);
  if (threadIdx.x == 0) atomicMax(D.rate, (unsigned long long)__double_as_longlong(bm));
}

// A caller-layout state (type S: energy as rho e) into the stored state of domain dm (type R,
// energy as rho e - e_ref of the level, the difference formed in FP64), with the CFL rate of
// the stored cells folded into the domain's rate slot: the state copy and the rate kernel in
// one pass. Items as in rate_kernel; VW consecutive cells of a level per thread, each field
// one aligned access (VW = 4 where every level starts on such a boundary, else 1).
template <class S, class R, class L, int VW>
__global__ void __launch_bounds__(256) load_rate_kernel(const S *src, const StageArgs a, int dm) {
  __shared__ double red[32];
  const DomDev &D = a.doms[dm];
  R *Y = reinterpret_cast<R *>(D.buf[0]);
  const long long plane = (long long)D.nx * D.ny, ncell = D.ncell;
  const long long span = (long long)blockDim.x * VW;
  const long long chunks = (plane + span - 1) / span;
  const long long items = chunks * D.nz;
  const CstT<R> &C = cst<R>(a);
  double r = 0.0;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int k = int(it / chunks);
    const long long p = (it - k * chunks) * span + (long long)threadIdx.x * VW;
    if (p < plane) {  // VW divides plane, so all VW cells lie in the level
      const long long c0 = k * plane + p;
      const double er = D.e_ref[k];
      R y[VW][L::NV];
#pragma unroll
      for (int v = 0; v < L::NV; ++v) {
        const Pack<S, VW> in = *reinterpret_cast<const Pack<S, VW> *>(src + v * ncell + c0);
        Pack<R, VW> out;
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          out.x[e] = v == L::IE ? R(double(in.x[e]) - er) : R(in.x[e]);
          y[e][v] = out.x[e];
        }
        *reinterpret_cast<Pack<R, VW> *>(Y + v * ncell + c0) = out;
      }
#pragma unroll
      for (int e = 0; e < VW; ++e)
        r = fmax(r, double(cell_rate_r<R, L>(C, y[e], Prof<R>::er(D, k), Prof<R>::ih(D, 0),
                                             Prof<R>::ih(D, 1), Prof<R>::ih(D, 2))));
    }
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
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < D.ncell;
       c += (long long)gridDim.x * blockDim.x) {
    R y[L::NV];
#pragma unroll
    for (int v = 0; v < L::NV; ++v) y[v] = Y[v * D.ncell + c];
    const double er = D.e_ref[c / ((long long)D.nx * D.ny)];
    const int it = satadj_cell<R, L>(a.ph, cst<R>(a), y, er,
                                     Prof<R>::er(D, int(c / ((long long)D.nx * D.ny))),
                                     a.ph.satadj_max_iter);
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
template <class R, class L, bool VISC, class T, bool MICRO = false>
struct Variant {
  using S = StageSmem<R, L, VISC, T>;
  static cudaError_t prepare() {
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<R, L, VISC, T, MICRO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(S::total));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(resident_step_kernel<R, L, VISC, T, MICRO>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::total));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_kernel<R, L, VISC, T, MICRO>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::total));
  }
  static int max_resident_tiles() {
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per, resident_step_kernel<R, L, VISC, T, MICRO>, T::NT, S::total) != cudaSuccess)
      return 0;
    return per * nsm;
  }
  static cudaError_t resident(const StageArgs &a, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(T::NT);
    cfg.dynamicSmemBytes = S::total;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, resident_step_kernel<R, L, VISC, T, MICRO>, a);
  }
  static cudaError_t stage(const StageArgs &a, int grid, cudaStream_t s) {
    stage_kernel<R, L, VISC, T, MICRO><<<grid, T::NT, S::total, s>>>(a);
    return cudaGetLastError();
  }
  static int max_resident_blocks() {
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step_kernel<R, L, VISC, T, MICRO>, T::NT,
                                                      S::total) != cudaSuccess)
      return 0;
    return per * nsm;
  }
  static cudaError_t step(const StageArgs &a, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(T::NT);
    cfg.dynamicSmemBytes = S::total;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, step_kernel<R, L, VISC, T, MICRO>, a);
  }
  static TileVariant get() {
    TileVariant v;
    v.tile[0] = T::TX;
    v.tile[1] = T::TY;
    v.tile[2] = T::TZ;
    v.threads = T::NT;
    v.smem_stage = S::total;
    v.stage = &stage;
    v.step = &step;
    v.max_resident_blocks = &max_resident_blocks;
    v.prepare = &prepare;
    v.resident = &resident;
    v.max_resident_tiles = &max_resident_tiles;
    return v;
  }
};

template <class R, class L>
struct Family {
  static cudaError_t rate(const StageArgs &a, int dm, int buf, cudaStream_t s) {
    rate_kernel<R, L><<<304, 256, 0, s>>>(a, dm, buf);
    return cudaGetLastError();
  }
  template <class S>
  static cudaError_t load_typed(const void *src, const StageArgs &a, int dm, long long plane,
                                long long nz, cudaStream_t s) {
    const long long span = 256ll * 4, chunks = (plane + span - 1) / span;
    const long long items = chunks * nz;
    const int grid = int(items < 1216 ? items : 1216);
    if (plane % 4 == 0 && (uintptr_t)src % (4 * sizeof(S)) == 0)
      load_rate_kernel<S, R, L, 4><<<grid, 256, 0, s>>>((const S *)src, a, dm);
    else
      load_rate_kernel<S, R, L, 1><<<grid, 256, 0, s>>>((const S *)src, a, dm);
    return cudaGetLastError();
  }
  static cudaError_t load(const void *src, int src_f32, const StageArgs &a, int dm,
                          long long plane, long long nz, cudaStream_t s) {
    return src_f32 ? load_typed<float>(src, a, dm, plane, nz, s)
                   : load_typed<double>(src, a, dm, plane, nz, s);
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
  // The tile shapes offered to the autotuner; the first is the default.
  template <bool VISC, class... Ts>
  static KernelSet set() {
    KernelSet k;
    k.nvariants = 0;
    TileVariant vs[] = {Variant<R, L, VISC, Ts>::get()...};
    for (const TileVariant &v : vs) k.var[k.nvariants++] = v;
    k.rate = &rate;
    k.load = &load;
    k.budget = &budget;
    k.satadj = &satadj;
    return k;
  }
  // kernels with the sedimentation fluxes and the Kessler scheme compiled in (inviscid)
  template <class... Ts>
  static KernelSet set_micro() {
    KernelSet k;
    k.nvariants = 0;
    TileVariant vs[] = {Variant<R, L, false, Ts, true>::get()...};
    for (const TileVariant &v : vs) k.var[k.nvariants++] = v;
    k.rate = &rate;
    k.load = &load;
    k.budget = &budget;
    k.satadj = &satadj;
    return k;
  }
};

}  // namespace snap
