// snap_adjoint.cuh -- discrete adjoint of one Runge-Kutta stage of the inviscid step (the
// transpose of stage_tiles in snap_stage.cuh): reverse of the saturation adjustment (App. D,
// by the derivative of its equilibrium), of the SSP-RK3 combine (Sec. 4.3), of the flux
// divergence and gravity source (Eq. forward, Eq. mom3), of LMARS (Eqs. rp, ru), of WENO5
// (Eq. weno5) and of the primitive map (App. B, Eq. p2). The upwind branch of LMARS is held
// fixed, except at u* = 0 where the mean of both one-sided derivatives is used; which vapours
// keep cloud is held fixed; the time step is a given constant.
//
// Per stage, deterministic (no atomics):
//   adj_satadj_kernel (moist layouts): one thread per cell maps the adjoint of the adjusted
//     state to that of the state before the adjustment (temperature inversion in FP64);
//   adj_face_kernel (FP32; one launch for the faces of every direction): one thread per face
//     recomputes the face states from its six-cell stencil, transposes LMARS and WENO5, and
//     writes the contribution of the face to each of its six stencil cells into
//     G[d][face][s][v] (v padded to a 16-byte vector, so that each slot moves as one access);
//   FP64 instead: adj_prim_kernel (primitives of every cell once), adj_weno_kernel (every
//     five-cell window once: both face states it yields and their gradients, sharing the
//     smoothness indicators) and adj_face_w_kernel (LMARS transposed from the stored states,
//     the same G) -- about a third less work on the slow FP64 pipe;
//   adj_cell_kernel: one thread per cell gathers the contributions of every face whose
//     stencil holds the cell (or a ghost image of it), transposes the primitive map and the
//     gravity source, and forms the stage combine.
#pragma once
#include "snap_stage.cuh"

namespace snap {

// Face contributions are stored per face and stencil slot as NVP values (the field count
// padded to a multiple of one 16-byte vector: 4 floats or 2 doubles).
template <class R>
struct GVec;
template <>
struct GVec<float> {
  using V = float4;
  static constexpr int W = 4;
  static __device__ __forceinline__ float get(const V &x, int e) {
    return e == 0 ? x.x : (e == 1 ? x.y : (e == 2 ? x.z : x.w));
  }
  static __device__ __forceinline__ V make(const float *p) { return make_float4(p[0], p[1], p[2], p[3]); }
};
template <>
struct GVec<double> {
  using V = double2;
  static constexpr int W = 2;
  static __device__ __forceinline__ double get(const V &x, int e) { return e == 0 ? x.x : x.y; }
  static __device__ __forceinline__ V make(const double *p) { return make_double2(p[0], p[1]); }
};
template <class R, int NV>
constexpr int g_stride() {
  return (NV + GVec<R>::W - 1) / GVec<R>::W * GVec<R>::W;
}

template <class R>
__device__ __forceinline__ const CstT<R> &acst(const AdjArgs &a);
template <>
__device__ __forceinline__ const CstT<float> &acst<float>(const AdjArgs &a) { return a.cf; }
template <>
__device__ __forceinline__ const CstT<double> &acst<double>(const AdjArgs &a) { return a.cd; }

// The shared reciprocal of the FP64 window transpose to ~1e-12 relative: the hardware's
// approximate FP64 reciprocal (about 1e-6) and one Newton-Raphson step, which squares its
// error (the adjoint is held to 1e-10 of the oracle's); FP32 as the forward kernels.
template <class R>
__device__ __forceinline__ R adj_rcp(R x) {
  if constexpr (sizeof(R) == 8) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return fma(y, fma(-x, y, 1.0), y);
  } else {
    return Ar<R>::rcp(x);
  }
}

// WENO5 value of the left state from (a..e) and its gradient (Jiang-Shu weights):
// dI/dq_j = sum_k w_k dv_k/dq_j + sum_k (v_k - I)/S (-2 alpha_k/(eps+beta_k)) dbeta_k/dq_j.
template <class R>
__device__ __forceinline__ R weno5_grad(const R q[5], R eps, R g[5]) {
  R t1, t2, b[3], db[3][5];
  t1 = q[0] - R(2) * q[1] + q[2];
  t2 = q[0] - R(4) * q[1] + R(3) * q[2];
  b[0] = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
  db[0][0] = R(13.0 / 6.0) * t1 + R(0.5) * t2;
  db[0][1] = R(-13.0 / 3.0) * t1 - R(2) * t2;
  db[0][2] = R(13.0 / 6.0) * t1 + R(1.5) * t2;
  db[0][3] = R(0);
  db[0][4] = R(0);
  t1 = q[1] - R(2) * q[2] + q[3];
  t2 = q[1] - q[3];
  b[1] = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
  db[1][0] = R(0);
  db[1][1] = R(13.0 / 6.0) * t1 + R(0.5) * t2;
  db[1][2] = R(-13.0 / 3.0) * t1;
  db[1][3] = R(13.0 / 6.0) * t1 - R(0.5) * t2;
  db[1][4] = R(0);
  t1 = q[2] - R(2) * q[3] + q[4];
  t2 = R(3) * q[2] - R(4) * q[3] + q[4];
  b[2] = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
  db[2][0] = R(0);
  db[2][1] = R(0);
  db[2][2] = R(13.0 / 6.0) * t1 + R(1.5) * t2;
  db[2][3] = R(-13.0 / 3.0) * t1 - R(2) * t2;
  db[2][4] = R(13.0 / 6.0) * t1 + R(0.5) * t2;
  const R d[3] = {R(0.1), R(0.6), R(0.3)};
  R al[3], v[3], S = R(0);
  v[0] = q[0] * R(1.0 / 3.0) - R(7.0 / 6.0) * q[1] + R(11.0 / 6.0) * q[2];
  v[1] = -q[1] * R(1.0 / 6.0) + R(5.0 / 6.0) * q[2] + q[3] * R(1.0 / 3.0);
  v[2] = q[2] * R(1.0 / 3.0) + R(5.0 / 6.0) * q[3] - q[4] * R(1.0 / 6.0);
  R ib[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ib[k] = Ar<R>::rcp(eps + b[k]);
    al[k] = d[k] * ib[k] * ib[k];
    S += al[k];
  }
  const R iS = Ar<R>::rcp(S);
  R I = (al[0] * v[0] + al[1] * v[1] + al[2] * v[2]) * iS;
  const R dv[3][5] = {{R(1.0 / 3.0), R(-7.0 / 6.0), R(11.0 / 6.0), R(0), R(0)},
                      {R(0), R(-1.0 / 6.0), R(5.0 / 6.0), R(1.0 / 3.0), R(0)},
                      {R(0), R(0), R(1.0 / 3.0), R(5.0 / 6.0), R(-1.0 / 6.0)}};
  R cb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) cb[k] = (v[k] - I) * iS * R(-2) * al[k] * ib[k];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    R gj = R(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) gj += al[k] * iS * dv[k][j] + cb[k] * db[k][j];
    g[j] = gj;
  }
  return I;
}

// weno5_grad<float> of two variables at once on the packed FP32x2 pipe (reciprocals scalar).
__device__ __forceinline__ float2 weno5_grad2(const float2 q[5], float eps, float2 g[5]) {
  const float2 k1312 = f2c(13.0f / 12.0f), kq = f2c(0.25f), k136 = f2c(13.0f / 6.0f);
  const float2 k133 = f2c(-13.0f / 3.0f), kh = f2c(0.5f);
  float2 b[3], db[3][5], t1, t2;
  // beta_0 over (q0, q1, q2)
  t1 = __ffma2_rn(f2c(-2.0f), q[1], __fadd2_rn(q[0], q[2]));
  t2 = __ffma2_rn(f2c(-4.0f), q[1], __ffma2_rn(f2c(3.0f), q[2], q[0]));
  b[0] = __ffma2_rn(__fmul2_rn(kq, t2), t2, __fmul2_rn(__fmul2_rn(k1312, t1), t1));
  db[0][0] = __ffma2_rn(k136, t1, __fmul2_rn(kh, t2));
  db[0][1] = __ffma2_rn(k133, t1, __fmul2_rn(f2c(-2.0f), t2));
  db[0][2] = __ffma2_rn(k136, t1, __fmul2_rn(f2c(1.5f), t2));
  // beta_1 over (q1, q2, q3)
  t1 = __ffma2_rn(f2c(-2.0f), q[2], __fadd2_rn(q[1], q[3]));
  t2 = __ffma2_rn(f2c(-1.0f), q[3], q[1]);
  b[1] = __ffma2_rn(__fmul2_rn(kq, t2), t2, __fmul2_rn(__fmul2_rn(k1312, t1), t1));
  db[1][1] = __ffma2_rn(k136, t1, __fmul2_rn(kh, t2));
  db[1][2] = __fmul2_rn(k133, t1);
  db[1][3] = __ffma2_rn(k136, t1, __fmul2_rn(f2c(-0.5f), t2));
  // beta_2 over (q2, q3, q4)
  t1 = __ffma2_rn(f2c(-2.0f), q[3], __fadd2_rn(q[2], q[4]));
  t2 = __ffma2_rn(f2c(3.0f), q[2], __ffma2_rn(f2c(-4.0f), q[3], q[4]));
  b[2] = __ffma2_rn(__fmul2_rn(kq, t2), t2, __fmul2_rn(__fmul2_rn(k1312, t1), t1));
  db[2][2] = __ffma2_rn(k136, t1, __fmul2_rn(f2c(1.5f), t2));
  db[2][3] = __ffma2_rn(k133, t1, __fmul2_rn(f2c(-2.0f), t2));
  db[2][4] = __ffma2_rn(k136, t1, __fmul2_rn(kh, t2));
  // candidates and weights
  float2 v[3];
  v[0] = __ffma2_rn(f2c(1.0f / 3.0f), q[0], __ffma2_rn(f2c(-7.0f / 6.0f), q[1], __fmul2_rn(f2c(11.0f / 6.0f), q[2])));
  v[1] = __ffma2_rn(f2c(-1.0f / 6.0f), q[1], __ffma2_rn(f2c(5.0f / 6.0f), q[2], __fmul2_rn(f2c(1.0f / 3.0f), q[3])));
  v[2] = __ffma2_rn(f2c(1.0f / 3.0f), q[2], __ffma2_rn(f2c(5.0f / 6.0f), q[3], __fmul2_rn(f2c(-1.0f / 6.0f), q[4])));
  const float2 ke = f2c(eps);
  float2 ib[3], al[3];
  const float dk[3] = {0.1f, 0.6f, 0.3f};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ib[k] = f2rcp(__fadd2_rn(ke, b[k]));
    al[k] = __fmul2_rn(__fmul2_rn(f2c(dk[k]), ib[k]), ib[k]);
  }
  const float2 S = __fadd2_rn(__fadd2_rn(al[0], al[1]), al[2]);
  const float2 iS = f2rcp(S);
  const float2 I = __fmul2_rn(__ffma2_rn(al[0], v[0], __ffma2_rn(al[1], v[1], __fmul2_rn(al[2], v[2]))), iS);
  float2 w[3], cb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    w[k] = __fmul2_rn(al[k], iS);
    // (v_k - I)/S (-2 alpha_k / (eps + beta_k))
    cb[k] = __fmul2_rn(__fmul2_rn(__ffma2_rn(f2c(-1.0f), I, v[k]), iS),
                       __fmul2_rn(__fmul2_rn(f2c(-2.0f), al[k]), ib[k]));
  }
  // g_j = sum_k w_k dv_k/dq_j + cb_k dbeta_k/dq_j (zero entries skipped)
  g[0] = __ffma2_rn(w[0], f2c(1.0f / 3.0f), __fmul2_rn(cb[0], db[0][0]));
  g[1] = __ffma2_rn(w[0], f2c(-7.0f / 6.0f), __ffma2_rn(w[1], f2c(-1.0f / 6.0f),
         __ffma2_rn(cb[0], db[0][1], __fmul2_rn(cb[1], db[1][1]))));
  g[2] = __ffma2_rn(w[0], f2c(11.0f / 6.0f), __ffma2_rn(w[1], f2c(5.0f / 6.0f),
         __ffma2_rn(w[2], f2c(1.0f / 3.0f), __ffma2_rn(cb[0], db[0][2],
         __ffma2_rn(cb[1], db[1][2], __fmul2_rn(cb[2], db[2][2]))))));
  g[3] = __ffma2_rn(w[1], f2c(1.0f / 3.0f), __ffma2_rn(w[2], f2c(5.0f / 6.0f),
         __ffma2_rn(cb[1], db[1][3], __fmul2_rn(cb[2], db[2][3]))));
  g[4] = __ffma2_rn(w[2], f2c(-1.0f / 6.0f), __fmul2_rn(cb[2], db[2][4]));
  return I;
}

// Both WENO5 states that the five-cell window q[0..4] (cells c-2 .. c+2 along a direction)
// produces, with their gradients (FP64 adjoint): QL, the left state of face c+1/2 (the window
// in order), and QR, the right state of face c-1/2 (the window reversed). gL[t] = dQL/dq[t]
// and gR[t] = dQR/dq[4-t], the gradient in the reversed window's own order as weno5_grad
// returns it. The mirrored window visits the same three sub-stencils in reverse order, so the
// smoothness indicators and their derivatives are formed once; the linear weights swap ends
// (0.3, 0.6, 0.1 over the sub-stencils in the window's order). The normalised Jiang-Shu
// weights of both states, and 1/(eps + beta_k) in the indicator terms of the gradients, come
// from one reciprocal through a common denominator: with e_k = eps + beta_k, m_k the product
// of the other two e and P = e0 e1 e2, alpha_k = d_k m_k^2 / P^2 and 1/e_k = m_k / P.
template <class R>
__device__ __forceinline__ void weno5_pair_grad(const R q[5], R eps, R &QL, R &QR, R gL[5],
                                                R gR[5]) {
  // sub-stencils A = (q0, q1, q2), B = (q1, q2, q3), C = (q2, q3, q4)
  const R tA = q[0] - R(2) * q[1] + q[2], sA = q[0] - R(4) * q[1] + R(3) * q[2];
  const R tB = q[1] - R(2) * q[2] + q[3], sB = q[1] - q[3];
  const R tC = q[2] - R(2) * q[3] + q[4], sC = R(3) * q[2] - R(4) * q[3] + q[4];
  // eps + beta and d beta / d q are both taken 12/13 times (beta = t^2 + 3/13 s^2 against
  // eps 12/13) and the linear weights 10 times: the weights w_k do not change, and each
  // indicator term below pairs a 13/12 larger factor 1 / e_k with a 12/13 smaller d beta
  constexpr R k3 = R(3.0 / 13.0);
  eps *= R(12.0 / 13.0);
  const R e0 = fma(tA, tA, fma(k3 * sA, sA, eps));
  const R e1 = fma(tB, tB, fma(k3 * sB, sB, eps));
  const R e2 = fma(tC, tC, fma(k3 * sC, sC, eps));
  // d beta / d q over each sub-stencil's own cells, but for the centre q2 (see below)
  const R dA0 = R(2) * tA + R(6.0 / 13.0) * sA, dA1 = R(-4) * tA - R(24.0 / 13.0) * sA;
  const R dB1 = R(2) * tB + R(6.0 / 13.0) * sB;
  const R dB3 = R(2) * tB - R(6.0 / 13.0) * sB;
  const R dC3 = R(-4) * tC - R(24.0 / 13.0) * sC;
  const R dC4 = R(2) * tC + R(6.0 / 13.0) * sC;
  const R m0 = e1 * e2, m1 = e0 * e2, m2 = e0 * e1, P = e0 * m0;
  const R s0 = m0 * m0, s1 = m1 * m1, s2 = m2 * m2;
  const R nL0 = s0, n1 = R(6) * s1, nL2 = R(3) * s2;
  const R nR0 = R(3) * s0, nR2 = s2;
  const R nL1 = n1, nR1 = n1;
  const R AL = nL0 + n1 + nL2, AR = nR0 + n1 + nR2;
  R iAL, iAR, iP;
  const R Z = adj_rcp<R>(AL * AR * P);  // NaN outside the normal range: the test below fails
  bool finite_pos;
  if constexpr (sizeof(R) == 8) {
    // 0 < Z < infinity (and not a NaN) from the high word, off the FP64 pipe: sign clear,
    // exponent below all ones, not zero (a Z below 2^-1022 takes the division path)
    finite_pos = (unsigned)__double2hiint(double(Z)) - 1u < 0x7fefffffu;
  } else {
    finite_pos = Z > R(0) && Z < R(INFINITY);
  }
  if (finite_pos) {
    iAL = AR * P * Z;
    iAR = AL * P * Z;
    iP = AL * AR * Z;
  } else {  // the triple product left the exponent range (a tiny eps): one division each
    iAL = R(1) / AL;
    iAR = R(1) / AR;
    iP = R(1) / P;
  }
  const R wL0 = nL0 * iAL, wL1 = nL1 * iAL, wL2 = nL2 * iAL;
  const R wR0 = nR0 * iAR, wR1 = nR1 * iAR, wR2 = nR2 * iAR;
  // candidates as offsets from the centre value q2, from the same second differences t and
  // first-difference combinations s as the indicators: the left state's on A, B, C are
  // q2 + t/12 + s/4, q2 + t/12 - s/4, q2 + t/12 - s/4; the right state's q2 + t/12 - s/4,
  // q2 + t/12 + s/4, q2 + t/12 + s/4
  const R SA = sA * R(0.25), SB = sB * R(0.25), SC = sC * R(0.25);
  const R dL0 = fma(tA, R(1.0 / 12.0), SA), dL1 = fma(tB, R(1.0 / 12.0), -SB);
  const R dL2 = fma(tC, R(1.0 / 12.0), -SC);
  const R dR0 = fma(tA, R(1.0 / 12.0), -SA), dR1 = fma(tB, R(1.0 / 12.0), SB);
  const R dR2 = fma(tC, R(1.0 / 12.0), SC);
  const R DL = wL0 * dL0 + wL1 * dL1 + wL2 * dL2, DR = wR0 * dR0 + wR1 * dR1 + wR2 * dR2;
  QL = q[2] + DL;
  QR = q[2] + DR;
  // indicator terms: (v_k - Q) dw_k/dbeta_k = -2 (v_k - Q) w_k / e_k
  const R m2iP = R(-2) * iP;
  const R cL0 = (dL0 - DL) * wL0 * m0 * m2iP, cL1 = (dL1 - DL) * wL1 * m1 * m2iP;
  const R cL2 = (dL2 - DL) * wL2 * m2 * m2iP;
  const R cR0 = (dR0 - DR) * wR0 * m0 * m2iP, cR1 = (dR1 - DR) * wR1 * m1 * m2iP;
  const R cR2 = (dR2 - DR) * wR2 * m2 * m2iP;
  gL[0] = wL0 * R(1.0 / 3.0) + cL0 * dA0;
  gL[1] = wL0 * R(-7.0 / 6.0) + wL1 * R(-1.0 / 6.0) + cL0 * dA1 + cL1 * dB1;
  gL[3] = wL1 * R(1.0 / 3.0) + wL2 * R(5.0 / 6.0) + cL1 * dB3 + cL2 * dC3;
  gL[4] = wL2 * R(-1.0 / 6.0) + cL2 * dC4;
  // dQR/dq[t], stored at gR[4 - t]
  gR[4] = wR0 * R(-1.0 / 6.0) + cR0 * dA0;
  gR[3] = wR0 * R(5.0 / 6.0) + wR1 * R(1.0 / 3.0) + cR0 * dA1 + cR1 * dB1;
  gR[1] = wR1 * R(-1.0 / 6.0) + wR2 * R(-7.0 / 6.0) + cR1 * dB3 + cR2 * dC3;
  gR[0] = wR2 * R(1.0 / 3.0) + cR2 * dC4;
  // a constant added to the whole window shifts each state by that constant (the indicators
  // do not change), so each gradient sums to one: the centre entries follow from the others
  gL[2] = R(1) - ((gL[0] + gL[1]) + (gL[3] + gL[4]));
  gR[2] = R(1) - ((gR[0] + gR[1]) + (gR[3] + gR[4]));
}

// Transpose of mix_factors<>: adds the adjoint of (num, den) to the tracer entries of Xb.
template <class R, class L>
__device__ __forceinline__ void mix_factors_adj(const CstT<R> &C, R numb, R denb, R *Xb) {
#pragma unroll
  for (int i = 0; i < L::NVAP; ++i) {
    Xb[1 + i] += numb * C.sigv_m1[i] + denb * C.ieps_m1[i];
#pragma unroll
    for (int j = 0; j < L::NCOND; ++j) Xb[L::cond(i, j)] += numb * C.sigc_m1[i][j] - denb;
  }
}

static __device__ __forceinline__ float adj_rsqrt(float x) { return rsqrtf(x); }
static __device__ __forceinline__ double adj_rsqrt(double x) { return rsqrt(x); }

// Transpose of lmars<>: accumulates XLb, XRb from Fb (forward values recomputed first, then
// each assignment of lmars<> reversed in the opposite order). Each side's sound speed comes
// from one reciprocal square root r = (gamma p rho)^(-1/2): c = gamma p r, and the factors of
// its derivative follow without further division, dc/dp = gamma r / 2, dc/drho = -c^2 r / 2
// (1/rho = c r) and dc/dgamma = p r / 2; the star-state terms share one reciprocal of rho c.
template <class R, class L>
__device__ __forceinline__ void lmars_adj(const CstT<R> &C, const R *XL, const R *XR, int dir,
                                          R pref, const R *Fb, R *XLb, R *XRb) {
  constexpr int NV = L::NV, IE = L::IE, IM0 = L::IM0, NM = L::NMOM;
  const int mn = L::mom(dir);
  const R gm1 = C.gm1, igm1 = C.igm1;
  R numL, denL, numR, denR;
  mix_factors<R, L>(C, XL, numL, denL);
  mix_factors<R, L>(C, XR, numR, denR);
  const R pL = pref + XL[IE], pR = pref + XR[IE];
  R gamL, gamR, inL = R(1), inR = R(1);
  if constexpr (L::NVAP == 0) {
    gamL = gamR = C.gamma_d;
  } else {
    inL = Ar<R>::rcp(numL);
    inR = Ar<R>::rcp(numR);
    gamL = R(1) + gm1 * (denL * inL);
    gamR = R(1) + gm1 * (denR * inR);
  }
  const R rsL = adj_rsqrt(gamL * pL * XL[0]), rsR = adj_rsqrt(gamR * pR * XR[0]);
  const R cL = gamL * pL * rsL, cR = gamR * pR * rsR;
  const R rhoc = R(0.5) * (XL[0] + XR[0]) * R(0.5) * (cL + cR);
  const R irc = Ar<R>::rcp(rhoc), i2rc = R(0.5) * irc;
  const R uL = XL[mn], uR = XR[mn];
  const R us = R(0.5) * (uL + uR) - (XR[IE] - XL[IE]) * i2rc;
  R usb = R(0), numLb = R(0), denLb = R(0), numRb = R(0), denRb = R(0);
  const R psb = Fb[mn];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const bool use_left = side == 0;
    const R wgt = us > R(0) ? (use_left ? R(1) : R(0))
                            : (us < R(0) ? (use_left ? R(0) : R(1)) : R(0.5));
    if (wgt == R(0)) continue;
    R XS[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) XS[v] = use_left ? XL[v] : XR[v];
    const R numS = use_left ? numL : numR, denS = use_left ? denL : denR;
    const R pS = use_left ? pL : pR, rhoS = XS[0], mf = us * rhoS;
    R qsum = R(0), u2 = R(0), muq = R(0);
#pragma unroll
    for (int t = 1; t < IM0; ++t) qsum += XS[t];
#pragma unroll
    for (int m = 0; m < NM; ++m) u2 += XS[IM0 + m] * XS[IM0 + m];
#pragma unroll
    for (int i = 0; i < L::NVAP; ++i)
#pragma unroll
      for (int j = 0; j < L::NCOND; ++j) muq += C.mu[i][j] * XS[L::cond(i, j)];
    const R K = R(0.5) * rhoS * u2;
    R rS = R(1), iden = R(1);
    if constexpr (L::NVAP > 0) {
      iden = Ar<R>::rcp(denS);
      rS = numS * iden;
    }
    const R rhoe = rS * pS * igm1 + K + rhoS * muq;
    // F[E] = u* (rho e + p_S), rho e = (num/den) p_S / (gamma_d - 1) + K + A
    usb += wgt * Fb[IE] * (rhoe + pS);
    const R rhoeb = wgt * Fb[IE] * us;
    const R pSb = rhoeb + rhoeb * rS * igm1;
    if constexpr (L::NVAP > 0) {
      const R rb = rhoeb * pS * igm1;
      if (use_left) {
        numLb += rb * iden;
        denLb -= rb * numS * iden * iden;
      } else {
        numRb += rb * iden;
        denRb -= rb * numS * iden * iden;
      }
    }
    R rhoSb = rhoeb * (R(0.5) * u2 + muq);
    R bS[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) bS[v] = R(0);
#pragma unroll
    for (int i = 0; i < L::NVAP; ++i)
#pragma unroll
      for (int j = 0; j < L::NCOND; ++j) bS[L::cond(i, j)] += rhoeb * rhoS * C.mu[i][j];
    // F[t] = mf q_t, F[0] = mf (1 - sum q), F[m] = mf u_m, mf = u* rho_S
    R mfb = Fb[0] * (R(1) - qsum);
#pragma unroll
    for (int t = 1; t < IM0; ++t) {
      mfb += Fb[t] * XS[t];
      bS[t] += wgt * (Fb[t] - Fb[0]) * mf;
    }
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      mfb += Fb[IM0 + m] * XS[IM0 + m];
      bS[IM0 + m] += wgt * Fb[IM0 + m] * mf + rhoeb * rhoS * XS[IM0 + m];
    }
    usb += wgt * mfb * rhoS;
    rhoSb += wgt * mfb * us;
    bS[0] += rhoSb;
    bS[IE] += pSb;
    if (use_left) {
#pragma unroll
      for (int v = 0; v < NV; ++v) XLb[v] += bS[v];
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) XRb[v] += bS[v];
    }
  }
  R rhocb = R(0);
  XLb[mn] += R(0.5) * usb;
  XRb[mn] += R(0.5) * usb;
  XRb[IE] -= usb * i2rc;
  XLb[IE] += usb * i2rc;
  rhocb += usb * (XR[IE] - XL[IE]) * i2rc * irc;
  XLb[IE] += R(0.5) * psb;
  XRb[IE] += R(0.5) * psb;
  rhocb -= R(0.5) * (uR - uL) * psb;
  XRb[mn] -= R(0.5) * rhoc * psb;
  XLb[mn] += R(0.5) * rhoc * psb;
  XLb[0] += R(0.25) * (cL + cR) * rhocb;
  XRb[0] += R(0.25) * (cL + cR) * rhocb;
  const R cb = R(0.25) * (XL[0] + XR[0]) * rhocb;
  const R hL = R(0.5) * cb * rsL, hR = R(0.5) * cb * rsR;
  XLb[IE] += hL * gamL;
  XLb[0] -= hL * cL * cL;
  XRb[IE] += hR * gamR;
  XRb[0] -= hR * cR * cR;
  if constexpr (L::NVAP > 0) {
    // gamma = 1 + (gamma_d - 1) den / num
    const R gLb = hL * pL, gRb = hR * pR;
    denLb += gLb * gm1 * inL;
    numLb -= gLb * gm1 * denL * inL * inL;
    denRb += gRb * gm1 * inR;
    numRb -= gRb * gm1 * denR * inR * inR;
    mix_factors_adj<R, L>(C, numLb, denLb, XLb);
    mix_factors_adj<R, L>(C, numRb, denRb, XRb);
  }
}

// Adjoint of face f of direction DIR (face index in [nz'][ny'][nx'] order of that direction).
template <class R, class L, int DIR>
__device__ __forceinline__ void adj_face(const AdjArgs &a, const DomDev &D, const CstT<R> &C,
                                         long long f) {
  constexpr int NV = L::NV, MN = L::mom(DIR);
  constexpr int fx = DIR == 0, fy = DIR == 1, fz = DIR == 2;
  const int nx = D.nx, ny = D.ny, nz = D.nz;
  const long long ncell = D.ncell;
  const int nfx = nx + fx, nfy = ny + fy;
  const long long nf = (long long)nfx * nfy * (nz + fz);
  const R *Ys = reinterpret_cast<const R *>(a.Ys);
  const R *lo = reinterpret_cast<const R *>(a.lam_out);
  R *G = reinterpret_cast<R *>(a.G[DIR]);
  const R bdt = R(a.b * a.dt), bih = bdt * Prof<R>::ih(D, DIR);
  const R hgb = fz ? R(0.5) * Prof<R>::grav(D) * bdt : R(0);
  const int nd = DIR == 0 ? nx : (DIR == 1 ? ny : nz);
  const int bclo = D.bc[2 * DIR], bchi = D.bc[2 * DIR + 1];
  const int i = int(f % nfx), j = int((f / nfx) % nfy), k = int(f / ((long long)nfx * nfy));
  const int pos = DIR == 0 ? i : (DIR == 1 ? j : k);
  // Fbar = (mu_right - mu_left) / h with mu = b dt lam_out, plus the gravity-energy term
  R Fb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Fb[v] = R(0);
  R Fbz = R(0);
  if (pos > 0) {
    const long long c = ((long long)(k - fz) * ny + (j - fy)) * nx + (i - fx);
#pragma unroll
    for (int v = 0; v < NV; ++v) Fb[v] -= bih * lo[v * ncell + c];
    if (fz) Fbz -= hgb * lo[L::IE * ncell + c];
  }
  if (pos < nd) {
    const long long c = ((long long)k * ny + j) * nx + i;
#pragma unroll
    for (int v = 0; v < NV; ++v) Fb[v] += bih * lo[v * ncell + c];
    if (fz) Fbz -= hgb * lo[L::IE * ncell + c];
  }
  if (fz) {
#pragma unroll
    for (int s = 0; s < L::IM0; ++s) Fb[s] += Fbz;
  }
  // stencil primitives, cells pos-3 .. pos+2 along DIR (ghosts mirrored or wrapped)
  R X[6][NV];
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    bool flip = false;
    const int p = map_index(pos - 3 + s, nd, bclo, bchi, flip);
    const int ci = fx ? p : i, cj = fy ? p : j, ck = fz ? p : k;
    const long long c = ((long long)ck * ny + cj) * nx + ci;
    R y[NV], pt, Tt;
#pragma unroll
    for (int v = 0; v < NV; ++v) y[v] = Ys[v * ncell + c];
    cons_to_prim<R, L>(a.ph, C, D, ck, y, X[s], pt, Tt);
    if (flip) X[s][MN] = -X[s][MN];
  }
  R QL[NV], QR[NV], gL[NV][5], gR[NV][5], QLb[NV], QRb[NV];
  const R weps = C.weno_eps;
  constexpr int NPACK = sizeof(R) == 4 ? NV / 2 * 2 : 0;  // variables done in FP32x2 pairs
  if constexpr (NPACK > 0) {
#pragma unroll
    for (int v = 0; v < NPACK; v += 2) {
      float2 q[5], g[5], I;
#pragma unroll
      for (int s = 0; s < 5; ++s) q[s] = make_float2(X[s][v], X[s][v + 1]);
      I = weno5_grad2(q, weps, g);
      QL[v] = I.x;
      QL[v + 1] = I.y;
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        gL[v][s] = g[s].x;
        gL[v + 1][s] = g[s].y;
      }
#pragma unroll
      for (int s = 0; s < 5; ++s) q[s] = make_float2(X[5 - s][v], X[5 - s][v + 1]);
      I = weno5_grad2(q, weps, g);
      QR[v] = I.x;
      QR[v + 1] = I.y;
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        gR[v][s] = g[s].x;
        gR[v + 1][s] = g[s].y;
      }
    }
  }
#pragma unroll
  for (int v = NPACK; v < NV; ++v) {
    R q[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) q[s] = X[s][v];
    QL[v] = weno5_grad<R>(q, weps, gL[v]);
#pragma unroll
    for (int s = 0; s < 5; ++s) q[s] = X[5 - s][v];
    QR[v] = weno5_grad<R>(q, weps, gR[v]);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) QLb[v] = QRb[v] = R(0);
  const R pref = fz ? Prof<R>::pf(D, k) : Prof<R>::pc(D, k);
  lmars_adj<R, L>(C, QL, QR, DIR, pref, Fb, QLb, QRb);
  constexpr int NVP = g_stride<R, NV>(), W = GVec<R>::W;
  using Vec = typename GVec<R>::V;
  Vec *Gf = reinterpret_cast<Vec *>(G + f * 6 * NVP);
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    R g[NVP];
#pragma unroll
    for (int v = 0; v < NVP; ++v) {
      g[v] = R(0);
      if (v < NV) {
        if (s <= 4) g[v] += QLb[v] * gL[v][s];
        if (s >= 1) g[v] += QRb[v] * gR[v][5 - s];
      }
    }
#pragma unroll
    for (int c = 0; c < NVP / W; ++c) Gf[s * (NVP / W) + c] = GVec<R>::make(g + c * W);
  }
  (void)nf;
}

// One thread per face; the faces of x, then y (3-D), then z.
template <class R, class L>
__global__ void __launch_bounds__(128, (sizeof(R) == 4 && !L::MOIST && !L::D3) ? 7 : 0)
    adj_face_kernel(const AdjArgs a) {
  const DomDev &D = a.doms[0];
  const CstT<R> &C = acst<R>(a);
  const int nx = D.nx, ny = D.ny, nz = D.nz;
  const long long n0 = (long long)(nx + 1) * ny * nz;
  const long long n1 = L::D3 ? (long long)nx * (ny + 1) * nz : 0ll;
  const long long ntot = n0 + n1 + (long long)nx * ny * (nz + 1);
  for (long long gf = blockIdx.x * (long long)blockDim.x + threadIdx.x; gf < ntot;
       gf += (long long)gridDim.x * blockDim.x) {
    if (gf < n0) {
      adj_face<R, L, 0>(a, D, C, gf);
    } else if (L::D3 && gf < n0 + n1) {
      if constexpr (L::D3) adj_face<R, L, 1>(a, D, C, gf - n0);
    } else {
      adj_face<R, L, 2>(a, D, C, gf - n0 - n1);
    }
  }
}

// ---- FP64 path: window-centred WENO transpose ------------------------------------------
// On the FP64 pipe the face kernel above is bound by arithmetic, most of it the two WENO5
// gradients of each face, whose windows (centred on the two cells beside the face) are each
// evaluated twice over the grid, and six primitive conversions per face. The FP64 adjoint
// splits the work: adj_prim_kernel converts every cell once; adj_weno_kernel evaluates every
// window once (both of its states, weno5_pair_grad); adj_face_w_kernel transposes LMARS at
// each face from the stored states and writes the same G as adj_face_kernel.

// Window centres of direction DIR: the cells -1 .. n_d along DIR (a ghost centre at each end
// holds the window of a boundary face's outer state), all cells across.
template <int DIR>
__device__ __forceinline__ long long n_centres(const DomDev &D) {
  return (long long)(D.nx + 2 * (DIR == 0)) * (D.ny + 2 * (DIR == 1)) * (D.nz + 2 * (DIR == 2));
}

template <class R, class L>
__global__ void __launch_bounds__(128) adj_prim_kernel(const AdjArgs a) {
  constexpr int NV = L::NV;
  const DomDev &D = a.doms[0];
  const CstT<R> &C = acst<R>(a);
  const long long ncell = D.ncell, plane = (long long)D.nx * D.ny;
  const R *Ys = reinterpret_cast<const R *>(a.Ys);
  R *X = reinterpret_cast<R *>(a.X);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    R y[NV], x[NV], pt, Tt;
#pragma unroll
    for (int v = 0; v < NV; ++v) y[v] = Ys[v * ncell + c];
    cons_to_prim<R, L>(a.ph, C, D, int(c / plane), y, x, pt, Tt);
#pragma unroll
    for (int v = 0; v < NV; ++v) X[v * ncell + c] = x[v];
  }
}

// Window centre e of direction DIR: reads the primitives of cells pos-2 .. pos+2 (ghosts
// mirrored, the normal velocity negated, or wrapped) and writes, per field v, at W[q][e]:
// q = v the left state of face pos+1/2, NV + v the right state of face pos-1/2, 2 NV + t NV + v
// the left state's gradient gL[t], 7 NV + t NV + v the right state's gR[t].
template <class R, class L, int DIR>
__device__ __forceinline__ void adj_window(const AdjArgs &a, const DomDev &D, long long e) {
  constexpr int NV = L::NV, MN = L::mom(DIR);
  constexpr int fx = DIR == 0, fy = DIR == 1, fz = DIR == 2;
  const int nx = D.nx, ny = D.ny;
  const int ex = nx + 2 * fx, ey = ny + 2 * fy;
  const int i = int(e % ex), j = int((e / ex) % ey), k = int(e / ((long long)ex * ey));
  const int pos = (DIR == 0 ? i : (DIR == 1 ? j : k)) - 1;
  const int nd = DIR == 0 ? nx : (DIR == 1 ? ny : D.nz);
  const int bclo = D.bc[2 * DIR], bchi = D.bc[2 * DIR + 1];
  const long long ncell = D.ncell, nc = n_centres<DIR>(D);
  const R *X = reinterpret_cast<const R *>(a.X);
  R *W = reinterpret_cast<R *>(a.W[DIR]);
  long long cs[5];
  bool fl[5];
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    const int p = map_index(pos - 2 + t, nd, bclo, bchi, fl[t]);
    const int ci = fx ? p : i, cj = fy ? p : j, ck = fz ? p : k;
    cs[t] = ((long long)ck * ny + cj) * nx + ci;
  }
  const R weps = acst<R>(a).weno_eps;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    R q[5], QL, QR, gL[5], gR[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      const R x = X[v * ncell + cs[t]];
      q[t] = (v == MN && fl[t]) ? -x : x;
    }
    weno5_pair_grad<R>(q, weps, QL, QR, gL, gR);
    W[v * nc + e] = QL;
    W[(NV + v) * nc + e] = QR;
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      W[(2 * NV + t * NV + v) * nc + e] = gL[t];
      W[(7 * NV + t * NV + v) * nc + e] = gR[t];
    }
  }
}

template <class R, class L>
__global__ void __launch_bounds__(128) adj_weno_kernel(const AdjArgs a) {
  const DomDev &D = a.doms[0];
  const long long n0 = n_centres<0>(D), n1 = L::D3 ? n_centres<1>(D) : 0ll;
  const long long ntot = n0 + n1 + n_centres<2>(D);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ntot;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < n0) {
      adj_window<R, L, 0>(a, D, e);
    } else if (L::D3 && e < n0 + n1) {
      if constexpr (L::D3) adj_window<R, L, 1>(a, D, e - n0);
    } else {
      adj_window<R, L, 2>(a, D, e - n0 - n1);
    }
  }
}

// Face f of direction DIR from the stored window results: the left state comes from the
// window centred on cell pos-1, the right state from the one centred on cell pos.
template <class R, class L, int DIR>
__device__ __forceinline__ void adj_face_w(const AdjArgs &a, const DomDev &D, const CstT<R> &C,
                                           long long f) {
  constexpr int NV = L::NV;
  constexpr int fx = DIR == 0, fy = DIR == 1, fz = DIR == 2;
  const int nx = D.nx, ny = D.ny, nz = D.nz;
  const long long ncell = D.ncell, nc = n_centres<DIR>(D);
  const int nfx = nx + fx, nfy = ny + fy;
  const R *lo = reinterpret_cast<const R *>(a.lam_out);
  const R *Wd = reinterpret_cast<const R *>(a.W[DIR]);
  R *G = reinterpret_cast<R *>(a.G[DIR]);
  const R bdt = R(a.b * a.dt), bih = bdt * Prof<R>::ih(D, DIR);
  const R hgb = fz ? R(0.5) * Prof<R>::grav(D) * bdt : R(0);
  const int nd = DIR == 0 ? nx : (DIR == 1 ? ny : nz);
  const int i = int(f % nfx), j = int((f / nfx) % nfy), k = int(f / ((long long)nfx * nfy));
  const int pos = DIR == 0 ? i : (DIR == 1 ? j : k);
  R Fb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Fb[v] = R(0);
  R Fbz = R(0);
  if (pos > 0) {
    const long long c = ((long long)(k - fz) * ny + (j - fy)) * nx + (i - fx);
#pragma unroll
    for (int v = 0; v < NV; ++v) Fb[v] -= bih * lo[v * ncell + c];
    if (fz) Fbz -= hgb * lo[L::IE * ncell + c];
  }
  if (pos < nd) {
    const long long c = ((long long)k * ny + j) * nx + i;
#pragma unroll
    for (int v = 0; v < NV; ++v) Fb[v] += bih * lo[v * ncell + c];
    if (fz) Fbz -= hgb * lo[L::IE * ncell + c];
  }
  if (fz) {
#pragma unroll
    for (int s = 0; s < L::IM0; ++s) Fb[s] += Fbz;
  }
  // centre index of the window on cell pos-1; the one on cell pos is a stride further
  const int ex = nx + 2 * fx, ey = ny + 2 * fy;
  const long long eL = ((long long)k * ey + j) * ex + i;
  const long long eR = eL + (DIR == 0 ? 1ll : (DIR == 1 ? (long long)ex : (long long)ex * ey));
  R QL[NV], QR[NV], QLb[NV], QRb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    QL[v] = Wd[v * nc + eL];
    QR[v] = Wd[(NV + v) * nc + eR];
    QLb[v] = QRb[v] = R(0);
  }
  const R pref = fz ? Prof<R>::pf(D, k) : Prof<R>::pc(D, k);
  lmars_adj<R, L>(C, QL, QR, DIR, pref, Fb, QLb, QRb);
  constexpr int NVP = g_stride<R, NV>(), W = GVec<R>::W;
  using Vec = typename GVec<R>::V;
  Vec *Gf = reinterpret_cast<Vec *>(G + f * 6 * NVP);
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    R g[NVP];
#pragma unroll
    for (int v = 0; v < NVP; ++v) {
      g[v] = R(0);
      if (v < NV) {
        if (s <= 4) g[v] += QLb[v] * Wd[(2 * NV + s * NV + v) * nc + eL];
        if (s >= 1) g[v] += QRb[v] * Wd[(7 * NV + (5 - s) * NV + v) * nc + eR];
      }
    }
#pragma unroll
    for (int c = 0; c < NVP / W; ++c) Gf[s * (NVP / W) + c] = GVec<R>::make(g + c * W);
  }
}

template <class R, class L>
__global__ void __launch_bounds__(128) adj_face_w_kernel(const AdjArgs a) {
  const DomDev &D = a.doms[0];
  const CstT<R> &C = acst<R>(a);
  const int nx = D.nx, ny = D.ny, nz = D.nz;
  const long long n0 = (long long)(nx + 1) * ny * nz;
  const long long n1 = L::D3 ? (long long)nx * (ny + 1) * nz : 0ll;
  const long long ntot = n0 + n1 + (long long)nx * ny * (nz + 1);
  for (long long gf = blockIdx.x * (long long)blockDim.x + threadIdx.x; gf < ntot;
       gf += (long long)gridDim.x * blockDim.x) {
    if (gf < n0) {
      adj_face_w<R, L, 0>(a, D, C, gf);
    } else if (L::D3 && gf < n0 + n1) {
      if constexpr (L::D3) adj_face_w<R, L, 1>(a, D, C, gf - n0);
    } else {
      adj_face_w<R, L, 2>(a, D, C, gf - n0 - n1);
    }
  }
}

// Adds to Xb the contributions of the faces of direction DIR whose stencil slot holds the
// position ipos along DIR (the cell itself or a ghost image of it), with the normal velocity
// entry multiplied by sg (-1 for a mirror image).
template <class R, class L, int DIR>
__device__ __forceinline__ void gather_image(const AdjArgs &a, const DomDev &D, int i, int j,
                                             int k, int ipos, R sg, R (&Xb)[L::NV]) {
  constexpr int fx = DIR == 0, fy = DIR == 1, fz = DIR == 2, MN = L::mom(DIR);
  const int nx = D.nx, ny = D.ny, nz = D.nz;
  const int nfx = nx + fx, nfy = ny + fy;
  const long long nf = (long long)nfx * nfy * (nz + fz);
  const int nd = DIR == 0 ? nx : (DIR == 1 ? ny : nz);
  constexpr int NVP = g_stride<R, L::NV>(), W = GVec<R>::W;
  using Vec = typename GVec<R>::V;
  const Vec *G = reinterpret_cast<const Vec *>(a.G[DIR]);
  (void)nf;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const int fpos = ipos + 3 - s;  // face whose stencil slot s is this position
    if (fpos < 0 || fpos > nd) continue;
    const int fi = fx ? fpos : i, fj = fy ? fpos : j, fk = fz ? fpos : k;
    const long long f = ((long long)fk * nfy + fj) * nfx + fi;
#pragma unroll
    for (int c = 0; c < NVP / W; ++c) {
      const Vec gv = G[(f * 6 + s) * (NVP / W) + c];
#pragma unroll
      for (int e = 0; e < W; ++e) {
        const int v = c * W + e;
        if (v < L::NV) {
          const R g = GVec<R>::get(gv, e);
          Xb[v] += v == MN ? sg * g : g;
        }
      }
    }
  }
}

template <class R, class L, int DIR>
__device__ __forceinline__ void gather_dir(const AdjArgs &a, const DomDev &D, int i, int j,
                                           int k, R (&Xb)[L::NV]) {
  const int nd = DIR == 0 ? D.nx : (DIR == 1 ? D.ny : D.nz);
  const int pos = DIR == 0 ? i : (DIR == 1 ? j : k);
  const int bclo = D.bc[2 * DIR], bchi = D.bc[2 * DIR + 1];
  gather_image<R, L, DIR>(a, D, i, j, k, pos, R(1), Xb);
  // ghost images within three cells of a boundary: a periodic copy, or a mirror image
  if (bclo == 1) {
    if (pos - nd >= -3) gather_image<R, L, DIR>(a, D, i, j, k, pos - nd, R(1), Xb);
  } else if (pos <= 2) {
    gather_image<R, L, DIR>(a, D, i, j, k, -1 - pos, R(-1), Xb);
  }
  if (bchi == 1) {
    if (pos + nd <= nd + 2) gather_image<R, L, DIR>(a, D, i, j, k, pos + nd, R(1), Xb);
  } else if (pos >= nd - 3) {
    gather_image<R, L, DIR>(a, D, i, j, k, 2 * nd - 1 - pos, R(-1), Xb);
  }
}

template <class R, class L>
__global__ void __launch_bounds__(128) adj_cell_kernel(const AdjArgs a) {
  constexpr int NV = L::NV, IE = L::IE, IM0 = L::IM0;
  const DomDev &D = a.doms[0];
  const CstT<R> &C = acst<R>(a);
  const int nx = D.nx, ny = D.ny;
  const long long ncell = D.ncell;
  const R *Ys = reinterpret_cast<const R *>(a.Ys);
  const R *lo = reinterpret_cast<const R *>(a.lam_out);
  R *ls = reinterpret_cast<R *>(a.lam_s);
  R *ln = reinterpret_cast<R *>(a.lam_n);
  // the forward combine is Y^n + b (s1 - Y^n): the weights of Y^n and s1 are 1 - b and b in
  // the kernel's type, summing to exactly one
  const R grav = Prof<R>::grav(D), bdt = R(a.b * a.dt), bv = R(a.b), av = R(1) - bv;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = int(c % nx), j = int((c / nx) % ny), k = int(c / ((long long)nx * ny));
    R Xb[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Xb[v] = R(0);
    gather_dir<R, L, 0>(a, D, i, j, k, Xb);
    if constexpr (L::D3) gather_dir<R, L, 1>(a, D, i, j, k, Xb);
    gather_dir<R, L, 2>(a, D, i, j, k, Xb);
    // transpose of the primitive map (App. B: rho, q_t = y_t / rho, u_m = y_m / rho,
    // p = (gamma_d - 1) (den/num) U with U = rho e - K - A) and of the gravity source
    R y[NV], Yb[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      y[v] = Ys[v * ncell + c];
      Yb[v] = R(0);
    }
    R rho = y[0];
#pragma unroll
    for (int t = 1; t < IM0; ++t) rho += y[t];
    const R ir = Ar<R>::rcp(rho);
    R u2 = R(0);
#pragma unroll
    for (int m = 0; m < L::NMOM; ++m) u2 += (y[IM0 + m] * ir) * (y[IM0 + m] * ir);
    const R pb = Xb[IE];
    R Ub = pb * C.gm1;
    R Qb[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) Qb[t] = t >= 1 && t < IM0 ? Xb[t] : R(0);
    if constexpr (L::NVAP > 0) {
      R x[NV], num, den, A = R(0);
#pragma unroll
      for (int t = 1; t < IM0; ++t) x[t] = y[t] * ir;
      mix_factors<R, L>(C, x, num, den);
#pragma unroll
      for (int i2 = 0; i2 < L::NVAP; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < L::NCOND; ++j2) A += C.mu[i2][j2] * y[L::cond(i2, j2)];
      const R U = (y[IE] + Prof<R>::er(D, k)) - R(0.5) * rho * u2 - A;
      const R inum = Ar<R>::rcp(num), rb = pb * C.gm1 * U;
      Ub = pb * C.gm1 * den * inum;
      mix_factors_adj<R, L>(C, -rb * den * inum * inum, rb * inum, Qb);
#pragma unroll
      for (int i2 = 0; i2 < L::NVAP; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < L::NCOND; ++j2) Yb[L::cond(i2, j2)] -= Ub * C.mu[i2][j2];
    }
    Yb[IE] += Ub;
    const R Kb = -Ub;
    R rhob = Xb[0] - Kb * R(0.5) * u2;
#pragma unroll
    for (int m = 0; m < L::NMOM; ++m) {
      const R u = y[IM0 + m] * ir;
      Yb[IM0 + m] += Kb * u + Xb[IM0 + m] * ir;
      rhob -= Xb[IM0 + m] * u * ir;
    }
#pragma unroll
    for (int t = 1; t < IM0; ++t) {
      Yb[t] += Qb[t] * ir;
      rhob -= Qb[t] * (y[t] * ir) * ir;
    }
    // momentum source -(rho - rho_bar) g on rho w, rho the sum of the densities
    rhob -= grav * bdt * lo[L::mom(2) * ncell + c];
#pragma unroll
    for (int t = 0; t < IM0; ++t) Yb[t] += rhob;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R l = lo[v * ncell + c];
      const R s = bv * l + Yb[v];
      if (a.mode == 2) {
        ln[v * ncell + c] = av * l;
        ls[v * ncell + c] = s;
      } else if (a.mode == 1) {
        ln[v * ncell + c] += av * l;
        ls[v * ncell + c] = s;
      } else {
        ls[v * ncell + c] = ln[v * ncell + c] + s;
      }
    }
  }
}

// Transpose of the saturation adjustment of one cell, in FP64, at its adjusted state y (the
// stage output): the adjustment converges to the equilibrium in which a vapour that keeps
// cloud holds rho*_i(T) = p*_i(T) / (R_i T) and its cloud the rest of the species total, a
// vapour without cloud the whole total; T follows from the conserved energy through
// F(T) = T C_v(T) + A(T) - (rho e - K) = 0. Hence dT/dy = -(dF/dy) / (dF/dT) with
// dF/dT = C_v + sum over saturated i of rho*_i' (T (c_vi - c_i1) - mu_i1) and, at fixed T,
// dF/dy = -1 (rho e), u_m (momenta), T c_vd - |u|^2/2 (rho_d), T c_i1 + mu_i1 - |u|^2/2
// (total of a saturated species), T c_vi - |u|^2/2 (an unsaturated one), T c_ij + mu_ij -
// |u|^2/2 (other condensates). lam (in place): (dY_out/dY_in)^T lam.
template <class R, class L>
__device__ __forceinline__ void satadj_adj_cell(const Phys &ph, const CstT<R> &C, const R *y,
                                                double eref, R *lam) {
  constexpr int NV = L::NV, IM0 = L::IM0;
  // T from the conserved energy in FP64 (the inversion cancels large terms); the derivative
  // itself in the kernel's type
  double Td, pd;
  cell_Tp<R, L>(ph, y, eref, Td, pd);
  const R T = R(Td), cvd = C.R_d * C.igm1;
  R rho = R(0), u2 = R(0), Cv = y[0];
#pragma unroll
  for (int s = 0; s < IM0; ++s) rho += y[s];
  const R ir = Ar<R>::rcp(rho);
#pragma unroll
  for (int m = 0; m < L::NMOM; ++m) u2 += (y[IM0 + m] * ir) * (y[IM0 + m] * ir);
#pragma unroll
  for (int i = 0; i < L::NVAP; ++i) {
    Cv += C.sig_v[i] * y[1 + i];
#pragma unroll
    for (int j = 0; j < L::NCOND; ++j) Cv += C.sig_c[i][j] * y[L::cond(i, j)];
  }
  Cv *= cvd;
  R dF[NV], li[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) li[v] = lam[v];
  dF[0] = T * cvd - R(0.5) * u2;
#pragma unroll
  for (int m = 0; m < L::NMOM; ++m) dF[IM0 + m] = y[IM0 + m] * ir;
  dF[L::IE] = R(-1);
  R dFdT = Cv, gT = R(0);
#pragma unroll
  for (int i = 0; i < L::NVAP; ++i) {
    const int vi = 1 + i, ci = L::cond(i, 0);
    const R c_v = C.sig_v[i] * cvd, c_c = C.sig_c[i][0] * cvd, mu_c = C.mu[i][0];
#pragma unroll
    for (int j = 1; j < L::NCOND; ++j)
      dF[L::cond(i, j)] = T * C.sig_c[i][j] * cvd + C.mu[i][j] - R(0.5) * u2;
    if (y[ci] > R(0)) {
      const R t = T * C.inv_Tref[i], it = Ar<R>::rcp(t), iT = Ar<R>::rcp(T);
      const R ps = C.pref[i] * Ar<R>::exp_(C.beta[i] * (R(1) - it) - C.delta[i] * Ar<R>::log_(t));
      const R rs = ps * C.eps[i] * C.iR_d * iT;  // p* / (R_i T), R_i = R_d / eps_i
      const R drs = rs * ((C.beta[i] * it - C.delta[i]) - R(1)) * iT;
      dFdT += drs * (T * (c_v - c_c) - mu_c);
      gT += drs * (lam[vi] - lam[ci]);
      dF[vi] = dF[ci] = T * c_c + mu_c - R(0.5) * u2;
      li[vi] = li[ci] = lam[ci];
    } else {
      dF[vi] = dF[ci] = T * c_v - R(0.5) * u2;
      li[vi] = li[ci] = lam[vi];
    }
  }
  const R coef = -gT * Ar<R>::rcp(dFdT);
#pragma unroll
  for (int v = 0; v < NV; ++v) lam[v] = li[v] + coef * dF[v];
}

// lam_s <- (dY_out / dY_in)^T lam_s of the adjustment, at the stage output a.Ys.
template <class R, class L>
__global__ void __launch_bounds__(128) adj_satadj_kernel(const AdjArgs a) {
  const DomDev &D = a.doms[0];
  const long long ncell = D.ncell, plane = (long long)D.nx * D.ny;
  const R *Yo = reinterpret_cast<const R *>(a.Ys);
  R *lam = reinterpret_cast<R *>(a.lam_s);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    R y[L::NV], l[L::NV];
#pragma unroll
    for (int v = 0; v < L::NV; ++v) {
      y[v] = Yo[v * ncell + c];
      l[v] = lam[v * ncell + c];
    }
    satadj_adj_cell<R, L>(a.ph, acst<R>(a), y, D.e_ref[c / plane], l);
#pragma unroll
    for (int v = 0; v < L::NV; ++v) lam[v * ncell + c] = l[v];
  }
}

template <class R, class L>
struct AdjFamily {
  // FP32: one face launch (latency-bound at the sizes an adjoint runs); FP64: primitives,
  // windows, then faces (see adj_weno_kernel)
  static cudaError_t face(const AdjArgs &a, long long nfaces, cudaStream_t s) {
    if constexpr (sizeof(R) == 8) {
      const long long ncell = (long long)a.nx * a.ny * a.nz;
      const long long ncent = (long long)(a.nx + 2) * a.ny * a.nz +
                              (L::D3 ? (long long)a.nx * (a.ny + 2) * a.nz : 0ll) +
                              (long long)a.nx * a.ny * (a.nz + 2);
      long long g = (ncell + 127) / 128;
      adj_prim_kernel<R, L><<<int(g < 9728 ? g : 9728), 128, 0, s>>>(a);
      g = (ncent + 127) / 128;
      adj_weno_kernel<R, L><<<int(g < 9728 ? g : 9728), 128, 0, s>>>(a);
      g = (nfaces + 127) / 128;
      adj_face_w_kernel<R, L><<<int(g < 9728 ? g : 9728), 128, 0, s>>>(a);
    } else {
      long long g = (nfaces + 127) / 128;
      adj_face_kernel<R, L><<<int(g < 9728 ? g : 9728), 128, 0, s>>>(a);
    }
    return cudaGetLastError();
  }
  static cudaError_t cell(const AdjArgs &a, long long ncell, cudaStream_t s) {
    long long g = (ncell + 127) / 128;
    adj_cell_kernel<R, L><<<int(g < 9728 ? g : 9728), 128, 0, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t satadj(const AdjArgs &a, long long ncell, cudaStream_t s) {
    long long g = (ncell + 127) / 128;
    adj_satadj_kernel<R, L><<<int(g < 9728 ? g : 9728), 128, 0, s>>>(a);
    return cudaGetLastError();
  }
  static AdjKernels get() {
    AdjKernels k;
    k.face = &face;
    k.cell = &cell;
    k.satadj = L::MOIST ? &satadj : nullptr;
    return k;
  }
};

}  // namespace snap
