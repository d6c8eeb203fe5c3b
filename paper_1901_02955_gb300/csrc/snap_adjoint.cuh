// snap_adjoint.cuh -- discrete adjoint of one Runge-Kutta stage of the dry, inviscid step
// (the transpose of stage_tiles in snap_stage.cuh): reverse of the SSP-RK3 combine
// (Sec. 4.3), of the flux divergence and gravity source (Eq. forward, Eq. mom3), of LMARS
// (Eqs. rp, ru), of WENO5 (Eq. weno5) and of the primitive map (App. B). The upwind branch
// of LMARS is held fixed, except at u* = 0 where the mean of both one-sided derivatives is
// used; the time step is a given constant.
//
// Two kernels per stage, deterministic (no atomics):
//   adj_face_kernel (one launch for the faces of every direction): one thread per face
//     recomputes the face states from its six-cell stencil, transposes LMARS and WENO5, and
//     writes the contribution of the face to each of its six stencil cells into
//     G[d][v][s][face];
//   adj_cell_kernel: one thread per cell gathers the contributions of every face whose
//     stencil holds the cell (or a ghost image of it), transposes the primitive map and the
//     gravity source, and forms the stage combine.
#pragma once
#include "snap_stage.cuh"

namespace snap {

template <class R>
__device__ __forceinline__ const CstT<R> &acst(const AdjArgs &a);
template <>
__device__ __forceinline__ const CstT<float> &acst<float>(const AdjArgs &a) { return a.cf; }
template <>
__device__ __forceinline__ const CstT<double> &acst<double>(const AdjArgs &a) { return a.cd; }

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

// Transpose of lmars<> for a dry gas: accumulates XLb, XRb from Fb.
template <class R, class L>
__device__ __forceinline__ void lmars_adj(const CstT<R> &C, const R *XL, const R *XR, int dir,
                                          R pref, const R *Fb, R *XLb, R *XRb) {
  static_assert(L::NVAP == 0, "the adjoint is built for a dry gas");
  constexpr int NV = L::NV, IE = L::IE, IM0 = L::IM0, NM = L::NMOM;
  const int mn = L::mom(dir);
  const R gam = C.gamma_d, igm1 = C.igm1;
  const R pL = pref + XL[IE], pR = pref + XR[IE];
  const R cL = Ar<R>::sqrt_pos(gam * pL * Ar<R>::rcp(XL[0]));
  const R cR = Ar<R>::sqrt_pos(gam * pR * Ar<R>::rcp(XR[0]));
  const R rhoc = R(0.5) * (XL[0] + XR[0]) * R(0.5) * (cL + cR);
  const R uL = XL[mn], uR = XR[mn];
  const R us = R(0.5) * (uL + uR) - Ar<R>::div(XR[IE] - XL[IE], R(2) * rhoc);
  R usb = R(0);
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
    const R pS = use_left ? pL : pR, rhoS = XS[0], mf = us * rhoS;
    R u2 = R(0), mfb = Fb[0];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      u2 += XS[IM0 + m] * XS[IM0 + m];
      mfb += Fb[IM0 + m] * XS[IM0 + m];
    }
    const R rhoe = pS * igm1 + R(0.5) * rhoS * u2;
    usb += wgt * (mfb * rhoS + Fb[IE] * (rhoe + pS));
    const R rhoeb = Fb[IE] * us;
    const R pSb = Fb[IE] * us + rhoeb * igm1;
    R b0 = wgt * (mfb * us + rhoeb * R(0.5) * u2);
    R bp = wgt * pSb;
    R bm[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) bm[m] = wgt * (Fb[IM0 + m] * mf + rhoeb * rhoS * XS[IM0 + m]);
    if (use_left) {
      XLb[0] += b0;
      XLb[IE] += bp;
#pragma unroll
      for (int m = 0; m < NM; ++m) XLb[IM0 + m] += bm[m];
    } else {
      XRb[0] += b0;
      XRb[IE] += bp;
#pragma unroll
      for (int m = 0; m < NM; ++m) XRb[IM0 + m] += bm[m];
    }
  }
  R rhocb = R(0);
  const R i2rc = Ar<R>::rcp(R(2) * rhoc);
  XLb[mn] += R(0.5) * usb;
  XRb[mn] += R(0.5) * usb;
  XRb[IE] -= usb * i2rc;
  XLb[IE] += usb * i2rc;
  rhocb += usb * (XR[IE] - XL[IE]) * i2rc * Ar<R>::rcp(rhoc);
  XLb[IE] += R(0.5) * psb;
  XRb[IE] += R(0.5) * psb;
  rhocb -= R(0.5) * (uR - uL) * psb;
  XRb[mn] -= R(0.5) * rhoc * psb;
  XLb[mn] += R(0.5) * rhoc * psb;
  XLb[0] += R(0.25) * (cL + cR) * rhocb;
  XRb[0] += R(0.25) * (cL + cR) * rhocb;
  const R cb = R(0.25) * (XL[0] + XR[0]) * rhocb;
  XLb[IE] += cb * cL * Ar<R>::rcp(R(2) * pL);
  XLb[0] -= cb * cL * Ar<R>::rcp(R(2) * XL[0]);
  XRb[IE] += cb * cR * Ar<R>::rcp(R(2) * pR);
  XRb[0] -= cb * cR * Ar<R>::rcp(R(2) * XR[0]);
}

// primitives of a stored dry state (p' = (gamma_d - 1)(y_E - K), y_E = rho e - e_ref)
template <class R, class L>
__device__ __forceinline__ void dry_prim(const CstT<R> &C, const R *y, R *x) {
  const R ir = Ar<R>::rcp(y[0]);
  x[0] = y[0];
  R K = R(0);
#pragma unroll
  for (int m = 0; m < L::NMOM; ++m) {
    x[L::IM0 + m] = y[L::IM0 + m] * ir;
    K += y[L::IM0 + m] * x[L::IM0 + m];
  }
  x[L::IE] = C.gm1 * (y[L::IE] - R(0.5) * K);
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
  const R bdt = R(a.b * a.dt), ih = Prof<R>::ih(D, DIR);
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
    for (int v = 0; v < NV; ++v) Fb[v] -= bdt * lo[v * ncell + c] * ih;
    if (fz) Fbz -= R(0.5) * Prof<R>::grav(D) * bdt * lo[L::IE * ncell + c];
  }
  if (pos < nd) {
    const long long c = ((long long)k * ny + j) * nx + i;
#pragma unroll
    for (int v = 0; v < NV; ++v) Fb[v] += bdt * lo[v * ncell + c] * ih;
    if (fz) Fbz -= R(0.5) * Prof<R>::grav(D) * bdt * lo[L::IE * ncell + c];
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
    R y[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) y[v] = Ys[v * ncell + c];
    dry_prim<R, L>(C, y, X[s]);
    if (flip) X[s][MN] = -X[s][MN];
  }
  R QL[NV], QR[NV], gL[NV][5], gR[NV][5], QLb[NV], QRb[NV];
  const R weps = C.weno_eps;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    R q[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) q[s] = X[s][v];
    QL[v] = weno5_grad<R>(q, weps, gL[v]);
#pragma unroll
    for (int s = 0; s < 5; ++s) q[s] = X[5 - s][v];
    QR[v] = weno5_grad<R>(q, weps, gR[v]);
    QLb[v] = QRb[v] = R(0);
  }
  const R pref = fz ? Prof<R>::pf(D, k) : Prof<R>::pc(D, k);
  lmars_adj<R, L>(C, QL, QR, DIR, pref, Fb, QLb, QRb);
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      R g = R(0);
      if (s <= 4) g += QLb[v] * gL[v][s];
      if (s >= 1) g += QRb[v] * gR[v][5 - s];
      G[((long long)v * 6 + s) * nf + f] = g;
    }
}

// One thread per face; the faces of x, then y (3-D), then z.
template <class R, class L>
__global__ void __launch_bounds__(128) adj_face_kernel(const AdjArgs a) {
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
  const R *G = reinterpret_cast<const R *>(a.G[DIR]);
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const int fpos = ipos + 3 - s;  // face whose stencil slot s is this position
    if (fpos < 0 || fpos > nd) continue;
    const int fi = fx ? fpos : i, fj = fy ? fpos : j, fk = fz ? fpos : k;
    const long long f = ((long long)fk * nfy + fj) * nfx + fi;
#pragma unroll
    for (int v = 0; v < L::NV; ++v) {
      const R g = G[((long long)v * 6 + s) * nf + f];
      Xb[v] += v == MN ? sg * g : g;
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
  const R grav = Prof<R>::grav(D), bdt = R(a.b * a.dt), av = R(a.a), bv = R(a.b);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = int(c % nx), j = int((c / nx) % ny), k = int(c / ((long long)nx * ny));
    R Xb[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Xb[v] = R(0);
    gather_dir<R, L, 0>(a, D, i, j, k, Xb);
    if constexpr (L::D3) gather_dir<R, L, 1>(a, D, i, j, k, Xb);
    gather_dir<R, L, 2>(a, D, i, j, k, Xb);
    // transpose of the primitive map and of the gravity source
    R y[NV], Yb[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) y[v] = Ys[v * ncell + c];
    const R rho = y[0], ir = Ar<R>::rcp(rho);
    R r0 = Xb[0], u2 = R(0);
#pragma unroll
    for (int m = 0; m < L::NMOM; ++m) {
      const R u = y[IM0 + m] * ir;
      r0 -= Xb[IM0 + m] * u * ir;
      u2 += u * u;
      Yb[IM0 + m] = Xb[IM0 + m] * ir - Xb[IE] * C.gm1 * u;
    }
    r0 += Xb[IE] * C.gm1 * R(0.5) * u2;
    Yb[0] = r0 - grav * bdt * lo[L::mom(2) * ncell + c];
    Yb[IE] = Xb[IE] * C.gm1;
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

template <class R, class L>
struct AdjFamily {
  static cudaError_t face(const AdjArgs &a, long long nfaces, cudaStream_t s) {
    long long g = (nfaces + 127) / 128;
    adj_face_kernel<R, L><<<int(g < 9728 ? g : 9728), 128, 0, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t cell(const AdjArgs &a, long long ncell, cudaStream_t s) {
    long long g = (ncell + 127) / 128;
    adj_cell_kernel<R, L><<<int(g < 9728 ? g : 9728), 128, 0, s>>>(a);
    return cudaGetLastError();
  }
  static AdjKernels get() {
    AdjKernels k;
    k.face = &face;
    k.cell = &cell;
    return k;
  }
};

}  // namespace snap
