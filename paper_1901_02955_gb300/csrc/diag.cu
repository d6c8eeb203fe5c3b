// diag.cu -- diagnostics of a state on the device (not part of the time step).
//
// Equivalent potential temperature (App. A, Eq. theta_e, Emanuel's 4.5.11) of each cell of a
// state with one vapour whose first condensate is the cloud:
//   theta_e = T (p0/p_d)^(R_d q_d / c) exp(L q_v / (c T)),  c = c_pd q_d + c_l q_t,
// q the mass fractions of the total density, q_t = q_v + q_cloud, p_d = rho_d R_d T, L = L^r -
// (c_l - c_pv)(T - T^r) (Eq. latent), p0 = 1e5 Pa. T comes from the conserved energy in FP64;
// the output is FP64.
#include <cuda_runtime.h>

#include "snap_internal.h"

namespace snap {

template <class R>
__global__ void __launch_bounds__(256) theta_e_kernel(const DomDev *doms, int dm, Phys ph, int nv,
                                                      int nmom, double *out) {
  const DomDev &D = doms[dm];
  const R *Y = reinterpret_cast<const R *>(D.buf[0]);
  const long long ncell = D.ncell, plane = (long long)D.nx * D.ny;
  const int im0 = 1 + ph.nvap + ph.nvap * ph.ncond;
  const double cvd = ph.c_vd, cpd = ph.c_pd, cl = ph.sig_c[0][0] * cvd;
  const double dc = cl - (ph.sig_v[0] * cvd + ph.R_v[0]);
  const double Lr = -ph.mu[0][0] - dc * ph.Tref[0];  // mu = -(L^r + dc T^r)
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    double rho = 0.0, m2 = 0.0, A = 0.0, Cv = 0.0;
    for (int s = 0; s < im0; ++s) rho += double(Y[s * ncell + c]);
    for (int m = 0; m < nmom; ++m) {
      const double y = double(Y[(im0 + m) * ncell + c]);
      m2 += y * y;
    }
    const double rd = double(Y[c]), rv = double(Y[ncell + c]);
    Cv = rd + ph.sig_v[0] * rv;
    for (int j = 0; j < ph.ncond; ++j) {
      const double rc = double(Y[(2 + j) * ncell + c]);
      Cv += ph.sig_c[0][j] * rc;
      A += ph.mu[0][j] * rc;
    }
    const double U = (double(Y[(nv - 1) * ncell + c]) + D.e_ref[c / plane]) - 0.5 * m2 / rho - A;
    const double T = U / (Cv * cvd);
    const double qd = rd / rho, qv = rv / rho, qt = (rv + double(Y[2 * ncell + c])) / rho;
    const double pd = rd * ph.R_d * T;
    const double L = Lr - dc * (T - ph.Tref[0]);
    const double cc = cpd * qd + cl * qt;
    out[c] = T * pow(1e5 / pd, ph.R_d * qd / cc) * exp(L * qv / (cc * T));
  }
}

cudaError_t launch_theta_e(const DomDev *doms_dev, int dm, long long ncell, const Phys &ph,
                           int f32, int nv, int nmom, double *out, cudaStream_t s) {
  long long g = (ncell + 255) / 256;
  const int grid = int(g < 2432 ? g : 2432);
  if (f32)
    theta_e_kernel<float><<<grid, 256, 0, s>>>(doms_dev, dm, ph, nv, nmom, out);
  else
    theta_e_kernel<double><<<grid, 256, 0, s>>>(doms_dev, dm, ph, nv, nmom, out);
  return cudaGetLastError();
}

}  // namespace snap
