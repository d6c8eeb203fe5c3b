// kern_moist2d.cu -- stage and adjoint kernels for one vapour with cloud and precipitation,
// x-z plane.
#include "snap_adjoint.cuh"

namespace snap {

bool find_kernels_moist2d(int f32, int visc, int micro, KernelSet *out) {
  using L = Lay<1, 2, false>;
  using A = TileT<32, 1, 14, 256, 3>;  // FP32: 3 CTAs per SM (85 registers)
  using A64 = TileT<32, 1, 14>;
  using B = TileT<64, 1, 6>;
  using C = TileT<16, 1, 30>;
  if (visc) return false;
  if (micro)  // sedimentation and the Kessler scheme compiled in, default tile only
    *out = f32 ? Family<float, L>::set_micro<A>() : Family<double, L>::set_micro<A64>();
  else
    *out = f32 ? Family<float, L>::set<false, A, B, C>() : Family<double, L>::set<false, A64>();
  return true;
}

bool find_adjoint_kernels_moist2d(int f32, AdjKernels *out) {
  using L = Lay<1, 2, false>;
  *out = f32 ? AdjFamily<float, L>::get() : AdjFamily<double, L>::get();
  return true;
}

}  // namespace snap
