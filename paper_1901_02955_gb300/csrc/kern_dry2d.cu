// kern_dry2d.cu -- stage kernels for a dry gas in the x-z plane (optional viscosity).
#include "snap_adjoint.cuh"

namespace snap {

bool find_kernels_dry2d(int f32, int visc, KernelSet *out) {
  using L = Lay<0, 0, false>;
  using A = TileT<32, 1, 14>;
  using B = TileT<64, 1, 6>;
  using C = TileT<16, 1, 30>;
  if (f32)
    *out = visc ? Family<float, L>::set<true, A, B, C>() : Family<float, L>::set<false, A, B, C>();
  else
    *out = visc ? Family<double, L>::set<true, A>() : Family<double, L>::set<false, A>();
  return true;
}

bool find_adjoint_kernels_dry2d(int f32, AdjKernels *out) {
  using L = Lay<0, 0, false>;
  *out = f32 ? AdjFamily<float, L>::get() : AdjFamily<double, L>::get();
  return true;
}

}  // namespace snap
