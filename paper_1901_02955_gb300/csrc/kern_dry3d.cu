// kern_dry3d.cu -- stage kernels for a dry gas in three dimensions (optional viscosity).
#include "snap_adjoint.cuh"

namespace snap {

bool find_kernels_dry3d(int f32, int visc, KernelSet *out) {
  using L = Lay<0, 0, true>;
  using A = TileT<8, 8, 4>;
  using B = TileT<16, 8, 2>;
  if (f32)
    *out = visc ? Family<float, L>::set<true, A, B>() : Family<float, L>::set<false, A, B>();
  else
    *out = visc ? Family<double, L>::set<true, A>() : Family<double, L>::set<false, A>();
  return true;
}

bool find_adjoint_kernels_dry3d(int f32, AdjKernels *out) {
  using L = Lay<0, 0, true>;
  *out = f32 ? AdjFamily<float, L>::get() : AdjFamily<double, L>::get();
  return true;
}

}  // namespace snap
