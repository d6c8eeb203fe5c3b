// kern_dry2d.cu -- stage kernels for a dry gas in the x-z plane (optional viscosity).
#include "snap_adjoint.cuh"

namespace snap {

bool find_kernels_dry2d(int f32, int visc, KernelSet *out) {
  using L = Lay<0, 0, false>;
  using A = TileT<32, 1, 14, 256, 4>;  // FP32: compiled for 4 CTAs per SM (64 registers)
  using A64 = TileT<32, 1, 14, 256, 2>;  // FP64: 2 CTAs per SM (128 registers)
  using B = TileT<64, 1, 6>;
  using C = TileT<16, 1, 30>;
  if (f32)
    *out = visc ? Family<float, L>::set<true, A, B, C>() : Family<float, L>::set<false, A, B, C>();
  else
    *out = visc ? Family<double, L>::set<true, A64>() : Family<double, L>::set<false, A64>();
  return true;
}

bool find_adjoint_kernels_dry2d(int f32, AdjKernels *out) {
  using L = Lay<0, 0, false>;
  *out = f32 ? AdjFamily<float, L>::get() : AdjFamily<double, L>::get();
  return true;
}

}  // namespace snap
