// kern_dry2d.cu -- stage kernels for a dry gas in the x-z plane (optional viscosity).
#include "snap_adjoint.cuh"

namespace snap {

bool find_kernels_dry2d(int f32, int visc, KernelSet *out) {
  using L = Lay<0, 0, false>;
  // FP32 default: 64 x 14 cells, 512 threads, 2 CTAs per SM (64 registers). Against the
  // 32 x 14 tile at 4 CTAs per SM the wider halo-to-interior ratio (1.56 vs 1.70 boxed cells
  // per owned cell) saves ~4 % of the step on the 1024 x 256 density current; the others are
  // autotuner candidates.
  using A = TileT<64, 1, 14, 512, 2>;
  using B = TileT<32, 1, 14, 256, 4>;
  using C = TileT<128, 1, 14, 1024, 1>;
  using D = TileT<64, 1, 28, 1024, 1>;
  // FP64 default: 32 x 28 cells, 512 threads, 1 CTA per SM (128 registers); the 32 x 14 tile
  // at 2 CTAs per SM is ~4 % slower on the same workload.
  using A64 = TileT<32, 1, 28, 512, 1>;
  using B64 = TileT<32, 1, 14, 256, 2>;
  if (f32)
    *out = visc ? Family<float, L>::set<true, A, B, C, D>()
                : Family<float, L>::set<false, A, B, C, D>();
  else
    *out = visc ? Family<double, L>::set<true, A64, B64>()
                : Family<double, L>::set<false, A64, B64>();
  return true;
}

bool find_adjoint_kernels_dry2d(int f32, AdjKernels *out) {
  using L = Lay<0, 0, false>;
  *out = f32 ? AdjFamily<float, L>::get() : AdjFamily<double, L>::get();
  return true;
}

}  // namespace snap
