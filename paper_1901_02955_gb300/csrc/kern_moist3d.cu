// kern_moist3d.cu -- stage kernels for two vapours with cloud and precipitation, 3-D.
#include "snap_stage.cuh"

namespace snap {

bool find_kernels_moist3d(int f32, int visc, int micro, KernelSet *out) {
  using L = Lay<2, 2, true>;
  // FP32: 8 x 8 x 4 cells, 256 threads, registers capped for 3 CTAs per SM (the compact
  // shared-memory cross fits three); 16 x 8 x 2 for two; FP64 uncapped
  using A = TileT<8, 8, 4, 256, 3>;
  using A64 = TileT<8, 8, 4>;
  using B = TileT<16, 8, 2, 256, 2>;
  if (visc) return false;
  if (micro)  // sedimentation and the Kessler scheme compiled in, default tile only
    *out = f32 ? Family<float, L>::set_micro<A>() : Family<double, L>::set_micro<A64>();
  else
    *out = f32 ? Family<float, L>::set<false, A, B>() : Family<double, L>::set<false, A64>();
  return true;
}

}  // namespace snap
