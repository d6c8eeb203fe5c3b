// kern_moist3d.cu -- stage kernels for two vapours with cloud and precipitation, 3-D.
#include "snap_stage.cuh"

namespace snap {

bool find_kernels_moist3d(int f32, int visc, int micro, KernelSet *out) {
  using L = Lay<2, 2, true>;
  using A = TileT<8, 8, 4>;
  using B = TileT<16, 8, 2>;
  if (visc) return false;
  if (micro)  // sedimentation and the Kessler scheme compiled in, default tile only
    *out = f32 ? Family<float, L>::set_micro<A>() : Family<double, L>::set_micro<A>();
  else
    *out = f32 ? Family<float, L>::set<false, A, B>() : Family<double, L>::set<false, A>();
  return true;
}

}  // namespace snap
