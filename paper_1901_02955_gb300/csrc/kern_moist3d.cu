// kern_moist3d.cu -- instantiation of the stage kernels for n_vapor = 2, n_cond = 2,
// three-dimensional = true.
#include "snap_stage.cuh"

namespace snap {

bool find_kernels_moist3d(int f32, int visc, KernelSet *out) {
  using L = Lay<2, 2, true>;
  if (visc) return false;
  *out = f32 ? Family<float, L, false>::set() : Family<double, L, false>::set();
  return true;
}

}  // namespace snap
