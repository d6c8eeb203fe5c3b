// kern_moist2d.cu -- instantiation of the stage kernels for n_vapor = 1, n_cond = 2,
// three-dimensional = false.
#include "snap_stage.cuh"

namespace snap {

bool find_kernels_moist2d(int f32, int visc, KernelSet *out) {
  using L = Lay<1, 2, false>;
  if (visc) return false;
  *out = f32 ? Family<float, L, false>::set() : Family<double, L, false>::set();
  return true;
}

}  // namespace snap
