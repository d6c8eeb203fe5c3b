// kern_dry3d.cu -- instantiation of the stage kernels for n_vapor = 0, n_cond = 0,
// three-dimensional = true.
#include "snap_stage.cuh"

namespace snap {

bool find_kernels_dry3d(int f32, int visc, KernelSet *out) {
  using L = Lay<0, 0, true>;
  if (f32)
    *out = visc ? Family<float, L, true>::set() : Family<float, L, false>::set();
  else
    *out = visc ? Family<double, L, true>::set() : Family<double, L, false>::set();
  return true;
}

}  // namespace snap
