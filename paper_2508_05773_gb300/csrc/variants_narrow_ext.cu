// variants_narrow_ext.cu -- solve-kernel instantiations carrying the optional
// terms (moving and e = 4 obstacles, collision cost, buffer cost), with 1
// or 2 lanes per sample.
#include "launch.h"

namespace brmppi {

const Variant* variants_narrow_ext(int* n) {
  static const Variant v[] = {
      {1, 1, true, &solve_kernel<1, 1, true>},
      {1, 2, true, &solve_kernel<1, 2, true>},
      {1, 3, true, &solve_kernel<1, 3, true>},
      {1, 4, true, &solve_kernel<1, 4, true>},
      {1, 5, true, &solve_kernel<1, 5, true>},
      {1, 6, true, &solve_kernel<1, 6, true>},
      {1, 8, true, &solve_kernel<1, 8, true>},
      {2, 1, true, &solve_kernel<2, 1, true>},
      {2, 2, true, &solve_kernel<2, 2, true>},
      {2, 3, true, &solve_kernel<2, 3, true>},
      {2, 4, true, &solve_kernel<2, 4, true>},
  };
  *n = static_cast<int>(sizeof(v) / sizeof(v[0]));
  return v;
}

}  // namespace brmppi
