// variants_latency_ext.cu -- exact-rows single-solve instantiations of the
// family with the optional terms (moving and e = 4 obstacles, collision and
// buffer costs, footprint discs, third-order rows, the jerk-input model):
// 4 lanes per sample, 1 to 4 rows a lane.
#include "launch.h"

namespace brmppi {

const Variant* variants_latency_ext(int* n) {
  static const Variant v[] = {
      {4, 1, true, &solve_kernel<4, 1, true, 1>, 1}, {4, 1, true, &solve_kernel<4, 1, true, 2>, 2},
      {4, 1, true, &solve_kernel<4, 1, true, 3>, 3}, {4, 1, true, &solve_kernel<4, 1, true, 4>, 4},
  };
  *n = static_cast<int>(sizeof(v) / sizeof(v[0]));
  return v;
}

}  // namespace brmppi
