// variants_latency.cu -- solve-kernel instantiations for single solves on
// the noise-warp shapes with an exact number of constraint rows per lane
// (2, 4 or 8 lanes per sample, 1 to 4 rows a lane): the step then runs
// without a branch on the row count.
#include "launch.h"

namespace brmppi {

const Variant* variants_latency(int* n) {
  static const Variant v[] = {
      {2, 1, false, &solve_kernel<2, 1, false, 1>, 1}, {2, 1, false, &solve_kernel<2, 1, false, 2>, 2},
      {2, 1, false, &solve_kernel<2, 1, false, 3>, 3}, {2, 1, false, &solve_kernel<2, 1, false, 4>, 4},
      {4, 1, false, &solve_kernel<4, 1, false, 1>, 1}, {4, 1, false, &solve_kernel<4, 1, false, 2>, 2},
      {4, 1, false, &solve_kernel<4, 1, false, 3>, 3}, {4, 1, false, &solve_kernel<4, 1, false, 4>, 4},
      {8, 1, false, &solve_kernel<8, 1, false, 1>, 1}, {8, 1, false, &solve_kernel<8, 1, false, 2>, 2},
      {8, 1, false, &solve_kernel<8, 1, false, 3>, 3}, {8, 1, false, &solve_kernel<8, 1, false, 4>, 4},
  };
  *n = static_cast<int>(sizeof(v) / sizeof(v[0]));
  return v;
}

}  // namespace brmppi
