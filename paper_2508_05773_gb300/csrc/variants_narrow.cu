// variants_narrow.cu -- solve-kernel instantiations with 1 or 2 lanes per
// sample (the throughput shapes of batches and serving).
#include "launch.h"

namespace brmppi {

const Variant* variants_narrow(int* n) {
  static const Variant v[] = {
      {1, 1, false, &solve_kernel<1, 1, false>}, {1, 2, false, &solve_kernel<1, 2, false>}, {1, 3, false, &solve_kernel<1, 3, false>},
      {1, 4, false, &solve_kernel<1, 4, false>}, {1, 5, false, &solve_kernel<1, 5, false>}, {1, 6, false, &solve_kernel<1, 6, false>},
      {1, 8, false, &solve_kernel<1, 8, false>}, {2, 1, false, &solve_kernel<2, 1, false>}, {2, 2, false, &solve_kernel<2, 2, false>},
      {2, 3, false, &solve_kernel<2, 3, false>}, {2, 4, false, &solve_kernel<2, 4, false>},
  };
  *n = static_cast<int>(sizeof(v) / sizeof(v[0]));
  return v;
}

}  // namespace brmppi
