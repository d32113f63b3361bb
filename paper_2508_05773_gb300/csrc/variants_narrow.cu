// variants_narrow.cu -- solve-kernel instantiations with 1 or 2 lanes per
// sample (the throughput shapes of batches and serving).
#include "launch.h"

namespace brmppi {

const Variant* variants_narrow(int* n) {
  static const Variant v[] = {
      {1, 1, &solve_kernel<1, 1>}, {1, 2, &solve_kernel<1, 2>}, {1, 3, &solve_kernel<1, 3>},
      {1, 4, &solve_kernel<1, 4>}, {1, 5, &solve_kernel<1, 5>}, {1, 6, &solve_kernel<1, 6>},
      {1, 8, &solve_kernel<1, 8>}, {2, 1, &solve_kernel<2, 1>}, {2, 2, &solve_kernel<2, 2>},
      {2, 3, &solve_kernel<2, 3>}, {2, 4, &solve_kernel<2, 4>},
  };
  *n = static_cast<int>(sizeof(v) / sizeof(v[0]));
  return v;
}

}  // namespace brmppi
