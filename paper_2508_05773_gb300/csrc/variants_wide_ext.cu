// variants_wide_ext.cu -- solve-kernel instantiations carrying the optional
// terms (moving and e = 4 obstacles, collision cost, buffer cost), with 4
// to 32 lanes per sample.
#include "launch.h"

namespace brmppi {

const Variant* variants_wide_ext(int* n) {
  static const Variant v[] = {
      {4, 1, true, &solve_kernel<4, 1, true>},
      {4, 2, true, &solve_kernel<4, 2, true>}, {4, 3, true, &solve_kernel<4, 3, true>},
      {4, 4, true, &solve_kernel<4, 4, true>},
      {8, 1, true, &solve_kernel<8, 1, true>},
      {8, 2, true, &solve_kernel<8, 2, true>}, {8, 3, true, &solve_kernel<8, 3, true>},
      {8, 4, true, &solve_kernel<8, 4, true>},
      {16, 1, true, &solve_kernel<16, 1, true>},
      {16, 2, true, &solve_kernel<16, 2, true>},
      {32, 1, true, &solve_kernel<32, 1, true>},
  };
  *n = static_cast<int>(sizeof(v) / sizeof(v[0]));
  return v;
}

}  // namespace brmppi
