// variants_wide.cu -- solve-kernel instantiations with 4 to 32 lanes per
// sample (the latency shapes of single solves).
#include "launch.h"

namespace brmppi {

const Variant* variants_wide(int* n) {
  static const Variant v[] = {
      {4, 1, false, &solve_kernel<4, 1, false>},   {4, 2, false, &solve_kernel<4, 2, false>}, {4, 3, false, &solve_kernel<4, 3, false>},   {4, 4, false, &solve_kernel<4, 4, false>},
      {8, 1, false, &solve_kernel<8, 1, false>},   {8, 2, false, &solve_kernel<8, 2, false>}, {8, 3, false, &solve_kernel<8, 3, false>},   {8, 4, false, &solve_kernel<8, 4, false>},
      {16, 1, false, &solve_kernel<16, 1, false>}, {16, 2, false, &solve_kernel<16, 2, false>}, {32, 1, false, &solve_kernel<32, 1, false>},
  };
  *n = static_cast<int>(sizeof(v) / sizeof(v[0]));
  return v;
}

}  // namespace brmppi
