// variants_wide.cu -- solve-kernel instantiations with 4 to 32 lanes per
// sample (the latency shapes of single solves).
#include "launch.h"

namespace brmppi {

const Variant* variants_wide(int* n) {
  static const Variant v[] = {
      {4, 1, &solve_kernel<4, 1>},   {4, 2, &solve_kernel<4, 2>},   {4, 4, &solve_kernel<4, 4>},
      {8, 1, &solve_kernel<8, 1>},   {8, 2, &solve_kernel<8, 2>},   {8, 4, &solve_kernel<8, 4>},
      {16, 1, &solve_kernel<16, 1>}, {16, 2, &solve_kernel<16, 2>}, {32, 1, &solve_kernel<32, 1>},
  };
  *n = static_cast<int>(sizeof(v) / sizeof(v[0]));
  return v;
}

}  // namespace brmppi
