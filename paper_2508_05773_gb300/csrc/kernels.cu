// kernels.cu -- instantiations of the solve kernel and their dispatch.
#include "launch.h"

namespace brmppi {

using KernelFn = void (*)(const KConst, const LaunchDesc);

namespace {

struct Variant {
  int tps, bpt;
  KernelFn fn;
};

#define BRMPPI_VARIANT(T, B) Variant{T, B, &solve_kernel<T, B>}
const Variant kVariants[] = {
    BRMPPI_VARIANT(1, 1),  BRMPPI_VARIANT(1, 2),  BRMPPI_VARIANT(1, 4),  BRMPPI_VARIANT(1, 8),
    BRMPPI_VARIANT(2, 1),  BRMPPI_VARIANT(2, 2),  BRMPPI_VARIANT(2, 4),
    BRMPPI_VARIANT(4, 1),  BRMPPI_VARIANT(4, 2),  BRMPPI_VARIANT(4, 4),
    BRMPPI_VARIANT(8, 1),  BRMPPI_VARIANT(8, 2),  BRMPPI_VARIANT(8, 4),
    BRMPPI_VARIANT(16, 1), BRMPPI_VARIANT(16, 2), BRMPPI_VARIANT(32, 1),
};
#undef BRMPPI_VARIANT

const Variant* find(int tps, int bpt) {
  for (const Variant& v : kVariants)
    if (v.tps == tps && v.bpt == bpt) return &v;
  return nullptr;
}

}  // namespace

bool variant_exists(int tps, int bpt) { return find(tps, bpt) != nullptr; }

cudaError_t set_smem_limit(size_t bytes) {
  for (const Variant& v : kVariants) {
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(v.fn),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int variant_occupancy(int tps, int bpt, int threads, size_t smem) {
  const Variant* v = find(tps, bpt);
  if (!v) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, v->fn, threads, smem) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_solve(int tps, int bpt, int blocks, int threads, size_t smem, cudaStream_t stream,
                         const KConst& k, const LaunchDesc& L) {
  const Variant* v = find(tps, bpt);
  if (!v) return cudaErrorInvalidValue;
  v->fn<<<blocks, threads, smem, stream>>>(k, L);
  return cudaGetLastError();
}

}  // namespace brmppi
