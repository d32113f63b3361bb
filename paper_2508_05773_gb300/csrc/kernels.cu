// kernels.cu -- dispatch over the solve-kernel instantiations.
#include "launch.h"

namespace brmppi {

namespace {

template <typename F>
void for_each_variant(F f) {
  int n = 0;
  const Variant* a = variants_narrow(&n);
  for (int i = 0; i < n; ++i) f(a[i]);
  const Variant* b = variants_wide(&n);
  for (int i = 0; i < n; ++i) f(b[i]);
}

const Variant* find(int tps, int bpt) {
  const Variant* hit = nullptr;
  for_each_variant([&](const Variant& v) {
    if (v.tps == tps && v.bpt == bpt) hit = &v;
  });
  return hit;
}

}  // namespace

bool variant_exists(int tps, int bpt) { return find(tps, bpt) != nullptr; }

cudaError_t set_smem_limit(size_t bytes) {
  cudaError_t err = cudaSuccess;
  for_each_variant([&](const Variant& v) {
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(v.fn),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
    if (e != cudaSuccess && err == cudaSuccess) err = e;
  });
  return err;
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
