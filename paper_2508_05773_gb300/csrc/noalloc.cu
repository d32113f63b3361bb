// noalloc.cu -- a solve entry point that allocates nothing.
//
// Some callers cannot allocate device memory at solve time: code running
// inside a CUDA graph that is being captured, or an embedded controller or
// safety process whose memory is fixed when it starts (no cudaMalloc,
// cudaFree or allocating library after start-up), cannot create a
// brmppi_ctx.  This entry point runs the same solve kernel with its
// scratch (softmin partials, the applied-input history and two counters)
// in a file-scope device array of fixed size instead.  Every device that
// loads the library holds that array (about 3.1 MiB) until the process
// exits.
//
// The array is shared by all calls on a device and keeps the contents of the
// last call: the counters that must start at zero are cleared (memset on the
// caller's stream) before each launch; the other regions are fully written
// before they are read.  Calls whose work overlaps on the GPU (different
// streams, or host threads racing) corrupt each other: serialise them.
#include <cmath>
#include <mutex>
#include <string>

#include "internal.h"

namespace brmppi_host {
// defined in api.cu
std::string check_params(const brmppi_params* p);
brmppi::KConst make_kconst(const brmppi_params& q);
brmppi::SmemCaps make_caps(int n_obs, int n_rows, int n_pts, int H, int tps);
size_t smem_bytes(const brmppi::SmemCaps& c, int spb);
brmppi::Inst make_inst(const double* x0, const float* U_nom, const float* obs, int n_obs, const float* path,
                       int n_pts, float ds, int S, int H, uint64_t seed, uint64_t counter, float* U_out,
                       float* traj_out, float* J_out, float* U_next, int32_t* status, float* part,
                       unsigned int* sync, int spb, int n_discs);
}  // namespace brmppi_host

namespace {

// Stated maxima of the allocation-free solve.
constexpr int kNaMaxS = 4096;
constexpr int kNaMaxH = 64;
constexpr int kNaMaxObstacles = 16;
constexpr int kNaMaxPathPts = 4096;
// Fixed launch shape: 4 lanes per sample, 128-thread CTAs (32 samples each).
constexpr int kNaTps = 4;
constexpr int kNaThreads = 128;
constexpr int kNaSpb = kNaThreads / kNaTps;
constexpr int kNaMaxTiles = (kNaMaxS + kNaSpb - 1) / kNaSpb;
constexpr int kNaPartStride = ((3 + 3 * kNaMaxH + 1) + 3) / 4 * 4;
constexpr size_t kNaSyncFloats = 64;  // [0] finished tiles, [1] error bits, rest padding
constexpr size_t kNaPartFloats = static_cast<size_t>(kNaMaxTiles) * kNaPartStride;
constexpr size_t kNaHistFloats = static_cast<size_t>(kNaMaxTiles) * 3 * kNaMaxH * kNaSpb;
constexpr size_t kNaScratchFloats = kNaSyncFloats + kNaPartFloats + kNaHistFloats;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float* g_scratch_ptr[kMaxDevices] = {};
size_t g_smem_optin[kMaxDevices] = {};

}  // namespace

// The scratch of the allocation-free solve (one per device that loads the
// library; host code must use the address from cudaGetSymbolAddress).
static __device__ __align__(256) float g_noalloc_scratch[kNaScratchFloats];

namespace {

// With the device current: the device address of the scratch array and the
// device's opt-in shared-memory limit.  The first call on a device also
// raises the kernel variants' shared-memory limit.  The address is looked up
// again on every call (a host-side query, no allocation): after a
// cudaDeviceReset the device's module, and with it the array, may move, and
// a changed address repeats the set-up.
brmppi_status scratch_for_current_device(float** out, size_t* smem_optin) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return brmppi_host::cuda_fail(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return brmppi_host::fail(nullptr, BRMPPI_EINVAL, "device index out of range");
  void* ptr = nullptr;
  if ((e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch)) != cudaSuccess)
    return brmppi_host::cuda_fail(nullptr, e, "cudaGetSymbolAddress(no-alloc scratch)");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (g_scratch_ptr[dev] != static_cast<float*>(ptr)) {
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
      return brmppi_host::cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
    g_smem_optin[dev] = static_cast<size_t>(optin) - 1024;  // static shared memory of the kernel
    if ((e = brmppi::set_smem_limit(g_smem_optin[dev])) != cudaSuccess)
      return brmppi_host::cuda_fail(nullptr, e, "cudaFuncSetAttribute");
    g_scratch_ptr[dev] = static_cast<float*>(ptr);
  }
  *out = g_scratch_ptr[dev];
  *smem_optin = g_smem_optin[dev];
  return BRMPPI_OK;
}

}  // namespace

extern "C" brmppi_status brmppi_solve_device_noalloc(const brmppi_params* p, const double* x0_dev,
                                                     const float* U_nom_dev, const float* obs_dev, int32_t n_obs,
                                                     const float* path_dev, int32_t n_pts, float ds, uint64_t seed,
                                                     uint64_t counter, float* U_out_dev, float* traj_out_dev,
                                                     float* J_out_dev, float* U_next_dev, int32_t* status_dev,
                                                     void* stream) {
  using namespace brmppi_host;
  const std::string bad = check_params(p);
  if (!bad.empty()) return fail(nullptr, BRMPPI_EINVAL, bad);
  if (p->S > kNaMaxS)
    return fail(nullptr, BRMPPI_EINVAL, "no-alloc solve: S = " + std::to_string(p->S) + " exceeds its maximum 4096");
  if (p->H > kNaMaxH)
    return fail(nullptr, BRMPPI_EINVAL, "no-alloc solve: H = " + std::to_string(p->H) + " exceeds its maximum 64");
  if (n_obs < 0 || n_obs > kNaMaxObstacles)
    return fail(nullptr, BRMPPI_EINVAL, "no-alloc solve: n_obs out of [0, 16]");
  if (n_pts < 2 || n_pts > kNaMaxPathPts) return fail(nullptr, BRMPPI_EINVAL, "no-alloc solve: n_pts out of [2, 4096]");
  if (!(ds > 0.f) || !std::isfinite(ds)) return fail(nullptr, BRMPPI_EINVAL, "no-alloc solve: ds must be positive");
  if (!x0_dev || !U_nom_dev || !path_dev || !U_out_dev || (n_obs > 0 && !obs_dev))
    return fail(nullptr, BRMPPI_EINVAL, "no-alloc solve: NULL buffer");
  float* scratch = nullptr;
  size_t smem_optin = 0;
  brmppi_status st = scratch_for_current_device(&scratch, &smem_optin);
  if (st != BRMPPI_OK) return st;
  int bpt = 0;
  const int n_rows = rows_of(*p, n_obs);
  if (!pick_bpt(kNaTps, philox_blocks(n_rows), &bpt)) return fail(nullptr, BRMPPI_EINVAL, "no-alloc solve: no variant");
  brmppi::LaunchDesc L{};
  unsigned int* sync = reinterpret_cast<unsigned int*>(scratch);
  float* part = scratch + kNaSyncFloats;
  L.single = make_inst(x0_dev, U_nom_dev, obs_dev, n_obs, path_dev, n_pts, ds, p->S, p->H, seed, counter, U_out_dev,
                       traj_out_dev, J_out_dev, U_next_dev, status_dev, part, sync, kNaSpb, p->n_discs);
  L.caps = make_caps(n_obs, n_rows, n_pts, p->H, kNaTps);
  L.uh = part + kNaPartFloats;
  L.uh_stride = 3 * p->H * kNaSpb;
  Shape sh;
  sh.tps = kNaTps;
  sh.bpt = bpt;
  sh.threads = kNaThreads;
  const brmppi::KConst k = make_kconst(*p);
  single_launch_options(L, sh, k, n_rows, p->H, smem_optin);
  const size_t smem = smem_bytes(L.caps, kNaSpb);
  if (smem > smem_optin)
    return fail(nullptr, BRMPPI_EINVAL,
                "no-alloc solve: shared memory need " + std::to_string(smem) + " B exceeds the device limit " +
                    std::to_string(smem_optin) + " B");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(float) * kNaSyncFloats, s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "no-alloc solve: clearing counters");
  e = brmppi::launch_solve(kNaTps, bpt, L.single.tiles, kNaThreads, smem, s, k, L, L.single.P);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "no-alloc solve: kernel launch");
  return BRMPPI_OK;
}
