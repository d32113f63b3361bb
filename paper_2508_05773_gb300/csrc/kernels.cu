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
  const Variant* c = variants_narrow_ext(&n);
  for (int i = 0; i < n; ++i) f(c[i]);
  const Variant* d = variants_wide_ext(&n);
  for (int i = 0; i < n; ++i) f(d[i]);
  const Variant* e = variants_latency(&n);
  for (int i = 0; i < n; ++i) f(e[i]);
  const Variant* g = variants_latency_ext(&n);
  for (int i = 0; i < n; ++i) f(g[i]);
}

// rows = 0: the general instantiation of a shape; rows > 0: the one with
// exactly that many constraint rows a lane (null if not compiled)
const Variant* find(int tps, int bpt, bool ext, int rows = 0) {
  const Variant* hit = nullptr;
  for_each_variant([&](const Variant& v) {
    if (v.tps == tps && v.bpt == bpt && v.ext == ext && v.rows == rows) hit = &v;
  });
  return hit;
}

// One state per thread: the hitch stabilizer on (x_i, u_ref_i).
__global__ void __launch_bounds__(256) stabilize_kernel(const KConst k, const double* x, const float* u_ref, int n,
                                                        float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int nx = k.jerk ? 8 : 7;
  const double* xi = x + nx * static_cast<size_t>(i);
  const float* ur = u_ref + 3 * static_cast<size_t>(i);
  float o[4];
  hitch_stabilize(k, static_cast<float>(xi[3] - xi[2]), static_cast<float>(xi[4]), static_cast<float>(xi[5]),
                  k.jerk ? static_cast<float>(xi[7]) : 0.f, ur[0], ur[1], ur[2], o);
  float* dst = out + 4 * static_cast<size_t>(i);
  dst[0] = o[0];
  dst[1] = o[1];
  dst[2] = o[2];
  dst[3] = o[3];
}

// One instance per thread: the hitch stabilizer on (x0, U*[0]) of every
// instance of a table that asks for it.  Runs after the solve on the same
// stream (kept out of the solve kernel: the unused code cost the solve time).
__global__ void __launch_bounds__(128) stabilize_table_kernel(const KConst k, const Inst* table, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Inst in = table[i];
  if (!in.u_safe) return;
  hitch_stabilize(k, static_cast<float>(in.x0[3] - in.x0[2]), static_cast<float>(in.x0[4]),
                  static_cast<float>(in.x0[5]), k.jerk ? static_cast<float>(in.x0[7]) : 0.f, in.U_out[0],
                  in.U_out[1], in.U_out[2], in.u_safe);
}

// One Philox block per thread: the words and normals the solve kernel draws
// for block b of step tau of sample s (the same device functions), at index
// ((s * H + tau) * n_blocks + b) * 4 + j.
__global__ void __launch_bounds__(256) noise_blocks_kernel(uint32_t key0, uint32_t key1, uint32_t ctr, int n_samples,
                                                           int H, int n_blocks, uint32_t* words, float* normals) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long n = static_cast<long long>(n_samples) * H * n_blocks;
  if (i >= n) return;
  const int b = static_cast<int>(i % n_blocks);
  const long long st = i / n_blocks;
  const int tau = static_cast<int>(st % H);
  const int s = static_cast<int>(st / H);
  const uint4 w = philox4x32_10(
      make_uint4(static_cast<uint32_t>(b), static_cast<uint32_t>(tau), static_cast<uint32_t>(s), ctr), key0, key1);
  if (words) reinterpret_cast<uint4*>(words)[i] = w;
  if (normals) {
    float4 g;
    box_muller(w.x, w.y, g.x, g.y);
    box_muller(w.z, w.w, g.z, g.w);
    reinterpret_cast<float4*>(normals)[i] = g;
  }
}

}  // namespace

cudaError_t launch_noise_blocks(uint64_t seed, uint64_t counter, int n_samples, int H, int n_blocks, uint32_t* words,
                                float* normals, cudaStream_t stream) {
  const long long n = static_cast<long long>(n_samples) * H * n_blocks;
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const long long grid = (n + threads - 1) / threads;
  noise_blocks_kernel<<<static_cast<unsigned>(grid), threads, 0, stream>>>(
      static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), static_cast<uint32_t>(counter), n_samples, H,
      n_blocks, words, normals);
  return cudaGetLastError();
}

cudaError_t launch_merge_tiles(const KConst& k, const Inst& in, const SmemCaps& caps, size_t smem,
                               cudaStream_t stream) {
  if (needs_ext(k)) {
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&merge_tiles_kernel<true>),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    merge_tiles_kernel<true><<<1, 256, smem, stream>>>(k, in, caps);
  } else {
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&merge_tiles_kernel<false>),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    merge_tiles_kernel<false><<<1, 256, smem, stream>>>(k, in, caps);
  }
  return cudaGetLastError();
}

cudaError_t launch_stabilize_table(const KConst& k, const Inst* d_table, int n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  stabilize_table_kernel<<<(n + 127) / 128, 128, 0, stream>>>(k, d_table, n);
  return cudaGetLastError();
}

cudaError_t launch_stabilize(const KConst& k, const double* x, const float* u_ref, int n, float* out,
                             cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  stabilize_kernel<<<(n + threads - 1) / threads, threads, 0, stream>>>(k, x, u_ref, n, out);
  return cudaGetLastError();
}

bool variant_exists(int tps, int bpt) { return find(tps, bpt, false) != nullptr && find(tps, bpt, true) != nullptr; }

cudaError_t set_smem_limit(size_t bytes) {
  cudaError_t err = cudaSuccess;
  for_each_variant([&](const Variant& v) {
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(v.fn),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
    if (e != cudaSuccess && err == cudaSuccess) err = e;
  });
  return err;
}

int noise_warps(int tps, int bpt, int threads, int P) {
  if (tps <= 1 || bpt > 2) return 0;  // the team's lanes draw (or stage) the blocks themselves
  const int blocks_per_step = P * (threads / tps);
  int w = (blocks_per_step + 63) / 64;  // at most two Philox blocks per producer lane and step
  // and at least one producer per compute warp: warps go to the four
  // schedulers round-robin, so each compute warp then shares its scheduler
  // with the same producer load (two producers for four compute warps left
  // two schedulers slower, and the step barrier waits for the slowest)
  if (w < threads / 32) w = threads / 32;
  const int room = (kMaxBlockThreads - threads) / 32;
  w = w > 4 ? 4 : w;
  w = w > room ? room : w;
  return w < 1 ? 1 : w;
}

int block_threads(int tps, int bpt, int threads, int P) { return threads + 32 * noise_warps(tps, bpt, threads, P); }

int exact_rows_variant(int tps, int bpt, const KConst& k, int n_rows) {
  if (!k.proj || tps <= 1 || bpt > 2 || n_rows <= 0) return 0;
  const int rows = (n_rows + tps - 1) / tps;
  return find(tps, 1, needs_ext(k), rows) ? rows : 0;
}

int variant_occupancy(int tps, int bpt, int threads, size_t smem, bool ext, int P) {
  const Variant* v = find(tps, bpt, ext);
  if (!v || block_threads(tps, bpt, threads, P) > kMaxBlockThreads) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, v->fn, block_threads(tps, bpt, threads, P), smem) !=
      cudaSuccess)
    return 0;
  return n;
}

cudaError_t launch_solve(int tps, int bpt, int blocks, int threads, size_t smem, cudaStream_t stream,
                         const KConst& k, const LaunchDesc& L, int P) {
  const Variant* v = find(tps, bpt, needs_ext(k));
  if (!v || block_threads(tps, bpt, threads, P) > kMaxBlockThreads) return cudaErrorInvalidValue;
  if (L.rows > 0) {
    // the exact-rows variants merge in shared memory: the launch must have
    // reserved the room for the instance's partials
    v = (L.work || (!L.single.no_merge && L.caps.merge < L.single.tiles * L.single.part_stride) ||
         L.caps.uh_per_team < 3 * L.single.H)
            ? nullptr
            : find(tps, 1, needs_ext(k), L.rows);
    if (!v) return cudaErrorInvalidValue;
  }
  LaunchDesc D = L;
  D.noise_warps = noise_warps(tps, bpt, threads, P);
  v->fn<<<blocks, block_threads(tps, bpt, threads, P), smem, stream>>>(k, D);
  return cudaGetLastError();
}

}  // namespace brmppi
