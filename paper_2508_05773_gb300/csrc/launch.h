// launch.h -- host-side interface between the C ABI and the solve kernels.
#pragma once

#include <cuda_runtime.h>

#include "rollout.cuh"

namespace brmppi {

using KernelFn = void (*)(const KConst, const LaunchDesc);

struct Variant {
  int tps, bpt;
  bool ext;  // carries the optional terms (BRMPPI_FLAG_COLLISION_COST, _OBS8, _ALPHA_BUFFER,
             // footprint discs other than the rear-axle point)
  KernelFn fn;
  int rows = 0;  // > 0: exactly this many constraint rows a lane (single solves)
};

// Instantiations, one translation unit per group of team widths and family
// (compiled in parallel); each returns its table and its length.  Both
// families hold the same (tps, bpt) pairs.
const Variant* variants_narrow(int* n);      // 1 and 2 lanes per sample
const Variant* variants_wide(int* n);        // 4 .. 32 lanes per sample
const Variant* variants_narrow_ext(int* n);  // the same, with the optional terms
const Variant* variants_wide_ext(int* n);
const Variant* variants_latency(int* n);     // exact rows a lane, noise-warp shapes
const Variant* variants_latency_ext(int* n); // the same with the optional terms (4 lanes)

// Whether a launch with these constants needs the family with the optional terms.
inline bool needs_ext(const KConst& k) { return k.coll || k.obs8 || k.abuf || k.discs || k.third || k.jerk; }

// Threads of a launch: `threads` roll out samples; teams wider than one lane
// with at most two Philox blocks per lane add warps that produce the noise,
// enough for two blocks per producer lane and step where the CTA has room
// (up to four; P blocks per sample).  Other variants draw on their own
// lanes (0 noise warps).  At most kMaxBlockThreads (the kernels' launch
// bound).
constexpr int kMaxBlockThreads = 512;
constexpr int kMaxRowsBlockThreads = 384;  // the exact-rows instantiations' launch bound
int noise_warps(int tps, int bpt, int threads, int P);
int block_threads(int tps, int bpt, int threads, int P);

// The rows a lane holds in a single solve of n_rows constraint rows on a
// noise-warp shape, if the instantiation with exactly that many is compiled
// (LaunchDesc::rows), else 0.
int exact_rows_variant(int tps, int bpt, const KConst& k, int n_rows);

// Supported (threads per sample, Philox blocks per lane) pairs.
bool variant_exists(int tps, int bpt);

// Raise the dynamic shared-memory limit of every variant to `bytes`.
cudaError_t set_smem_limit(size_t bytes);

// CTAs of a variant resident per SM for a launch shape (0 if it cannot run).
int variant_occupancy(int tps, int bpt, int threads, size_t smem, bool ext, int P);

// Enqueue the hitch stabilizer for n states (out: n x 4 floats).
cudaError_t launch_stabilize(const KConst& k, const double* x, const float* u_ref, int n, float* out,
                             cudaStream_t stream);

// Enqueue the hitch stabilizer for the instances of a device table whose
// u_safe is set (after their solve, on the same stream).
cudaError_t launch_stabilize_table(const KConst& k, const Inst* d_table, int n, cudaStream_t stream);

// Enqueue the noise-table kernel: Philox words and Box-Muller normals of
// samples < n_samples, steps < H, blocks < n_blocks (words or normals may
// be null).
cudaError_t launch_noise_blocks(uint64_t seed, uint64_t counter, int n_samples, int H, int n_blocks, uint32_t* words,
                                float* normals, cudaStream_t stream);

// Enqueue the one-CTA merge of an instance's gathered tile partials
// (in.part, in.tiles; caps: the instance's tables; smem: their bytes).
cudaError_t launch_merge_tiles(const KConst& k, const Inst& in, const SmemCaps& caps, size_t smem,
                               cudaStream_t stream);

// Enqueue one launch of the solve kernel.
cudaError_t launch_solve(int tps, int bpt, int blocks, int threads, size_t smem, cudaStream_t stream,
                         const KConst& k, const LaunchDesc& L, int P);

}  // namespace brmppi
