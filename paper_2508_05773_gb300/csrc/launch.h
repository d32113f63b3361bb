// launch.h -- host-side interface between the C ABI and the solve kernels.
#pragma once

#include <cuda_runtime.h>

#include "rollout.cuh"

namespace brmppi {

using KernelFn = void (*)(const KConst, const LaunchDesc);

struct Variant {
  int tps, bpt;
  KernelFn fn;
};

// Instantiations, one translation unit per group of team widths (compiled
// in parallel); each returns its table and its length.
const Variant* variants_narrow(int* n);  // 1 and 2 lanes per sample
const Variant* variants_wide(int* n);    // 4 .. 32 lanes per sample

// Supported (threads per sample, Philox blocks per lane) pairs.
bool variant_exists(int tps, int bpt);

// Raise the dynamic shared-memory limit of every variant to `bytes`.
cudaError_t set_smem_limit(size_t bytes);

// CTAs of a variant resident per SM for a launch shape (0 if it cannot run).
int variant_occupancy(int tps, int bpt, int threads, size_t smem);

// Enqueue one launch of the solve kernel.
cudaError_t launch_solve(int tps, int bpt, int blocks, int threads, size_t smem, cudaStream_t stream,
                         const KConst& k, const LaunchDesc& L);

}  // namespace brmppi
