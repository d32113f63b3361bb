// launch.h -- host-side interface between the C ABI and the rollout kernels.
#pragma once

#include <cuda_runtime.h>

#include "rollout.cuh"

namespace brmppi {

// Supported (threads per sample, Philox blocks per lane) pairs.
bool variant_exists(int tps, int bpt);
// Largest Philox-block count (ceil(d/4)) a tps can serve.
int variant_max_blocks(int tps);

// Shared memory a launch needs, in bytes.
size_t smem_bytes(int n_obs, int n_pts, int H, int spb);

// Raise the dynamic shared-memory limit of every variant to `bytes`.
cudaError_t set_smem_limit(size_t bytes);

// Enqueue one solve kernel.
cudaError_t launch_rollout(int tps, int bpt, int blocks, int threads, size_t smem, cudaStream_t stream,
                           const KParams& p, const KIO& io);

}  // namespace brmppi
