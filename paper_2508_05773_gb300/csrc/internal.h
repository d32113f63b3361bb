// internal.h -- private host-side structures of libbrmppi.so, shared by the
// C-ABI translation unit (api.cu) and the serving loop (serve.cu).
#pragma once

#include <cmath>
#include <cstdint>
#include <map>
#include <string>

#include "brmppi.h"
#include "launch.h"

namespace brmppi_host {

constexpr int kMaxObstacles = 124;  // ceil((4 + n)/4) <= 32 Philox blocks
constexpr int kMaxPathPts = 8192;  // 5 floats a row in shared memory
constexpr int kMaxH = 1024;
constexpr int kMinThreads = 64;
constexpr int kMaxThreads = 512;
constexpr int kMinBatchSpb = 16;  // smallest tile of a batch launch
constexpr int kMaxResidentThreads = 2048;

// Doubles of a state (the jerk-input model adds the acceleration).
inline int state_dim(const brmppi_params& p) { return (p.flags & BRMPPI_FLAG_JERK_MODEL) ? 8 : 7; }

// Constraint rows of obstacles: each obstacle seen from every footprint disc.
inline int rows_of(const brmppi_params& p, int n_obs) { return n_obs * p.n_discs; }

// Floats per obstacle row, and the exponents a row may carry.
inline int obs_floats(const brmppi_params& p) { return (p.flags & BRMPPI_FLAG_OBS8) ? 8 : 6; }
inline bool exponent_ok(const brmppi_params& p, float e) {
  return e == 2.0f || ((p.flags & BRMPPI_FLAG_OBS8) && e == 4.0f);
}

// Consecutive path headings at most pi/4 apart (and finite): the kernel
// turns each row's heading direction by the interpolation angle.
inline bool path_turns_ok(const float* path, int n_pts) {
  for (int j = 0; j + 1 < n_pts; ++j)
    if (!(std::fabs(path[3 * j + 5] - path[3 * j + 2]) <= 0.78539816339744831f)) return false;
  return true;
}

struct Shape {
  int tps = 0, bpt = 0, threads = 0;
};

// Everything one in-flight batch launch needs: instance table, work list,
// per-tile partial pool, per-instance counters, per-CTA input history, host
// staging of the table and list, and the events that guard their reuse.
struct Lane {
  brmppi::Inst* d_inst = nullptr;
  int2* d_work = nullptr;
  unsigned int* d_work_ctr = nullptr;
  float* d_bpart = nullptr;
  unsigned int* d_bsync = nullptr;
  float* d_buh = nullptr;
  brmppi::Inst* h_inst = nullptr;
  int2* h_work = nullptr;
  cudaEvent_t upload_done = nullptr;  // host staging free again
  cudaEvent_t batch_done = nullptr;   // device table free again
  cudaStream_t stream = nullptr;      // owned when the lane belongs to the server
  bool pending = false;
  int max_batch = 0;
  size_t bpart_floats = 0, buh_floats = 0, max_work = 0;
};

struct BatchPlan {
  Shape shape;
  int n_inst = 0, n_work = 0, grid = 0, Hmax = 0;
  bool any_u_safe = false;  // some instance asks for the stabilized input
  int P = 1;                // Philox blocks per step the launch is shaped for
  brmppi::SmemCaps caps{};
  size_t smem = 0;
};

struct Server;

}  // namespace brmppi_host

struct brmppi_ctx {
  brmppi_params prm{};
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  size_t smem_limit = 0;
  // plain solves
  unsigned char* d_in = nullptr;  // x0 | U_nom | obs | path
  float* d_J = nullptr;
  float* d_part = nullptr;
  unsigned int* d_sync = nullptr;  // finished tiles, error bits
  float* d_uh = nullptr;
  unsigned char* h_in = nullptr;
  float* h_out = nullptr;          // U | traj | status of brmppi_solve (written by the kernel)
  float* d_out = nullptr;          // the same on the device: the autotuner's scratch
  size_t off_unom = 0, off_obs = 0, off_path = 0, in_bytes = 0, out_floats = 0;
  size_t part_stride = 0, part_tiles = 0, uh_floats = 0;
  std::map<int, brmppi_host::Shape> tuned;  // obstacle count -> fastest plain shape
  // batches
  brmppi_host::Lane batch;
  bool batch_tuned = false;
  brmppi_host::Shape batch_shape;
  // serving
  brmppi_host::Server* server = nullptr;
  std::string err;
};

struct brmppi_graph {
  brmppi_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  brmppi::Inst* h_inst = nullptr;
  int2* h_work = nullptr;
};

namespace brmppi_host {

size_t align_up(size_t v, size_t a);

// Every device and pinned-host allocation of the library goes through these
// two.  A test hook (brmppi_inject_alloc_failure) makes the n-th allocation
// from then on fail with cudaErrorMemoryAllocation without calling CUDA, so
// that the out-of-memory paths (BRMPPI_ENOMEM, clean unwinding) can be
// exercised without exhausting a device.
cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t host_alloc(void** p, size_t bytes);
template <typename T>
cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_alloc(reinterpret_cast<void**>(p), bytes);
}
template <typename T>
cudaError_t host_alloc(T** p, size_t bytes) {
  return host_alloc(reinterpret_cast<void**>(p), bytes);
}

// Bounded waits of the host threads: poll an event or a stream until it
// completes (cudaSuccess), fails (its error) or `timeout_ms` passes
// (cudaErrorNotReady).
cudaError_t wait_event(cudaEvent_t ev, int timeout_ms);
cudaError_t wait_stream(cudaStream_t s, int timeout_ms);
// The host-wait limit of a context (params.wait_timeout_ms, 0 = 10 s).
inline int wait_limit_ms(const brmppi_params& p) { return p.wait_timeout_ms > 0 ? p.wait_timeout_ms : 10000; }
brmppi_status fail(brmppi_ctx* c, brmppi_status st, const std::string& msg);
brmppi_status cuda_fail(brmppi_ctx* c, cudaError_t e, const char* what);
int philox_blocks(int n_rows);  // per step, for n_rows obstacle rows
bool pick_bpt(int tps, int P, int* bpt);
int part_stride_for(int H);
// Team width of batches and serving when the optional terms are on: at most
// two Philox blocks per lane.
int ext_team_width(int P);
brmppi_status check_sizes(brmppi_ctx* c, int32_t n_obs, int32_t n_pts, float ds);
// Options of a single (non-batch) solve launch: the exact-rows variant, with
// the applied-input history and the merge of the tile partials in shared
// memory, when the variant exists and the room fits (L.rows,
// L.caps.uh_per_team, L.caps.merge); L.caps and L.single must be set.
void single_launch_options(brmppi::LaunchDesc& L, const Shape& sh, const brmppi::KConst& k, int n_rows, int H,
                           size_t smem_limit);

// Allocate / free the buffers of a lane for max_batch instances of at most
// S samples and H steps.
cudaError_t lane_alloc(Lane& L, int max_batch, size_t S, size_t H, int num_sms, size_t part_stride);
// Free a lane; false (nothing freed) if its last batch did not finish within
// timeout_ms.
bool lane_free(Lane& L, int timeout_ms);

// Validate instances and fill a lane's host staging (table + longest-first
// work list); `forced` fixes the launch shape (else the context's batch shape).
brmppi_status plan_batch(brmppi_ctx* c, Lane& L, const brmppi_instance* inst, int32_t n, const Shape* forced,
                         brmppi::Inst* h_inst, int2* h_work, BatchPlan* plan);
// Upload the staging and launch on `stream` (waits for the lane's previous batch).
brmppi_status upload_and_launch(brmppi_ctx* c, Lane& L, const BatchPlan& plan, const brmppi::Inst* h_inst,
                                const int2* h_work, cudaStream_t stream);

// Serving loop (serve.cu).
brmppi_status server_create(brmppi_ctx* c);
// Stop and free the serving loop; false if a lane did not finish within the
// context's wait limit (its buffers are then left allocated).
bool server_destroy(brmppi_ctx* c);

}  // namespace brmppi_host
