// cupso_internal.h -- host-side launch wrappers shared by the C-ABI layer.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cupso.h"
#include "cupso_device.cuh"

namespace cupso {

constexpr int kBlock = 256;             // threads per CTA of the streaming kernels
constexpr int kPerThread = 4;           // particles per thread (one float4)
constexpr int kTile = kBlock * kPerThread;
constexpr int kPad = 128;               // Np = N rounded up to a multiple of this

__host__ __device__ inline int tiles_of(int Np) { return (Np + kTile - 1) / kTile; }

// All wrappers return a cudaError_t of the launch.
cudaError_t launch_init(const SwarmDev& s, int fid, int grid, cudaStream_t st);
cudaError_t launch_sync_step(const SwarmDev& s, int fid, int grid, cudaStream_t st);
cudaError_t launch_tree_step(const SwarmDev& s, int fid, bool unrolled, cudaStream_t st);
// ASYNC: `block` threads per CTA (a multiple of 32, <= kBlock), each CTA a
// tile of 4 * block particles per pass.
cudaError_t launch_async(const SwarmDev& s, int fid, int grid, int block, uint32_t t_first, int iters,
                         int hold_lock, cudaStream_t st);
cudaError_t launch_recompute(const SwarmDev& s, uint32_t t, cudaStream_t st);

// Pipelined fused step (kernels_pipelined.cu): `stages`-deep cp.async ring.
bool pipelined_supported(int stages, int D);
cudaError_t prepare_pipelined(int D);   // raise the dynamic shared-memory limit; call outside capture
// ppt: particles per thread (4, 2 or 1); a warp takes units of 32 * ppt particles.
int pipelined_blocks_per_sm(int stages, int fid, int D, int ppt);
cudaError_t launch_sync_pipelined(const SwarmDev& s, int fid, int stages, int ppt, int grid, cudaStream_t st);
// Write back the pbest rows the pipelined step left pending (lazy pbest) and clear the flags.
cudaError_t launch_materialize(const SwarmDev& s, int grid, cudaStream_t st);

// Batched step (kernels_batch.cu): one iteration of every swarm of a batch.
cudaError_t prepare_batch();
// Shapes: (stages, minb) in {(3, 2), (3, 3), (4, 2)}; minb = CTAs per SM the
// register budget is sized for.
int batch_blocks_per_sm(int stages, int minb);
cudaError_t launch_batch_step(const BatchDev& b, int stages, int minb, int grid, cudaStream_t st);
// Step 1 (t = 0) of every swarm of a batch in one launch, over the same units;
// per swarm the same bits as launch_init. Needs gkey = all ones, done and
// pflag zero.
cudaError_t launch_batch_init(const BatchDev& b, int grid, cudaStream_t st);

// Fused SYNC step on the panel layout (kernels_panel.cu): element (d, i) of
// x, v, pb at ((d / W) * Np + i) * W + d % W, panel width W = 8 or 16, ring
// depth 3 or 5 panels.
bool panel_supported(int width, int stages, int D);
cudaError_t prepare_panel(int D);
int panel_blocks_per_sm(int width, int stages, int fid, int D);
// Iterations of one panel launch; more than one is a cooperative launch with a
// grid barrier per iteration (every CTA resident; see kernels_panel.cu).
constexpr int kPanelMaxIters = 4096;
cudaError_t launch_sync_panel(const SwarmDev& s, int fid, int width, int stages, int grid, int iters,
                              bool stall_barrier, cudaStream_t st);
cudaError_t launch_materialize_panel(const SwarmDev& s, int width, int grid, cudaStream_t st);
// dst = src in the other layout (dimension-major <-> panel of width W); D % W == 0.
cudaError_t launch_relayout(const float* src, float* dst, int D, int Np, int width, bool to_panel, int grid,
                            cudaStream_t st);

// Resident CTAs per SM of the persistent kernels (for grid sizing).
int sync_blocks_per_sm(int fid, int D);
int async_blocks_per_sm(int fid, int D);

// Record an error message for cupso_last_error() on the calling thread.
void set_last_error(const char* msg);
void set_cuda_error(cudaError_t e, const char* where);

// Host-side argument check of one problem (CUPSO_OK or CUPSO_ERR_INVALID_ARG).
int check_problem_args(int D, int N, const cupso_bounds* b, float w, float c1, float c2, int fid);
// Solve one problem through its own handle (create, iters steps, gbest, destroy).
int solve_one_plain(const cupso_problem& p, int iters, cupso_result& r, cudaStream_t stream);

// On-chip variant: whole swarm in the shared memory of one thread-block
// cluster, many iterations per launch.
bool onchip_fits(int N, int D, int* cluster_out, int* per_cta_out);
cudaError_t launch_onchip(const SwarmDev& s, int fid, int iters, cudaStream_t st);

}  // namespace cupso
