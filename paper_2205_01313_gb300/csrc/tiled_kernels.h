// tiled_kernels.h -- host interface of kernels_tiled.cu: the synchronous FP32
// iteration with a tile of particles and all their dimensions per block.
#pragma once

#include <cuda_runtime.h>

#include "cupso_device.cuh"

namespace cupso {

constexpr int kTiledItems = 4096;   // P * D per tile at most (x' and the fitness terms in shared memory)

// Particles per tile for (N, D) on num_sms SMs: a power of two up to 32, at
// most kTiledItems / D, and (down to 4) small enough that the tiles cover the
// SMs twice over. 0 when D > kTiledItems.
int tiled_particles(int N, int D, int num_sms);

// One iteration (Steps 2-5) with tiles of P particles; `grid` blocks walk the
// tiles (at most one block per tile).
cudaError_t launch_sync_tiled(const SwarmDev& s, int fid, int P, int grid, cudaStream_t st);

// Resident blocks per SM of the tiled kernel for (fitness, P, D).
int tiled_blocks_per_sm(int fid, int P, int D);

}  // namespace cupso
