// tiled_kernels.h -- host interface of kernels_tiled.cu: the synchronous FP32
// iteration with a tile of particles and all their dimensions per block.
#pragma once

#include <cuda_runtime.h>

#include "cupso_device.cuh"

namespace cupso {

constexpr int kTiledItems = 4096;   // P * D per tile at most (x' and the fitness terms in shared memory)
constexpr int kTiledMaxP = 256;     // particles per tile at most (one per thread)

// The tiles of a batch: (swarm, tile) units in hand-out order, and per swarm
// its particles per tile and tile count.
struct BatchTiles {
    const uint2* units;
    unsigned int nunits;
    const int* P;
    const unsigned int* ntiles;
};

// Particles per tile for (N, D) on num_sms SMs: a power of two up to
// kTiledMaxP, at most kTiledItems / D, and (down to 4) small enough that the
// tiles cover the SMs twice over. 0 when D > kTiledItems.
int tiled_particles(int N, int D, int num_sms);

// Particles per tile of a batch swarm with D dimensions: the largest power of
// two up to kTiledMaxP with P * D <= kTiledItems (tiles of similar cost).
int batch_tile_particles(int D);

// The asynchronous mode in tiles: the record prologue, then `iters`
// iterations of persistent CTAs with no grid barrier (iterations t_first ...).
cudaError_t launch_async_tiled(const SwarmDev& s, int fid, int P, int grid, uint32_t t_first, int iters,
                               int hold_lock, cudaStream_t st);
int async_tiled_blocks_per_sm(int P, int D);

// The record prologue of the asynchronous kernels (kernels_stream.cu):
// gbest into the lock-protected record, lock released (or held, a test hook).
cudaError_t launch_async_prologue(const SwarmDev& s, int hold_lock, cudaStream_t st);

// One iteration of every swarm of a batch, in tiles; `grid` CTAs.
cudaError_t launch_batch_tiled(const BatchDev& b, const BatchTiles& bt, int grid, cudaStream_t st);
int batch_tiled_blocks_per_sm();

// One iteration (Steps 2-5) with tiles of P particles; `grid` blocks walk the
// tiles (at most one block per tile).
cudaError_t launch_sync_tiled(const SwarmDev& s, int fid, int P, int grid, cudaStream_t st);

// Resident blocks per SM of the tiled kernel for (fitness, P, D).
int tiled_blocks_per_sm(int fid, int P, int D);

}  // namespace cupso
