// kernels_stream.cu -- PSO iteration kernels that stream the swarm through HBM.
//
// One CTA of 256 threads moves a tile of 1024 particles; each thread owns
// four consecutive particles and walks the dimensions two at a time (one
// Philox call yields r1, r2 for two dimensions of one particle).
//
//  * init_kernel        Step 1 of Alg. 1 (Sec. 2.1) on the device.
//  * sync_step_kernel   Steps 2-5 fused into one launch. Global best by the
//                       paper's conditional update (Sec. 3.1: only particles
//                       that beat the current best compete), done as a warp
//                       shuffle argmin and one 64-bit atomicMin on a packed
//                       (fitness key, index); the last CTA to finish gathers
//                       gbest_pos (index first, position after, Sec. 4.3).
//  * tree_k1 / tree_k2  The parallel-reduction baseline of Sec. 2.2 (Fig. 1):
//                       block tree reduction into auxiliary arrays, then a
//                       second one-block kernel. `unrolled` is the loop-
//                       unrolling variant of the same section.
//  * async_kernel       Sec. 3.2 (Alg. 3) taken to its asynchronous end (the
//                       future work of Sec. 6): persistent CTAs iterate on
//                       their own particles with no grid barrier, against a
//                       lock-protected global best read under a sequence lock
//                       (async_common.cuh). Large swarms and D = 1; smaller
//                       ones run the tiled form (kernels_tiled.cu).
//  * recompute_kernel   gbest from pbest after the host loads a state.
#include <cuda_runtime.h>

#include "cupso_device.cuh"
#include "async_common.cuh"
#include "cupso_internal.h"
#include "stream_common.cuh"
#include "tiled_kernels.h"

namespace cupso {

// ---------------------------------------------------------------------------
// Step 1 (t = 0): pos0 = min_pos + u (max_pos - min_pos), v0 = -max_v + u 2 max_v,
// fitness, pbest = pos0, gbest = argmin. Keys of every particle compete.
// ---------------------------------------------------------------------------
template <int FIT>
__global__ void __launch_bounds__(kBlock) init_kernel(const __grid_constant__ SwarmDev s) {
    __shared__ unsigned long long red[kBlock / 32];
    const size_t Np = (size_t)s.Np;
    const float span = __fsub_rn(s.hi, s.lo);
    const float vspan = __fmul_rn(2.0f, s.vmax);
    unsigned long long best = kKeyNone;
    bool nan = false;
    const int ntiles = tiles_of(s.Np);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t i0 = (uint32_t)tile * kTile + threadIdx.x * kPerThread;
        if (i0 >= (uint32_t)s.Np) continue;
        FitAcc<FIT> acc[4];
        for (int d0 = 0; d0 < s.D; d0 += 2) {
            uint4 r[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                r[j] = philox4x32_10(make_uint4((uint32_t)(d0 >> 1), i0 + j, 0u, s.swarm), s.key0, s.key1);
            for (int h = 0; h < 2 && d0 + h < s.D; ++h) {
                const int d = d0 + h;
                float4 X, V;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float xj = clampf(__fmaf_rn(u01(word(r[j], 2 * h)), span, s.lo), s.lo, s.hi);
                    const float vj = clampf(__fmaf_rn(u01(word(r[j], 2 * h + 1)), vspan, -s.vmax),
                                            -s.vmax, s.vmax);
                    set_lane(X, j, xj);
                    set_lane(V, j, vj);
                    acc[j].add(d, xj);
                }
                const size_t off = (size_t)d * Np + i0;
                st4(s.x + off, X);
                st4(s.v + off, V);
                st4(s.pb + off, X);
            }
        }
        float4 PF;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float f = acc[j].finish(s.D);
            set_lane(PF, j, f);
            if (i0 + j < (uint32_t)s.N) {
                const unsigned long long k = pack_key(f, i0 + j);
                best = k < best ? k : best;
                nan |= (f != f);
            }
        }
        st4(s.pf + i0, PF);
    }
    best = block_min(best, red);
    if (threadIdx.x == 0 && best != kKeyNone) atomicMin(s.gkey + 0, best);
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
    // t = 0 lives in slot 0; the epilogue copies it to slot 1 as well.
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(s.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const unsigned long long k0 = __ldcg(s.gkey + 0);
    const uint32_t g = (uint32_t)(k0 & 0xFFFFFFFFull);
    for (int d = threadIdx.x; d < s.D; d += blockDim.x) s.G[d] = __ldcg(s.pb + (size_t)d * Np + g);
    if (threadIdx.x == 0) {
        s.gkey[1] = k0;
        *s.t_dev = 0u;
        *s.ticket = 0u;
    }
}

// ---------------------------------------------------------------------------
// Synchronous fused iteration: Steps 2-5 in one launch.
// ---------------------------------------------------------------------------
template <int FIT>
__global__ void __launch_bounds__(kBlock) sync_step_kernel(const __grid_constant__ SwarmDev s) {
    extern __shared__ float Gs[];
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    const uint32_t t = t_prev + 1u;
    const unsigned long long K = __ldcg(s.gkey + cur);   // gbest at the end of t-1
    for (int d = threadIdx.x; d < s.D; d += blockDim.x) Gs[d] = __ldcg(s.G + (size_t)cur * s.D + d);
    __syncthreads();

    unsigned long long best = kKeyNone;
    bool nan = false;
    const int ntiles = tiles_of(s.Np);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t i0 = (uint32_t)tile * kTile + threadIdx.x * kPerThread;
        if (i0 >= (uint32_t)s.Np) continue;
        float f[4], pf[4];
        move4<FIT>(s, i0, t, Gs, f);
        const unsigned mask = pbest4(s, i0, f, pf);
        // Step 5, conditional: only a particle that just improved and now beats
        // the current gbest can change it (Sec. 3.1).
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (mask & (1u << j)) {
                const unsigned long long k = pack_key(f[j], i0 + j);
                if (k < K && k < best) best = k;
            }
        }
        nan |= any_nan4(s, i0, f);
    }
    best = warp_min_u64(best);
    if ((threadIdx.x & 31) == 0 && best < K) atomicMin(s.gkey + nxt, best);
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
    finish_iteration(s, cur, nxt, t);
}

// ---------------------------------------------------------------------------
// Tree-reduction baseline (Sec. 2.2, Fig. 1): first kernel = per-particle work
// plus a block tree reduction over every particle's pbest into aux[block];
// second kernel = one block reduces aux and gathers gbest_pos.
// ---------------------------------------------------------------------------
template <int FIT, bool UNROLLED>
__global__ void __launch_bounds__(kBlock) tree_k1(const __grid_constant__ SwarmDev s) {
    extern __shared__ float Gs[];
    __shared__ unsigned long long red[kBlock];
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur = (int)(t_prev & 1u);
    const uint32_t t = t_prev + 1u;
    for (int d = threadIdx.x; d < s.D; d += blockDim.x) Gs[d] = __ldcg(s.G + (size_t)cur * s.D + d);
    __syncthreads();

    const uint32_t i0 = (uint32_t)blockIdx.x * kTile + threadIdx.x * kPerThread;
    unsigned long long best = kKeyNone;
    bool nan = false;
    if (i0 < (uint32_t)s.Np) {
        float f[4], pf[4];
        move4<FIT>(s, i0, t, Gs, f);
        pbest4(s, i0, f, pf);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (i0 + j < (uint32_t)s.N) {
                const unsigned long long k = pack_key(pf[j], i0 + j);
                best = k < best ? k : best;
            }
        }
        nan = any_nan4(s, i0, f);
    }
    red[threadIdx.x] = best;
    __syncthreads();
    if (!UNROLLED) {
        // classic shared-memory tree: halve the active range every step
        for (unsigned stride = blockDim.x / 2; stride > 0; stride >>= 1) {
            if (threadIdx.x < stride) {
                const unsigned long long o = red[threadIdx.x + stride];
                if (o < red[threadIdx.x]) red[threadIdx.x] = o;
            }
            __syncthreads();
        }
    } else {
        // unrolled: fixed strides down to one warp, then shuffles (no barriers)
#pragma unroll
        for (unsigned stride = kBlock / 2; stride >= 32; stride >>= 1) {
            if (threadIdx.x < stride) {
                const unsigned long long o = red[threadIdx.x + stride];
                if (o < red[threadIdx.x]) red[threadIdx.x] = o;
            }
            __syncthreads();
        }
        if (threadIdx.x < 32) {
            const unsigned long long k = warp_min_u64(red[threadIdx.x]);
            if (threadIdx.x == 0) red[0] = k;
        }
    }
    if (threadIdx.x == 0) s.aux[blockIdx.x] = red[0];
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
}

__global__ void __launch_bounds__(1024) tree_k2(const __grid_constant__ SwarmDev s, int nblocks) {
    __shared__ unsigned long long red[1024];
    __shared__ uint32_t s_g;
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    unsigned long long k = kKeyNone;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const unsigned long long o = __ldcg(s.aux + b);
        k = o < k ? o : k;
    }
    red[threadIdx.x] = k;
    __syncthreads();
    for (unsigned stride = blockDim.x / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride) {
            const unsigned long long o = red[threadIdx.x + stride];
            if (o < red[threadIdx.x]) red[threadIdx.x] = o;
        }
        __syncthreads();
    }
    const unsigned long long knew = red[0];
    if (threadIdx.x == 0) s_g = (uint32_t)(knew & 0xFFFFFFFFull);
    __syncthreads();
    const uint32_t g = s_g;
    if (g < (uint32_t)s.N)
        for (int d = threadIdx.x; d < s.D; d += blockDim.x)
            s.G[(size_t)nxt * s.D + d] = __ldcg(s.pb + (size_t)d * s.Np + g);
    if (threadIdx.x == 0) {
        s.gkey[0] = knew;
        s.gkey[1] = knew;
        *s.t_dev = t_prev + 1u;
    }
}

// ---------------------------------------------------------------------------
// Asynchronous variant. Every wait is bounded by s.wait_limit_ns; on expiry the
// kernel sets kStatusTimeout and every CTA stops at its next iteration.
// ---------------------------------------------------------------------------
__global__ void async_prologue(const __grid_constant__ SwarmDev s, int hold_lock) {
    const uint32_t t = __ldcg(s.t_dev);
    const int cur = (int)(t & 1u);
    for (int d = threadIdx.x; d < s.D; d += blockDim.x) s.Grec[d] = s.G[(size_t)cur * s.D + d];
    if (threadIdx.x == 0) {
        const unsigned long long k = s.gkey[cur];
        *s.reckey = k;
        *s.claim = k;
        *s.seq = 0u;
        *s.lock = hold_lock ? 1u : 0u;  // a held lock is a fault-injection hook: waits must expire
        *s.ticket = 0u;
    }
}

template <int FIT>
__global__ void __launch_bounds__(kBlock) async_kernel(const __grid_constant__ SwarmDev s, uint32_t t_first,
                                                       int iters) {
    extern __shared__ float Gs[];
    __shared__ unsigned long long red[kBlock / 32];
    __shared__ int s_stop;
    // Tiles follow the block size, so small swarms still spread over many CTAs.
    const uint32_t tile_sz = blockDim.x * kPerThread;
    const int ntiles = (int)(((uint32_t)s.Np + tile_sz - 1) / tile_sz);
    for (int k = 0; k < iters; ++k) {
        const uint32_t t = t_first + (uint32_t)k;
        if (threadIdx.x == 0) s_stop = (__ldcg(s.status) & kStatusTimeout) != 0u;
        __syncthreads();
        if (s_stop) break;
        if (!read_record(s, Gs)) {
            if (threadIdx.x == 0) atomicOr(s.status, kStatusTimeout);
            break;
        }
        const unsigned long long K = __ldcg(s.claim);
        unsigned long long best = kKeyNone;
        bool nan = false;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const uint32_t i0 = (uint32_t)tile * tile_sz + threadIdx.x * kPerThread;
            if (i0 >= (uint32_t)s.Np) continue;
            float f[4], pf[4];
            move4<FIT>(s, i0, t, Gs, f);
            const unsigned mask = pbest4(s, i0, f, pf);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (mask & (1u << j)) {
                    const unsigned long long kk = pack_key(f[j], i0 + j);
                    if (kk < K && kk < best) best = kk;
                }
            }
            nan |= any_nan4(s, i0, f);
        }
        if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
        best = block_min(best, red);   // ends with a barrier: pbest writes are visible
        if (best != kKeyNone && threadIdx.x < 32) {
            if (!publish(s, best) && threadIdx.x == 0) atomicOr(s.status, kStatusTimeout);
        }
        __syncthreads();
    }
    // The last CTA to finish hands the record back to the synchronous state.
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(s.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const uint32_t t_end = t_first - 1u + (uint32_t)iters;
    const int cur = (int)(t_end & 1u);
    for (int d = threadIdx.x; d < s.D; d += blockDim.x) s.G[(size_t)cur * s.D + d] = __ldcg(s.Grec + d);
    if (threadIdx.x == 0) {
        const unsigned long long k = __ldcg(s.reckey);
        s.gkey[0] = k;
        s.gkey[1] = k;
        *s.t_dev = t_end;
        *s.ticket = 0u;
    }
}

// ---------------------------------------------------------------------------
// gbest = lexicographic argmin over (pbest_fit, index), one block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) recompute_kernel(const __grid_constant__ SwarmDev s, uint32_t t) {
    __shared__ unsigned long long red[32];
    unsigned long long k = kKeyNone;
    bool nan = false;
    for (int i = threadIdx.x; i < s.N; i += blockDim.x) {
        const float f = s.pf[i];
        const unsigned long long kk = pack_key(f, (uint32_t)i);
        k = kk < k ? kk : k;
        nan |= (f != f);
    }
    k = block_min(k, red);
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
    const int cur = (int)(t & 1u);
    const uint32_t g = (uint32_t)(k & 0xFFFFFFFFull);
    for (int d = threadIdx.x; d < s.D; d += blockDim.x) s.G[(size_t)cur * s.D + d] = s.pb[(size_t)d * s.Np + g];
    if (threadIdx.x == 0) {
        s.gkey[0] = k;
        s.gkey[1] = k;
        *s.t_dev = t;
        *s.ticket = 0u;
    }
}

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
#define CUPSO_DISPATCH_FIT(fid, KERNEL_CALL)                       \
    switch (fid) {                                                 \
        case kSphere: { constexpr int F = kSphere; KERNEL_CALL; } break;         \
        case kRastrigin: { constexpr int F = kRastrigin; KERNEL_CALL; } break;   \
        case kAckley: { constexpr int F = kAckley; KERNEL_CALL; } break;         \
        case kRosenbrock: { constexpr int F = kRosenbrock; KERNEL_CALL; } break; \
        case kCubicMax: { constexpr int F = kCubicMax; KERNEL_CALL; } break;     \
        default: return cudaErrorInvalidValue;                     \
    }

// Step 1 also covers the least-squares fitness (its values come later).
#define CUPSO_DISPATCH_FIT_INIT(fid, KERNEL_CALL)                  \
    if (fid == kLsq) { constexpr int F = kLsq; KERNEL_CALL; } else CUPSO_DISPATCH_FIT(fid, KERNEL_CALL)

cudaError_t launch_init(const SwarmDev& s, int fid, int grid, cudaStream_t st) {
    CUPSO_DISPATCH_FIT_INIT(fid, (init_kernel<F><<<grid, kBlock, 0, st>>>(s)));
    return cudaGetLastError();
}

cudaError_t launch_sync_step(const SwarmDev& s, int fid, int grid, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)s.D;
    CUPSO_DISPATCH_FIT(fid, (sync_step_kernel<F><<<grid, kBlock, smem, st>>>(s)));
    return cudaGetLastError();
}

cudaError_t launch_tree_step(const SwarmDev& s, int fid, bool unrolled, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)s.D;
    const int nb = tiles_of(s.Np);
    if (unrolled) {
        CUPSO_DISPATCH_FIT(fid, (tree_k1<F, true><<<nb, kBlock, smem, st>>>(s)));
    } else {
        CUPSO_DISPATCH_FIT(fid, (tree_k1<F, false><<<nb, kBlock, smem, st>>>(s)));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tree_k2<<<1, 1024, 0, st>>>(s, nb);
    return cudaGetLastError();
}

cudaError_t launch_async_prologue(const SwarmDev& s, int hold_lock, cudaStream_t st) {
    async_prologue<<<1, 256, 0, st>>>(s, hold_lock);
    return cudaGetLastError();
}

cudaError_t launch_async(const SwarmDev& s, int fid, int grid, int block, uint32_t t_first, int iters,
                         int hold_lock, cudaStream_t st) {
    async_prologue<<<1, 256, 0, st>>>(s, hold_lock);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(float) * (size_t)s.D;
    CUPSO_DISPATCH_FIT(fid, (async_kernel<F><<<grid, block, smem, st>>>(s, t_first, iters)));
    return cudaGetLastError();
}

cudaError_t launch_recompute(const SwarmDev& s, uint32_t t, cudaStream_t st) {
    recompute_kernel<<<1, 1024, 0, st>>>(s, t);
    return cudaGetLastError();
}

namespace {
template <typename K>
int blocks_per_sm(K kernel, int D) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kBlock, sizeof(float) * (size_t)D) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}
}  // namespace

int sync_blocks_per_sm(int fid, int D) {
    switch (fid) {
        case kSphere: return blocks_per_sm(sync_step_kernel<kSphere>, D);
        case kRastrigin: return blocks_per_sm(sync_step_kernel<kRastrigin>, D);
        case kAckley: return blocks_per_sm(sync_step_kernel<kAckley>, D);
        case kRosenbrock: return blocks_per_sm(sync_step_kernel<kRosenbrock>, D);
        default: return blocks_per_sm(sync_step_kernel<kCubicMax>, D);
    }
}

int async_blocks_per_sm(int fid, int D) {
    switch (fid) {
        case kSphere: return blocks_per_sm(async_kernel<kSphere>, D);
        case kRastrigin: return blocks_per_sm(async_kernel<kRastrigin>, D);
        case kAckley: return blocks_per_sm(async_kernel<kAckley>, D);
        case kRosenbrock: return blocks_per_sm(async_kernel<kRosenbrock>, D);
        default: return blocks_per_sm(async_kernel<kCubicMax>, D);
    }
}

}  // namespace cupso
