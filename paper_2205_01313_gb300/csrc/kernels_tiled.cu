// kernels_tiled.cu -- the synchronous FP32 iteration for swarms too small to
// fill the GPU when each thread walks a particle's dimensions in order.
//
// The streaming kernels give each thread whole particles and run over d
// inside the thread; a swarm of some 10^4 particles then leaves most warp
// slots empty and every thread waits on D dependent row loads. Here a block
// takes a tile of P particles with all D dimensions and spreads the
// (dimension pair, particle) items of Eq. 1 and Eq. 2 over its threads, so
// every load of a tile is in flight at once. The fitness (Step 3) keeps its
// order: the per-dimension terms are formed in parallel, and one thread per
// particle adds them for d = 0 .. D-1 with the same operations as the
// streaming kernels. Steps 4-5 as in the fused step: strict pbest, the
// conditional atomicMin on the packed key, the last CTA gathers gbest_pos.
#include <cuda_runtime.h>

#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "stream_common.cuh"
#include "tiled_kernels.h"

namespace cupso {

namespace {

constexpr int kTiledThreads = 256;
constexpr int kChunk = 4;     // items whose loads a thread issues together

// Fitness from per-dimension terms; sum() equals FitAcc<FIT> over d in order.
template <int FIT>
struct FitTerms {
    // Rosenbrock's term d pairs x_d with x_{d+1}
    static constexpr bool kNeedsNext = (FIT == kRosenbrock);
    // no term array: the sum fuses x * x itself
    static constexpr bool kNoTerm = (FIT == kSphere);
    __device__ static __forceinline__ float term(float x, float xn) {
        if constexpr (FIT == kRastrigin) {
            return __fmaf_rn(x, x, __fmaf_rn(-10.0f, cos2pi(x), 10.0f));
        } else if constexpr (FIT == kAckley) {
            return cos2pi(x);
        } else if constexpr (FIT == kRosenbrock) {
            const float p = __fmaf_rn(-x, x, xn);
            const float q = __fsub_rn(1.0f, x);
            return __fmaf_rn(__fmul_rn(100.0f, p), p, __fmul_rn(q, q));
        } else if constexpr (FIT == kCubicMax) {
            return __fmaf_rn(__fmaf_rn(__fsub_rn(x, 0.8f), x, -1000.0f), x, 8000.0f);
        } else {
            return 0.0f;
        }
    }
    // particle column p (stride P) of X and H
    __device__ static __forceinline__ float sum(const float* X, const float* H, int P, int p, int D) {
        FitAcc<FIT> a;
        if constexpr (FIT == kSphere) {
#pragma unroll 8
            for (int d = 0; d < D; ++d) {
                const float x = X[d * P + p];
                a.acc = __fmaf_rn(x, x, a.acc);
            }
        } else if constexpr (FIT == kAckley) {
#pragma unroll 8
            for (int d = 0; d < D; ++d) {
                const float x = X[d * P + p];
                a.acc = __fmaf_rn(x, x, a.acc);
                a.acc2 = __fadd_rn(a.acc2, H[d * P + p]);
            }
        } else {
            const int n = FIT == kRosenbrock ? D - 1 : D;
#pragma unroll 8
            for (int d = 0; d < n; ++d) a.acc = __fadd_rn(a.acc, H[d * P + p]);
        }
        return a.finish(D);
    }
};

template <int FIT, bool FAST>
__global__ void __launch_bounds__(kTiledThreads) sync_tiled_kernel(const __grid_constant__ SwarmDev s, int P) {
    __shared__ float X[kTiledItems];
    __shared__ float H[kTiledItems];
    __shared__ unsigned long long red[kTiledThreads / 32];
    __shared__ int imp[32];
    const uint32_t t_prev = __ldcg(s.t_dev);
    const uint32_t t = t_prev + 1u;
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    const unsigned long long K = __ldcg(s.gkey + cur);   // gbest at the end of t-1
    const int tid = threadIdx.x;
    const int D = s.D, npairs = (D + 1) >> 1;
    const size_t Np = (size_t)s.Np;
    const float* G = s.G + (size_t)cur * D;
    // Every thread keeps one particle lane p of the tile; blockDim is a
    // multiple of 32, so P (a power of two up to 32) divides it.
    const int p = tid & (P - 1);
    const int row0 = tid / P, rows = blockDim.x / P;
    const int ntiles = (s.N + P - 1) / P;

    unsigned long long best = kKeyNone;
    bool nan = false;
    // persistent: the block walks the tiles with a stride of the grid
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int base = tile * P;
        const int n = min(P, s.N - base);
        const bool live = p < n;
        const uint32_t i = (uint32_t)(base + p);
        // Steps 2 (Eq. 1, Eq. 2): one Philox call per (dimension pair, particle).
        // A thread loads the rows of kChunk pairs before it computes any of them,
        // so that all of those loads are in flight together.
        for (int g0 = row0; g0 < npairs; g0 += kChunk * rows) {
            float xs[kChunk][2], vs[kChunk][2], ps[kChunk][2];
#pragma unroll
            for (int c = 0; c < kChunk; ++c) {
                const int g = g0 + c * rows;
                if (live && g < npairs) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int d = min(2 * g + h, D - 1);
                        const size_t off = (size_t)d * Np + i;
                        xs[c][h] = s.x[off];
                        vs[c][h] = s.v[off];
                        ps[c][h] = s.pb[off];
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < kChunk; ++c) {
                const int g = g0 + c * rows;
                if (!live || g >= npairs) break;
                const uint4 r = philox4x32_10(make_uint4((uint32_t)g, i, t, s.swarm), s.key0, s.key1);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int d = 2 * g + h;
                    if (d >= D) break;
                    const size_t off = (size_t)d * Np + i;
                    float x = xs[c][h], v = vs[c][h];
                    if constexpr (FAST)
                        move_one_fast(x, v, ps[c][h], G[d], hi24(word(r, 2 * h)), hi24(word(r, 2 * h + 1)), s);
                    else
                        move_one(x, v, ps[c][h], G[d], u01(word(r, 2 * h)), u01(word(r, 2 * h + 1)), s);
                    s.x[off] = x;
                    s.v[off] = v;
                    X[d * P + p] = x;
                    if constexpr (!FitTerms<FIT>::kNeedsNext && !FitTerms<FIT>::kNoTerm)
                        H[d * P + p] = FitTerms<FIT>::term(x, 0.0f);
                }
            }
        }
        __syncthreads();
        if constexpr (FitTerms<FIT>::kNeedsNext) {
            if (live)
                for (int d = row0; d + 1 < D; d += rows) H[d * P + p] = FitTerms<FIT>::term(X[d * P + p], X[(d + 1) * P + p]);
            __syncthreads();
        }
        // Steps 3-4; the candidates of Step 5 (improved and below the current gbest key)
        if (tid < n) {
            const float f = FitTerms<FIT>::sum(X, H, P, tid, D);
            const uint32_t ip = (uint32_t)(base + tid);
            nan |= (f != f);
            const bool better = f < s.pf[ip];
            imp[tid] = better ? 1 : 0;
            if (better) {
                s.pf[ip] = f;
                const unsigned long long k = pack_key(f, ip);
                if (k < K && k < best) best = k;
            }
        }
        __syncthreads();
        if (live && imp[p])
            for (int d = row0; d < D; d += rows) s.pb[(size_t)d * Np + i] = X[d * P + p];
        __syncthreads();   // X, H and imp are reused by the next tile
    }
    best = block_min(best, red);
    if (tid == 0 && best != kKeyNone) atomicMin(s.gkey + nxt, best);
    if (__syncthreads_or(nan) && tid == 0) atomicOr(s.status, kStatusNaN);
    finish_iteration(s, cur, nxt, t);
}

#define CUPSO_TILED_DISPATCH(fid, FASTV, CALL)                                   \
    switch (fid) {                                                              \
        case kSphere: { constexpr int F = kSphere; CALL; break; }                \
        case kRastrigin: { constexpr int F = kRastrigin; CALL; break; }          \
        case kAckley: { constexpr int F = kAckley; CALL; break; }                \
        case kRosenbrock: { constexpr int F = kRosenbrock; CALL; break; }        \
        case kCubicMax: { constexpr int F = kCubicMax; CALL; break; }            \
        default: return cudaErrorInvalidValue;                                  \
    }

}  // namespace

int tiled_particles(int N, int D, int num_sms) {
    if (D > kTiledItems) return 0;
    int P = 32;
    while (P > 1 && (P * D > kTiledItems || (P > 4 && (long long)N < 2ll * num_sms * P))) P >>= 1;
    return P;
}

cudaError_t launch_sync_tiled(const SwarmDev& s, int fid, int P, int grid, cudaStream_t st) {
    if (P < 1 || P > 32 || P * s.D > kTiledItems) return cudaErrorInvalidValue;
    const int tiles = (s.N + P - 1) / P;
    const int work = P * ((s.D + 1) / 2);
    const int threads = work >= kTiledThreads ? kTiledThreads : (work + 31) / 32 * 32;
    const int g = grid < 1 ? 1 : (grid < tiles ? grid : tiles);
    if (s.fast_cr && s.fast_clamp) {
        CUPSO_TILED_DISPATCH(fid, true, (sync_tiled_kernel<F, true><<<g, threads, 0, st>>>(s, P)));
    } else {
        CUPSO_TILED_DISPATCH(fid, false, (sync_tiled_kernel<F, false><<<g, threads, 0, st>>>(s, P)));
    }
    return cudaGetLastError();
}

int tiled_blocks_per_sm(int fid, int P, int D) {
    const int work = P * ((D + 1) / 2);
    const int threads = work >= kTiledThreads ? kTiledThreads : (work + 31) / 32 * 32;
    int n = 0;
    cudaError_t e = cudaSuccess;
    switch (fid) {
        case kSphere: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sync_tiled_kernel<kSphere, true>, threads, 0); break;
        case kRastrigin: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sync_tiled_kernel<kRastrigin, true>, threads, 0); break;
        case kAckley: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sync_tiled_kernel<kAckley, true>, threads, 0); break;
        case kRosenbrock: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sync_tiled_kernel<kRosenbrock, true>, threads, 0); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sync_tiled_kernel<kCubicMax, true>, threads, 0); break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n < 1 ? 1 : n;
}

}  // namespace cupso
