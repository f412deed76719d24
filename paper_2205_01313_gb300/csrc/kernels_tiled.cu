// kernels_tiled.cu -- the FP32 iteration in tiles, for swarms too small to
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
// streaming kernels. The tile step serves three kernels:
//  * sync_tiled_kernel   SYNC: Steps 4-5 as in the fused step (strict pbest,
//                        conditional atomicMin on the packed key, the last
//                        CTA gathers gbest_pos);
//  * async_tiled_kernel  ASYNC: persistent CTAs own fixed tiles and iterate
//                        with no grid barrier against the lock-protected
//                        gbest record;
//  * batch_tiled_kernel  a batch: (swarm, tile) units of all swarms per launch.
#include <cuda_runtime.h>

#include "async_common.cuh"
#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "pdl.cuh"
#include "stream_common.cuh"
#include "tiled_kernels.h"

namespace cupso {

namespace {

constexpr int kTiledThreads = 256;
constexpr int kChunk = 4;     // dimension pairs whose loads a thread issues together

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

// Fitness chosen at run time (a batch mixes them): FIT = kAnyFit dispatches on
// `fid`, uniformly for a whole tile; a fixed FIT compiles to its own code.
constexpr int kAnyFit = -1;

template <int FIT>
__device__ __forceinline__ bool needs_next(int fid) {
    if constexpr (FIT != kAnyFit) return FitTerms<FIT>::kNeedsNext;
    else return fid == kRosenbrock;
}

template <int FIT>
__device__ __forceinline__ bool has_term(int fid) {
    if constexpr (FIT != kAnyFit) return !FitTerms<FIT>::kNoTerm;
    else return fid != kSphere;
}

template <int FIT>
__device__ __forceinline__ float tile_term(int fid, float x, float xn) {
    if constexpr (FIT != kAnyFit) {
        return FitTerms<FIT>::term(x, xn);
    } else {
        switch (fid) {
            case kRastrigin: return FitTerms<kRastrigin>::term(x, xn);
            case kAckley: return FitTerms<kAckley>::term(x, xn);
            case kRosenbrock: return FitTerms<kRosenbrock>::term(x, xn);
            case kCubicMax: return FitTerms<kCubicMax>::term(x, xn);
            default: return 0.0f;
        }
    }
}

template <int FIT>
__device__ __forceinline__ float tile_sum(int fid, const float* X, const float* H, int P, int p, int D) {
    if constexpr (FIT != kAnyFit) {
        return FitTerms<FIT>::sum(X, H, P, p, D);
    } else {
        switch (fid) {
            case kSphere: return FitTerms<kSphere>::sum(X, H, P, p, D);
            case kRastrigin: return FitTerms<kRastrigin>::sum(X, H, P, p, D);
            case kAckley: return FitTerms<kAckley>::sum(X, H, P, p, D);
            case kRosenbrock: return FitTerms<kRosenbrock>::sum(X, H, P, p, D);
            default: return FitTerms<kCubicMax>::sum(X, H, P, p, D);
        }
    }
}

// A swarm as the tile step sees it (one swarm of SwarmDev, or of a batch).
struct TileSwarm {
    float *x, *v, *pb, *pf;
    unsigned char* pflag;   // lazy-pbest flags left by the streaming kernels, or null
    const float* G;         // gbest_pos at the end of the previous iteration [D]
    int N, D, Np;
    float lo, hi, vmax, w, c1, c2, c1s, c2s;
    uint32_t key0, key1, swarm;
};

// Eq. 1 and Eq. 2 for one element; FAST: c * r as one FMA of c 2^-24 with the
// 24-bit integer of the draw and min/max clamps (bit-identical when valid).
template <bool FAST>
__device__ __forceinline__ void move_tile(float& x, float& v, float pb, float g, uint32_t w1, uint32_t w2,
                                          const TileSwarm& s) {
    const float cognitive = __fsub_rn(pb, x);
    const float social = __fsub_rn(g, x);
    float vel = __fmul_rn(s.w, v);
    if constexpr (FAST) {
        vel = __fmaf_rn(__fmaf_rn(s.c1s, hi24(w1), s.c1s), cognitive, vel);
        vel = __fmaf_rn(__fmaf_rn(s.c2s, hi24(w2), s.c2s), social, vel);
        v = clampf_minmax(vel, -s.vmax, s.vmax);
        x = clampf_minmax(__fadd_rn(x, v), s.lo, s.hi);
    } else {
        vel = __fmaf_rn(__fmul_rn(s.c1, u01(w1)), cognitive, vel);
        vel = __fmaf_rn(__fmul_rn(s.c2, u01(w2)), social, vel);
        v = clampf(vel, -s.vmax, s.vmax);
        x = clampf(__fadd_rn(x, v), s.lo, s.hi);
    }
}

// Steps 2-4 for the tile of P particles starting at `base` (all D dimensions)
// at iteration t; the tile's Step-5 candidates (improved and below K) are
// folded into `best`. Every thread of the block calls it; it ends with a
// barrier, so X, H and imp can be reused at once.
template <int FIT, bool FAST>
__device__ __forceinline__ void process_tile(const TileSwarm& s, int fid, int P, int base, uint32_t t,
                                             unsigned long long K, float* X, float* H, int* imp,
                                             unsigned long long& best, bool& nan) {
    const int tid = threadIdx.x;
    const int D = s.D, npairs = (D + 1) >> 1;
    const size_t Np = (size_t)s.Np;
    // every thread keeps one particle lane p; P (a power of two) divides blockDim
    const int p = tid & (P - 1);
    const int row0 = tid / P, rows = blockDim.x / P;
    const int n = min(P, s.N - base);
    const bool live = p < n;
    const uint32_t i = (uint32_t)(base + p);
    // a particle flagged by the lazy write-back has pbest_pos == pos: use and write it
    const bool lazy = live && s.pflag && s.pflag[i];
    // Step 2 (Eq. 1, Eq. 2): one Philox call per (dimension pair, particle). A
    // thread loads the rows of kChunk pairs before it computes any of them, so
    // that all of those loads are in flight together.
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
                    ps[c][h] = lazy ? xs[c][h] : s.pb[off];
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
                if (lazy) s.pb[off] = ps[c][h];
                float x = xs[c][h], v = vs[c][h];
                move_tile<FAST>(x, v, ps[c][h], s.G[d], word(r, 2 * h), word(r, 2 * h + 1), s);
                s.x[off] = x;
                s.v[off] = v;
                X[d * P + p] = x;
                if (!needs_next<FIT>(fid) && has_term<FIT>(fid)) H[d * P + p] = tile_term<FIT>(fid, x, 0.0f);
            }
        }
    }
    __syncthreads();
    if (needs_next<FIT>(fid)) {
        if (live)
            for (int d = row0; d + 1 < D; d += rows)
                H[d * P + p] = tile_term<FIT>(fid, X[d * P + p], X[(d + 1) * P + p]);
        __syncthreads();
    }
    // Steps 3-4: the ordered sum, strict improvement, the candidate
    if (tid < n) {
        const float f = tile_sum<FIT>(fid, X, H, P, tid, D);
        const uint32_t ip = (uint32_t)(base + tid);
        nan |= (f != f);
        const bool better = f < s.pf[ip];
        imp[tid] = better ? 1 : 0;
        if (better) {
            s.pf[ip] = f;
            const unsigned long long k = pack_key(f, ip);
            if (k < K && k < best) best = k;
        }
        if (s.pflag && s.pflag[ip]) s.pflag[ip] = 0;
    }
    __syncthreads();
    if (live && imp[p])
        for (int d = row0; d < D; d += rows) s.pb[(size_t)d * Np + i] = X[d * P + p];
    __syncthreads();
}

template <int FIT, bool FAST>
__global__ void __launch_bounds__(kTiledThreads) sync_tiled_kernel(const __grid_constant__ SwarmDev s, int P) {
    __shared__ float X[kTiledItems];
    __shared__ float H[kTiledItems];
    __shared__ unsigned long long red[kTiledThreads / 32];
    __shared__ int imp[kTiledMaxP];
    pdl_wait();
    const uint32_t t_prev = __ldcg(s.t_dev);
    const uint32_t t = t_prev + 1u;
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    const unsigned long long K = __ldcg(s.gkey + cur);   // gbest at the end of t-1
    const TileSwarm ts{s.x, s.v, s.pb, s.pf, nullptr, s.G + (size_t)cur * s.D, s.N, s.D, s.Np, s.lo, s.hi, s.vmax,
                       s.w, s.c1, s.c2, s.c1s, s.c2s, s.key0, s.key1, s.swarm};
    const int ntiles = (s.N + P - 1) / P;
    unsigned long long best = kKeyNone;
    bool nan = false;
    // persistent: the block walks the tiles with a stride of the grid
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        process_tile<FIT, FAST>(ts, FIT, P, tile * P, t, K, X, H, imp, best, nan);
    // The next iteration may start launching now: its blocks would otherwise
    // take SM slots while this one still has tiles to run.
    pdl_launch_next();
    best = block_min(best, red);
    if (threadIdx.x == 0 && best != kKeyNone) atomicMin(s.gkey + nxt, best);
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
    finish_iteration(s, cur, nxt, t);
}

// The asynchronous variant in tiles (Sec. 3.2 taken to its end, Sec. 6): a
// persistent CTA owns the tiles blockIdx.x, blockIdx.x + gridDim.x, ... and
// iterates over them with no grid barrier. Each of its iterations reads the
// latest gbest record (sequence lock), runs the tile step over its tiles and
// publishes its best improvement under the lock. Random draws stay keyed on
// (t, particle), so only the gbest each particle sees depends on timing; with
// one CTA the run is the synchronous one.
// Register budget for 4 CTAs per SM: with no grid barrier, more resident CTAs
// hide each other's ordered sums and lock waits (measured: 53 -> 44 us per
// iteration on Rastrigin 65536 x 128; the synchronous kernel is faster at 3).
template <int FIT, bool FAST>
__global__ void __launch_bounds__(kTiledThreads, 4) async_tiled_kernel(const __grid_constant__ SwarmDev s, int P,
                                                                   uint32_t t_first, int iters) {
    __shared__ float X[kTiledItems];
    __shared__ float H[kTiledItems];
    __shared__ unsigned long long red[kTiledThreads / 32];
    __shared__ int imp[kTiledMaxP];
    __shared__ int s_stop;
    __shared__ int s_last;
    extern __shared__ float Gs[];   // [D] the gbest this CTA's iteration uses
    const int tid = threadIdx.x;
    const int ntiles = (s.N + P - 1) / P;
    const TileSwarm ts{s.x, s.v, s.pb, s.pf, nullptr, Gs, s.N, s.D, s.Np, s.lo, s.hi, s.vmax,
                       s.w, s.c1, s.c2, s.c1s, s.c2s, s.key0, s.key1, s.swarm};
    for (int k = 0; k < iters; ++k) {
        const uint32_t t = t_first + (uint32_t)k;
        if (tid == 0) s_stop = (__ldcg(s.status) & kStatusTimeout) != 0u;
        __syncthreads();
        if (s_stop) break;
        if (!read_record(s, Gs)) {
            if (tid == 0) atomicOr(s.status, kStatusTimeout);
            break;
        }
        const unsigned long long K = __ldcg(s.claim);
        unsigned long long best = kKeyNone;
        bool nan = false;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
            process_tile<FIT, FAST>(ts, FIT, P, tile * P, t, K, X, H, imp, best, nan);
        if (__syncthreads_or(nan) && tid == 0) atomicOr(s.status, kStatusNaN);
        best = block_min(best, red);   // ends with a barrier: the pbest writes are visible
        if (best != kKeyNone && tid < 32) {
            if (!publish(s, best) && tid == 0) atomicOr(s.status, kStatusTimeout);
        }
        __syncthreads();
    }
    // The last CTA to finish hands the record back to the synchronous state.
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(s.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const uint32_t t_end = t_first - 1u + (uint32_t)iters;
    const int cur = (int)(t_end & 1u);
    for (int d = tid; d < s.D; d += blockDim.x) s.G[(size_t)cur * s.D + d] = __ldcg(s.Grec + d);
    if (tid == 0) {
        const unsigned long long kk = __ldcg(s.reckey);
        s.gkey[0] = kk;
        s.gkey[1] = kk;
        *s.t_dev = t_end;
        *s.ticket = 0u;
    }
}

// One iteration of every swarm of a batch, in tiles: CTAs take (swarm, tile)
// units from a counter (the order is the host's: costliest first); each unit
// ends with the swarm's conditional atomicMin, and the CTA that completes a
// swarm's last tile gathers that swarm's gbest_pos. The kernel boundary is the
// only barrier between iterations, so every swarm follows its own
// synchronous trajectory.
__global__ void __launch_bounds__(kTiledThreads, 3) batch_tiled_kernel(const __grid_constant__ BatchDev b,
                                                                   const __grid_constant__ BatchTiles bt) {
    __shared__ float X[kTiledItems];
    __shared__ float H[kTiledItems];
    __shared__ unsigned long long red[kTiledThreads / 32];
    __shared__ int imp[kTiledMaxP];
    __shared__ uint2 s_unit;
    __shared__ int s_last;
    const uint32_t t_prev = __ldcg(b.t_dev);
    const uint32_t t = t_prev + 1u;
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    unsigned* work = b.work + (t & 1u);
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            const unsigned k = atomicAdd(work, 1u);
            s_unit = k < bt.nunits ? bt.units[k] : make_uint2(0xFFFFFFFFu, 0u);
        }
        __syncthreads();
        const uint2 un = s_unit;
        if (un.x == 0xFFFFFFFFu) break;
        const BatchSwarm& w = b.swarms[un.x];
        const int P = bt.P[un.x];
        const unsigned long long K = __ldcg(w.gkey + cur);
        const TileSwarm ts{w.x, w.v, w.pb, w.pf, w.pflag, w.G + (size_t)cur * w.D, w.N, w.D, w.Np, w.lo, w.hi,
                           w.vmax, w.w, w.c1, w.c2, w.c1s, w.c2s, w.key0, w.key1, w.swarm};
        unsigned long long best = kKeyNone;
        bool nan = false;
        if (w.fast) process_tile<kAnyFit, true>(ts, w.fid, P, (int)un.y * P, t, K, X, H, imp, best, nan);
        else process_tile<kAnyFit, false>(ts, w.fid, P, (int)un.y * P, t, K, X, H, imp, best, nan);
        best = block_min(best, red);
        const bool any_nan = __syncthreads_or(nan);
        // publish, then count the tile; the CTA that completes the swarm gathers its gbest
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            if (best < K) atomicMin(w.gkey + nxt, best);
            if (any_nan) atomicOr(w.status, kStatusNaN);
            __threadfence();
            s_last = atomicAdd(w.done, 1u) == bt.ntiles[un.x] - 1u;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            const unsigned long long knew = __ldcg(w.gkey + nxt);
            const uint32_t gi = (uint32_t)(knew & 0xFFFFFFFFull);
            if (gi < (uint32_t)w.N)
                for (int d = tid; d < w.D; d += blockDim.x)
                    w.G[(size_t)nxt * w.D + d] = __ldcg(w.pb + (size_t)d * w.Np + gi);
            __syncthreads();
            if (tid == 0) {
                w.gkey[cur] = knew;
                *w.done = 0u;
            }
        }
        __syncthreads();
    }
    // The last CTA rolls the batch forward: the next launch counts on the other counter.
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(b.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (s_last && tid == 0) {
        b.work[(t + 1u) & 1u] = 0u;
        *b.ticket = 0u;
        *b.t_dev = t;
    }
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
    int P = kTiledMaxP;
    while (P > 1 && (P * D > kTiledItems || (P > 4 && (long long)N < 2ll * num_sms * P))) P >>= 1;
    return P;
}

int batch_tile_particles(int D) {
    if (D > kTiledItems) return 0;
    int P = kTiledMaxP;
    while (P > 1 && P * D > kTiledItems) P >>= 1;
    return P;
}

namespace {
// Threads of a tile block: enough for the tile's (pair, particle) items, a
// multiple of 32 (so that P divides it) and at least P.
int tile_threads(int P, int D) {
    const int work = P * ((D + 1) / 2);
    int th = work >= kTiledThreads ? kTiledThreads : (work + 31) / 32 * 32;
    return th < P ? P : th;
}
}  // namespace

cudaError_t launch_sync_tiled(const SwarmDev& s, int fid, int P, int grid, cudaStream_t st) {
    if (P < 1 || P > kTiledMaxP || (P & (P - 1)) || P * s.D > kTiledItems) return cudaErrorInvalidValue;
    const int tiles = (s.N + P - 1) / P;
    const int threads = tile_threads(P, s.D);
    const int g = grid < 1 ? 1 : (grid < tiles ? grid : tiles);
    if (s.fast_cr && s.fast_clamp) {
        CUPSO_TILED_DISPATCH(fid, true, return launch_pdl(sync_tiled_kernel<F, true>, dim3(g), dim3(threads), 0, st, s, P));
    } else {
        CUPSO_TILED_DISPATCH(fid, false, return launch_pdl(sync_tiled_kernel<F, false>, dim3(g), dim3(threads), 0, st, s, P));
    }
    return cudaErrorInvalidValue;
}

int tiled_blocks_per_sm(int fid, int P, int D) {
    const int threads = tile_threads(P, D);
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

cudaError_t launch_async_tiled(const SwarmDev& s, int fid, int P, int grid, uint32_t t_first, int iters,
                               int hold_lock, cudaStream_t st) {
    if (P < 1 || P > kTiledMaxP || (P & (P - 1)) || P * s.D > kTiledItems) return cudaErrorInvalidValue;
    cudaError_t e = launch_async_prologue(s, hold_lock, st);
    if (e != cudaSuccess) return e;
    const int tiles = (s.N + P - 1) / P;
    const int threads = tile_threads(P, s.D);
    const int g = grid < 1 ? 1 : (grid < tiles ? grid : tiles);
    const size_t smem = sizeof(float) * (size_t)s.D;
    if (s.fast_cr && s.fast_clamp) {
        CUPSO_TILED_DISPATCH(fid, true, (async_tiled_kernel<F, true><<<g, threads, smem, st>>>(s, P, t_first, iters)));
    } else {
        CUPSO_TILED_DISPATCH(fid, false, (async_tiled_kernel<F, false><<<g, threads, smem, st>>>(s, P, t_first, iters)));
    }
    return cudaGetLastError();
}

int async_tiled_blocks_per_sm(int P, int D) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, async_tiled_kernel<kRastrigin, true>, tile_threads(P, D),
                                                      sizeof(float) * (size_t)D) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n < 1 ? 1 : n;
}

int batch_tiled_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_tiled_kernel, kTiledThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n < 1 ? 1 : n;
}

cudaError_t launch_batch_tiled(const BatchDev& b, const BatchTiles& bt, int grid, cudaStream_t st) {
    batch_tiled_kernel<<<grid, kTiledThreads, 0, st>>>(b, bt);
    return cudaGetLastError();
}

}  // namespace cupso
