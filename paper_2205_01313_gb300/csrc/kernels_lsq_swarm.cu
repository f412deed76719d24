// kernels_lsq_swarm.cu -- one PSO iteration of a swarm with the least-squares
// fitness ||A x - b||^2.
//
// The fitness of the whole swarm is one matrix product (kernels_lsq.cu), so the
// iteration runs as separate launches: move (Eq. 1, Eq. 2 and their clamps),
// fitness, then Steps 4-5. With the plain FP32 fitness Steps 4-5 are those of
// the synchronous kernels (strict pbest, conditional atomicMin, last CTA
// gathers gbest_pos): bit-exact with the oracle. With the BF16/FP8 fitness the
// pbest decisions use the approximate values, but no global best is accepted
// on them: the (up to) 16 improved particles with the lowest approximate
// fitness are rescored in extended precision (float-float or FP64 Gram form,
// FP64 residuals when D > M) and the best of them replaces gbest only if its
// rescored fitness is lower than gbest's (ties to the lower index).
//
// Every kernel reads the iteration counter from device memory, so a chain of
// iterations can be captured in a CUDA graph.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "lsq_internal.h"
#include "stream_common.cuh"
#include "tma_common.cuh"

#include <algorithm>
#include <cstring>

namespace cupso {

namespace {

constexpr int kCand = 16;   // candidates rescored per iteration

}  // namespace

// Steps 2 of every particle at iteration t = *t_dev + 1 (the fitness is a
// separate matrix product). No fitness runs along d here, so the work is
// spread over (4-particle group, dimension pair) items.
__global__ void __launch_bounds__(kBlock) lsq_move_kernel(const __grid_constant__ SwarmDev s) {
    extern __shared__ float Gs[];
    const uint32_t t_prev = __ldcg(s.t_dev);
    const uint32_t t = t_prev + 1u;
    const int cur = (int)(t_prev & 1u);
    for (int d = threadIdx.x; d < s.D; d += blockDim.x) Gs[d] = __ldcg(s.G + (size_t)cur * s.D + d);
    __syncthreads();
    const size_t groups = (size_t)s.Np / 4;
    const int npairs = (s.D + 1) / 2;
    const size_t items = groups * (size_t)npairs;
    const size_t Np = (size_t)s.Np;
    for (size_t it = (size_t)blockIdx.x * blockDim.x + threadIdx.x; it < items; it += (size_t)gridDim.x * blockDim.x) {
        const int g = (int)(it / groups);
        const uint32_t i0 = (uint32_t)(it % groups) * 4u;
        uint4 r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) r[j] = philox4x32_10_rk(make_uint4((uint32_t)g, i0 + j, t, s.swarm), s.rk0, s.rk1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int d = 2 * g + h;
            if (d >= s.D) break;
            const size_t off = (size_t)d * Np + i0;
            float4 X = ld4(s.x + off), V = ld4(s.v + off);
            const float4 P = ld4(s.pb + off);
            const float gd = Gs[d];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float xj = lane(X, j), vj = lane(V, j);
                move_one(xj, vj, lane(P, j), gd, u01(word(r[j], 2 * h)), u01(word(r[j], 2 * h + 1)), s);
                set_lane(X, j, xj);
                set_lane(V, j, vj);
            }
            st4(s.x + off, X);
            st4(s.v + off, V);
        }
    }
}

// Step 2 fused with the tensor-core operand of the fitness product: the same
// moves as lsq_move_kernel, and each new position's displacement from the
// iteration's gbest_pos g (the reference point of the fitness, see
// lsq_offset_kernel) lands in Xq[i][k] (row-major, row length Kp): x'_k - g_k,
// computed in FP32, rounded to BF16, or multiplied by sx and rounded to FP8
// e4m3 with saturation (|x' - g| <= max_pos - min_pos, so sx = 448 / (max_pos -
// min_pos) never saturates); zero for i >= N and k >= D.
// One CTA per SM walks tiles of 64 particles x 64 dimensions (tile b, b +
// gridDim.x, ...). Thread 0 keeps a ring of kMoveStages tiles in flight: per
// tile, three 2-D tensor copies (pos, v, pbest_pos; rows past D read as zeros)
// and one bulk copy of the tile's 64 improvement flags, all completing on the
// stage's mbarrier; a stage is refilled as soon as every thread is done with
// it. Thread q takes 4 particles x one dimension pair of the tile; new pos and
// v go straight back to global memory; the operand's transposition goes
// through shared memory, so its rows are written in whole segments.
// Lazy pbest: a particle flagged in s.pflag improved in the previous
// iteration, so its pbest_pos is the position loaded here; that row is written
// back on the way. Every wait is bounded: on a timeout the CTA sets
// kStatusTimeout, waits (bounded) for the copies it has in flight and stops.
struct MoveMaps {
    CUtensorMap m[3];   // pos, v, pbest_pos
};
constexpr int kMoveThreads = 512;
constexpr int kMoveStages = 3;
constexpr int kMoveBox = 64 * 64 * 4;   // one array's tile
constexpr int kMoveStageBytes = (3 * kMoveBox + 64 + 127) / 128 * 128;
constexpr uint32_t kMoveTx = 3 * kMoveBox + 64;

template <bool FP8>
__global__ void __launch_bounds__(kMoveThreads, 1) lsq_move_q_kernel(const __grid_constant__ SwarmDev s,
                                                                     const __grid_constant__ MoveMaps maps,
                                                                     void* __restrict__ Xq, int Kp, float sx) {
    extern __shared__ unsigned char msm_raw[];   // kMoveStages stages, 128-byte aligned below
    __shared__ uint32_t S[32][65];               // [dimension pair][particle]: the pair's two operand values
    __shared__ __align__(8) uint64_t full[kMoveStages];
    const uint32_t raw = smem_u32(msm_raw);
    const uint32_t sbase = (raw + 127u) & ~127u;
    unsigned char* msm = msm_raw + (sbase - raw);
    const uint32_t t_prev = __ldcg(s.t_dev);
    const uint32_t t = t_prev + 1u;
    const float* G = s.G + (size_t)(t_prev & 1u) * s.D;
    const size_t Np = (size_t)s.Np;
    const int ptiles = s.Np / 64, ntiles = ptiles * (Kp / 64);
    const int mine = (int)blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    // tile k of this CTA into stage k % kMoveStages (thread 0)
    auto issue = [&](int k) {
        const int tile = (int)blockIdx.x + k * (int)gridDim.x;
        const int p0 = (tile % ptiles) * 64, d0 = (tile / ptiles) * 64;
        const int st = k % kMoveStages;
        const uint32_t bar = smem_u32(&full[st]), dst = sbase + (uint32_t)(st * kMoveStageBytes);
        mbar_expect_tx(bar, kMoveTx);
#pragma unroll
        for (int a = 0; a < 3; ++a) tma_load_2d_cta(dst + (uint32_t)(a * kMoveBox), &maps.m[a], p0, d0, bar);
        bulk_load_cta(dst + 3u * kMoveBox, s.pflag + p0, 64u, bar);
    };
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) prefetch_tensormap(&maps.m[a]);
        for (int st = 0; st < kMoveStages; ++st) mbar_init(smem_u32(&full[st]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async_smem();
        for (int k = 0; k < mine && k < kMoveStages; ++k) issue(k);
    }
    __syncthreads();
    const int q = (int)threadIdx.x, grp = q & 15, gl = q >> 4;
    for (int k = 0; k < mine; ++k) {
        const int st = k % kMoveStages;
        const bool ok = mbar_wait(smem_u32(&full[st]), (uint32_t)((k / kMoveStages) & 1), s.wait_limit_ns);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(s.status, kStatusTimeout);
                // the copies still in flight land before the CTA leaves
                for (int kk = k; kk < mine && kk < k + kMoveStages; ++kk)
                    mbar_wait(smem_u32(&full[kk % kMoveStages]), (uint32_t)((kk / kMoveStages) & 1), s.wait_limit_ns);
            }
            break;
        }
        const int tile = (int)blockIdx.x + k * (int)gridDim.x;
        const uint32_t p0 = (uint32_t)(tile % ptiles) * 64u;
        const int dt = tile / ptiles;
        const float* tx = reinterpret_cast<const float*>(msm + st * kMoveStageBytes);   // [64 dims][64 particles]
        const float* tv = tx + 64 * 64;
        const float* tp = tv + 64 * 64;
        const uint32_t* tfl = reinterpret_cast<const uint32_t*>(tp + 64 * 64);          // 16 groups of 4 flag bytes
        const int g = dt * 32 + gl;
        const uint32_t i0 = p0 + 4u * (uint32_t)grp;
        float xn[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        if (2 * g < s.D) {
            const uint32_t fl = tfl[grp];
            uint4 r[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                r[j] = philox4x32_10_rk(make_uint4((uint32_t)g, i0 + j, t, s.swarm), s.rk0, s.rk1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int d = 2 * g + h;
                if (d >= s.D) break;
                const int row = (2 * gl + h) * 64 + 4 * grp;
                const size_t off = (size_t)d * Np + i0;
                float4 Xh = *reinterpret_cast<const float4*>(tx + row);
                float4 Vh = *reinterpret_cast<const float4*>(tv + row);
                float4 Ph = *reinterpret_cast<const float4*>(tp + row);
                if (fl) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if ((fl >> (8 * j)) & 1u) set_lane(Ph, j, lane(Xh, j));
                    st4(s.pb + off, Ph);
                }
                const float gd = __ldg(G + d);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float xj = lane(Xh, j), vj = lane(Vh, j);
                    move_one(xj, vj, lane(Ph, j), gd, u01(word(r[j], 2 * h)), u01(word(r[j], 2 * h + 1)), s);
                    set_lane(Xh, j, xj);
                    set_lane(Vh, j, vj);
                    xn[h][j] = __fsub_rn(xj, gd);
                }
                st4(s.x + off, Xh);
                st4(s.v + off, Vh);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool real = i0 + j < (uint32_t)s.N;
            const float a = real ? xn[0][j] : 0.0f, b = real ? xn[1][j] : 0.0f;
            uint32_t wq;
            if constexpr (FP8) {
                const __nv_fp8x2_e4m3 q2(make_float2(__fmul_rn(a, sx), __fmul_rn(b, sx)));
                wq = (uint32_t)q2.__x;
            } else {
                const __nv_bfloat162 q2 = __floats2bfloat162_rn(a, b);
                wq = *reinterpret_cast<const uint32_t*>(&q2);
            }
            S[gl][4 * grp + j] = wq;
        }
        __syncthreads();   // stage st read by every thread, S complete
        if (threadIdx.x == 0 && k + kMoveStages < mine) {
            fence_proxy_async_smem();
            issue(k + kMoveStages);
        }
        char* row0 = static_cast<char*>(Xq) + (size_t)p0 * Kp * (FP8 ? 1 : 2);
        if constexpr (FP8) {
            // 64 rows x 4 pieces of 16 dimensions (16 B)
            if (threadIdx.x < 256) {
                const int c = threadIdx.x & 3, pl = threadIdx.x >> 2;
                uint4 u;
                u.x = (S[8 * c + 0][pl] & 0xFFFFu) | (S[8 * c + 1][pl] << 16);
                u.y = (S[8 * c + 2][pl] & 0xFFFFu) | (S[8 * c + 3][pl] << 16);
                u.z = (S[8 * c + 4][pl] & 0xFFFFu) | (S[8 * c + 5][pl] << 16);
                u.w = (S[8 * c + 6][pl] & 0xFFFFu) | (S[8 * c + 7][pl] << 16);
                *reinterpret_cast<uint4*>(row0 + (size_t)pl * Kp + dt * 64 + 16 * c) = u;
            }
        } else {
            // 64 rows x 8 pieces of 8 dimensions (16 B): one per thread
            const int c = threadIdx.x & 7, pl = threadIdx.x >> 3;
            const uint4 u = make_uint4(S[4 * c][pl], S[4 * c + 1][pl], S[4 * c + 2][pl], S[4 * c + 3][pl]);
            *reinterpret_cast<uint4*>(row0 + ((size_t)pl * Kp + dt * 64 + 8 * c) * 2) = u;
        }
        __syncthreads();   // S free for the next tile
    }
}

// pbest_pos[d][i] = pos[d][i] for every particle flagged as improved (one
// float4 group of particles per item, all dimensions in parallel).
__global__ void __launch_bounds__(kBlock) lsq_copy_pbest_kernel(const __grid_constant__ SwarmDev s,
                                                                const unsigned int* __restrict__ flags) {
    const size_t groups = (size_t)s.Np / 4;
    const size_t items = groups * (size_t)s.D;
    const size_t Np = (size_t)s.Np;
    for (size_t it = (size_t)blockIdx.x * blockDim.x + threadIdx.x; it < items; it += (size_t)gridDim.x * blockDim.x) {
        const size_t q = it % groups;
        const uint32_t fl = __ldg(flags + q);
        if (!fl) continue;
        const size_t off = (it / groups) * Np + 4 * q;
        const float4 X = ld4(s.x + off);
        if (fl == 0x01010101u) {
            st4(s.pb + off, X);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((fl >> (8 * j)) & 1u) s.pb[off + j] = lane(X, j);
        }
    }
}

// Step 4 for every particle: strict improvement of pbest_fit, and the flag
// that its pbest_pos must become its pos (copied by lsq_copy_pbest_kernel).
// Returns the improvement mask of the 4 particles at i0.
__device__ __forceinline__ unsigned lsq_pf4(const SwarmDev& s, uint32_t i0, const float f[4],
                                            unsigned int* __restrict__ flags) {
    float4 PF = ld4(s.pf + i0);
    unsigned mask = 0, fl = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if ((i0 + j) < (uint32_t)s.N && f[j] < lane(PF, j)) {
            mask |= 1u << j;
            fl |= 1u << (8 * j);
            set_lane(PF, j, f[j]);
        }
    }
    if (mask) st4(s.pf + i0, PF);
    flags[i0 / 4] = fl;
    return mask;
}

// Steps 4-5 with the exact FP32 fitness: strict pbest, then the conditional
// atomicMin on the packed key (only particles that improved and beat gbest).
__global__ void __launch_bounds__(kBlock) lsq_select_exact_kernel(const __grid_constant__ SwarmDev s,
                                                                  const float* __restrict__ fit,
                                                                  unsigned int* __restrict__ flags) {
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    const unsigned long long K = __ldcg(s.gkey + cur);
    unsigned long long best = kKeyNone;
    bool nan = false;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < (uint32_t)s.Np / 4; q += gridDim.x * blockDim.x) {
        const uint32_t i0 = 4 * q;
        float f[4];
        const float4 F = ld4(fit + i0);
        f[0] = F.x; f[1] = F.y; f[2] = F.z; f[3] = F.w;
        const unsigned mask = lsq_pf4(s, i0, f, flags);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (mask & (1u << j)) {
                const unsigned long long k = pack_key(f[j], i0 + j);
                if (k < K && k < best) best = k;
            }
        nan |= any_nan4(s, i0, f);
    }
    best = warp_min_u64(best);
    if ((threadIdx.x & 31) == 0 && best < K) atomicMin(s.gkey + nxt, best);
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
}

// After the pbest copy: gbest_pos from pbest_pos at the winning index; roll t.
__global__ void lsq_gather_kernel(const __grid_constant__ SwarmDev s) {
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    const unsigned long long knew = __ldcg(s.gkey + nxt);
    const uint32_t g = (uint32_t)(knew & 0xFFFFFFFFull);
    if (g < (uint32_t)s.N)
        for (int d = threadIdx.x; d < s.D; d += blockDim.x)
            s.G[(size_t)nxt * s.D + d] = __ldcg(s.pb + (size_t)d * s.Np + g);
    __syncthreads();
    if (threadIdx.x == 0) {
        s.gkey[cur] = knew;
        *s.t_dev = t_prev + 1u;
    }
}

// The 16 smallest keys a warp holds, ascending, into out[0..15] (lane 0
// writes): round r takes the smallest key above round r-1's (keys are unique:
// the particle index is in the low bits; kKeyNone fills the rounds past the
// last key). item(q) is the lane's q-th key, q < n (N > 0: n = N, unrolled).
template <int N, typename Item>
__device__ __forceinline__ void warp_top(Item item, int n, unsigned long long* out) {
    unsigned long long last = 0;
    for (int r = 0; r < kCand; ++r) {
        unsigned long long lm = kKeyNone;
        if constexpr (N > 0) {
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const unsigned long long k = item(q);
                if ((r == 0 || k > last) && k < lm) lm = k;
            }
        } else {
            for (int q = 0; q < n; ++q) {
                const unsigned long long k = item(q);
                if ((r == 0 || k > last) && k < lm) lm = k;
            }
        }
        const unsigned long long m = warp_min_u64(lm);
        if ((threadIdx.x & 31) == 0) out[r] = m;
        last = m;
    }
}

// Step 4 with an approximate fitness, and the 16 lowest keys among the
// particles that improved (all particles when `all` is set: the first gbest).
// One particle per thread, blocks of kSel threads (small, so that even a swarm
// of a few thousand particles spreads over most SMs). Each thread loads all
// its partial sums at once (with its pbest_fit) and adds them in k order; each
// warp sorts its 32 keys with a bitonic network of lane exchanges and writes
// its 16 lowest as one ascending list (cand[list][16], list = 2 block + warp).
// The last block to finish merges all lists into top[16], ascending (kKeyNone
// where fewer): for up to 32 * kMergeLists lists, a k-way merge (the first
// kStageDepth keys of every list staged in shared memory in one round, then
// merged by warp 0 alone: each lane holds the heads of kMergeLists lists, a
// warp minimum per round, no block barrier between rounds; a list's deeper
// keys, needed only when it gives up more than kStageDepth of the 16, come
// from global memory), else a selection over all their keys. The fitness
// comes from `fit`, or, with `part`, as the sum of the product's nparts
// partial sums in their order.
constexpr int kSel = 64;
constexpr int kSelWarps = kSel / 32;
constexpr int kMergeLists = 8;     // lists per lane of the last block's k-way merge
constexpr int kStageDepth = 4;     // keys of each list staged for the merge
// top[16] = the 16 lowest keys of the nl ascending lists cand[list][16]
// (kKeyNone where fewer), by one block of kSel threads.
__device__ __forceinline__ void merge_lists(const unsigned long long* __restrict__ cand, int nl,
                                         unsigned long long* __restrict__ top) {
    __shared__ unsigned long long stage[32 * kMergeLists * kStageDepth];
    __shared__ unsigned long long wtop[kSelWarps][kCand];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = nl * kCand;
    const int tid = (int)threadIdx.x;
    if (nl <= 32 * kMergeLists) {
        // k-way merge of the ascending lists: lane l of warp 0 owns lists l,
        // l + 32, ...; each round the smallest head over the warp is taken and
        // its list advances (keys are unique, so one owner moves)
        constexpr int kPer = 32 * kMergeLists * kStageDepth / kSel;
        unsigned long long v[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int e = tid + kSel * j, l = e / kStageDepth;
            v[j] = l < nl ? __ldcg(cand + (size_t)l * kCand + e % kStageDepth) : kKeyNone;
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j) stage[tid + kSel * j] = v[j];
        __syncthreads();
        if (warp == 0) {
            int head[kMergeLists];
            unsigned long long hv[kMergeLists];
#pragma unroll
            for (int q = 0; q < kMergeLists; ++q) {
                head[q] = 0;
                hv[q] = stage[(lane + 32 * q) * kStageDepth];
            }
            for (int r = 0; r < kCand; ++r) {
                unsigned long long lm = kKeyNone;
#pragma unroll
                for (int q = 0; q < kMergeLists; ++q) lm = hv[q] < lm ? hv[q] : lm;
                const unsigned long long m = warp_min_u64(lm);
                if (lane == 0) top[r] = m;
                if (m != kKeyNone) {
#pragma unroll
                    for (int q = 0; q < kMergeLists; ++q)
                        if (hv[q] == m) {
                            const int b = lane + 32 * q, h = ++head[q];
                            hv[q] = h < kStageDepth ? stage[b * kStageDepth + h]
                                    : h < kCand   ? __ldcg(cand + (size_t)b * kCand + h)
                                                  : kKeyNone;
                        }
                }
            }
        }
    } else {
        // many lists: a selection over all their keys, per warp then over the
        // warps' lists
        const int per = tid < n ? (n - tid + kSel - 1) / kSel : 0;   // this thread's entries: tid + kSel q
        warp_top<0>([&](int q) { return __ldcg(cand + (size_t)tid + (size_t)kSel * q); }, per, wtop[warp]);
        __syncthreads();
        constexpr int kPerLane = kSelWarps * kCand / 32;
        const unsigned long long* flat = &wtop[0][0];
        if (warp == 0) warp_top<kPerLane>([&](int q) { return flat[lane + 32 * q]; }, kPerLane, top);
    }
}

__global__ void __launch_bounds__(kSel) lsq_select_cand_kernel(const __grid_constant__ SwarmDev s,
                                                               const float* __restrict__ fit,
                                                               const float* __restrict__ part, int nparts,
                                                               int all,
                                                               unsigned long long* __restrict__ cand,
                                                               unsigned int* __restrict__ flags,
                                                               unsigned long long* __restrict__ top,
                                                               unsigned int* __restrict__ ticket) {
    __shared__ int s_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t i = (uint32_t)blockIdx.x * kSel + threadIdx.x;
    unsigned long long key = kKeyNone;
    bool nan = false;
    if (i < (uint32_t)s.Np) {
        const bool real = i < (uint32_t)s.N;
        const float pf = (!all && real) ? s.pf[i] : 0.0f;
        float f = 0.0f;
        if (part) {
            // in k order; up to 32 loads in flight
            for (int k0 = 0; k0 < nparts; k0 += 32) {
                float v[32];
#pragma unroll
                for (int e = 0; e < 32; ++e) v[e] = k0 + e < nparts ? __ldcg(part + (size_t)(k0 + e) * s.Np + i) : 0.0f;
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    if (k0 + e < nparts) f = __fadd_rn(f, v[e]);
            }
        } else {
            f = fit[i];
        }
        // strict improvement; the byte flag tells the next move (or the
        // pbest copy) that pbest_pos must become pos
        unsigned char fl = 0;
        if (!all && real && f < pf) {
            s.pf[i] = f;
            fl = 1;
        }
        reinterpret_cast<unsigned char*>(flags)[i] = fl;
        if (real && (all || fl)) key = pack_key(f, i);
        nan = real && (f != f);
    }
    if (__any_sync(0xFFFFFFFFu, nan) && lane == 0) atomicOr(s.status, kStatusNaN);
    // the warp's keys ascending over its lanes: for each size k of the bitonic
    // sequences, exchanges at distances k/2 .. 1; the lower lane of a pair keeps
    // the smaller key where its k-block ascends, the larger where it descends
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, key, j);
            const bool lower = (lane & j) == 0, asc = (lane & k) == 0;
            key = (lower == asc) ? (o < key ? o : key) : (o > key ? o : key);
        }
    }
    if (lane < kCand) cand[((size_t)blockIdx.x * kSelWarps + warp) * kCand + lane] = key;
    // the last block merges: the lists are written (barrier), thread 0 releases
    // them with its ticket and, in the last block, acquires all the others
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        if (s_last) asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
    __syncthreads();
    if (!s_last) return;
    merge_lists(cand, (int)gridDim.x * kSelWarps, top);
    if (threadIdx.x == 0) *ticket = 0u;
}

// Accepts the best rescored candidate if its rescored value beats gbest's; rolls t.
// Run by the last block of the rescoring kernel (any block size that is a
// multiple of 32): warp w sums candidates w, w + warps, ... (lane l takes
// chunks l, l + 32, ... in order, then a fixed butterfly); thread 0 compares.
// When it accepts one, *stale is set: the reference point of the tensor-core
// fitness moved, so its residual offsets must be recomputed.
__device__ void accept_best(const SwarmDev& s, const float* __restrict__ src, const unsigned long long* __restrict__ top,
                            const double* __restrict__ partial, int chunks, double* __restrict__ g64,
                            int* __restrict__ stale) {
    __shared__ double fsum[kCand];
    __shared__ unsigned long long skey[kCand];
    __shared__ int s_best;
    __shared__ double s_f, s_g64;
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
    // the candidate list, gbest's FP64 value and the candidates' partial sums,
    // read at once (up to 256 pieces per candidate: 8 loads per lane for each
    // of the warp's two candidates in flight together); a candidate's sum
    // runs over its pieces lane + 32 k in k order, then a fixed butterfly.
    // Absent candidates (past the first kKeyNone) are summed but never read.
    if (threadIdx.x < kCand) skey[threadIdx.x] = top[threadIdx.x];
    if (threadIdx.x == 32) s_g64 = __ldcg(g64);
    for (int c0 = warp; c0 < kCand; c0 += 2 * nw) {
        const int c1 = c0 + nw < kCand ? c0 + nw : -1;
        double f0 = 0.0, f1 = 0.0;
        if (chunks <= 256) {
            double v0[8], v1[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int h = lane + 32 * k;
                v0[k] = h < chunks ? __ldcg(partial + (size_t)c0 * chunks + h) : 0.0;
                v1[k] = (c1 >= 0 && h < chunks) ? __ldcg(partial + (size_t)c1 * chunks + h) : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                f0 += v0[k];
                f1 += v1[k];
            }
        } else {
            for (int h = lane; h < chunks; h += 32) {
                f0 += __ldcg(partial + (size_t)c0 * chunks + h);
                if (c1 >= 0) f1 += __ldcg(partial + (size_t)c1 * chunks + h);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            f0 += __shfl_xor_sync(0xFFFFFFFFu, f0, o);
            f1 += __shfl_xor_sync(0xFFFFFFFFu, f1, o);
        }
        if (lane == 0) {
            fsum[c0] = f0;
            if (c1 >= 0) fsum[c1] = f1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = -1;
        double bf = 0.0;
        for (int c = 0; c < kCand; ++c) {
            const unsigned long long k = skey[c];
            if (k == kKeyNone) break;
            const double f = fsum[c];
            const int i = (int)(k & 0xFFFFFFFFull);
            if (f == f && (best < 0 || f < bf || (f == bf && i < best))) {
                best = i;
                bf = f;
            }
        }
        s_best = (best >= 0 && bf < s_g64) ? best : -1;
        s_f = bf;
    }
    __syncthreads();
    const int best = s_best;
    for (int d = threadIdx.x; d < s.D; d += blockDim.x)
        s.G[(size_t)nxt * s.D + d] = best >= 0 ? __ldcg(src + (size_t)d * s.Np + best) : s.G[(size_t)cur * s.D + d];
    if (threadIdx.x == 0) {
        if (best >= 0) {
            *g64 = s_f;
            const unsigned long long k = pack_key((float)s_f, (uint32_t)best);
            s.gkey[0] = k;
            s.gkey[1] = k;
            if (stale) *stale = 1;
        } else {
            s.gkey[nxt] = s.gkey[cur];
        }
        *s.t_dev = t_prev + 1u;
    }
}

// The rescoring blocks' hand-off: the last block to finish (ticket) runs the
// acceptance; a null ticket skips it (a plain FP64 evaluation).
struct AcceptArgs {
    unsigned int* ticket;
    const float* src;
    const unsigned long long* top;
    const double* partial;
    int chunks;
    double* g64;
    int* stale;
};

__device__ __forceinline__ void last_block_accepts(const SwarmDev& s, const AcceptArgs& a) {
    if (!a.ticket) return;
    __shared__ int s_last;
    // the block's partial sums are written (barrier); thread 0 releases them
    // with its ticket and, in the last block, acquires the others' for all
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        s_last = atomicAdd(a.ticket, 1u) == gridDim.x * gridDim.y - 1;
        if (s_last) asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
    __syncthreads();
    if (!s_last) return;
    accept_best(s, a.src, a.top, a.partial, a.chunks, a.g64, a.stale);
    if (threadIdx.x == 0) *a.ticket = 0u;
}

// FP64 rescoring: partial[c][chunk] = sum over rows m of the chunk of
// (sum_d A[m][d] src[d][i_c] - b[m])^2 in double, i_c = index of top[c], src
// the candidates' pbest_pos (or their positions, which equal it when they
// improved in this iteration). One warp per row at a time, lanes over d;
// fixed reduction order throughout.
__global__ void __launch_bounds__(256) lsq_rescore_kernel(const __grid_constant__ SwarmDev s,
                                                          const float* __restrict__ src,
                                                          const float* __restrict__ A, const float* __restrict__ b,
                                                          int M, const unsigned long long* __restrict__ top,
                                                          int rows_per_chunk, double* __restrict__ partial,
                                                          const AcceptArgs acc_args) {
    extern __shared__ double xc[];            // [D]
    __shared__ double wsum[8];
    const int c = blockIdx.x, chunk = blockIdx.y;
    const unsigned long long key = top[c];
    double* out = partial + ((size_t)c * gridDim.y + chunk);
    if (key == kKeyNone) {
        if (threadIdx.x == 0) *out = __longlong_as_double(0x7FF8000000000000ll);   // no candidate
        last_block_accepts(s, acc_args);
        return;
    }
    const uint32_t i = (uint32_t)(key & 0xFFFFFFFFull);
    for (int d = threadIdx.x; d < s.D; d += blockDim.x) xc[d] = (double)src[(size_t)d * s.Np + i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = chunk * rows_per_chunk, m1 = min(M, m0 + rows_per_chunk);
    double acc = 0.0;   // this warp's rows, in order
    for (int m = m0 + warp; m < m1; m += 8) {
        const float* row = A + (size_t)m * s.D;
        // four independent chains per lane (d = lane + 32 (4k + j)), summed in a fixed order
        double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
        int d = lane;
        for (; d + 96 < s.D; d += 128) {
            p0 = fma((double)row[d], xc[d], p0);
            p1 = fma((double)row[d + 32], xc[d + 32], p1);
            p2 = fma((double)row[d + 64], xc[d + 64], p2);
            p3 = fma((double)row[d + 96], xc[d + 96], p3);
        }
        for (; d < s.D; d += 32) p0 = fma((double)row[d], xc[d], p0);
        double p = (p0 + p1) + (p2 + p3);
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xFFFFFFFFu, p, o);
        const double r = p - (double)b[m];
        acc = fma(r, r, acc);
    }
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += wsum[w];
        *out = tot;
    }
    last_block_accepts(s, acc_args);
}

// FP64 Gram form of the rescoring, for D <= M: with Gm = A^T A, c = A^T b,
// bb = b^T b (all FP64, computed once), f(x) = x^T Gm x - 2 c^T x + bb. Gm is
// symmetric, so only its upper triangle is read:
//   f(x) = sum_r x_r (Gm_rr x_r + 2 sum_{c>r} Gm_rc x_c - 2 c_r) + bb.
// Rows are taken in pairs (q, D-1-q), whose upper parts hold D-1 entries
// together, so every warp gets the same work. Block (group, chunk) handles 4
// candidates (group 4g..4g+3) and the pairs of its chunk:
// partial[cand][chunk] = its rows' terms (+ bb in chunk 0): per warp, each lane
// sums x_r times its columns of row r over the warp's rows, lanes take the
// diagonal and linear terms row by row, and one butterfly over the warp adds
// them; warps in a fixed order.
__global__ void __launch_bounds__(256) lsq_rescore_gram_kernel(const __grid_constant__ SwarmDev s,
                                                               const float* __restrict__ src,
                                                               const double* __restrict__ Gm,
                                                               const double* __restrict__ cvec, double bb,
                                                               const unsigned long long* __restrict__ top,
                                                               int pairs_per_chunk, int chunks,
                                                               double* __restrict__ partial,
                                                               const AcceptArgs acc_args) {
    extern __shared__ double xg[];            // [4][D]
    __shared__ double wsum[8][4];
    const int grp = blockIdx.x, chunk = blockIdx.y;
    const int D = s.D;
    bool live[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned long long key = top[grp * 4 + q];
        live[q] = key != kKeyNone;
        const uint32_t i = live[q] ? (uint32_t)(key & 0xFFFFFFFFull) : 0u;
        for (int d = threadIdx.x; d < D; d += blockDim.x)
            xg[q * D + d] = live[q] ? (double)src[(size_t)d * s.Np + i] : 0.0;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int npairs = (D + 1) / 2;
    const int p0 = chunk * pairs_per_chunk, p1 = min(npairs, p0 + pairs_per_chunk);
    // off[q]: this lane's share of sum_r x_r sum_{c>r} Gm_rc x_c over the warp's
    // rows (its columns of each row); reduced over the warp once, at the end
    double off[4] = {0.0, 0.0, 0.0, 0.0};
    int nrows = 0;   // rows of this warp, in order
    for (int pr = p0 + warp; pr < p1; pr += 8) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int r = side == 0 ? pr : D - 1 - pr;
            if (side == 1 && r == pr) break;   // the middle row of an odd D
            ++nrows;
            const double* row = Gm + (size_t)r * D;
            double y[4] = {0.0, 0.0, 0.0, 0.0};
            int c = r + 1 + lane;
            // four row loads in flight per lane (the loop is bound by their latency)
            for (; c + 96 < D; c += 128) {
                const double g0 = row[c], g1 = row[c + 32], g2 = row[c + 64], g3 = row[c + 96];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double* xq = xg + q * D + c;
                    y[q] = fma(g0, xq[0], y[q]);
                    y[q] = fma(g1, xq[32], y[q]);
                    y[q] = fma(g2, xq[64], y[q]);
                    y[q] = fma(g3, xq[96], y[q]);
                }
            }
            for (; c < D; c += 32) {
                const double g = row[c];
#pragma unroll
                for (int q = 0; q < 4; ++q) y[q] = fma(g, xg[q * D + c], y[q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) off[q] = fma(xg[q * D + r], y[q], off[q]);
        }
    }
    // diagonal and linear terms x_r (Gm_rr x_r - 2 c_r) of the warp's rows:
    // item t * 4 + q (row t of the warp, candidate q) on lane item % 32, so a
    // lane's items all belong to candidate lane % 4
    double dg = 0.0;
    for (int item = lane; item < nrows * 4; item += 32) {
        const int t = item >> 2, q = item & 3;
        const int pr = p0 + warp + 8 * (t >> 1);
        const int r = (t & 1) == 0 ? pr : D - 1 - pr;
        const double xr = xg[q * D + r];
        dg = fma(xr, fma(Gm[(size_t)r * D + r], xr, -2.0 * cvec[r]), dg);
    }
    double acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double v = fma(2.0, off[q], (lane & 3) == q ? dg : 0.0);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        acc[q] = v;
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) wsum[warp][q] = acc[q];
    __syncthreads();
    if (threadIdx.x < 4) {
        const int q = threadIdx.x;
        double tot = chunk == 0 ? bb : 0.0;
        for (int w = 0; w < 8; ++w) tot += wsum[w][q];
        partial[(size_t)(grp * 4 + q) * chunks + chunk] =
            live[q] ? tot : __longlong_as_double(0x7FF8000000000000ll);
    }
    last_block_accepts(s, acc_args);
}

// (hi, lo) += p + e: Knuth's TwoSum of hi and p (exact: hi' + t = hi + p), the
// error t and e collected in lo. Rounded operations only, none contracted.
__device__ __forceinline__ void ff_acc(float& hi, float& lo, float p, float e) {
    const float s = __fadd_rn(hi, p);
    const float z = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(p, z));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(t, e));
}

// The Gram-form rescoring of lsq_rescore_gram_kernel with the off-diagonal
// part in float-float arithmetic (unevaluated sums hi + lo of two binary32
// values, Dekker 1971), which the GB300 runs on its binary32 pipes, 64 times
// its binary64 rate. Each entry Gm_rc is held as gh + gl (gh = Gm_rc rounded
// to binary32, gl = the rest, rounded): x_r gh = p + e exactly (e by one fma),
// p enters the running hi by TwoSum, e and x_r gl the running lo. Per column c
// and quarter of a tile's rows the sum runs in float-float, is multiplied by
// x_c the same way, and a candidate's pieces are added in float-float in a
// fixed order (a reduce-scatter over each warp's lanes, then the warps in
// order) before one conversion to FP64. The diagonal and linear terms
// x_r (Gm_rr x_r - 2 c_r) stay in FP64 (D per candidate). Relative to the sum
// of the terms' magnitudes the result is within a few units of 2^-44, beside
// the FP64 Gram form's own cancellation error, which near a minimum dominates
// both.
//
// Block = (tile (tr, tc), tr <= tc, of the upper triangle in kFfTile squares;
// candidate quarter cq): blocks 4 k .. 4 k + 3 share tile k, so that a GPU of
// 152 SMs holds several blocks per SM and no SM gets a whole tile more than
// another. Thread (rq = tid / 64, c = tid % 64) takes column c of the tile,
// rows 16 rq .. 16 rq + 15, and the block's 4 candidates at once (one Gram
// entry and one float4 of coordinates from shared memory serve 4 terms).
// Entries on or below the diagonal of a diagonal tile are zeroed in shared
// memory (their terms are then exact zeros); the diagonal tile also adds the
// FP64 diagonal and linear terms of its rows, and tile 0 adds bb.
// partial[cand][tile].
__global__ void __launch_bounds__(256) lsq_rescore_gram_ff_kernel(const __grid_constant__ SwarmDev s,
                                                                  const float* __restrict__ src,
                                                                  const float2* __restrict__ Gff, int ldf,
                                                                  const double* __restrict__ Gm,
                                                                  const double* __restrict__ cvec, double bb,
                                                                  const unsigned long long* __restrict__ top,
                                                                  int ntiles, double* __restrict__ partial,
                                                                  const AcceptArgs acc_args) {
    constexpr int T = kFfTile, Q = 4, RQ = 4;
    static_assert(T == 64 && kCand == 4 * Q, "thread layout: 64 columns x 4 row quarters, 4 candidates each");
    __shared__ __align__(16) float2 gt[T][T];   // (gh, gl) of the tile, row-major
    __shared__ __align__(16) float4 xr[T], xc[T];   // the 4 candidates' coordinates of the tile's rows / columns
    __shared__ uint32_t cid[Q];
    __shared__ float rh[8][Q], rl[8][Q];        // per warp
    __shared__ double rd[8][Q];
    const int D = s.D;
    const int nt = ldf / T;
    const int tile = (int)blockIdx.x >> 2, cq = (int)blockIdx.x & 3;
    int tr = 0, k = tile;
    while (k >= nt - tr) {
        k -= nt - tr;
        ++tr;
    }
    const int tc = tr + k;
    const bool diag = tr == tc;
    const int r0 = tr * T, c0 = tc * T;
    if (threadIdx.x < Q) {
        const unsigned long long key = top[Q * cq + threadIdx.x];
        cid[threadIdx.x] = key == kKeyNone ? 0xFFFFFFFFu : (uint32_t)(key & 0xFFFFFFFFull);
    }
    __syncthreads();
    {
        // the tile: 64 rows x 32 float4 (two entries each); the 4 candidates'
        // coordinates of its rows and columns: 2 x 4 x 64 gathered values
        float4 g[8];
        float xv[2];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int e = (int)threadIdx.x + 256 * j;
            g[j] = *reinterpret_cast<const float4*>(Gff + (size_t)(r0 + (e >> 5)) * ldf + c0 + 2 * (e & 31));
        }
        const int q = (int)threadIdx.x >> 6, dd = (int)threadIdx.x & 63;
        const uint32_t i = cid[q];
#pragma unroll
        for (int j = 0; j < 2; ++j) {   // j = 0: rows, 1: columns
            const int d = (j ? c0 : r0) + dd;
            xv[j] = (i != 0xFFFFFFFFu && d < D) ? __ldcg(src + (size_t)d * s.Np + i) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int e = (int)threadIdx.x + 256 * j;
            const int rr = e >> 5, cc = 2 * (e & 31);
            float4 v = g[j];
            if (diag && cc <= rr) v.x = v.y = 0.0f;
            if (diag && cc + 1 <= rr) v.z = v.w = 0.0f;
            *reinterpret_cast<float4*>(&gt[rr][cc]) = v;
        }
        reinterpret_cast<float*>(&xr[dd])[q] = xv[0];
        reinterpret_cast<float*>(&xc[dd])[q] = xv[1];
    }
    __syncthreads();
    const int rq = (int)threadIdx.x >> 6, c = (int)threadIdx.x & 63;
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    float wh[Q] = {0.f, 0.f, 0.f, 0.f}, wl[Q] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int j = 0; j < T / RQ; ++j) {
        const int r = rq * (T / RQ) + j;
        const float4 x4 = xr[r];
        const float2 gv = gt[r][c];
        const float xq[Q] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const float p = __fmul_rn(xq[q], gv.x);
            const float e = __fmaf_rn(xq[q], gv.x, -p);   // exact: x gh = p + e
            ff_acc(wh[q], wl[q], p, __fmaf_rn(xq[q], gv.y, e));
        }
    }
    // times x_c
    float sh[Q], sl[Q];
    {
        const float4 x4 = xc[c];
        const float xq[Q] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            sh[q] = __fmul_rn(wh[q], xq[q]);
            sl[q] = __fmaf_rn(wl[q], xq[q], __fmaf_rn(wh[q], xq[q], -sh[q]));
        }
    }
    // the warp's 32 columns, a fixed pattern: lanes l and l ^ 1 split the 4
    // candidates (the lower lane keeps 0 and 1), lanes l and l ^ 2 split those
    // two, then three butterfly levels; lane 4 q' + 2 b + a ends with candidate
    // 2 a + b's sum over the warp (lanes 0, 1, 2, 3 hold candidates 0, 2, 1, 3)
    const bool up1 = (lane & 1) != 0, up2 = (lane & 2) != 0;
    // level 1: keep candidates 2 up1 + {0, 1}, send the other pair
    float a0h = up1 ? sh[2] : sh[0], a0l = up1 ? sl[2] : sl[0];
    float a1h = up1 ? sh[3] : sh[1], a1l = up1 ? sl[3] : sl[1];
    {
        const float g0h = up1 ? sh[0] : sh[2], g0l = up1 ? sl[0] : sl[2];
        const float g1h = up1 ? sh[1] : sh[3], g1l = up1 ? sl[1] : sl[3];
        const float o0h = __shfl_xor_sync(0xFFFFFFFFu, g0h, 1), o0l = __shfl_xor_sync(0xFFFFFFFFu, g0l, 1);
        const float o1h = __shfl_xor_sync(0xFFFFFFFFu, g1h, 1), o1l = __shfl_xor_sync(0xFFFFFFFFu, g1l, 1);
        ff_acc(a0h, a0l, o0h, o0l);
        ff_acc(a1h, a1l, o1h, o1l);
    }
    // level 2: keep candidate 2 up1 + up2, send the other one
    float h1 = up2 ? a1h : a0h, l1 = up2 ? a1l : a0l;
    {
        const float gh = up2 ? a0h : a1h, gl = up2 ? a0l : a1l;
        const float oh = __shfl_xor_sync(0xFFFFFFFFu, gh, 2), ol = __shfl_xor_sync(0xFFFFFFFFu, gl, 2);
        ff_acc(h1, l1, oh, ol);
    }
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
        const float oh = __shfl_xor_sync(0xFFFFFFFFu, h1, o), ol = __shfl_xor_sync(0xFFFFFFFFu, l1, o);
        ff_acc(h1, l1, oh, ol);
    }
    // x_r (Gm_rr x_r - 2 c_r) of row r0 + c for the 4 candidates, in the
    // diagonal tile's warps 0 and 1, summed over each warp
    double dq[Q] = {0.0, 0.0, 0.0, 0.0};
    if (diag && rq == 0) {
        const int d = r0 + c;
        const float4 x4 = xr[c];
        const float xq[Q] = {x4.x, x4.y, x4.z, x4.w};
        if (d < D) {
            const double gdd = __ldg(Gm + (size_t)d * D + d), c2 = -2.0 * __ldg(cvec + d);
#pragma unroll
            for (int q = 0; q < Q; ++q) dq[q] = (double)xq[q] * fma(gdd, (double)xq[q], c2);
        }
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dq[q] += __shfl_xor_sync(0xFFFFFFFFu, dq[q], o);
    }
    if (lane < 4) {
        const int q = 2 * (lane & 1) + (lane >> 1);   // the candidate lane `lane` holds
        rh[warp][q] = h1;
        rl[warp][q] = l1;
        rd[warp][q] = q == 0 ? dq[0] : q == 1 ? dq[1] : q == 2 ? dq[2] : dq[3];
    }
    __syncthreads();
    if (threadIdx.x < Q) {
        const int q = (int)threadIdx.x;
        float h = rh[0][q], l = rl[0][q];
        double dsum = rd[0][q];
#pragma unroll
        for (int w = 1; w < 8; ++w) {
            ff_acc(h, l, rh[w][q], rl[w][q]);
            dsum += rd[w][q];
        }
        double tot = fma(2.0, (double)h + (double)l, dsum);
        if (tile == 0) tot += bb;
        partial[(size_t)(Q * cq + q) * ntiles + tile] =
            cid[q] != 0xFFFFFFFFu ? tot : __longlong_as_double(0x7FF8000000000000ll);
    }
    last_block_accepts(s, acc_args);
}

// Gm = A^T A (D x D), cvec = A^T b, in FP64 (one-time setup). 32 x 32 output
// tile per block, rows of A in order.
__global__ void __launch_bounds__(256) lsq_gram_kernel(const float* __restrict__ A, const float* __restrict__ b,
                                                       int M, int D, double* __restrict__ Gm,
                                                       double* __restrict__ cvec, float2* __restrict__ Gff, int ldf) {
    __shared__ double ta[32][33], tb[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int m0 = 0; m0 < M; m0 += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int mm = e / 32, cc = e % 32;
            const int m = m0 + mm;
            ta[mm][cc] = (m < M && r0 + cc < D) ? (double)A[(size_t)m * D + r0 + cc] : 0.0;
            tb[mm][cc] = (m < M && c0 + cc < D) ? (double)A[(size_t)m * D + c0 + cc] : 0.0;
        }
        __syncthreads();
        for (int mm = 0; mm < 32; ++mm) {
            const double bv = tb[mm][tx];
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] = fma(ta[mm][ty * 4 + k], bv, acc[k]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = r0 + ty * 4 + k, c = c0 + tx;
        if (r < D && c < D) {
            Gm[(size_t)r * D + c] = acc[k];
            // the same entry as hi + lo in binary32 for the float-float rescoring
            const float hi = __double2float_rn(acc[k]);
            Gff[(size_t)r * ldf + c] = make_float2(hi, __double2float_rn(acc[k] - (double)hi));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const int r = r0 + threadIdx.x;
        if (r < D) {
            double v = 0.0;
            for (int m = 0; m < M; ++m) v = fma((double)A[(size_t)m * D + r], (double)b[m], v);
            cvec[r] = v;
        }
    }
}

// Error-free transformations in FP32 (Knuth's TwoSum; the product's error by
// one fma), for the compensated dot product of lsq_offset_kernel.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// The residual offsets of the reference point: off[m] = sum_d A[m][d] g[d] -
// b[m] for the gbest_pos g that the next iteration moves towards (the tensor-
// core fitness of a displacement y = x - g is then sum_m (A y + off)_m^2 =
// ||A x - b||^2). Each dot product is the compensated Dot2 of Ogita, Rump and
// Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005):
// as accurate as if accumulated in twice the FP32 precision, then rounded,
// which an FP32 sum of ~D terms of |A x| ~ 1 would not be next to residuals
// near the noise level. One warp per row: each lane keeps (sum, error) over
// its columns, the lanes are combined by the same transformation in a fixed
// tree, and the result, with b subtracted, is rounded once to float. Runs only
// when *stale is set (the accept kernel sets it when gbest moved) and clears it.
__global__ void __launch_bounds__(256) lsq_offset_kernel(const __grid_constant__ SwarmDev s,
                                                         const float* __restrict__ A, const float* __restrict__ b,
                                                         int M, float* __restrict__ off, int* __restrict__ stale) {
    extern __shared__ float gs[];   // gbest_pos [D]
    if (__ldcg(stale) == 0) return;
    const uint32_t t = __ldcg(s.t_dev);
    const float* g = s.G + (size_t)(t & 1u) * s.D;
    const int D = s.D;
    for (int d = threadIdx.x; d < D; d += blockDim.x) gs[d] = __ldcg(g + d);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = (int)(gridDim.x * blockDim.x) >> 5;
    // rows as float4 when they are 16-byte aligned: eight loads in flight per lane
    const bool vec = (D & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    for (int m = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); m < M; m += warps) {
        const float* row = A + (size_t)m * D;
        float p = 0.0f, c = 0.0f;   // running sum and its accumulated error
        auto term = [&](float a, float x) {
            const float h = __fmul_rn(a, x);
            const float r = __fmaf_rn(a, x, -h);   // exact: a x = h + r
            float q;
            two_sum(p, h, p, q);
            c = __fadd_rn(c, __fadd_rn(q, r));
        };
        if (vec) {
            const int nv = D >> 2;
            for (int v0 = 0; v0 < nv; v0 += 256) {
                float4 a4[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int v = v0 + lane + 32 * k;
                    a4[k] = v < nv ? __ldg(reinterpret_cast<const float4*>(row) + v) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int v = v0 + lane + 32 * k;
                    if (v < nv) {
                        term(a4[k].x, gs[4 * v]);
                        term(a4[k].y, gs[4 * v + 1]);
                        term(a4[k].z, gs[4 * v + 2]);
                        term(a4[k].w, gs[4 * v + 3]);
                    }
                }
            }
        } else {
            for (int d = lane; d < D; d += 32) term(__ldg(row + d), gs[d]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float p2 = __shfl_xor_sync(0xFFFFFFFFu, p, o), c2 = __shfl_xor_sync(0xFFFFFFFFu, c, o);
            // the same operands on both lanes of a pair, in a fixed order, so every lane ends with the same bits
            const float lo_p = lane & o ? p2 : p, hi_p = lane & o ? p : p2;
            const float lo_c = lane & o ? c2 : c, hi_c = lane & o ? c : c2;
            float q;
            two_sum(lo_p, hi_p, p, q);
            c = __fadd_rn(__fadd_rn(lo_c, hi_c), q);
        }
        if (lane == 0) off[m] = __double2float_rn(((double)p + (double)c) - (double)b[m]);
    }
    // every block has read *stale above; the last one to finish clears it
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(reinterpret_cast<unsigned int*>(stale) + 1, 1u) == gridDim.x - 1) {
            stale[1] = 0;
            stale[0] = 0;
        }
    }
}

// *g64 = sum over chunks of candidate 0's partial sums (fixed order).
__global__ void lsq_sum_one_kernel(const double* __restrict__ partial, int chunks, double* __restrict__ g64) {
    if (threadIdx.x == 0) {
        double f = 0.0;
        for (int h = 0; h < chunks; ++h) f += partial[h];
        *g64 = f;
    }
}

// Copies f into pbest_fit for real particles (the first evaluation: pbest = pos).
__global__ void lsq_set_pf_kernel(const __grid_constant__ SwarmDev s, const float* __restrict__ fit) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.N; i += gridDim.x * blockDim.x) s.pf[i] = fit[i];
}

// gbest recomputed from scratch in the approximate modes: all particles are
// candidates; the acceptance compares against +inf. Leaves t unchanged.
__global__ void lsq_keep_t_kernel(const __grid_constant__ SwarmDev s, uint32_t t) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *s.t_dev = t;
}

// ---------------------------------------------------------------------------

cudaError_t lsq_launch_move(const SwarmDev& s, int grid, cudaStream_t st) {
    lsq_move_kernel<<<grid, kBlock, sizeof(float) * (size_t)s.D, st>>>(s);
    return cudaGetLastError();
}

cudaError_t lsq_launch_move_q(const SwarmDev& s, const unsigned char (*maps)[128], void* Xq, int Kp, bool fp8,
                              float sx, int num_sms, cudaStream_t st) {
    if (s.Np % 64 != 0 || Kp % 64 != 0 || Kp < s.D || num_sms < 1 || !maps ||
        (reinterpret_cast<uintptr_t>(s.pflag) & 15) != 0)
        return cudaErrorInvalidValue;
    const int ntiles = (s.Np / 64) * (Kp / 64);
    const size_t smem = (size_t)kMoveStages * kMoveStageBytes + 128;
    MoveMaps mm;
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    for (int a = 0; a < 3; ++a) std::memcpy(&mm.m[a], maps[a], sizeof(CUtensorMap));
    // one CTA per SM walks the tiles
    const int grid = std::min(num_sms, ntiles);
    cudaError_t e = cudaFuncSetAttribute(fp8 ? (const void*)lsq_move_q_kernel<true> : (const void*)lsq_move_q_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (fp8) lsq_move_q_kernel<true><<<grid, kMoveThreads, smem, st>>>(s, mm, Xq, Kp, sx);
    else lsq_move_q_kernel<false><<<grid, kMoveThreads, smem, st>>>(s, mm, Xq, Kp, sx);
    return cudaGetLastError();
}

cudaError_t lsq_launch_select_exact(const SwarmDev& s, const float* fit, unsigned int* flags, int grid,
                                    cudaStream_t st) {
    const int g1 = std::max(1, std::min(grid, (s.Np / 4 + kBlock - 1) / kBlock));
    lsq_select_exact_kernel<<<g1, kBlock, 0, st>>>(s, fit, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lsq_copy_pbest_kernel<<<grid, kBlock, 0, st>>>(s, flags);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lsq_gather_kernel<<<1, 256, 0, st>>>(s);
    return cudaGetLastError();
}

int lsq_cand_lists(int Np) { return (Np + kSel - 1) / kSel * kSelWarps; }

cudaError_t lsq_launch_gram(const float* A, const float* b, int M, int D, double* Gm, double* cvec, float2* Gff,
                            int ldf, cudaStream_t st) {
    if (D > kGramMaxD || ldf < D || ldf % kFfTile != 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(Gff, 0, sizeof(float2) * (size_t)ldf * ldf, st);
    if (e != cudaSuccess) return e;
    lsq_gram_kernel<<<dim3((D + 31) / 32, (D + 31) / 32), 256, 0, st>>>(A, b, M, D, Gm, cvec, Gff, ldf);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the rescoring keeps 4 candidates x D doubles in shared memory: past the
    // default 48 KB from D = 1537 on
    return cudaFuncSetAttribute(lsq_rescore_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * 4 * (size_t)D));
}

// cand: [lists * 16] + [16] + ticket; partial: [16 * chunks]; flags: [Np / 4].
// With Gm set (D <= M) the rescoring uses the Gram form (float-float when
// gram.ff, else FP64); without it the FP64 residuals row by row.
cudaError_t lsq_launch_offsets(const SwarmDev& s, const float* A, const float* b, int M, float* off, int* stale,
                               int num_sms, cudaStream_t st) {
    const int grid = std::max(1, std::min(num_sms * 4, (M + 7) / 8));
    const size_t smem = sizeof(float) * (size_t)s.D;   // gbest_pos in shared memory
    if (smem > 48 * 1024) {
        if (smem > 227 * 1024) return cudaErrorInvalidValue;
        const cudaError_t e = cudaFuncSetAttribute(lsq_offset_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    lsq_offset_kernel<<<grid, 256, smem, st>>>(s, A, b, M, off, stale);
    return cudaGetLastError();
}

cudaError_t lsq_launch_gbest_approx(const SwarmDev& s, const float* fit, const float* part, int nparts, int all,
                                    bool lazy, const float* A, const float* b, int M, unsigned long long* cand,
                                    double* partial, int chunks, double* g64, unsigned int* flags, int grid,
                                    const LsqGram& gram, float* off, int* stale, int num_sms, cudaStream_t st) {
    const int nblk = (s.Np + kSel - 1) / kSel;
    unsigned long long* top = cand + (size_t)lsq_cand_lists(s.Np) * kCand;
    unsigned int* ticket = reinterpret_cast<unsigned int*>(top + kCand);
    lsq_select_cand_kernel<<<nblk, kSel, 0, st>>>(s, fit, part, nparts, all, cand, flags, top, ticket);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (!all && !lazy) {
        lsq_copy_pbest_kernel<<<grid, kBlock, 0, st>>>(s, flags);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // the candidates improved in this iteration (or, with `all`, are every
    // pbest): their pbest_pos is the position, pending write-back when lazy
    const float* src = (lazy && !all) ? s.x : s.pb;
    // the last rescoring block accepts the best candidate (ticket: stale[2])
    const AcceptArgs acc{reinterpret_cast<unsigned int*>(stale + 2), src, top, partial, chunks, g64, stale};
    if (gram.Gm && gram.ff) {
        const int nt = lsq_ff_tiles(s.D);
        const AcceptArgs acc_ff{acc.ticket, src, top, partial, nt, g64, stale};
        lsq_rescore_gram_ff_kernel<<<4 * nt, 256, 0, st>>>(s, src, gram.Gff, gram.ldf, gram.Gm, gram.cvec, gram.bb,
                                                           top, nt, partial, acc_ff);
    } else if (gram.Gm) {
        const int pairs = ((s.D + 1) / 2 + chunks - 1) / chunks;
        lsq_rescore_gram_kernel<<<dim3(kCand / 4, chunks), 256, sizeof(double) * 4 * (size_t)s.D, st>>>(
            s, src, gram.Gm, gram.cvec, gram.bb, top, pairs, chunks, partial, acc);
    } else {
        const int rows = (M + chunks - 1) / chunks;
        lsq_rescore_kernel<<<dim3(kCand, chunks), 256, sizeof(double) * (size_t)s.D, st>>>(s, src, A, b, M, top,
                                                                                          rows, partial, acc);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess || !off) return e;
    return lsq_launch_offsets(s, A, b, M, off, stale, num_sms, st);
}

// FP64 fitness of pbest_pos of the particle in `key` into *g64 (one candidate).
cudaError_t lsq_rescore_one(const SwarmDev& s, const float* A, const float* b, int M, unsigned long long key,
                            unsigned long long* scratch, double* partial, int chunks, double* g64, cudaStream_t st) {
    unsigned long long top[kCand];
    for (int c = 0; c < kCand; ++c) top[c] = c == 0 ? key : kKeyNone;
    cudaError_t e = cudaMemcpyAsync(scratch, top, sizeof(top), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const int rows = (M + chunks - 1) / chunks;
    const AcceptArgs none{nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr};
    lsq_rescore_kernel<<<dim3(kCand, chunks), 256, sizeof(double) * (size_t)s.D, st>>>(s, s.pb, A, b, M, scratch,
                                                                                      rows, partial, none);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lsq_sum_one_kernel<<<1, 32, 0, st>>>(partial, chunks, g64);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

cudaError_t lsq_launch_set_pf(const SwarmDev& s, const float* fit, cudaStream_t st) {
    lsq_set_pf_kernel<<<std::max(1, std::min(1024, (s.N + 255) / 256)), 256, 0, st>>>(s, fit);
    return cudaGetLastError();
}

cudaError_t lsq_launch_set_t(const SwarmDev& s, uint32_t t, cudaStream_t st) {
    lsq_keep_t_kernel<<<1, 32, 0, st>>>(s, t);
    return cudaGetLastError();
}

}  // namespace cupso
