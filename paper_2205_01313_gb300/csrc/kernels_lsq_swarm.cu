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
// fitness are rescored in FP64 and the best of them replaces gbest only if its
// FP64 fitness is lower than gbest's (ties to the lower index).
//
// Every kernel reads the iteration counter from device memory, so a chain of
// iterations can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "stream_common.cuh"

#include <algorithm>

namespace cupso {

namespace {

constexpr int kCand = 16;   // candidates rescored in FP64 per iteration

__device__ __forceinline__ unsigned long long my_min4(const unsigned long long k[4]) {
    unsigned long long m = k[0];
#pragma unroll
    for (int j = 1; j < 4; ++j) m = k[j] < m ? k[j] : m;
    return m;
}

}  // namespace

// Steps 2 of every particle at iteration t = *t_dev + 1 (no fitness here).
__global__ void __launch_bounds__(kBlock) lsq_move_kernel(const __grid_constant__ SwarmDev s) {
    extern __shared__ float Gs[];
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur = (int)(t_prev & 1u);
    for (int d = threadIdx.x; d < s.D; d += blockDim.x) Gs[d] = __ldcg(s.G + (size_t)cur * s.D + d);
    __syncthreads();
    const int ntiles = tiles_of(s.Np);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t i0 = (uint32_t)tile * kTile + threadIdx.x * kPerThread;
        if (i0 >= (uint32_t)s.Np) continue;
        float f[4];
        move4<kLsq>(s, i0, t_prev + 1u, Gs, f);
    }
}

// Steps 4-5 with the exact FP32 fitness f: as in sync_step_kernel.
__global__ void __launch_bounds__(kBlock) lsq_select_exact_kernel(const __grid_constant__ SwarmDev s,
                                                                  const float* __restrict__ fit) {
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    const unsigned long long K = __ldcg(s.gkey + cur);
    unsigned long long best = kKeyNone;
    bool nan = false;
    const int ntiles = tiles_of(s.Np);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t i0 = (uint32_t)tile * kTile + threadIdx.x * kPerThread;
        if (i0 >= (uint32_t)s.Np) continue;
        float f[4], pf[4];
        const float4 F = ld4(fit + i0);
        f[0] = F.x; f[1] = F.y; f[2] = F.z; f[3] = F.w;
        const unsigned mask = pbest4(s, i0, f, pf);
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
    finish_iteration(s, cur, nxt, t_prev + 1u);
}

// Step 4 with an approximate fitness, and each block's 16 lowest keys among the
// particles that improved (all particles when `all` is set: the first gbest).
// One 1024-particle tile per block; cand[block][16] (kKeyNone where fewer).
__global__ void __launch_bounds__(kBlock) lsq_select_cand_kernel(const __grid_constant__ SwarmDev s,
                                                                 const float* __restrict__ fit, int all,
                                                                 unsigned long long* __restrict__ cand) {
    __shared__ unsigned long long red[kBlock / 32];
    const uint32_t i0 = (uint32_t)blockIdx.x * kTile + threadIdx.x * kPerThread;
    unsigned long long k4[4] = {kKeyNone, kKeyNone, kKeyNone, kKeyNone};
    bool nan = false;
    if (i0 < (uint32_t)s.Np) {
        float f[4], pf[4];
        const float4 F = ld4(fit + i0);
        f[0] = F.x; f[1] = F.y; f[2] = F.z; f[3] = F.w;
        const unsigned mask = all ? 0u : pbest4(s, i0, f, pf);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool real = (i0 + j) < (uint32_t)s.N;
            if (real && (all || (mask & (1u << j)))) k4[j] = pack_key(f[j], i0 + j);
        }
        nan = any_nan4(s, i0, f);
    }
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
    // 16 rounds: the block minimum, removed by its owner
    for (int r = 0; r < kCand; ++r) {
        const unsigned long long m = block_min(my_min4(k4), red);
        if (threadIdx.x == 0) cand[(size_t)blockIdx.x * kCand + r] = m;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (k4[j] == m) k4[j] = kKeyNone;
    }
}

// The 16 lowest keys over all blocks' candidate lists, ascending, into top[16].
// Keys are unique (the index is in the low bits), so round r takes the
// smallest key above round r-1's.
__global__ void __launch_bounds__(1024) lsq_merge_cand_kernel(const unsigned long long* __restrict__ cand, int n,
                                                              unsigned long long* __restrict__ top) {
    __shared__ unsigned long long red[32];
    unsigned long long last = 0;
    for (int r = 0; r < kCand; ++r) {
        unsigned long long lm = kKeyNone;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const unsigned long long k = cand[e];
            if ((r == 0 || k > last) && k < lm) lm = k;
        }
        const unsigned long long m = block_min(lm, red);
        if (threadIdx.x == 0) top[r] = m;
        last = m;
        if (m == kKeyNone) {
            for (int q = r + 1 + (int)threadIdx.x; q < kCand; q += blockDim.x) top[q] = kKeyNone;
            break;
        }
    }
}

// FP64 rescoring: partial[c][chunk] = sum over rows m of the chunk of
// (sum_d A[m][d] pbest_pos[d][i_c] - b[m])^2 in double, i_c = index of top[c].
// One warp per row at a time, lanes over d; fixed reduction order throughout.
__global__ void __launch_bounds__(256) lsq_rescore_kernel(const __grid_constant__ SwarmDev s,
                                                          const float* __restrict__ A, const float* __restrict__ b,
                                                          int M, const unsigned long long* __restrict__ top,
                                                          int rows_per_chunk, double* __restrict__ partial) {
    extern __shared__ double xc[];            // [D]
    __shared__ double wsum[8];
    const int c = blockIdx.x, chunk = blockIdx.y;
    const unsigned long long key = top[c];
    double* out = partial + ((size_t)c * gridDim.y + chunk);
    if (key == kKeyNone) {
        if (threadIdx.x == 0) *out = __longlong_as_double(0x7FF8000000000000ll);   // no candidate
        return;
    }
    const uint32_t i = (uint32_t)(key & 0xFFFFFFFFull);
    for (int d = threadIdx.x; d < s.D; d += blockDim.x) xc[d] = (double)s.pb[(size_t)d * s.Np + i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = chunk * rows_per_chunk, m1 = min(M, m0 + rows_per_chunk);
    double acc = 0.0;   // this warp's rows, in order
    for (int m = m0 + warp; m < m1; m += 8) {
        const float* row = A + (size_t)m * s.D;
        double p = 0.0;
        for (int d = lane; d < s.D; d += 32) p = fma((double)row[d], xc[d], p);
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
}

// Accepts the best rescored candidate if it beats gbest in FP64; rolls t.
__global__ void lsq_accept_kernel(const __grid_constant__ SwarmDev s, const unsigned long long* __restrict__ top,
                                  const double* __restrict__ partial, int chunks, double* __restrict__ g64) {
    __shared__ int s_best;
    __shared__ double s_f;
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    if (threadIdx.x == 0) {
        int best = -1;
        double bf = 0.0;
        for (int c = 0; c < kCand; ++c) {
            const unsigned long long k = top[c];
            if (k == kKeyNone) break;
            double f = 0.0;
            for (int h = 0; h < chunks; ++h) f += partial[(size_t)c * chunks + h];
            const int i = (int)(k & 0xFFFFFFFFull);
            if (f == f && (best < 0 || f < bf || (f == bf && i < best))) {
                best = i;
                bf = f;
            }
        }
        s_best = (best >= 0 && bf < *g64) ? best : -1;
        s_f = bf;
    }
    __syncthreads();
    const int best = s_best;
    for (int d = threadIdx.x; d < s.D; d += blockDim.x)
        s.G[(size_t)nxt * s.D + d] = best >= 0 ? s.pb[(size_t)d * s.Np + best] : s.G[(size_t)cur * s.D + d];
    if (threadIdx.x == 0) {
        if (best >= 0) {
            *g64 = s_f;
            const unsigned long long k = pack_key((float)s_f, (uint32_t)best);
            s.gkey[0] = k;
            s.gkey[1] = k;
        } else {
            s.gkey[nxt] = s.gkey[cur];
        }
        *s.t_dev = t_prev + 1u;
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

cudaError_t lsq_launch_select_exact(const SwarmDev& s, const float* fit, int grid, cudaStream_t st) {
    lsq_select_exact_kernel<<<grid, kBlock, 0, st>>>(s, fit);
    return cudaGetLastError();
}

int lsq_cand_blocks(const SwarmDev& s) { return tiles_of(s.Np); }

// cand: [blocks * 16] + [16] scratch; partial: [16 * chunks].
cudaError_t lsq_launch_gbest_approx(const SwarmDev& s, const float* fit, int all, const float* A, const float* b,
                                    int M, unsigned long long* cand, double* partial, int chunks, double* g64,
                                    cudaStream_t st) {
    const int nblk = tiles_of(s.Np);
    unsigned long long* top = cand + (size_t)nblk * kCand;
    lsq_select_cand_kernel<<<nblk, kBlock, 0, st>>>(s, fit, all, cand);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lsq_merge_cand_kernel<<<1, 1024, 0, st>>>(cand, nblk * kCand, top);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int rows = (M + chunks - 1) / chunks;
    lsq_rescore_kernel<<<dim3(kCand, chunks), 256, sizeof(double) * (size_t)s.D, st>>>(s, A, b, M, top, rows, partial);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lsq_accept_kernel<<<1, 256, 0, st>>>(s, top, partial, chunks, g64);
    return cudaGetLastError();
}

// FP64 fitness of pbest_pos of the particle in `key` into *g64 (one candidate).
cudaError_t lsq_rescore_one(const SwarmDev& s, const float* A, const float* b, int M, unsigned long long key,
                            unsigned long long* scratch, double* partial, int chunks, double* g64, cudaStream_t st) {
    unsigned long long top[kCand];
    for (int c = 0; c < kCand; ++c) top[c] = c == 0 ? key : kKeyNone;
    cudaError_t e = cudaMemcpyAsync(scratch, top, sizeof(top), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const int rows = (M + chunks - 1) / chunks;
    lsq_rescore_kernel<<<dim3(kCand, chunks), 256, sizeof(double) * (size_t)s.D, st>>>(s, A, b, M, scratch, rows,
                                                                                      partial);
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
