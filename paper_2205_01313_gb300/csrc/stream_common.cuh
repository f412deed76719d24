// stream_common.cuh -- per-particle building blocks shared by the kernels that
// stream the swarm through HBM (kernels_stream.cu, kernels_pipelined.cu).
#pragma once

#include <cuda_runtime.h>

#include "cupso_device.cuh"
#include "cupso_internal.h"

namespace cupso {

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float lane(const float4& v, int j) {
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}
__device__ __forceinline__ void set_lane(float4& v, int j, float a) {
    if (j == 0) v.x = a; else if (j == 1) v.y = a; else if (j == 2) v.z = a; else v.w = a;
}
__device__ __forceinline__ uint32_t word(const uint4& r, int k) {
    return k == 0 ? r.x : (k == 1 ? r.y : (k == 2 ? r.z : r.w));
}

// Eq. 1 and Eq. 2 for one (particle, dimension), with the clamps of Alg. 1.
__device__ __forceinline__ void move_one(float& x, float& v, float pb, float g, float r1, float r2,
                                         const SwarmDev& s) {
    const float cognitive = __fsub_rn(pb, x);
    const float social = __fsub_rn(g, x);
    float vel = __fmul_rn(s.w, v);
    vel = __fmaf_rn(__fmul_rn(s.c1, r1), cognitive, vel);
    vel = __fmaf_rn(__fmul_rn(s.c2, r2), social, vel);
    v = clampf(vel, -s.vmax, s.vmax);
    x = clampf(__fadd_rn(x, v), s.lo, s.hi);
}

// The same update on the fast path: c * r as fma(cs, k, cs) with
// k = float(w >> 8) (the identical rounded product), clamps as min/max.
// Bit-identical to move_one when s.fast_cr and s.fast_clamp hold.
__device__ __forceinline__ void move_one_fast(float& x, float& v, float pb, float g, float k1, float k2,
                                              const SwarmDev& s) {
    const float cognitive = __fsub_rn(pb, x);
    const float social = __fsub_rn(g, x);
    float vel = __fmul_rn(s.w, v);
    vel = __fmaf_rn(__fmaf_rn(s.c1s, k1, s.c1s), cognitive, vel);
    vel = __fmaf_rn(__fmaf_rn(s.c2s, k2, s.c2s), social, vel);
    v = clampf_minmax(vel, -s.vmax, s.vmax);
    x = clampf_minmax(__fadd_rn(x, v), s.lo, s.hi);
}

__device__ __forceinline__ float hi24(uint32_t w) { return __uint2float_rn(w >> 8); }

// Steps 2-3 for the particles i0..i0+3 at iteration t: reads x, v, pb, writes
// x', v', returns the four fitness values. Gs is gbest_pos in shared memory.
template <int FIT>
__device__ __forceinline__ void move4(const SwarmDev& s, uint32_t i0, uint32_t t,
                                      const float* __restrict__ Gs, float f[4]) {
    const size_t Np = (size_t)s.Np;
    FitAcc<FIT> acc[4];
    const int D = s.D;
#pragma unroll 1
    for (int d0 = 0; d0 < D; d0 += 2) {
        uint4 r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            r[j] = philox4x32_10(make_uint4((uint32_t)(d0 >> 1), i0 + j, t, s.swarm), s.key0, s.key1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int d = d0 + h;
            if (h == 1 && d >= D) break;
            const size_t off = (size_t)d * Np + i0;
            float4 X = ld4(s.x + off), V = ld4(s.v + off);
            const float4 P = ld4(s.pb + off);
            const float g = Gs[d];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float xj = lane(X, j), vj = lane(V, j);
                move_one(xj, vj, lane(P, j), g, u01(word(r[j], 2 * h)), u01(word(r[j], 2 * h + 1)), s);
                set_lane(X, j, xj);
                set_lane(V, j, vj);
                acc[j].add(d, xj);
            }
            st4(s.x + off, X);
            st4(s.v + off, V);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) f[j] = acc[j].finish(D);
}

// Step 4 for the four particles: strict improvement, then pbest_fit and the
// improved columns of pbest_pos are written (x' is re-read, still in L2).
// Returns the improved mask; pf_out holds the (new) pbest_fit values.
__device__ __forceinline__ unsigned pbest4(const SwarmDev& s, uint32_t i0, const float f[4], float pf_out[4]) {
    float4 PF = ld4(s.pf + i0);
    unsigned mask = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool real = (i0 + j) < (uint32_t)s.N;
        if (real && f[j] < lane(PF, j)) {
            mask |= 1u << j;
            set_lane(PF, j, f[j]);
        }
        pf_out[j] = lane(PF, j);
    }
    if (mask) {
        st4(s.pf + i0, PF);
        const size_t Np = (size_t)s.Np;
        for (int d = 0; d < s.D; ++d) {
            const size_t off = (size_t)d * Np + i0;
            const float4 X = ld4(s.x + off);
            if (mask == 0xFu) {
                st4(s.pb + off, X);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (mask & (1u << j)) s.pb[off + j] = lane(X, j);
            }
        }
    }
    return mask;
}

__device__ __forceinline__ bool any_nan4(const SwarmDev& s, uint32_t i0, const float f[4]) {
    bool nan = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) nan |= ((i0 + j) < (uint32_t)s.N) && (f[j] != f[j]);
    return nan;
}

// Block-wide minimum of one key per thread (warp shuffles, then warp 0).
__device__ __forceinline__ unsigned long long block_min(unsigned long long k, unsigned long long* red) {
    k = warp_min_u64(k);
    const int lane_id = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane_id == 0) red[wid] = k;
    __syncthreads();
    if (wid == 0) {
        k = lane_id < (int)(blockDim.x >> 5) ? red[lane_id] : kKeyNone;
        k = warp_min_u64(k);
        if (lane_id == 0) red[0] = k;
    }
    __syncthreads();
    k = red[0];
    __syncthreads();
    return k;
}

// Last-CTA-done epilogue: the CTA that finishes last gathers gbest_pos from
// pbest_pos at the winning index and rolls the iteration state forward.
__device__ __forceinline__ void finish_iteration(const SwarmDev& s, int cur, int nxt, uint32_t t_new) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(s.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const unsigned long long knew = __ldcg(s.gkey + nxt);
    const uint32_t g = (uint32_t)(knew & 0xFFFFFFFFull);
    const size_t Np = (size_t)s.Np;
    if (g < (uint32_t)s.N) {
        // a particle whose pbest is not yet written back has pbest_pos == pos
        const bool lazy = s.pflag && ((__ldcg(reinterpret_cast<const unsigned int*>(s.pflag) + (g >> 2)) >>
                                       (8u * (g & 3u))) & 0xFFu);
        const float* src = lazy ? s.x : s.pb;
        for (int d = threadIdx.x; d < s.D; d += blockDim.x)
            s.G[(size_t)nxt * s.D + d] = __ldcg(src + (size_t)d * Np + g);
    }
    if (threadIdx.x == 0) {
        s.gkey[cur] = knew;
        *s.t_dev = t_new;
        *s.ticket = 0u;
        if (s.work) *s.work = 0u;
    }
}

}  // namespace cupso
