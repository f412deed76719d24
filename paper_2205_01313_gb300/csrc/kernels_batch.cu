// kernels_batch.cu -- many independent swarms of uneven size in one launch per
// iteration.
//
// Each launch advances every swarm of the batch by one synchronous iteration
// (Steps 2-5 of Alg. 1). The work is the union of all swarms' 128-particle
// units, handed to warps from one counter in a fixed order (swarms with the
// same fitness function together; within those the units with the most
// dimensions first, so that the short ones fill the tail). A unit is
// processed exactly like one unit of the pipelined single-swarm kernel, by a
// copy of the unit loop compiled for its swarm's fitness function: rows staged through a per-thread cp.async ring in shared
// memory, lazy pbest write-back, conditional atomicMin on the swarm's packed
// gbest key. Each swarm keeps its own gbest key and position; the warp that
// finishes a swarm's last unit gathers that swarm's gbest_pos. The kernel
// boundary between iterations is the only barrier, so every swarm follows the
// same synchronous trajectory as if it ran alone (its Philox counter carries
// its own swarm id).
#include <cuda_runtime.h>

#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "stream_common.cuh"

namespace cupso {

namespace {

constexpr int kUnitB = 128;

__device__ __forceinline__ void cp_async16b(float4* smem, const float* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit_b() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait_b() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One unit of work: (swarm index, unit within that swarm), 0xFFFFFFFF = none.
struct Unit {
    uint32_t sw, u;
};

__device__ __forceinline__ Unit fetch(const BatchDev& b, unsigned* work, int lane_id) {
    uint32_t k = 0;
    if (lane_id == 0) k = atomicAdd(work, 1u);
    k = __shfl_sync(0xFFFFFFFFu, k, 0);
    if (k >= b.nunits) return Unit{0xFFFFFFFFu, 0u};
    const uint2 e = __ldg(b.units + k);
    return Unit{e.x, e.y};
}

// Copies of pair g of unit u of swarm w into ring stage `stage`.
__device__ __forceinline__ void issue_rows(const BatchSwarm& w, float4* my, uint32_t u, int g, int stage,
                                           int lane_id) {
    const size_t col = (size_t)u * kUnitB + (size_t)lane_id * 4;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int d = 2 * g + r;
        if (d < w.D) {
            const size_t off = (size_t)d * (size_t)w.Np + col;
            cp_async16b(my + (stage * 6 + 0 + r) * kBlock, w.x + off);
            cp_async16b(my + (stage * 6 + 2 + r) * kBlock, w.v + off);
            cp_async16b(my + (stage * 6 + 4 + r) * kBlock, w.pb + off);
        }
    }
    cp_commit_b();
}

// The same for unit `un` of the batch (an empty group if there is none).
__device__ __forceinline__ void issue(const BatchDev& b, float4* my, Unit un, int g, int stage, int lane_id) {
    if (un.sw != 0xFFFFFFFFu) issue_rows(b.swarms[un.sw], my, un.u, g, stage, lane_id);
    else cp_commit_b();
}

// Eq. 1 and Eq. 2 for one element with the parameters of swarm w.
template <bool FAST>
__device__ __forceinline__ void move_w(float& x, float& v, float pb, float g, uint32_t w1, uint32_t w2,
                                       const BatchSwarm& w) {
    const float cognitive = __fsub_rn(pb, x);
    const float social = __fsub_rn(g, x);
    float vel = __fmul_rn(w.w, v);
    if constexpr (FAST) {
        vel = __fmaf_rn(__fmaf_rn(w.c1s, hi24(w1), w.c1s), cognitive, vel);
        vel = __fmaf_rn(__fmaf_rn(w.c2s, hi24(w2), w.c2s), social, vel);
        v = clampf_minmax(vel, -w.vmax, w.vmax);
        x = clampf_minmax(__fadd_rn(x, v), w.lo, w.hi);
    } else {
        vel = __fmaf_rn(__fmul_rn(w.c1, u01(w1)), cognitive, vel);
        vel = __fmaf_rn(__fmul_rn(w.c2, u01(w2)), social, vel);
        v = clampf(vel, -w.vmax, w.vmax);
        x = clampf(__fadd_rn(x, v), w.lo, w.hi);
    }
}

// The per-warp pipeline state carried from one unit to the next.
struct Pipe {
    Unit nxt;        // the unit after the current one (fetched when first needed)
    bool have_nxt;
    int ig;          // pair of the next issue, counted from the current unit
    int stage;       // ring stage of the pair being computed
};

// Process unit `cu` of the batch at iteration t; keeps STAGES-1 pairs in
// flight. One copy per (fitness, fast path), so the loop body carries no
// per-element branch and a thread's four particles interleave freely.
template <int STAGES, int FIT, bool FAST>
__device__ __forceinline__ void run_unit_t(const BatchDev& b, unsigned* work, float4* my, Unit cu, Pipe& pp,
                                           uint32_t t, int lane_id) {
    // A private copy of the descriptor: the unit's own stores cannot alias it,
    // so its fields stay in registers.
    const BatchSwarm w = b.swarms[cu.sw];
    const int D = w.D, npairs = (D + 1) >> 1;
    const size_t Np = (size_t)w.Np;
    const int cur = (int)((t - 1u) & 1u), nxt = cur ^ 1;
    const float* G = w.G + (size_t)cur * D;
    const unsigned long long K = __ldcg(w.gkey + cur);
    const uint32_t i0 = cu.u * kUnitB + (uint32_t)lane_id * 4;
    const uint32_t fl = __ldcg(reinterpret_cast<const unsigned int*>(w.pflag + i0));
    FitAcc<FIT> acc[4];
    float4 PF = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int g = 0; g < npairs; ++g) {
        {
            int ws = pp.stage + STAGES - 1;
            if (ws >= STAGES) ws -= STAGES;
            if (pp.ig < npairs) {
                issue_rows(w, my, cu.u, pp.ig, ws, lane_id);
                ++pp.ig;
            } else {
                if (!pp.have_nxt) {
                    pp.nxt = fetch(b, work, lane_id);
                    pp.have_nxt = true;
                }
                // every unit has >= STAGES-1 pairs, so the lookahead stays within
                // the next unit (or there is no next unit: an empty group)
                issue(b, my, pp.nxt, pp.ig - npairs, ws, lane_id);
                ++pp.ig;
            }
        }
        if (g == npairs - 1) PF = ld4(w.pf + i0);
        cp_wait_b<STAGES - 1>();
        const uint4 rr[4] = {philox4x32_10(make_uint4((uint32_t)g, i0 + 0, t, w.swarm), w.key0, w.key1),
                             philox4x32_10(make_uint4((uint32_t)g, i0 + 1, t, w.swarm), w.key0, w.key1),
                             philox4x32_10(make_uint4((uint32_t)g, i0 + 2, t, w.swarm), w.key0, w.key1),
                             philox4x32_10(make_uint4((uint32_t)g, i0 + 3, t, w.swarm), w.key0, w.key1)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int d = 2 * g + h;
            if (h == 1 && d >= D) break;
            float4 X = my[(pp.stage * 6 + 0 + h) * kBlock];
            float4 V = my[(pp.stage * 6 + 2 + h) * kBlock];
            float4 P = my[(pp.stage * 6 + 4 + h) * kBlock];
            const size_t off = (size_t)d * Np + i0;
            if (fl) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if ((fl >> (8 * j)) & 1u) set_lane(P, j, lane(X, j));
                st4(w.pb + off, P);
            }
            const float gd = __ldg(G + d);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float xj = lane(X, j), vj = lane(V, j);
                move_w<FAST>(xj, vj, lane(P, j), gd, word(rr[j], 2 * h), word(rr[j], 2 * h + 1), w);
                set_lane(X, j, xj);
                set_lane(V, j, vj);
                acc[j].add(d, xj);
            }
            st4(w.x + off, X);
            st4(w.v + off, V);
        }
        if (++pp.stage == STAGES) pp.stage = 0;
    }
    // Step 4 (lazy pbest) and the unit's Step-5 candidate.
    uint32_t fl_new = 0u;
    unsigned long long best = kKeyNone;
    bool nan = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float f = acc[j].finish(D);
        const bool real = (i0 + j) < (uint32_t)w.N;
        nan |= real && (f != f);
        if (real && f < lane(PF, j)) {
            fl_new |= 1u << (8 * j);
            set_lane(PF, j, f);
            const unsigned long long k = pack_key(f, i0 + j);
            if (k < K && k < best) best = k;
        }
    }
    if (fl_new) st4(w.pf + i0, PF);
    if (fl_new != fl) *reinterpret_cast<unsigned int*>(w.pflag + i0) = fl_new;
    const bool lane_cand = best < K;
    best = warp_min_u64(best);
    const bool any_nan = __any_sync(0xFFFFFFFFu, nan);
    // Publish, then count the unit; the warp that completes the swarm gathers
    // its gbest. The gather reads only the winner's row and improvement flag,
    // and the winner was a candidate below K in its unit, so only a lane that
    // holds such a candidate makes its stores visible before lane 0 counts
    // (a fence per unit in every lane stalled each warp on its own stores).
    if (lane_cand) __threadfence();
    __syncwarp();
    int last = 0;
    if (lane_id == 0) {
        if (best < K) {
            atomicMin(w.gkey + nxt, best);
            __threadfence();
        }
        if (any_nan) atomicOr(w.status, kStatusNaN);
        last = atomicAdd(w.done, 1u) == w.nunits - 1u;
        if (last) __threadfence();
    }
    last = __shfl_sync(0xFFFFFFFFu, last, 0);
    if (last) {
        const unsigned long long knew = __ldcg(w.gkey + nxt);
        const uint32_t gi = (uint32_t)(knew & 0xFFFFFFFFull);
        if (gi < (uint32_t)w.N) {
            const bool lazy = (__ldcg(reinterpret_cast<const unsigned int*>(w.pflag) + (gi >> 2)) >>
                               (8u * (gi & 3u))) & 0xFFu;
            const float* src = lazy ? w.x : w.pb;
            for (int d = lane_id; d < D; d += 32) w.G[(size_t)nxt * D + d] = __ldcg(src + (size_t)d * Np + gi);
        }
        __syncwarp();
        if (lane_id == 0) {
            w.gkey[cur] = knew;
            *w.done = 0u;
        }
    }
    pp.ig -= npairs;
}

template <int STAGES>
__device__ __forceinline__ void run_unit(const BatchDev& b, unsigned* work, float4* my, Unit cu, Pipe& pp,
                                         uint32_t t, int lane_id) {
    const BatchSwarm& w = b.swarms[cu.sw];
    const bool fast = w.fast != 0;
    switch (w.fid) {
        case kSphere:
            if (fast) run_unit_t<STAGES, kSphere, true>(b, work, my, cu, pp, t, lane_id);
            else run_unit_t<STAGES, kSphere, false>(b, work, my, cu, pp, t, lane_id);
            break;
        case kRastrigin:
            if (fast) run_unit_t<STAGES, kRastrigin, true>(b, work, my, cu, pp, t, lane_id);
            else run_unit_t<STAGES, kRastrigin, false>(b, work, my, cu, pp, t, lane_id);
            break;
        case kAckley:
            if (fast) run_unit_t<STAGES, kAckley, true>(b, work, my, cu, pp, t, lane_id);
            else run_unit_t<STAGES, kAckley, false>(b, work, my, cu, pp, t, lane_id);
            break;
        case kRosenbrock:
            if (fast) run_unit_t<STAGES, kRosenbrock, true>(b, work, my, cu, pp, t, lane_id);
            else run_unit_t<STAGES, kRosenbrock, false>(b, work, my, cu, pp, t, lane_id);
            break;
        default:  // kCubicMax (the host admits nothing else)
            if (fast) run_unit_t<STAGES, kCubicMax, true>(b, work, my, cu, pp, t, lane_id);
            else run_unit_t<STAGES, kCubicMax, false>(b, work, my, cu, pp, t, lane_id);
            break;
    }
}

// Step 1 (t = 0) for unit u of swarm w: each lane draws its four particles'
// positions and velocities over all dimensions, scores them, and the unit's
// best key competes for the swarm's gbest. The same arithmetic, in the same
// order, as the single-swarm init kernel.
template <int FIT>
__device__ __forceinline__ void init_unit(const BatchSwarm& wg, uint32_t u, int lane_id) {
    const BatchSwarm w = wg;
    const size_t Np = (size_t)w.Np;
    const float span = __fsub_rn(w.hi, w.lo);
    const float vspan = __fmul_rn(2.0f, w.vmax);
    const uint32_t i0 = u * kUnitB + (uint32_t)lane_id * 4;
    FitAcc<FIT> acc[4];
    for (int d0 = 0; d0 < w.D; d0 += 2) {
        uint4 r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            r[j] = philox4x32_10(make_uint4((uint32_t)(d0 >> 1), i0 + j, 0u, w.swarm), w.key0, w.key1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int d = d0 + h;
            if (h == 1 && d >= w.D) break;
            float4 X, V;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float xj = clampf(__fmaf_rn(u01(word(r[j], 2 * h)), span, w.lo), w.lo, w.hi);
                const float vj = clampf(__fmaf_rn(u01(word(r[j], 2 * h + 1)), vspan, -w.vmax), -w.vmax, w.vmax);
                set_lane(X, j, xj);
                set_lane(V, j, vj);
                acc[j].add(d, xj);
            }
            const size_t off = (size_t)d * Np + i0;
            st4(w.x + off, X);
            st4(w.v + off, V);
            st4(w.pb + off, X);
        }
    }
    float4 PF;
    unsigned long long best = kKeyNone;
    bool nan = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float f = acc[j].finish(w.D);
        set_lane(PF, j, f);
        if (i0 + j < (uint32_t)w.N) {
            const unsigned long long k = pack_key(f, i0 + j);
            best = k < best ? k : best;
            nan |= (f != f);
        }
    }
    st4(w.pf + i0, PF);
    best = warp_min_u64(best);
    const bool any_nan = __any_sync(0xFFFFFFFFu, nan);
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane_id == 0) {
        if (best != kKeyNone) atomicMin(w.gkey + 0, best);
        if (any_nan) atomicOr(w.status, kStatusNaN);
        __threadfence();
        last = atomicAdd(w.done, 1u) == w.nunits - 1u;
        if (last) __threadfence();
    }
    last = __shfl_sync(0xFFFFFFFFu, last, 0);
    if (last) {
        // t = 0 lives in slot 0; slot 1 gets the same key (the step's invariant)
        const unsigned long long k0 = __ldcg(w.gkey + 0);
        const uint32_t g = (uint32_t)(k0 & 0xFFFFFFFFull);
        for (int d = lane_id; d < w.D; d += 32) w.G[d] = __ldcg(w.pb + (size_t)d * Np + g);
        __syncwarp();
        if (lane_id == 0) {
            w.gkey[1] = k0;
            *w.done = 0u;
        }
    }
}

}  // namespace

// One iteration of every swarm of the batch. Iteration t = *t_dev + 1.
// Requires (D + 1) / 2 >= STAGES - 1 for every swarm of the batch.
// MINB: CTAs per SM the register budget is sized for (a tuning choice).
template <int STAGES, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) batch_step_kernel(const __grid_constant__ BatchDev b) {
    extern __shared__ float4 ring_b[];
    const uint32_t t_prev = __ldcg(b.t_dev);
    const uint32_t t = t_prev + 1u;
    unsigned* work = b.work + (t & 1u);
    const int lane_id = threadIdx.x & 31;
    float4* my = ring_b + threadIdx.x;

    Pipe pp;
    Unit cu = fetch(b, work, lane_id);
    pp.have_nxt = false;
    pp.stage = 0;
    // prologue: the first STAGES-1 pairs of the first unit
#pragma unroll
    for (int j = 0; j < STAGES - 1; ++j) issue(b, my, cu, j, j, lane_id);
    pp.ig = STAGES - 1;
    while (cu.sw != 0xFFFFFFFFu) {
        run_unit<STAGES>(b, work, my, cu, pp, t, lane_id);
        if (!pp.have_nxt) {
            pp.nxt = fetch(b, work, lane_id);
        }
        cu = pp.nxt;
        pp.have_nxt = false;
    }
    cp_wait_b<0>();
    // The last CTA rolls the batch forward: next launch counts on the other counter.
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(b.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        b.work[(t + 1u) & 1u] = 0u;
        *b.ticket = 0u;
        *b.t_dev = t;
    }
}

// Step 1 of every swarm: the batch's units dealt to warps round-robin.
__global__ void __launch_bounds__(kBlock) batch_init_kernel(const __grid_constant__ BatchDev b) {
    const int lane_id = threadIdx.x & 31;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    for (unsigned k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < b.nunits; k += nwarps) {
        const uint2 e = __ldg(b.units + k);
        const BatchSwarm& w = b.swarms[e.x];
        switch (w.fid) {
            case kSphere: init_unit<kSphere>(w, e.y, lane_id); break;
            case kRastrigin: init_unit<kRastrigin>(w, e.y, lane_id); break;
            case kAckley: init_unit<kAckley>(w, e.y, lane_id); break;
            case kRosenbrock: init_unit<kRosenbrock>(w, e.y, lane_id); break;
            default: init_unit<kCubicMax>(w, e.y, lane_id); break;   // the host admits nothing else
        }
    }
}

namespace {
template <int STAGES>
size_t batch_smem() {
    return sizeof(float4) * (size_t)STAGES * 6 * kBlock;
}

const void* batch_kernel(int stages, int minb) {
    if (stages == 3 && minb == 2) return (const void*)batch_step_kernel<3, 2>;
    if (stages == 3 && minb == 3) return (const void*)batch_step_kernel<3, 3>;
    if (stages == 4 && minb == 2) return (const void*)batch_step_kernel<4, 2>;
    return nullptr;
}

size_t batch_smem_of(int stages) { return stages == 3 ? batch_smem<3>() : batch_smem<4>(); }
}  // namespace

cudaError_t prepare_batch() {
    const int shapes[3][2] = {{3, 2}, {3, 3}, {4, 2}};
    for (const auto& sh : shapes) {
        cudaError_t e = cudaFuncSetAttribute(batch_kernel(sh[0], sh[1]), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)batch_smem_of(sh[0]));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int batch_blocks_per_sm(int stages, int minb) {
    const void* k = batch_kernel(stages, minb);
    int n = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kBlock, batch_smem_of(stages)) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_batch_init(const BatchDev& b, int grid, cudaStream_t st) {
    if (grid < 1) return cudaErrorInvalidValue;
    batch_init_kernel<<<grid, kBlock, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_batch_step(const BatchDev& b, int stages, int minb, int grid, cudaStream_t st) {
    const void* k = batch_kernel(stages, minb);
    if (!k) return cudaErrorInvalidValue;
    void* args[] = {const_cast<BatchDev*>(&b)};
    return cudaLaunchKernel(k, dim3(grid), dim3(kBlock), args, batch_smem_of(stages), st);
}

}  // namespace cupso
