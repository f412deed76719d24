// kernels_pipelined.cu -- the fused synchronous iteration with its HBM reads
// staged through shared memory ahead of use.
//
// Same arithmetic and the same aggregation as sync_step_kernel (Steps 2-5 in
// one launch; conditional warp argmin + one 64-bit atomicMin; last CTA gathers
// gbest_pos), organised for bandwidth:
//  * each thread copies its own float4 of pos, v and pbest_pos rows into a
//    private slot ring in shared memory with cp.async, STAGES-1 dimension
//    pairs ahead of the pair it computes on, so the bytes in flight per SM no
//    longer depend on how many registers hold loaded values (the structure-of-
//    arrays rows of Sec. 4.1 stay fully coalesced: a warp copies 512 B of one
//    row per instruction);
//  * no thread reads another thread's slots, so the ring needs no barrier;
//  * warps take 128-particle units from a counter, so work is balanced
//    across SMs to within one unit instead of one 1024-particle tile.
#include <cuda_runtime.h>

#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "stream_common.cuh"

namespace cupso {

namespace {

constexpr int kUnit = 128;  // particles per warp unit: 32 lanes x float4

__device__ __forceinline__ void cp_async16(float4* smem, const float* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint32_t fetch_unit(const SwarmDev& s, int lane_id) {
    uint32_t u = 0;
    if (lane_id == 0) u = atomicAdd(s.work, 1u);
    return __shfl_sync(0xFFFFFFFFu, u, 0);
}

// Copies of one step (unit u, dimension pair g) into ring stage `stage`:
// rows 2g and 2g+1 of pos, v and pbest_pos, one float4 per lane per row.
// Slot (stage, a, r) of this thread is my[(stage * 6 + 2 * a + r) * kBlock].
template <int STAGES>
__device__ __forceinline__ void issue_step(const SwarmDev& s, float4* my, uint32_t u, int g, int stage,
                                           uint32_t nunits, int lane_id) {
    if (u < nunits) {
        const size_t col = (size_t)u * kUnit + (size_t)lane_id * 4;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int d = 2 * g + r;
            if (d < s.D) {
                const size_t off = (size_t)d * (size_t)s.Np + col;
                cp_async16(my + (stage * 6 + 0 + r) * kBlock, s.x + off);
                cp_async16(my + (stage * 6 + 2 + r) * kBlock, s.v + off);
                cp_async16(my + (stage * 6 + 4 + r) * kBlock, s.pb + off);
            }
        }
    }
    cp_commit();  // an empty group when there is nothing left to copy
}

}  // namespace

// Requires (D + 1) / 2 >= STAGES - 1 (the host falls back to the register
// kernel otherwise) and Np a multiple of 128.
template <int FIT, int STAGES>
__global__ void __launch_bounds__(kBlock) sync_pipelined_kernel(const __grid_constant__ SwarmDev s) {
    extern __shared__ float4 ring[];  // [STAGES][6][kBlock] float4, then gbest_pos [D]
    float* Gs = reinterpret_cast<float*>(ring + STAGES * 6 * kBlock);
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    const uint32_t t = t_prev + 1u;
    const unsigned long long K = __ldcg(s.gkey + cur);  // gbest at the end of t-1
    for (int d = threadIdx.x; d < s.D; d += blockDim.x) Gs[d] = __ldcg(s.G + (size_t)cur * s.D + d);
    __syncthreads();

    const int lane_id = threadIdx.x & 31;
    const int D = s.D, npairs = (D + 1) >> 1;
    const uint32_t nunits = (uint32_t)s.Np / kUnit;
    const size_t Np = (size_t)s.Np;
    float4* my = ring + threadIdx.x;

    uint32_t u_cur = fetch_unit(s, lane_id);
    uint32_t u_nxt = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < STAGES - 1; ++j) issue_step<STAGES>(s, my, u_cur, j, j, nunits, lane_id);
    int ig = STAGES - 1;  // pair of the next issue, counted from the current unit
    int stage = 0;        // ring stage of the pair being computed

    unsigned long long best = kKeyNone;
    bool nan = false;
    while (u_cur < nunits) {
        const uint32_t i0 = u_cur * kUnit + (uint32_t)lane_id * 4;
        FitAcc<FIT> acc[4];
        for (int g = 0; g < npairs; ++g) {
            // keep STAGES-1 pairs in flight: issue the pair STAGES-1 ahead
            {
                int ws = stage + STAGES - 1;
                if (ws >= STAGES) ws -= STAGES;
                if (ig < npairs) {
                    issue_step<STAGES>(s, my, u_cur, ig, ws, nunits, lane_id);
                } else {
                    if (u_nxt == 0xFFFFFFFFu) u_nxt = fetch_unit(s, lane_id);
                    issue_step<STAGES>(s, my, u_nxt, ig - npairs, ws, nunits, lane_id);
                }
                ++ig;
            }
            cp_wait<STAGES - 1>();  // this thread's copies of the current pair have landed
            const uint4 rr[4] = {
                philox4x32_10(make_uint4((uint32_t)g, i0 + 0, t, s.swarm), s.key0, s.key1),
                philox4x32_10(make_uint4((uint32_t)g, i0 + 1, t, s.swarm), s.key0, s.key1),
                philox4x32_10(make_uint4((uint32_t)g, i0 + 2, t, s.swarm), s.key0, s.key1),
                philox4x32_10(make_uint4((uint32_t)g, i0 + 3, t, s.swarm), s.key0, s.key1)};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int d = 2 * g + h;
                if (h == 1 && d >= D) break;
                float4 X = my[(stage * 6 + 0 + h) * kBlock];
                float4 V = my[(stage * 6 + 2 + h) * kBlock];
                const float4 P = my[(stage * 6 + 4 + h) * kBlock];
                const float gd = Gs[d];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float xj = lane(X, j), vj = lane(V, j);
                    move_one(xj, vj, lane(P, j), gd, u01(word(rr[j], 2 * h)), u01(word(rr[j], 2 * h + 1)), s);
                    set_lane(X, j, xj);
                    set_lane(V, j, vj);
                    acc[j].add(d, xj);
                }
                const size_t off = (size_t)d * Np + i0;
                st4(s.x + off, X);
                st4(s.v + off, V);
            }
            if (++stage == STAGES) stage = 0;
        }
        // Steps 4 and 5 for the unit's particles.
        float f[4], pf[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) f[j] = acc[j].finish(D);
        const unsigned mask = pbest4(s, i0, f, pf);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (mask & (1u << j)) {
                const unsigned long long k = pack_key(f[j], i0 + j);
                if (k < K && k < best) best = k;
            }
        }
        nan |= any_nan4(s, i0, f);
        u_cur = u_nxt;
        u_nxt = 0xFFFFFFFFu;
        ig -= npairs;
    }
    cp_wait<0>();
    best = warp_min_u64(best);
    if (lane_id == 0 && best < K) atomicMin(s.gkey + nxt, best);
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
    finish_iteration(s, cur, nxt, t);
}

namespace {

template <int STAGES>
size_t pipelined_smem(int D) {
    return sizeof(float4) * (size_t)STAGES * 6 * kBlock + sizeof(float) * (size_t)D;
}

template <int STAGES>
cudaError_t launch_pipelined_t(const SwarmDev& s, int fid, int grid, cudaStream_t st) {
    const size_t smem = pipelined_smem<STAGES>(s.D);
    switch (fid) {
        case kSphere: sync_pipelined_kernel<kSphere, STAGES><<<grid, kBlock, smem, st>>>(s); break;
        case kRastrigin: sync_pipelined_kernel<kRastrigin, STAGES><<<grid, kBlock, smem, st>>>(s); break;
        case kAckley: sync_pipelined_kernel<kAckley, STAGES><<<grid, kBlock, smem, st>>>(s); break;
        case kRosenbrock: sync_pipelined_kernel<kRosenbrock, STAGES><<<grid, kBlock, smem, st>>>(s); break;
        case kCubicMax: sync_pipelined_kernel<kCubicMax, STAGES><<<grid, kBlock, smem, st>>>(s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int STAGES, typename F>
cudaError_t for_each_fit(F f) {
    cudaError_t e = f(sync_pipelined_kernel<kSphere, STAGES>);
    if (e == cudaSuccess) e = f(sync_pipelined_kernel<kRastrigin, STAGES>);
    if (e == cudaSuccess) e = f(sync_pipelined_kernel<kAckley, STAGES>);
    if (e == cudaSuccess) e = f(sync_pipelined_kernel<kRosenbrock, STAGES>);
    if (e == cudaSuccess) e = f(sync_pipelined_kernel<kCubicMax, STAGES>);
    return e;
}

template <int STAGES>
void* kernel_of(int fid) {
    switch (fid) {
        case kSphere: return (void*)sync_pipelined_kernel<kSphere, STAGES>;
        case kRastrigin: return (void*)sync_pipelined_kernel<kRastrigin, STAGES>;
        case kAckley: return (void*)sync_pipelined_kernel<kAckley, STAGES>;
        case kRosenbrock: return (void*)sync_pipelined_kernel<kRosenbrock, STAGES>;
        default: return (void*)sync_pipelined_kernel<kCubicMax, STAGES>;
    }
}

}  // namespace

bool pipelined_supported(int stages, int D) {
    return (stages == 3 || stages == 4) && (D + 1) / 2 >= stages - 1 && D <= 8192;
}

cudaError_t prepare_pipelined(int D) {
    cudaError_t e = for_each_fit<3>([&](auto k) {
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pipelined_smem<3>(D));
    });
    if (e != cudaSuccess) return e;
    return for_each_fit<4>([&](auto k) {
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pipelined_smem<4>(D));
    });
}

int pipelined_blocks_per_sm(int stages, int fid, int D) {
    int n = 0;
    const void* k = stages == 3 ? kernel_of<3>(fid) : kernel_of<4>(fid);
    const size_t smem = stages == 3 ? pipelined_smem<3>(D) : pipelined_smem<4>(D);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kBlock, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_sync_pipelined(const SwarmDev& s, int fid, int stages, int grid, cudaStream_t st) {
    if (!pipelined_supported(stages, s.D)) return cudaErrorInvalidValue;
    return stages == 3 ? launch_pipelined_t<3>(s, fid, grid, st) : launch_pipelined_t<4>(s, fid, grid, st);
}

}  // namespace cupso
