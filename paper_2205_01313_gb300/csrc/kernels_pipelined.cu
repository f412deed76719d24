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

// Lazy pbest: when particle i improves at iteration t its new pbest_pos is its
// new pos, which this kernel has just written to pos; instead of copying it to
// pbest_pos at once (a re-read of D values long evicted from L2), the kernel
// sets flag i. At iteration t+1 the flagged particle's pbest_pos is the pos it
// reads anyway: it uses that value (pbest - pos = 0 exactly, as with an
// explicit copy) and writes the pbest_pos row from it with full 16-byte
// stores. The arithmetic is unchanged; only when pbest_pos is stored differs.
__device__ __forceinline__ uint32_t flag_bit(uint32_t fl, int j) { return (fl >> (8 * j)) & 1u; }

__device__ __forceinline__ uint32_t load_flags(const SwarmDev& s, uint32_t i0) {
    return __ldcg(reinterpret_cast<const unsigned int*>(s.pflag + i0));
}

// Requires (D + 1) / 2 >= STAGES - 1 (the host falls back to the register
// kernel otherwise), Np a multiple of 128 and s.pflag set.
// FAST selects move_one_fast (requires s.fast_cr and s.fast_clamp).
template <int FIT, int STAGES, bool FAST>
__global__ void __launch_bounds__(kBlock, 3) sync_pipelined_kernel(const __grid_constant__ SwarmDev s) {
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
    uint32_t fl_cur = u_cur < nunits ? load_flags(s, u_cur * kUnit + (uint32_t)lane_id * 4) : 0u;
    uint32_t u_nxt = 0xFFFFFFFFu, fl_nxt = 0u;
#pragma unroll
    for (int j = 0; j < STAGES - 1; ++j) issue_step<STAGES>(s, my, u_cur, j, j, nunits, lane_id);
    int ig = STAGES - 1;  // pair of the next issue, counted from the current unit
    int stage = 0;        // ring stage of the pair being computed

    unsigned long long best = kKeyNone;
    bool nan = false;
    while (u_cur < nunits) {
        const uint32_t i0 = u_cur * kUnit + (uint32_t)lane_id * 4;
        FitAcc<FIT> acc[4];
        float4 PF = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int g = 0; g < npairs; ++g) {
            // keep STAGES-1 pairs in flight: issue the pair STAGES-1 ahead
            {
                int ws = stage + STAGES - 1;
                if (ws >= STAGES) ws -= STAGES;
                if (ig < npairs) {
                    issue_step<STAGES>(s, my, u_cur, ig, ws, nunits, lane_id);
                } else {
                    if (u_nxt == 0xFFFFFFFFu) {
                        u_nxt = fetch_unit(s, lane_id);
                        if (u_nxt < nunits) fl_nxt = load_flags(s, u_nxt * kUnit + (uint32_t)lane_id * 4);
                    }
                    issue_step<STAGES>(s, my, u_nxt, ig - npairs, ws, nunits, lane_id);
                }
                ++ig;
            }
            if (g == npairs - 1) PF = ld4(s.pf + i0);  // needed after the last pair
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
                float4 P = my[(stage * 6 + 4 + h) * kBlock];
                const size_t off = (size_t)d * Np + i0;
                if (fl_cur) {
                    // pbest_pos of a flagged particle is its pos: use it and write it back
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (flag_bit(fl_cur, j)) set_lane(P, j, lane(X, j));
                    st4(s.pb + off, P);
                }
                const float gd = Gs[d];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float xj = lane(X, j), vj = lane(V, j);
                    if constexpr (FAST)
                        move_one_fast(xj, vj, lane(P, j), gd, hi24(word(rr[j], 2 * h)), hi24(word(rr[j], 2 * h + 1)),
                                      s);
                    else
                        move_one(xj, vj, lane(P, j), gd, u01(word(rr[j], 2 * h)), u01(word(rr[j], 2 * h + 1)), s);
                    set_lane(X, j, xj);
                    set_lane(V, j, vj);
                    acc[j].add(d, xj);
                }
                st4(s.x + off, X);
                st4(s.v + off, V);
            }
            if (++stage == STAGES) stage = 0;
        }
        // Step 4 (strict improvement; the new pbest_pos is pos, flagged) and Step 5.
        uint32_t fl_new = 0u;
        float f[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            f[j] = acc[j].finish(D);
            if ((i0 + j) < (uint32_t)s.N && f[j] < lane(PF, j)) {
                fl_new |= 1u << (8 * j);
                set_lane(PF, j, f[j]);
                const unsigned long long k = pack_key(f[j], i0 + j);
                if (k < K && k < best) best = k;
            }
        }
        if (fl_new) st4(s.pf + i0, PF);
        if (fl_new != fl_cur) *reinterpret_cast<unsigned int*>(s.pflag + i0) = fl_new;
        nan |= any_nan4(s, i0, f);
        u_cur = u_nxt;
        fl_cur = fl_nxt;
        u_nxt = 0xFFFFFFFFu;
        fl_nxt = 0u;
        ig -= npairs;
    }
    cp_wait<0>();
    best = warp_min_u64(best);
    if (lane_id == 0 && best < K) atomicMin(s.gkey + nxt, best);
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
    finish_iteration(s, cur, nxt, t);
}

// Writes back every pending pbest_pos row (pbest_pos := pos where flagged) and
// clears the flags, so that kernels without lazy pbest see a complete pb.
__global__ void __launch_bounds__(kBlock) materialize_kernel(const __grid_constant__ SwarmDev s) {
    const uint32_t ngroups = (uint32_t)s.Np / 4;
    const size_t Np = (size_t)s.Np;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < ngroups; q += gridDim.x * blockDim.x) {
        unsigned int* fw = reinterpret_cast<unsigned int*>(s.pflag) + q;
        const uint32_t fl = *fw;
        if (!fl) continue;
        for (int d = 0; d < s.D; ++d) {
            const size_t off = (size_t)d * Np + 4 * (size_t)q;
            const float4 X = ld4(s.x + off);
            float4 P = ld4(s.pb + off);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (flag_bit(fl, j)) set_lane(P, j, lane(X, j));
            st4(s.pb + off, P);
        }
        *fw = 0u;
    }
}

namespace {

template <int STAGES>
size_t pipelined_smem(int D) {
    return sizeof(float4) * (size_t)STAGES * 6 * kBlock + sizeof(float) * (size_t)D;
}

// The kernel instance for (fitness, ring depth, fast path).
template <int STAGES, bool FAST>
const void* kernel_of_t(int fid) {
    switch (fid) {
        case kSphere: return (const void*)sync_pipelined_kernel<kSphere, STAGES, FAST>;
        case kRastrigin: return (const void*)sync_pipelined_kernel<kRastrigin, STAGES, FAST>;
        case kAckley: return (const void*)sync_pipelined_kernel<kAckley, STAGES, FAST>;
        case kRosenbrock: return (const void*)sync_pipelined_kernel<kRosenbrock, STAGES, FAST>;
        case kCubicMax: return (const void*)sync_pipelined_kernel<kCubicMax, STAGES, FAST>;
        default: return nullptr;
    }
}

const void* kernel_of(int stages, bool fast, int fid) {
    if (stages == 3) return fast ? kernel_of_t<3, true>(fid) : kernel_of_t<3, false>(fid);
    return fast ? kernel_of_t<4, true>(fid) : kernel_of_t<4, false>(fid);
}

size_t smem_of(int stages, int D) { return stages == 3 ? pipelined_smem<3>(D) : pipelined_smem<4>(D); }

}  // namespace

bool pipelined_supported(int stages, int D) {
    return (stages == 3 || stages == 4) && (D + 1) / 2 >= stages - 1 && D <= 8192;
}

cudaError_t prepare_pipelined(int D) {
    for (int stages = 3; stages <= 4; ++stages)
        for (int fast = 0; fast < 2; ++fast)
            for (int fid = kSphere; fid <= kCubicMax; ++fid) {
                cudaError_t e = cudaFuncSetAttribute(kernel_of(stages, fast != 0, fid),
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_of(stages, D));
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

int pipelined_blocks_per_sm(int stages, int fid, int D) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel_of(stages, true, fid), kBlock,
                                                      smem_of(stages, D)) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_materialize(const SwarmDev& s, int grid, cudaStream_t st) {
    if (!s.pflag) return cudaSuccess;
    materialize_kernel<<<grid, kBlock, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t launch_sync_pipelined(const SwarmDev& s, int fid, int stages, int grid, cudaStream_t st) {
    if (!pipelined_supported(stages, s.D) || !s.pflag) return cudaErrorInvalidValue;
    const void* k = kernel_of(stages, s.fast_cr && s.fast_clamp, fid);
    if (!k) return cudaErrorInvalidValue;
    void* args[] = {const_cast<SwarmDev*>(&s)};
    return cudaLaunchKernel(k, dim3(grid), dim3(kBlock), args, smem_of(stages, s.D), st);
}

}  // namespace cupso
