// kernels_panel.cu -- the fused synchronous iteration on the panel layout.
//
// The panel layout keeps the structure of arrays of Sec. 4.1 (one array per
// quantity, particles side by side) but groups dimensions by eight:
//   element (d, i) of pos, v, pbest_pos is at ((d / 8) * Np + i) * 8 + d % 8,
// so the eight values of one particle in one panel fill one 32-byte DRAM
// sector, and the 32 particles of a warp read 1 KB contiguous per panel.
//
// What that buys is the pbest write at particle granularity. With lazy pbest
// (a particle that improved in iteration t-1 has pbest_pos == pos, and its row
// is written during iteration t), a flagged particle's pbest_pos need not be
// read at all: its sectors are written from the pos just loaded instead. Every
// particle therefore moves exactly 20 bytes per dimension per iteration (read
// pos and v, read pbest_pos or write it, write pos and v), whatever fraction of
// the swarm improves. In the dimension-major layout eight particles share a
// sector of each row, so one improving particle among them costs a full
// sector write on top of the read, and early iterations -- where half the
// swarm improves -- move about a sixth more bytes.
//
// The arithmetic is unchanged: Eq. 1, Eq. 2 and the fitness terms in the
// oracle's order over d, with the same random words (counter (d >> 1, i, t,
// swarm)). Steps 4-5 are those of the other fused kernels: strict pbest, a
// conditional warp argmin and one 64-bit atomicMin on the packed key, and the
// last CTA gathers gbest_pos.
//
// Two lanes share a particle: lane 2p + h owns the half panel of dimensions
// 8q + 4h .. 8q + 4h + 3 of particle p of its warp's unit (16 particles), so
// the 32 lanes of a warp read and write 512 contiguous bytes per instruction,
// as with one float4 per lane in the dimension-major kernel. The fitness terms
// of a half panel (cos(2 pi x) included) are computed in both lanes at once;
// only their summation, which keeps the oracle's order over d, alternates
// between the two lanes, the running sum passed by a shuffle. Loads are staged
// through a per-thread cp.async ring of STAGES half panels (pos, v and
// pbest_pos: three 16-byte slots each), STAGES - 1 ahead of the one computed;
// warps take units of 16 particles from a counter.
#include <cuda_runtime.h>

#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "stream_common.cuh"

namespace cupso {

namespace {

__device__ __forceinline__ void cp16(float4* smem, const float* gmem) {
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

constexpr uint32_t kUnitP = 16;   // particles per warp unit (two lanes each)

// Offset of particle i's panel q.
__device__ __forceinline__ size_t panel_off(const SwarmDev& s, int q, uint32_t i) {
    return ((size_t)q * (size_t)s.Np + (size_t)i) * 8;
}

// Copies of panel q of unit u into ring stage `stage`: this lane's half of its
// particle's panel of pos and v, and of pbest_pos unless the particle's row is
// pending (then pbest_pos is the pos being loaded). Slot (stage, k) of this
// thread is my[(stage * 3 + k) * kBlock]: k = 0 pos, 1 v, 2 pbest_pos.
__device__ __forceinline__ void issue_panel(const SwarmDev& s, float4* my, uint32_t u, int q, int stage,
                                            uint32_t nunits, int lane_id, uint32_t pending) {
    if (u < nunits) {
        const size_t off = panel_off(s, q, u * kUnitP + (uint32_t)(lane_id >> 1)) + 4 * (lane_id & 1);
        float4* slot = my + (size_t)stage * 3 * kBlock;
        cp16(slot, s.x + off);
        cp16(slot + kBlock, s.v + off);
        if (!pending) cp16(slot + 2 * kBlock, s.pb + off);
    }
    cp_commit();  // an empty group when there is nothing left to copy
}

// The running fitness state of lane `src`, for the fields the function uses.
template <int FIT>
__device__ __forceinline__ void pull(FitAcc<FIT>& a, int src) {
    a.acc = __shfl_sync(0xFFFFFFFFu, a.acc, src);
    if constexpr (FIT == kAckley) a.acc2 = __shfl_sync(0xFFFFFFFFu, a.acc2, src);
    if constexpr (FIT == kRosenbrock) a.prev = __shfl_sync(0xFFFFFFFFu, a.prev, src);
}

// Adds the four fitness terms of this lane's half panel (dimensions d0 ..
// d0 + 3) in the oracle's order: the even lane of a pair continues the sum its
// odd partner ended the previous panel with, then the odd lane continues the
// even one's. Afterwards the odd lane holds the sum up to d0 + 3 of its half.
template <int FIT>
__device__ __forceinline__ void panel_sum(FitAcc<FIT>& a, const float4& X, int d0, int h, int lane_id) {
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if constexpr (FitAcc<FIT>::kNeedsCos) {
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = cos2pi(lane(X, k));
    }
    pull(a, lane_id | 1);
    if (h == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) a.add_c(d0 + k, lane(X, k), c[k]);
    }
    pull(a, lane_id & ~1);
    if (h == 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) a.add_c(d0 + k, lane(X, k), c[k]);
    }
}

// Last-CTA-done epilogue on the panel layout: gbest_pos from the winner's
// pbest_pos (or from pos when its row is still pending).
__device__ __forceinline__ void finish_iteration_panel(const SwarmDev& s, int cur, int nxt, uint32_t t_new) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(s.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const unsigned long long knew = __ldcg(s.gkey + nxt);
    const uint32_t g = (uint32_t)(knew & 0xFFFFFFFFull);
    if (g < (uint32_t)s.N) {
        const bool lazy = __ldcg(s.pflag + g) != 0;
        const float* src = lazy ? s.x : s.pb;
        for (int d = threadIdx.x; d < s.D; d += blockDim.x)
            s.G[(size_t)nxt * s.D + d] = __ldcg(src + panel_off(s, d >> 3, g) + (d & 7));
    }
    if (threadIdx.x == 0) {
        s.gkey[cur] = knew;
        *s.t_dev = t_new;
        *s.ticket = 0u;
        *s.work = 0u;
    }
}

}  // namespace

// Requires D % 8 == 0, D / 8 >= STAGES - 1, Np a multiple of 128 and s.pflag,
// s.work set (work zero at launch). FAST selects move_one_fast (requires
// s.fast_cr and s.fast_clamp).
template <int FIT, int STAGES, bool FAST>
__global__ void __launch_bounds__(kBlock, 3) sync_panel_kernel(const __grid_constant__ SwarmDev s) {
    extern __shared__ float4 ring[];  // [STAGES][3][kBlock], then gbest_pos [D]
    float* Gs = reinterpret_cast<float*>(ring + STAGES * 3 * kBlock);
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    const uint32_t t = t_prev + 1u;
    const unsigned long long K = __ldcg(s.gkey + cur);  // gbest at the end of t-1
    for (int d = threadIdx.x; d < s.D; d += blockDim.x) Gs[d] = __ldcg(s.G + (size_t)cur * s.D + d);
    __syncthreads();

    const int lane_id = threadIdx.x & 31, h = lane_id & 1;
    const uint32_t pl = (uint32_t)(lane_id >> 1);
    const int D = s.D, Dq = D >> 3;
    const uint32_t nunits = (uint32_t)s.Np / kUnitP;
    float4* my = ring + threadIdx.x;
    constexpr uint32_t kNone = 0xFFFFFFFFu;

    uint32_t u_cur = fetch_unit(s, lane_id);
    uint32_t fl_cur = u_cur < nunits ? (uint32_t)__ldcg(s.pflag + u_cur * kUnitP + pl) : 0u;
    uint32_t u_nxt = kNone, fl_nxt = 0u;
#pragma unroll
    for (int j = 0; j < STAGES - 1; ++j) issue_panel(s, my, u_cur, j, j, nunits, lane_id, fl_cur);
    int iq = STAGES - 1;  // panel of the next issue, counted from the current unit
    int stage = 0;        // ring stage of the panel being computed

    unsigned long long best = kKeyNone;
    bool nan = false;
    while (u_cur < nunits) {
        const uint32_t i = u_cur * kUnitP + pl;
        FitAcc<FIT> acc;
        float pf = 0.0f;
        for (int q = 0; q < Dq; ++q) {
            // keep STAGES-1 panels in flight: issue the panel STAGES-1 ahead
            {
                int ws = stage + STAGES - 1;
                if (ws >= STAGES) ws -= STAGES;
                if (iq < Dq) {
                    issue_panel(s, my, u_cur, iq, ws, nunits, lane_id, fl_cur);
                } else {
                    if (u_nxt == kNone) {
                        u_nxt = fetch_unit(s, lane_id);
                        if (u_nxt < nunits) fl_nxt = (uint32_t)__ldcg(s.pflag + u_nxt * kUnitP + pl);
                    }
                    issue_panel(s, my, u_nxt, iq - Dq, ws, nunits, lane_id, fl_nxt);
                }
                ++iq;
            }
            if (q == Dq - 1 && h == 1) pf = __ldcg(s.pf + i);  // needed after the last panel
            cp_wait<STAGES - 1>();  // this thread's copies of the current panel have landed
            const float4* slot = my + (size_t)stage * 3 * kBlock;
            float4 X = slot[0], V = slot[kBlock];
            float4 Pb;
            const int d0 = 8 * q + 4 * h;
            const size_t off = panel_off(s, q, i) + 4 * h;
            if (fl_cur) {
                // pbest_pos of a flagged particle is its pos: use it and write the row back
                Pb = X;
                st4(s.pb + off, X);
            } else {
                Pb = slot[2 * kBlock];
            }
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const uint4 r = philox4x32_10(make_uint4((uint32_t)((d0 >> 1) + g), i, t, s.swarm), s.key0, s.key1);
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int k = 2 * g + hh;
                    float xj = lane(X, k), vj = lane(V, k);
                    if constexpr (FAST)
                        move_one_fast(xj, vj, lane(Pb, k), Gs[d0 + k], hi24(word(r, 2 * hh)),
                                      hi24(word(r, 2 * hh + 1)), s);
                    else
                        move_one(xj, vj, lane(Pb, k), Gs[d0 + k], u01(word(r, 2 * hh)), u01(word(r, 2 * hh + 1)),
                                 s);
                    set_lane(X, k, xj);
                    set_lane(V, k, vj);
                }
            }
            st4(s.x + off, X);
            st4(s.v + off, V);
            panel_sum<FIT>(acc, X, d0, h, lane_id);
            if (++stage == STAGES) stage = 0;
        }
        // Step 4 (strict improvement; the new pbest_pos is pos, flagged) and
        // Step 5, in the odd lane of each pair, which holds the whole sum.
        if (h == 1) {
            const float f = acc.finish(D);
            const bool real = i < (uint32_t)s.N;
            nan |= real && (f != f);
            uint32_t fl_new = 0u;
            if (real && f < pf) {
                fl_new = 1u;
                s.pf[i] = f;
                const unsigned long long k = pack_key(f, i);
                if (k < K && k < best) best = k;
            }
            if (fl_new != fl_cur) s.pflag[i] = (unsigned char)fl_new;
        }
        u_cur = u_nxt;
        fl_cur = fl_nxt;
        u_nxt = kNone;
        fl_nxt = 0u;
        iq -= Dq;
    }
    cp_wait<0>();
    best = warp_min_u64(best);
    if (lane_id == 0 && best < K) atomicMin(s.gkey + nxt, best);
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
    finish_iteration_panel(s, cur, nxt, t);
}

// Writes back every pending pbest_pos row on the panel layout (pbest_pos :=
// pos where flagged) and clears the flags.
__global__ void __launch_bounds__(kBlock) materialize_panel_kernel(const __grid_constant__ SwarmDev s) {
    const int Dq = s.D >> 3;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (uint32_t)s.Np; i += gridDim.x * blockDim.x) {
        if (!s.pflag[i]) continue;
        for (int q = 0; q < Dq; ++q) {
            const size_t off = panel_off(s, q, i);
            st4(s.pb + off, ld4(s.x + off));
            st4(s.pb + off + 4, ld4(s.x + off + 4));
        }
        s.pflag[i] = 0;
    }
}

// dst = src converted between the dimension-major layout (d * Np + i) and the
// panel layout; one thread per (panel, particle), both sides coalesced.
__global__ void __launch_bounds__(kBlock) relayout_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                          int D, int Np, int to_panel) {
    const size_t items = (size_t)(D >> 3) * (size_t)Np;
    for (size_t it = (size_t)blockIdx.x * blockDim.x + threadIdx.x; it < items; it += (size_t)gridDim.x * blockDim.x) {
        const size_t q = it / (size_t)Np, i = it % (size_t)Np;
        const size_t poff = it * 8;   // (q * Np + i) * 8
        if (to_panel) {
            float v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = src[(q * 8 + k) * (size_t)Np + i];
            st4(dst + poff, make_float4(v[0], v[1], v[2], v[3]));
            st4(dst + poff + 4, make_float4(v[4], v[5], v[6], v[7]));
        } else {
            const float4 a = ld4(src + poff), b = ld4(src + poff + 4);
            const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) dst[(q * 8 + k) * (size_t)Np + i] = v[k];
        }
    }
}

namespace {

size_t panel_smem(int stages, int D) {
    return sizeof(float4) * (size_t)stages * 3 * kBlock + sizeof(float) * (size_t)D;
}

template <int STAGES, bool FAST>
const void* panel_kernel_t(int fid) {
    switch (fid) {
        case kSphere: return (const void*)sync_panel_kernel<kSphere, STAGES, FAST>;
        case kRastrigin: return (const void*)sync_panel_kernel<kRastrigin, STAGES, FAST>;
        case kAckley: return (const void*)sync_panel_kernel<kAckley, STAGES, FAST>;
        case kRosenbrock: return (const void*)sync_panel_kernel<kRosenbrock, STAGES, FAST>;
        case kCubicMax: return (const void*)sync_panel_kernel<kCubicMax, STAGES, FAST>;
        default: return nullptr;
    }
}

const void* panel_kernel(int stages, bool fast, int fid) {
    if (stages == 3) return fast ? panel_kernel_t<3, true>(fid) : panel_kernel_t<3, false>(fid);
    return fast ? panel_kernel_t<6, true>(fid) : panel_kernel_t<6, false>(fid);
}

}  // namespace

bool panel_supported(int stages, int D) {
    return (stages == 3 || stages == 6) && D % 8 == 0 && D / 8 >= stages - 1 && D <= 8192;
}

cudaError_t prepare_panel(int D) {
    for (int stages = 3; stages <= 6; stages += 3)
        for (int fast = 0; fast < 2; ++fast)
            for (int fid = kSphere; fid <= kCubicMax; ++fid) {
                cudaError_t e = cudaFuncSetAttribute(panel_kernel(stages, fast != 0, fid),
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)panel_smem(stages, D));
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

int panel_blocks_per_sm(int stages, int fid, int D) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, panel_kernel(stages, true, fid), kBlock,
                                                      panel_smem(stages, D)) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_sync_panel(const SwarmDev& s, int fid, int stages, int grid, cudaStream_t st) {
    if (!panel_supported(stages, s.D) || !s.pflag || !s.work || s.Np % 128 != 0) return cudaErrorInvalidValue;
    const void* k = panel_kernel(stages, s.fast_cr && s.fast_clamp, fid);
    if (!k) return cudaErrorInvalidValue;
    void* args[] = {const_cast<SwarmDev*>(&s)};
    return cudaLaunchKernel(k, dim3(grid), dim3(kBlock), args, panel_smem(stages, s.D), st);
}

cudaError_t launch_materialize_panel(const SwarmDev& s, int grid, cudaStream_t st) {
    if (!s.pflag || s.D % 8 != 0) return cudaErrorInvalidValue;
    materialize_panel_kernel<<<grid, kBlock, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t launch_relayout(const float* src, float* dst, int D, int Np, bool to_panel, int grid, cudaStream_t st) {
    if (D % 8 != 0) return cudaErrorInvalidValue;
    relayout_kernel<<<grid, kBlock, 0, st>>>(src, dst, D, Np, to_panel ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace cupso
