// kernels_panel.cu -- the fused synchronous iteration on the panel layout.
//
// The panel layout keeps the structure of arrays of Sec. 4.1 (one array per
// quantity, particles side by side) but groups dimensions by W (8 or 16):
//   element (d, i) of pos, v, pbest_pos is at ((d / W) * Np + i) * W + d % W,
// so the W values of one particle in one panel are contiguous: one 32-byte
// DRAM sector for W = 8, the 64 bytes a GB300 reads from HBM at a time for
// W = 16 (measured: with W = 8, a pbest row skipped for one particle of a
// 64-byte pair was read anyway).
//
// What that buys is the pbest write at particle granularity. With lazy pbest
// (a particle that improved in iteration t-1 has pbest_pos == pos, and its row
// is written during iteration t), a flagged particle's pbest_pos need not be
// read at all: its panels are written from the pos just loaded instead. Every
// particle therefore moves 20 bytes per dimension per iteration (read pos and
// v, read pbest_pos or write it, write pos and v), whatever fraction of the
// swarm improves. In the dimension-major layout eight particles share a sector
// of each row, so one improving particle among them costs a full sector write
// on top of the read, and early iterations -- where half the swarm improves --
// move about a sixth more bytes.
//
// The arithmetic is unchanged: Eq. 1, Eq. 2 and the fitness terms in the
// oracle's order over d, with the same random words (counter (d >> 1, i, t,
// swarm)). Steps 4-5 are those of the other fused kernels: strict pbest, a
// conditional warp argmin and one 64-bit atomicMin on the packed key, and the
// last CTA gathers gbest_pos.
//
// L = W / 4 lanes share a particle: lane L p + j owns dimensions W q + 4 j ..
// W q + 4 j + 3 of particle p of its warp's unit (32 / L particles), so the
// 32 lanes of a warp read and write 512 contiguous bytes per instruction, as
// with one float4 per lane in the dimension-major kernel (with one lane per
// particle, every 16-byte access hit a 32-byte stride and the kernel ran 30%
// slower). The fitness terms of a lane's four dimensions (cos(2 pi x)
// included) are computed in all lanes at once; only their summation, which
// keeps the oracle's order over d, passes from lane to lane of the particle,
// the running sum carried by a shuffle. Loads are staged through a per-thread
// cp.async ring of STAGES panels (pos, v and pbest_pos: three 16-byte slots
// each), STAGES - 1 ahead of the one computed; warps take units from a counter
// (two at a time when the swarm has many per warp).
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

// Offset of particle i's panel q in a layout of width W.
template <int W>
__device__ __forceinline__ size_t panel_off(const SwarmDev& s, int q, uint32_t i) {
    return ((size_t)q * (size_t)s.Np + (size_t)i) * W;
}

// Hands out the units after the warps' own first ones (units base, base + 1,
// ...; base = the number of warps). For a swarm with many units per warp, one
// counter increment per two units (fewer atomics on one address) until the
// last two units per warp, which go out one at a time: an iteration lasts as
// long as the warp with the most work, and a two-unit grain at the end would
// double that excess. A swarm with few units per warp gets single units only.
struct UnitFeed {
    uint32_t spare = 0xFFFFFFFFu;   // the second unit of the last fetch, if not yet taken
    uint32_t base;
    uint32_t npairs;                // fetches 0 .. npairs - 1 hand out two units
    __device__ __forceinline__ UnitFeed(uint32_t nunits, uint32_t nwarps) : base(nwarps), npairs(0u) {
        if (nunits >= 8u * nwarps) {
            const uint32_t dyn = nunits - nwarps, tail = 2u * nwarps;
            npairs = (dyn - tail) / 2u;
        }
    }
    __device__ __forceinline__ uint32_t next(const SwarmDev& s, int lane_id) {
        if (spare != 0xFFFFFFFFu) {
            const uint32_t u = spare;
            spare = 0xFFFFFFFFu;
            return u;
        }
        uint32_t k = 0;
        if (lane_id == 0) k = atomicAdd(s.work, 1u);
        k = __shfl_sync(0xFFFFFFFFu, k, 0);
        if (k >= npairs) return base + npairs + k;   // single units after the pairs: 2 npairs + (k - npairs)
        spare = base + 2u * k + 1u;
        return base + 2u * k;
    }
};

// Copies of panel q of unit u into ring stage `stage`: this lane's four values
// of its particle's panel of pos and v, and of pbest_pos unless the particle's
// row is pending (then pbest_pos is the pos being loaded). Slot (stage, k) of
// this thread is my[(stage * 3 + k) * kBlock]: k = 0 pos, 1 v, 2 pbest_pos.
template <int W>
__device__ __forceinline__ void issue_panel(const SwarmDev& s, float4* my, uint32_t u, int q, int stage,
                                            uint32_t nunits, int lane_id, uint32_t pending) {
    constexpr int L = W / 4;
    constexpr uint32_t PU = 32 / L;
    if (u < nunits) {
        const size_t off = panel_off<W>(s, q, u * PU + (uint32_t)(lane_id / L)) + 4 * (lane_id % L);
        float4* slot = my + (size_t)stage * 3 * kBlock;
        cp16(slot, s.x + off);
        cp16(slot + kBlock, s.v + off);
        if (!pending) cp16(slot + 2 * kBlock, s.pb + off);
    }
    cp_commit();  // an empty group when there is nothing left to copy
}

// The running fitness sums of lane `src`.
template <int FIT>
__device__ __forceinline__ void pull(FitAcc<FIT>& a, int src) {
    a.acc = __shfl_sync(0xFFFFFFFFu, a.acc, src);
    if constexpr (FIT == kAckley) a.acc2 = __shfl_sync(0xFFFFFFFFu, a.acc2, src);
}

// Adds the fitness terms of this lane's four dimensions (d0 .. d0 + 3) in the
// oracle's order. The terms themselves do not depend on the running sum
// (Rastrigin's x^2 - 10 cos 2 pi x + 10, Rosenbrock's 100 (x_{d+1} - x_d^2)^2 +
// (1 - x_d)^2, the cubic's Horner value), so every lane computes its own at
// once; only their folding into the sum, which keeps the order over d, passes
// from lane to lane of the particle: in phase k the particle's lane k continues
// the sum of lane k - 1 (lane 0 that of lane L - 1, which ended the previous
// panel). Sphere and Ackley fold x with an fma, as the oracle does. After the
// last phase, lane L - 1 of the particle holds the sum through its panel.
// `carry` is x_{d0 - 1} for the particle's lane 0 (the last value of the
// previous panel), updated here to this panel's last value.
template <int FIT, int L>
__device__ __forceinline__ void panel_sum(FitAcc<FIT>& a, const float4& X, int d0, int j, int lane_id, float& carry) {
    const float x[4] = {X.x, X.y, X.z, X.w};
    float t[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const int base = lane_id - j;
    if constexpr (FIT == kRastrigin) {
#pragma unroll
        for (int k = 0; k < 4; ++k) t[k] = __fmaf_rn(x[k], x[k], __fmaf_rn(-10.0f, cos2pi(x[k]), 10.0f));
    } else if constexpr (FIT == kAckley) {
#pragma unroll
        for (int k = 0; k < 4; ++k) t[k] = cos2pi(x[k]);
    } else if constexpr (FIT == kCubicMax) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            t[k] = __fmaf_rn(__fmaf_rn(__fsub_rn(x[k], 0.8f), x[k], -1000.0f), x[k], 8000.0f);
    } else if constexpr (FIT == kRosenbrock) {
        // term of dimension d (d >= 1) from x_{d-1} and x_d
        const float from_left = __shfl_sync(0xFFFFFFFFu, X.w, lane_id - 1 < base ? lane_id : lane_id - 1);
        float prev = j == 0 ? carry : from_left;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float pp = __fmaf_rn(-prev, prev, x[k]);
            const float qq = __fsub_rn(1.0f, prev);
            t[k] = __fmaf_rn(__fmul_rn(100.0f, pp), pp, __fmul_rn(qq, qq));
            prev = x[k];
        }
        carry = __shfl_sync(0xFFFFFFFFu, X.w, base + L - 1);
    }
#pragma unroll
    for (int ph = 0; ph < L; ++ph) {
        pull(a, base + (ph + L - 1) % L);
        if (j == ph) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if constexpr (FIT == kSphere) {
                    a.acc = __fmaf_rn(x[k], x[k], a.acc);
                } else if constexpr (FIT == kAckley) {
                    a.acc = __fmaf_rn(x[k], x[k], a.acc);
                    a.acc2 = __fadd_rn(a.acc2, t[k]);
                } else if constexpr (FIT == kRosenbrock) {
                    if (d0 + k > 0) a.acc = __fadd_rn(a.acc, t[k]);
                } else {
                    a.acc = __fadd_rn(a.acc, t[k]);
                }
            }
        }
    }
}

// gbest_pos of iteration parity nxt from the winner's pbest_pos, or from pos
// when its row is still pending -- exactly when the key improved in this
// iteration (K: the key it started from): the winner then improved its own
// pbest, and a gbest particle that did not improve has had its row written
// in this iteration. Run by the last CTA of an iteration.
template <int W>
__device__ __forceinline__ void gather_gbest_panel(const SwarmDev& s, int nxt, unsigned long long K) {
    const unsigned long long knew = __ldcg(s.gkey + nxt);
    const uint32_t g = (uint32_t)(knew & 0xFFFFFFFFull);
    if (g < (uint32_t)s.N) {
        const float* src = knew < K ? s.x : s.pb;
        for (int d = threadIdx.x; d < s.D; d += blockDim.x)
            s.G[(size_t)nxt * s.D + d] = __ldcg(src + panel_off<W>(s, d / W, g) + (d % W));
    }
}

__device__ __forceinline__ unsigned int ld_acquire_gpu_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// One iteration of a warp's units: first u_cur, whose first STAGES - 1 panels
// the ring already holds (fl_cur: its particles' pending flags), then those
// the feed hands out. Returns the lane's Step-5 candidate (a key below K, or
// none); the ring is empty on return.
template <int FIT, int W, int STAGES, bool FAST>
__device__ __forceinline__ unsigned long long panel_units(const SwarmDev& s, float4* my, const float* Gs,
                                                          UnitFeed& feed, uint32_t u_cur, uint32_t fl_cur,
                                                          uint32_t nunits, uint32_t t, unsigned long long K,
                                                          bool& nan) {
    constexpr int L = W / 4;              // lanes per particle
    constexpr uint32_t PU = 32 / L;       // particles per warp unit
    constexpr uint32_t kNone = 0xFFFFFFFFu;
    const int lane_id = threadIdx.x & 31, j = lane_id % L;
    const uint32_t pl = (uint32_t)(lane_id / L);
    const int D = s.D, Dq = D / W;
    uint32_t u_nxt = kNone, fl_nxt = 0u;
    int iq = STAGES - 1;  // panel of the next issue, counted from the current unit
    int stage = 0;        // ring stage of the panel being computed
    unsigned long long best = kKeyNone;
    while (u_cur < nunits) {
        const uint32_t i = u_cur * PU + pl;
        FitAcc<FIT> acc;
        float carry = 0.0f;   // Rosenbrock: x_{d-1} across panels
        float pf = 0.0f;
        for (int q = 0; q < Dq; ++q) {
            // keep STAGES-1 panels in flight: issue the panel STAGES-1 ahead
            {
                int ws = stage + STAGES - 1;
                if (ws >= STAGES) ws -= STAGES;
                if (iq < Dq) {
                    issue_panel<W>(s, my, u_cur, iq, ws, nunits, lane_id, fl_cur);
                } else {
                    if (u_nxt == kNone) {
                        u_nxt = feed.next(s, lane_id);
                        if (u_nxt < nunits) fl_nxt = (uint32_t)__ldcg(s.pflag + u_nxt * PU + pl);
                    }
                    issue_panel<W>(s, my, u_nxt, iq - Dq, ws, nunits, lane_id, fl_nxt);
                }
                ++iq;
            }
            if (q == Dq - 1 && j == L - 1) pf = __ldcg(s.pf + i);  // needed after the last panel
            cp_wait<STAGES - 1>();  // this thread's copies of the current panel have landed
            const float4* slot = my + (size_t)stage * 3 * kBlock;
            float4 X = slot[0], V = slot[kBlock];
            float4 Pb;
            const int d0 = W * q + 4 * j;
            const size_t off = panel_off<W>(s, q, i) + 4 * j;
            if (fl_cur) {
                // pbest_pos of a flagged particle is its pos: use it and write the row back
                Pb = X;
                st4(s.pb + off, X);
            } else {
                Pb = slot[2 * kBlock];
            }
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const uint4 r = philox4x32_10_rk(make_uint4((uint32_t)((d0 >> 1) + g), i, t, s.swarm), s.rk0, s.rk1);
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
            panel_sum<FIT, L>(acc, X, d0, j, lane_id, carry);
            if (++stage == STAGES) stage = 0;
        }
        // Step 4 (strict improvement; the new pbest_pos is pos, flagged) and
        // Step 5, in the particle's last lane, which holds the whole sum.
        if (j == L - 1) {
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
    return best;
}

}  // namespace

// `iters` synchronous iterations. Requires D % W == 0, D / W >= STAGES - 1,
// Np a multiple of 128, s.pflag, s.work and s.bar set, work and bar zero at
// launch. FAST selects move_one_fast (requires s.fast_cr and s.fast_clamp).
//
// Each warp takes unit (its warp index) first in every iteration, then units
// from the counter. With more than one iteration, every CTA must be resident
// (a cooperative launch): an iteration ends in a grid barrier on s.bar -- each
// CTA arrives once; the last to arrive gathers gbest_pos and releases the
// others -- and while a CTA waits, its warps already load the first panels of
// their own unit for the next iteration (rows they wrote themselves, so they
// need nothing from the barrier). The wait is bounded by s.wait_limit_ns: on
// expiry the timeout status is set and the CTA stops. `expect` is the number
// of arrivals that completes a barrier: gridDim.x (one more only to test that
// bound).
template <int FIT, int W, int STAGES, bool FAST>
__global__ void __launch_bounds__(kBlock, 3) sync_panel_kernel(const __grid_constant__ SwarmDev s, int iters,
                                                               unsigned int expect) {
    constexpr int L = W / 4;
    constexpr uint32_t PU = 32 / L;
    extern __shared__ float4 ring[];      // [STAGES][3][kBlock], then gbest_pos [D]
    float* Gs = reinterpret_cast<float*>(ring + STAGES * 3 * kBlock);
    __shared__ int s_last, s_ok;
    const int lane_id = threadIdx.x & 31;
    const uint32_t pl = (uint32_t)(lane_id / L);
    const uint32_t nunits = (uint32_t)s.Np / PU;
    const uint32_t nwarps = gridDim.x * (kBlock / 32);
    const uint32_t u0 = blockIdx.x * (kBlock / 32) + (uint32_t)(threadIdx.x >> 5);
    float4* my = ring + threadIdx.x;
    const uint32_t t_prev = __ldcg(s.t_dev);

    uint32_t fl0 = u0 < nunits ? (uint32_t)__ldcg(s.pflag + u0 * PU + pl) : 0u;
#pragma unroll
    for (int k = 0; k < STAGES - 1; ++k) issue_panel<W>(s, my, u0, k, k, nunits, lane_id, fl0);
    bool nan = false;
    for (int it = 0; it < iters; ++it) {
        const uint32_t t = t_prev + 1u + (uint32_t)it;
        const int cur = (int)((t - 1u) & 1u), nxt = cur ^ 1;
        const unsigned long long K = __ldcg(s.gkey + cur);  // gbest at the end of t-1
        for (int d = threadIdx.x; d < s.D; d += blockDim.x) Gs[d] = __ldcg(s.G + (size_t)cur * s.D + d);
        __syncthreads();
        UnitFeed feed(nunits, nwarps);
        unsigned long long best = panel_units<FIT, W, STAGES, FAST>(s, my, Gs, feed, u0, fl0, nunits, t, K, nan);
        best = warp_min_u64(best);
        if (lane_id == 0 && best < K) atomicMin(s.gkey + nxt, best);

        // arrival; the last CTA completes Step 5 and releases the barrier
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(s.bar, 1u) == (uint32_t)(it + 1) * (expect + 1u) - 2u;
        __syncthreads();
        const bool final_it = it + 1 == iters;
        if (s_last) {
            __threadfence();
            gather_gbest_panel<W>(s, nxt, K);
            __syncthreads();
            if (threadIdx.x == 0) {
                s.gkey[cur] = __ldcg(s.gkey + nxt);
                *s.t_dev = t;
                *s.work = 0u;
                if (final_it) *s.bar = 0u;
                __threadfence();
                if (!final_it) atomicAdd(s.bar, 1u);
            }
        }
        if (final_it) break;

        // the first panels of this warp's own unit for the next iteration
        fl0 = u0 < nunits ? (uint32_t)__ldcg(s.pflag + u0 * PU + pl) : 0u;
#pragma unroll
        for (int k = 0; k < STAGES - 1; ++k) issue_panel<W>(s, my, u0, k, k, nunits, lane_id, fl0);
        if (threadIdx.x == 0) {
            const uint32_t target = (uint32_t)(it + 1) * (expect + 1u);
            const long long deadline = global_ns() + s.wait_limit_ns;
            int ok = 1;
            while (ld_acquire_gpu_u32(s.bar) < target) {
                if (global_ns() > deadline) {
                    ok = 0;
                    atomicOr(s.status, kStatusTimeout);
                    break;
                }
                __nanosleep(32);
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) {
            cp_wait<0>();
            break;
        }
    }
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
}

// Writes back every pending pbest_pos row on the panel layout (pbest_pos :=
// pos where flagged) and clears the flags.
template <int W>
__global__ void __launch_bounds__(kBlock) materialize_panel_kernel(const __grid_constant__ SwarmDev s) {
    const int Dq = s.D / W;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (uint32_t)s.Np; i += gridDim.x * blockDim.x) {
        if (!s.pflag[i]) continue;
        for (int q = 0; q < Dq; ++q) {
            const size_t off = panel_off<W>(s, q, i);
#pragma unroll
            for (int k = 0; k < W; k += 4) st4(s.pb + off + k, ld4(s.x + off + k));
        }
        s.pflag[i] = 0;
    }
}

// dst = src converted between the dimension-major layout (d * Np + i) and the
// panel layout of width W; one thread per (panel, particle), both sides
// coalesced.
template <int W>
__global__ void __launch_bounds__(kBlock) relayout_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                          int D, int Np, int to_panel) {
    const size_t items = (size_t)(D / W) * (size_t)Np;
    for (size_t it = (size_t)blockIdx.x * blockDim.x + threadIdx.x; it < items; it += (size_t)gridDim.x * blockDim.x) {
        const size_t q = it / (size_t)Np, i = it % (size_t)Np;
        const size_t poff = it * W;   // (q * Np + i) * W
#pragma unroll
        for (int k0 = 0; k0 < W; k0 += 4) {
            if (to_panel) {
                float v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] = src[(q * W + k0 + k) * (size_t)Np + i];
                st4(dst + poff + k0, make_float4(v[0], v[1], v[2], v[3]));
            } else {
                const float4 a = ld4(src + poff + k0);
                const float v[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) dst[(q * W + k0 + k) * (size_t)Np + i] = v[k];
            }
        }
    }
}

namespace {

size_t panel_smem(int stages, int D) {
    return sizeof(float4) * (size_t)stages * 3 * kBlock + sizeof(float) * (size_t)D;
}

template <int W, int STAGES, bool FAST>
const void* panel_kernel_t(int fid) {
    switch (fid) {
        case kSphere: return (const void*)sync_panel_kernel<kSphere, W, STAGES, FAST>;
        case kRastrigin: return (const void*)sync_panel_kernel<kRastrigin, W, STAGES, FAST>;
        case kAckley: return (const void*)sync_panel_kernel<kAckley, W, STAGES, FAST>;
        case kRosenbrock: return (const void*)sync_panel_kernel<kRosenbrock, W, STAGES, FAST>;
        case kCubicMax: return (const void*)sync_panel_kernel<kCubicMax, W, STAGES, FAST>;
        default: return nullptr;
    }
}

template <int W>
const void* panel_kernel_w(int stages, bool fast, int fid) {
    if (stages == 3) return fast ? panel_kernel_t<W, 3, true>(fid) : panel_kernel_t<W, 3, false>(fid);
    return fast ? panel_kernel_t<W, 5, true>(fid) : panel_kernel_t<W, 5, false>(fid);
}

const void* panel_kernel(int width, int stages, bool fast, int fid) {
    return width == 16 ? panel_kernel_w<16>(stages, fast, fid) : panel_kernel_w<8>(stages, fast, fid);
}

}  // namespace

bool panel_supported(int width, int stages, int D) {
    return (width == 8 || width == 16) && (stages == 3 || stages == 5) && D % width == 0 &&
           D / width >= stages - 1 && D <= 8192;
}

cudaError_t prepare_panel(int D) {
    for (int width = 8; width <= 16; width += 8)
        for (int stages = 3; stages <= 5; stages += 2)
            for (int fast = 0; fast < 2; ++fast)
                for (int fid = kSphere; fid <= kCubicMax; ++fid) {
                    cudaError_t e = cudaFuncSetAttribute(panel_kernel(width, stages, fast != 0, fid),
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)panel_smem(stages, D));
                    if (e != cudaSuccess) return e;
                }
    return cudaSuccess;
}

int panel_blocks_per_sm(int width, int stages, int fid, int D) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, panel_kernel(width, stages, true, fid), kBlock,
                                                      panel_smem(stages, D)) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_sync_panel(const SwarmDev& s, int fid, int width, int stages, int grid, int iters,
                              bool stall_barrier, cudaStream_t st) {
    if (!panel_supported(width, stages, s.D) || !s.pflag || !s.work || !s.bar || s.Np % 128 != 0 || iters < 1 ||
        iters > kPanelMaxIters || grid < 1 || (unsigned long long)iters * ((unsigned long long)grid + 2ull) >= (1ull << 32))
        return cudaErrorInvalidValue;
    const void* k = panel_kernel(width, stages, s.fast_cr && s.fast_clamp, fid);
    if (!k) return cudaErrorInvalidValue;
    unsigned int expect = (unsigned int)grid + (stall_barrier ? 1u : 0u);
    void* args[] = {const_cast<SwarmDev*>(&s), &iters, &expect};
    if (iters == 1) return cudaLaunchKernel(k, dim3(grid), dim3(kBlock), args, panel_smem(stages, s.D), st);
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kBlock), args, panel_smem(stages, s.D), st);
}

cudaError_t launch_materialize_panel(const SwarmDev& s, int width, int grid, cudaStream_t st) {
    if (!s.pflag || (width != 8 && width != 16) || s.D % width != 0) return cudaErrorInvalidValue;
    if (width == 16) materialize_panel_kernel<16><<<grid, kBlock, 0, st>>>(s);
    else materialize_panel_kernel<8><<<grid, kBlock, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t launch_relayout(const float* src, float* dst, int D, int Np, int width, bool to_panel, int grid,
                            cudaStream_t st) {
    if ((width != 8 && width != 16) || D % width != 0) return cudaErrorInvalidValue;
    if (width == 16) relayout_kernel<16><<<grid, kBlock, 0, st>>>(src, dst, D, Np, to_panel ? 1 : 0);
    else relayout_kernel<8><<<grid, kBlock, 0, st>>>(src, dst, D, Np, to_panel ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace cupso
