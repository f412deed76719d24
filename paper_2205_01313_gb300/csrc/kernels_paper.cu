// kernels_paper.cu -- the paper's own GPU designs, one particle per thread,
// and the double-precision swarm.
//
// The paper maps one particle to one thread (Sec. 2.2) and compares four ways
// of finding the global best after Steps 2-4:
//  * reduction (Sec. 2.2, Fig. 1): every block reduces its particles' pbest
//    to one entry of an auxiliary array, a second kernel reduces that array;
//  * loop unrolling (Sec. 2.2): the same with the reduction loop unrolled;
//  * queue (Sec. 3.1, Alg. 2): only particles that beat the global best enter
//    a shared-memory queue through an atomic add, thread 0 scans the queue into
//    the block's auxiliary entry, and the second kernel does the same over the
//    blocks;
//  * queue lock (Sec. 3.2, Alg. 3): thread 0 takes a global lock and updates
//    the global best itself, so the second kernel disappears. The update is in
//    place: blocks that run later in the same launch already see it.
// Here they are rebuilt for both precisions, as comparison baselines beside
// the library's own kernels. The candidate order is lexicographic on
// (fitness key, index), so every variant but the queue lock gives the
// synchronous result exactly. Iterations read the counter from device memory
// (graph-capturable); the one-kernel variants roll it from the last block.
//
// The double-precision swarm runs the paper's workload in its precision:
// binary64 state, 53-bit uniforms, sphere / Rosenbrock / the cubic of Eq. 3.
// Besides the four designs above it has a fused one-launch synchronous step
// (block argmin, a short candidate list, the last block gathers gbest) and an
// on-chip kernel that keeps a small swarm in one CTA's shared memory for many
// iterations.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "paper_kernels.h"
#include "pdl.cuh"
#include "stream_common.cuh"

namespace cg = cooperative_groups;

namespace cupso {

namespace {

// ---------------------------------------------------------------------------
// Candidate keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ PKey key_none() { return PKey{~0ull, kNoIdx, 0u}; }

__device__ __forceinline__ bool key_less(const PKey& a, const PKey& b) {
    return a.k < b.k || (a.k == b.k && a.i < b.i);
}

__device__ __forceinline__ PKey warp_min_key(PKey a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        PKey b;
        b.k = __shfl_xor_sync(0xFFFFFFFFu, a.k, o);
        b.i = __shfl_xor_sync(0xFFFFFFFFu, a.i, o);
        b.pad = 0u;
        if (key_less(b, a)) a = b;
    }
    return a;
}

// Minimum over the block (every thread returns it). red: >= 32 entries.
__device__ __forceinline__ PKey block_min_key(PKey k, PKey* red) {
    k = warp_min_key(k);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = k;
    __syncthreads();
    if (threadIdx.x < 32) {
        PKey m = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : key_none();
        m = warp_min_key(m);
        if (threadIdx.x == 0) red[0] = m;
    }
    __syncthreads();
    const PKey r = red[0];
    __syncthreads();
    return r;
}

// Appends a block's candidate to the list; a push beyond the capacity is
// dropped and reported (launchers never start more blocks than list_cap).
__device__ __forceinline__ void push_candidate(const PaperBufs& b, const PKey& k, unsigned int* status) {
    const unsigned int slot = atomicAdd(b.list_n, 1u);
    if (slot < b.list_cap) b.list[slot] = k;
    else atomicOr(status, kStatusBadArg);
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// ---------------------------------------------------------------------------
// Double precision building blocks
// ---------------------------------------------------------------------------

// Two words -> (m + 1) 2^-53 with m = hi 2^21 + (lo >> 11), in (0, 1], times
// 2^k. The double is assembled from integer parts: exponent from the leading
// bit of v = m + 1 (plus k), the bits below it as the fraction (v <= 2^53, so
// it is exact; callers keep |k| <= 512, so the result stays normal).
__device__ __forceinline__ double u53_pow2(uint32_t hi, uint32_t lo, int k) {
    const unsigned long long v = (((unsigned long long)hi << 21) | (unsigned long long)(lo >> 11)) + 1ull;
    const int lz = __clzll((long long)v);
    const unsigned long long frac = ((v << lz) << 1) >> 12;
    const unsigned long long e = (unsigned long long)(1033 - lz + k);
    return __longlong_as_double((long long)((e << 52) | frac));
}

__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) { return u53_pow2(hi, lo, 0); }

// c * u53(hi, lo), rounded once: an exponent shift when c = 2^k (exact).
__device__ __forceinline__ double c_times_u53(double c, int cexp, uint32_t hi, uint32_t lo) {
    if (cexp != kNoExp) return u53_pow2(hi, lo, cexp);
    return __dmul_rn(c, u53(hi, lo));
}

// Closed clamp to [lo, hi] with a NaN going to lo, as comparisons of the
// values' order keys (klo, khi: keys of lo, hi). Equal to the floating-point
// comparison form for every a (-0 and +0 compare equal in both), but it runs
// on the integer pipes instead of the FP64 one.
__device__ __forceinline__ double clamp64(double a, double lo, double hi, long long klo, long long khi) {
    const long long b = __double_as_longlong(a);
    const long long mag = b & 0x7FFFFFFFFFFFFFFFll;
    if (mag > 0x7FF0000000000000ll) return lo;
    const long long k = b >= 0 ? b : -mag;
    return k < klo ? lo : (k > khi ? hi : a);
}

__device__ __forceinline__ unsigned long long fit_key64(double f) {
    if (f != f) return ~0ull;
    unsigned long long b = (unsigned long long)__double_as_longlong(f);
    if ((b << 1) == 0ull) b = 0ull;  // -0 -> +0
    return (b >> 63) ? ~b : (b | (1ull << 63));
}

template <int FIT>
struct FitAcc64 {
    double acc = 0.0;
    double prev = 0.0;
    __device__ __forceinline__ void add(int d, double x) {
        if constexpr (FIT == kSphere) {
            acc = __fma_rn(x, x, acc);
        } else if constexpr (FIT == kRosenbrock) {
            if (d > 0) {
                const double p = __fma_rn(-prev, prev, x);
                const double q = __dsub_rn(1.0, prev);
                acc = __dadd_rn(acc, __fma_rn(__dmul_rn(100.0, p), p, __dmul_rn(q, q)));
            }
            prev = x;
        } else if constexpr (FIT == kCubicMax) {
            const double h = __fma_rn(__fma_rn(__dsub_rn(x, 0.8), x, -1000.0), x, 8000.0);
            acc = __dadd_rn(acc, h);
        }
    }
    __device__ __forceinline__ double finish() const { return FIT == kCubicMax ? -acc : acc; }
};

// Eq. 1 and Eq. 2 in binary64 with the clamps of Alg. 1 (same order as FP32),
// from the dimension's Philox words. Products that are exact by construction
// (w v with w = 1, c r with c a power of two) are formed without the FP64 pipe.
__device__ __forceinline__ void move_one64(double& x, double& v, double pb, double g, uint4 r, const SwarmDev64& s) {
    const double cognitive = __dsub_rn(pb, x);
    const double social = __dsub_rn(g, x);
    double vel = s.w_one ? v : __dmul_rn(s.w, v);
    vel = __fma_rn(c_times_u53(s.c1, s.c1_exp, r.x, r.y), cognitive, vel);
    vel = __fma_rn(c_times_u53(s.c2, s.c2_exp, r.z, r.w), social, vel);
    v = clamp64(vel, -s.vmax, s.vmax, s.k_vlo, s.k_vhi);
    x = clamp64(__dadd_rn(x, v), s.lo, s.hi, s.k_lo, s.k_hi);
}

// ---------------------------------------------------------------------------
// Precision adapters: what the generic kernels need from each swarm type.
// ---------------------------------------------------------------------------
struct Fp32 {
    using Dev = SwarmDev;
    using T = float;

    // Steps 2-3 for particle i at iteration t: one Philox call per dimension pair.
    template <int FIT>
    __device__ static float step_particle(const SwarmDev& s, uint32_t i, uint32_t t, const float* G) {
        const size_t Np = (size_t)s.Np;
        FitAcc<FIT> acc;
        for (int d0 = 0; d0 < s.D; d0 += 2) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)(d0 >> 1), i, t, s.swarm), s.key0, s.key1);
            for (int h = 0; h < 2 && d0 + h < s.D; ++h) {
                const int d = d0 + h;
                const size_t off = (size_t)d * Np + i;
                float x = s.x[off], v = s.v[off];
                move_one(x, v, s.pb[off], G[d], u01(word(r, 2 * h)), u01(word(r, 2 * h + 1)), s);
                s.x[off] = x;
                s.v[off] = v;
                acc.add(d, x);
            }
        }
        return acc.finish(s.D);
    }
    __device__ static PKey key(float f, uint32_t i) { return PKey{(unsigned long long)fit_key(f), i, 0u}; }
    // fitness part of the current gbest key (a single 64-bit load)
    __device__ static unsigned long long gk(const SwarmDev& s, int par) { return ld_volatile_u64(s.gkey + par) >> 32; }
    __device__ static PKey load_gkey(const SwarmDev& s, int par) {
        const unsigned long long k = ld_volatile_u64(s.gkey + par);
        return PKey{k >> 32, (uint32_t)(k & 0xFFFFFFFFull), 0u};
    }
    __device__ static void store_gkey(const SwarmDev& s, int par, PKey k) {
        *reinterpret_cast<volatile unsigned long long*>(s.gkey + par) = (k.k << 32) | (unsigned long long)k.i;
    }
};

struct Fp64 {
    using Dev = SwarmDev64;
    using T = double;

    // Steps 2-3 for particle i at iteration t: one Philox call per dimension.
    template <int FIT>
    __device__ static double step_particle(const SwarmDev64& s, uint32_t i, uint32_t t, const double* G) {
        const size_t Np = (size_t)s.Np;
        FitAcc64<FIT> acc;
        for (int d = 0; d < s.D; ++d) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)d, i, t, s.swarm), s.key0, s.key1);
            const size_t off = (size_t)d * Np + i;
            double x = s.x[off], v = s.v[off];
            move_one64(x, v, s.pb[off], G[d], r, s);
            s.x[off] = x;
            s.v[off] = v;
            acc.add(d, x);
        }
        return acc.finish();
    }
    __device__ static PKey key(double f, uint32_t i) { return PKey{fit_key64(f), i, 0u}; }
    __device__ static unsigned long long gk(const SwarmDev64& s, int par) { return ld_volatile_u64(&s.gkey[par].k); }
    __device__ static PKey load_gkey(const SwarmDev64& s, int par) {
        const volatile PKey* p = s.gkey + par;
        return PKey{p->k, p->i, 0u};
    }
    __device__ static void store_gkey(const SwarmDev64& s, int par, PKey k) {
        volatile PKey* p = s.gkey + par;
        p->i = k.i;
        p->k = k.k;
    }
};

// ---------------------------------------------------------------------------
// Alg. 3: thread 0 of a block with a candidate takes the global lock (a
// bounded wait: on expiry the timeout status is set and the update skipped),
// re-checks against the global best and, if it is better, writes gbest_pos
// (from the candidate's pbest row: index first, position after) and the key.
// ---------------------------------------------------------------------------
template <class A>
__device__ void locked_update(const typename A::Dev& s, const PaperBufs& b, int cur, PKey best) {
    const long long deadline = global_ns() + s.wait_limit_ns;
    bool got = false;
    for (;;) {
        if (atomicCAS(b.lock, 0u, 1u) == 0u) {
            got = true;
            break;
        }
        if (global_ns() > deadline) break;
        __nanosleep(64);
    }
    if (!got) {
        atomicOr(s.status, kStatusTimeout);
        return;
    }
    __threadfence();
    const PKey K = A::load_gkey(s, cur);
    if (key_less(best, K)) {
        const size_t Np = (size_t)s.Np;
        for (int d = 0; d < s.D; ++d) s.G[(size_t)cur * s.D + d] = __ldcg(s.pb + (size_t)d * Np + best.i);
        __threadfence();
        A::store_gkey(s, cur, best);
        __threadfence();
    }
    atomicExch(b.lock, 0u);
}

// ---------------------------------------------------------------------------
// One iteration's first (or only) kernel: Steps 2-4 for one particle per
// thread, then the block's part of Step 5 in the chosen design.
// ---------------------------------------------------------------------------
template <class A, int FIT, int AGG>
__global__ void __launch_bounds__(kPaperBlock) paper_step_kernel(const __grid_constant__ typename A::Dev s,
                                                                 const __grid_constant__ PaperBufs b) {
    using T = typename A::T;
    __shared__ PKey red[kPaperBlock];   // tree operands, or the queue
    __shared__ unsigned int qn;
    __shared__ int s_last;
    pdl_wait();
    pdl_launch_next();
    const uint32_t t_prev = __ldcg(s.t_dev);
    const uint32_t t = t_prev + 1u;
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    const int tid = threadIdx.x;
    const uint32_t i = blockIdx.x * (uint32_t)kPaperBlock + (uint32_t)tid;
    const size_t Np = (size_t)s.Np;
    if (tid == 0) qn = 0u;
    __syncthreads();

    PKey mine = key_none();
    bool nan = false;
    if (i < (uint32_t)s.N) {
        const T f = A::template step_particle<FIT>(s, i, t, s.G + (size_t)cur * s.D);   // Steps 2-3
        nan = (f != f);
        const T pf = s.pf[i];
        const bool imp = f < pf;                                                         // Step 4
        if (imp) {
            s.pf[i] = f;
            for (int d = 0; d < s.D; ++d) s.pb[(size_t)d * Np + i] = s.x[(size_t)d * Np + i];
        }
        if constexpr (AGG == kAggReduce || AGG == kAggReduceUnrolled) {
            mine = A::key(imp ? f : pf, i);              // the reduction takes every particle
        } else if (imp) {
            // Sec. 3.1: only a particle that improved and can beat the global best
            // competes. Comparing the fitness key alone (<=) keeps every particle
            // that could win a tie on its index.
            const PKey k = A::key(f, i);
            if (k.k <= A::gk(s, cur)) mine = k;
        }
    }

    if constexpr (AGG == kAggReduce) {
        red[tid] = mine;
        __syncthreads();
        for (int st = kPaperBlock / 2; st > 0; st >>= 1) {
            if (tid < st && key_less(red[tid + st], red[tid])) red[tid] = red[tid + st];
            __syncthreads();
        }
        if (tid == 0) b.aux[blockIdx.x] = red[0];
    } else if constexpr (AGG == kAggReduceUnrolled) {
        red[tid] = mine;
        __syncthreads();
#pragma unroll
        for (int st = kPaperBlock / 2; st > 32; st >>= 1) {
            if (tid < st && key_less(red[tid + st], red[tid])) red[tid] = red[tid + st];
            __syncthreads();
        }
        if (tid < 32) {
            PKey k = red[tid];
            if (key_less(red[tid + 32], k)) k = red[tid + 32];
            k = warp_min_key(k);
            if (tid == 0) b.aux[blockIdx.x] = k;
        }
    } else if constexpr (AGG == kAggQueue || AGG == kAggQueueLock) {
        // Alg. 2: the rare candidates enter the block's queue in atomic order
        if (mine.i != kNoIdx) red[atomicAdd(&qn, 1u)] = mine;
        __syncthreads();
        if (tid == 0) {
            PKey best = key_none();
            const unsigned int n = qn;
            for (unsigned int j = 0; j < n; ++j)
                if (key_less(red[j], best)) best = red[j];
            if constexpr (AGG == kAggQueue) {
                b.aux[blockIdx.x] = best;
            } else if (best.i != kNoIdx) {
                locked_update<A>(s, b, cur, best);   // Alg. 3
            }
        }
    } else {  // kAggSyncList
        const PKey k = block_min_key(mine, red);
        if (tid == 0 && k.i != kNoIdx) push_candidate(b, k, s.status);
    }
    if (__syncthreads_or(nan) && tid == 0) atomicOr(s.status, kStatusNaN);

    if constexpr (AGG == kAggQueueLock || AGG == kAggSyncList) {
        // The last block to finish closes the iteration.
        __threadfence();
        __syncthreads();
        if (tid == 0) s_last = (atomicAdd(b.ticket, 1u) == gridDim.x - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        if constexpr (AGG == kAggQueueLock) {
            // the in-place gbest of this iteration is the next iteration's
            for (int d = tid; d < s.D; d += blockDim.x)
                s.G[(size_t)nxt * s.D + d] = __ldcg(s.G + (size_t)cur * s.D + d);
            if (tid == 0) A::store_gkey(s, nxt, A::load_gkey(s, cur));
        } else {
            const unsigned int n = min(__ldcg(b.list_n), b.list_cap);
            PKey k = tid == 0 ? A::load_gkey(s, cur) : key_none();
            for (unsigned int j = tid; j < n; j += blockDim.x) {
                PKey c;
                c.k = __ldcg(&b.list[j].k);
                c.i = __ldcg(&b.list[j].i);
                c.pad = 0u;
                if (key_less(c, k)) k = c;
            }
            const PKey best = block_min_key(k, red);
            if (best.i < (uint32_t)s.N)
                for (int d = tid; d < s.D; d += blockDim.x)
                    s.G[(size_t)nxt * s.D + d] = __ldcg(s.pb + (size_t)d * Np + best.i);
            if (tid == 0) {
                A::store_gkey(s, nxt, best);
                A::store_gkey(s, cur, best);
                *b.list_n = 0u;
            }
        }
        __syncthreads();
        if (tid == 0) {
            *b.ticket = 0u;
            *s.t_dev = t;
        }
    }
}

// ---------------------------------------------------------------------------
// Second kernel (one block): over the blocks' auxiliary entries. REDUCE and
// REDUCE_UNROLLED reduce all of them (every particle's pbest took part);
// QUEUE runs Alg. 2 once more: entries that beat the global best enter a
// queue that thread 0 scans. ADVANCE: this closes iteration t_prev + 1
// (gbest into the next parity, counter rolled); otherwise it sets the gbest
// of the current iteration (after the initialisation or a loaded state).
// ---------------------------------------------------------------------------
template <class A, int AGG, bool ADVANCE>
__global__ void __launch_bounds__(1024) paper_finish_kernel(const __grid_constant__ typename A::Dev s,
                                                            const __grid_constant__ PaperBufs b, int nblocks) {
    __shared__ PKey red[1024];
    __shared__ unsigned int qn;
    pdl_wait();
    pdl_launch_next();
    const int tid = threadIdx.x;
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur = (int)(t_prev & 1u);
    const int out = ADVANCE ? (cur ^ 1) : cur;
    PKey k = key_none();
    for (int j = tid; j < nblocks; j += blockDim.x) {
        PKey c;
        c.k = __ldcg(&b.aux[j].k);
        c.i = __ldcg(&b.aux[j].i);
        c.pad = 0u;
        if (key_less(c, k)) k = c;
    }
    PKey best;
    if constexpr (AGG == kAggQueue) {
        if (tid == 0) qn = 0u;
        __syncthreads();
        const PKey K = A::load_gkey(s, cur);
        if (k.i != kNoIdx && key_less(k, K)) red[atomicAdd(&qn, 1u)] = k;
        __syncthreads();
        if (tid == 0) {
            PKey m = K;
            const unsigned int n = qn;
            for (unsigned int j = 0; j < n; ++j)
                if (key_less(red[j], m)) m = red[j];
            red[0] = m;
        }
        __syncthreads();
        best = red[0];
    } else {
        red[tid] = k;
        __syncthreads();
        const int lim = AGG == kAggReduceUnrolled ? 32 : 0;
        for (int st = blockDim.x / 2; st > lim; st >>= 1) {
            if (tid < st && key_less(red[tid + st], red[tid])) red[tid] = red[tid + st];
            __syncthreads();
        }
        if (AGG == kAggReduceUnrolled && tid < 32) {
            PKey m = red[tid];
            if (key_less(red[tid + 32], m)) m = red[tid + 32];
            m = warp_min_key(m);
            if (tid == 0) red[0] = m;
        }
        __syncthreads();
        best = red[0];
    }
    const size_t Np = (size_t)s.Np;
    if (best.i < (uint32_t)s.N)
        for (int d = tid; d < s.D; d += blockDim.x) s.G[(size_t)out * s.D + d] = __ldcg(s.pb + (size_t)d * Np + best.i);
    if (tid == 0) {
        A::store_gkey(s, 0, best);
        A::store_gkey(s, 1, best);
        if (ADVANCE) *s.t_dev = t_prev + 1u;
    }
}

// ---------------------------------------------------------------------------
// FP64 Step 1 (t = 0) and the gbest of a loaded state.
// ---------------------------------------------------------------------------
template <int FIT>
__global__ void __launch_bounds__(kPaperBlock) init64_kernel(const __grid_constant__ SwarmDev64 s,
                                                             const __grid_constant__ PaperBufs b) {
    __shared__ PKey red[32];
    const uint32_t i = blockIdx.x * (uint32_t)kPaperBlock + threadIdx.x;
    const size_t Np = (size_t)s.Np;
    PKey mine = key_none();
    bool nan = false;
    if (i < (uint32_t)s.N) {
        const double span = __dsub_rn(s.hi, s.lo);
        const double vspan = __dmul_rn(2.0, s.vmax);
        FitAcc64<FIT> acc;
        for (int d = 0; d < s.D; ++d) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)d, i, 0u, s.swarm), s.key0, s.key1);
            const double x = clamp64(__fma_rn(u53(r.x, r.y), span, s.lo), s.lo, s.hi, s.k_lo, s.k_hi);
            const double v = clamp64(__fma_rn(u53(r.z, r.w), vspan, -s.vmax), -s.vmax, s.vmax, s.k_vlo, s.k_vhi);
            const size_t off = (size_t)d * Np + i;
            s.x[off] = x;
            s.v[off] = v;
            s.pb[off] = x;
            acc.add(d, x);
        }
        const double f = acc.finish();
        s.pf[i] = f;
        nan = (f != f);
        mine = Fp64::key(f, i);
    }
    const PKey k = block_min_key(mine, red);
    if (threadIdx.x == 0) b.aux[blockIdx.x] = k;
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
}

__global__ void __launch_bounds__(kPaperBlock) pbest_min64_kernel(const __grid_constant__ SwarmDev64 s,
                                                                  const __grid_constant__ PaperBufs b) {
    __shared__ PKey red[32];
    const uint32_t i = blockIdx.x * (uint32_t)kPaperBlock + threadIdx.x;
    PKey mine = key_none();
    bool nan = false;
    if (i < (uint32_t)s.N) {
        const double f = s.pf[i];
        nan = (f != f);
        mine = Fp64::key(f, i);
    }
    const PKey k = block_min_key(mine, red);
    if (threadIdx.x == 0) b.aux[blockIdx.x] = k;
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
}

// ---------------------------------------------------------------------------
// Fitness from per-dimension terms, for the kernels that spread a particle's
// dimensions over threads: the terms are formed in parallel, then one thread
// per particle adds them in order d = 0 .. D-1 (the same operations, in the
// same order, as FitAcc64).
// ---------------------------------------------------------------------------
template <int FIT>
struct FitTerms64 {
    static constexpr bool kNeedsNext = (FIT == kRosenbrock);
    // term of dimension d (x = x_d, xn = x_{d+1}); Rosenbrock: d < D - 1 only
    __device__ static __forceinline__ double term(double x, double xn) {
        if constexpr (FIT == kCubicMax) {
            return __fma_rn(__fma_rn(__dsub_rn(x, 0.8), x, -1000.0), x, 8000.0);
        } else if constexpr (FIT == kRosenbrock) {
            const double p = __fma_rn(-x, x, xn);
            const double q = __dsub_rn(1.0, x);
            return __fma_rn(__dmul_rn(100.0, p), p, __dmul_rn(q, q));
        } else {
            return 0.0;   // sphere: the sum fuses x * x, no separate term
        }
    }
    // sequential sum over d of particle column p (stride P) of X / H
    __device__ static __forceinline__ double sum(const double* X, const double* H, int P, int p, int D) {
        double acc = 0.0;
        if constexpr (FIT == kSphere) {
            for (int d = 0; d < D; ++d) {
                const double x = X[(size_t)d * P + p];
                acc = __fma_rn(x, x, acc);
            }
        } else {
            const int n = FIT == kRosenbrock ? D - 1 : D;
            for (int d = 0; d < n; ++d) acc = __dadd_rn(acc, H[(size_t)d * P + p]);
        }
        return FIT == kCubicMax ? -acc : acc;
    }
};

// ---------------------------------------------------------------------------
// On-chip FP64 swarm: a cluster of C CTAs (1 <= C <= 16). CTA r keeps the
// particles [r P, r P + n_r) -- x, v, pbest_pos and the fitness terms
// ([D][P]), pbest_fit and its copy of gbest -- in shared memory for `iters`
// iterations. Per iteration every CTA pushes its best candidate (key and
// position) into slot [parity][r] of every CTA of the cluster through
// distributed shared memory (index first, position after, Sec. 4.3); one
// cluster barrier replaces the paper's kernel boundary (Sec. 2.2), and every
// CTA reduces the same slots in the same order, so all hold the same gbest.
// ---------------------------------------------------------------------------
constexpr int kOnchip64Threads = 1024;
constexpr int kMaxCluster64 = 16;

struct Onchip64Layout {
    int P;                                  // particles per CTA
    size_t o_x, o_v, o_pb, o_h, o_pf, o_G, o_red, o_slots, slot, bytes;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) / 16 * 16; }

__host__ __device__ inline Onchip64Layout onchip64_layout(int N, int D, int C) {
    Onchip64Layout L;
    L.P = (N + C - 1) / C;
    const size_t plane = sizeof(double) * (size_t)L.P * (size_t)D;
    size_t o = 0;
    L.o_x = o; o = al16(o + plane);
    L.o_v = o; o = al16(o + plane);
    L.o_pb = o; o = al16(o + plane);
    L.o_h = o; o = al16(o + plane);
    L.o_pf = o; o = al16(o + sizeof(double) * (size_t)L.P);
    L.o_G = o; o = al16(o + sizeof(double) * (size_t)D);
    L.o_red = o; o = al16(o + sizeof(PKey) * 32);
    L.slot = al16(sizeof(PKey) + sizeof(double) * (size_t)D);
    L.o_slots = o; o += 2 * (size_t)C * L.slot;
    L.bytes = o;
    return L;
}

template <int FIT>
__global__ void __launch_bounds__(kOnchip64Threads) onchip64_kernel(const __grid_constant__ SwarmDev64 s, int iters) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int N = s.N, D = s.D;
    const Onchip64Layout L = onchip64_layout(N, D, C);
    const int P = L.P;
    const int base = rank * P;
    const int n = max(0, min(P, N - base));       // particles of this CTA
    double* x = reinterpret_cast<double*>(smem + L.o_x);    // [D][P]
    double* v = reinterpret_cast<double*>(smem + L.o_v);
    double* pb = reinterpret_cast<double*>(smem + L.o_pb);
    double* H = reinterpret_cast<double*>(smem + L.o_h);
    double* pf = reinterpret_cast<double*>(smem + L.o_pf);
    double* G = reinterpret_cast<double*>(smem + L.o_G);
    PKey* red = reinterpret_cast<PKey*>(smem + L.o_red);
    unsigned char* slots = smem + L.o_slots;
    const size_t Np = (size_t)s.Np;
    const int tid = threadIdx.x;
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur0 = (int)(t_prev & 1u);
    const int nD = n * D;

    for (int e = tid; e < nD; e += blockDim.x) {
        const int d = e / n, p = e - d * n;
        const size_t g = (size_t)d * Np + (size_t)(base + p);
        x[d * P + p] = s.x[g];
        v[d * P + p] = s.v[g];
        pb[d * P + p] = s.pb[g];
    }
    for (int p = tid; p < n; p += blockDim.x) pf[p] = s.pf[base + p];
    for (int d = tid; d < D; d += blockDim.x) G[d] = s.G[(size_t)cur0 * D + d];
    PKey K = Fp64::load_gkey(s, cur0);
    __syncthreads();

    bool nan = false;
    for (int k = 0; k < iters; ++k) {
        const uint32_t t = t_prev + 1u + (uint32_t)k;
        // Step 2 for every (dimension, particle); the fitness terms that need only x_d
        for (int e = tid; e < nD; e += blockDim.x) {
            const int d = e / n, p = e - d * n;
            const int j = d * P + p;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)d, (uint32_t)(base + p), t, s.swarm), s.key0, s.key1);
            double xx = x[j], vv = v[j];
            move_one64(xx, vv, pb[j], G[d], r, s);
            x[j] = xx;
            v[j] = vv;
            if constexpr (!FitTerms64<FIT>::kNeedsNext && FIT != kSphere) H[j] = FitTerms64<FIT>::term(xx, 0.0);
        }
        __syncthreads();
        if constexpr (FitTerms64<FIT>::kNeedsNext) {
            for (int e = tid; e < nD; e += blockDim.x) {
                const int d = e / n, p = e - d * n;
                if (d + 1 < D) H[d * P + p] = FitTerms64<FIT>::term(x[d * P + p], x[(d + 1) * P + p]);
            }
            __syncthreads();
        }
        // Steps 3-4 per particle; this CTA's Step-5 candidate
        PKey cand = key_none();
        for (int p = tid; p < n; p += blockDim.x) {
            const double f = FitTerms64<FIT>::sum(x, H, P, p, D);
            nan |= (f != f);
            if (f < pf[p]) {
                pf[p] = f;
                for (int d = 0; d < D; ++d) pb[d * P + p] = x[d * P + p];
                const PKey c = Fp64::key(f, (uint32_t)(base + p));
                if (key_less(c, K) && key_less(c, cand)) cand = c;
            }
        }
        const PKey best = block_min_key(cand, red);   // barriers inside
        // push (key, position) into slot [par][rank] of every CTA
        const int par = k & 1;
        const size_t my_slot = ((size_t)par * C + rank) * L.slot;
        if (tid < C) {
            unsigned char* remote = cluster.map_shared_rank(slots, tid);
            *reinterpret_cast<PKey*>(remote + my_slot) = best;
        }
        if (best.i != kNoIdx) {
            const int pc = (int)best.i - base;
            for (int e = tid; e < C * D; e += blockDim.x) {
                const int r = e / D, d = e - r * D;
                unsigned char* remote = cluster.map_shared_rank(slots, r);
                reinterpret_cast<double*>(remote + my_slot + sizeof(PKey))[d] = pb[d * P + pc];
            }
        }
        cluster.sync();
        // Step 5: the same reduction over the slots in every CTA
        PKey bk = K;
        int win = -1;
        for (int r = 0; r < C; ++r) {
            const PKey kk = *reinterpret_cast<const PKey*>(slots + ((size_t)par * C + r) * L.slot);
            if (key_less(kk, bk)) {
                bk = kk;
                win = r;
            }
        }
        if (win >= 0) {
            const double* row = reinterpret_cast<const double*>(slots + ((size_t)par * C + win) * L.slot + sizeof(PKey));
            for (int d = tid; d < D; d += blockDim.x) G[d] = row[d];
            K = bk;
        }
        __syncthreads();
    }
    for (int e = tid; e < nD; e += blockDim.x) {
        const int d = e / n, p = e - d * n;
        const size_t g = (size_t)d * Np + (size_t)(base + p);
        s.x[g] = x[d * P + p];
        s.v[g] = v[d * P + p];
        s.pb[g] = pb[d * P + p];
    }
    for (int p = tid; p < n; p += blockDim.x) s.pf[base + p] = pf[p];
    if (__syncthreads_or(nan) && tid == 0) atomicOr(s.status, kStatusNaN);
    if (rank == 0) {
        const int out = (int)((t_prev + (uint32_t)iters) & 1u);
        for (int d = tid; d < D; d += blockDim.x) s.G[(size_t)out * D + d] = G[d];
        if (tid == 0) {
            Fp64::store_gkey(s, 0, K);
            Fp64::store_gkey(s, 1, K);
            *s.t_dev = t_prev + (uint32_t)iters;
        }
    }
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
}

// ---------------------------------------------------------------------------
// FP64 synchronous step for many dimensions: a block takes a tile of P
// particles with all D dimensions and spreads its (dimension, particle) pairs
// over the threads (the one-particle-per-thread designs leave most SMs idle
// when N is small and D large). The fitness terms are formed in parallel, the
// ordered sum by one thread per particle; pbest rows are written by all
// threads. Step 5 as in the fused one-particle-per-thread step: block argmin,
// candidate list, the last block gathers gbest.
// ---------------------------------------------------------------------------
constexpr int kTileItems = 2048;     // P * D per block at most (32 KB of x' and terms)
constexpr int kTileMinD = 16;        // below this the one-particle-per-thread step is used
constexpr int kChunk64 = 1;          // items whose loads a thread issues together (more only costs occupancy: FP64-bound)

template <int FIT>
__global__ void __launch_bounds__(256) sync64_tile_kernel(const __grid_constant__ SwarmDev64 s,
                                                         const __grid_constant__ PaperBufs b, int P) {
    __shared__ double X[kTileItems];
    __shared__ double H[kTileItems];
    __shared__ PKey red[32];
    __shared__ int imp[32];
    __shared__ int s_last;
    pdl_wait();
    pdl_launch_next();
    const uint32_t t_prev = __ldcg(s.t_dev);
    const uint32_t t = t_prev + 1u;
    const int cur = (int)(t_prev & 1u), nxt = cur ^ 1;
    const int tid = threadIdx.x;
    const int D = s.D;
    const size_t Np = (size_t)s.Np;
    const int base = blockIdx.x * P;
    const int n = min(P, s.N - base);
    const int nD = n * D;
    const double* G = s.G + (size_t)cur * D;

    // a thread loads the rows of kChunk64 items before it computes any of them
    for (int e0 = tid; e0 < nD; e0 += kChunk64 * blockDim.x) {
        double xs[kChunk64], vs[kChunk64], ps[kChunk64];
#pragma unroll
        for (int c = 0; c < kChunk64; ++c) {
            const int e = e0 + c * blockDim.x;
            if (e < nD) {
                const int d = e / n, p = e - d * n;
                const size_t off = (size_t)d * Np + (size_t)(base + p);
                xs[c] = s.x[off];
                vs[c] = s.v[off];
                ps[c] = s.pb[off];
            }
        }
#pragma unroll
        for (int c = 0; c < kChunk64; ++c) {
            const int e = e0 + c * blockDim.x;
            if (e >= nD) break;
            const int d = e / n, p = e - d * n;
            const uint32_t i = (uint32_t)(base + p);
            const size_t off = (size_t)d * Np + i;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)d, i, t, s.swarm), s.key0, s.key1);
            double xx = xs[c], vv = vs[c];
            move_one64(xx, vv, ps[c], G[d], r, s);
            s.x[off] = xx;
            s.v[off] = vv;
            X[d * P + p] = xx;
            if constexpr (!FitTerms64<FIT>::kNeedsNext && FIT != kSphere) H[d * P + p] = FitTerms64<FIT>::term(xx, 0.0);
        }
    }
    __syncthreads();
    if constexpr (FitTerms64<FIT>::kNeedsNext) {
        for (int e = tid; e < nD; e += blockDim.x) {
            const int d = e / n, p = e - d * n;
            if (d + 1 < D) H[d * P + p] = FitTerms64<FIT>::term(X[d * P + p], X[(d + 1) * P + p]);
        }
        __syncthreads();
    }
    PKey cand = key_none();
    bool nan = false;
    if (tid < n) {
        const uint32_t i = (uint32_t)(base + tid);
        const double f = FitTerms64<FIT>::sum(X, H, P, tid, D);
        nan = (f != f);
        const bool better = f < s.pf[i];
        imp[tid] = better ? 1 : 0;
        if (better) {
            s.pf[i] = f;
            const PKey c = Fp64::key(f, i);
            if (c.k <= Fp64::gk(s, cur)) cand = c;
        }
    }
    __syncthreads();
    for (int e = tid; e < nD; e += blockDim.x) {
        const int d = e / n, p = e - d * n;
        if (imp[p]) s.pb[(size_t)d * Np + (size_t)(base + p)] = X[d * P + p];
    }
    const PKey k = block_min_key(cand, red);
    if (tid == 0 && k.i != kNoIdx) push_candidate(b, k, s.status);
    if (__syncthreads_or(nan) && tid == 0) atomicOr(s.status, kStatusNaN);

    // the last block to finish closes the iteration
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(b.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const unsigned int nl = min(__ldcg(b.list_n), b.list_cap);
    PKey m = tid == 0 ? Fp64::load_gkey(s, cur) : key_none();
    for (unsigned int j = tid; j < nl; j += blockDim.x) {
        PKey c;
        c.k = __ldcg(&b.list[j].k);
        c.i = __ldcg(&b.list[j].i);
        c.pad = 0u;
        if (key_less(c, m)) m = c;
    }
    const PKey best = block_min_key(m, red);
    if (best.i < (uint32_t)s.N)
        for (int d = tid; d < D; d += blockDim.x)
            s.G[(size_t)nxt * D + d] = __ldcg(s.pb + (size_t)d * Np + best.i);
    __syncthreads();
    if (tid == 0) {
        Fp64::store_gkey(s, nxt, best);
        Fp64::store_gkey(s, cur, best);
        *b.list_n = 0u;
        *b.ticket = 0u;
        *s.t_dev = t;
    }
}

// Particles per tile of sync64_tile_kernel: a power of two, at most 32 and
// kTileItems / D, and small enough that the tiles cover the SMs twice over.
int tile_particles(int N, int D, int num_sms) {
    int P = 32;
    while (P > 1 && (P * D > kTileItems || (long long)N < 2ll * num_sms * P)) P >>= 1;
    return P;
}

// ---------------------------------------------------------------------------
// Persistent FP64 swarm (a cooperative launch, so every block is resident):
// `iters` iterations, each ending with a grid barrier instead of a kernel
// boundary. A block's Step-5 candidate goes to its own slot of a list
// double-buffered by parity; after the barrier every block reduces the same
// slots in the same order, so all hold the same gbest.
// ---------------------------------------------------------------------------
constexpr int kPersistThreads = 128;

// Bounded grid barrier: thread 0 of every block arrives on a counter; the last
// one resets it and advances the generation the others wait on. A wait past
// the limit sets the timeout status and returns false.
__device__ bool grid_barrier(const PaperBufs& b, unsigned int nblocks, long long limit_ns, unsigned int* status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int g = *reinterpret_cast<volatile unsigned int*>(b.bar_gen);
        __threadfence();
        if (atomicAdd(b.bar_count, 1u) == nblocks - 1u) {
            *reinterpret_cast<volatile unsigned int*>(b.bar_count) = 0u;
            __threadfence();
            atomicAdd(b.bar_gen, 1u);
        } else {
            const long long deadline = global_ns() + limit_ns;
            while (*reinterpret_cast<volatile unsigned int*>(b.bar_gen) == g) {
                if (global_ns() > deadline) {
                    ok = 0;
                    atomicOr(status, kStatusTimeout);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <int FIT>
__global__ void __launch_bounds__(kPersistThreads) persist64_kernel(const __grid_constant__ SwarmDev64 s,
                                                                   const __grid_constant__ PaperBufs b, int iters) {
    extern __shared__ double Gsh[];   // [D] the current gbest
    __shared__ PKey red[32];
    const int tid = threadIdx.x;
    const size_t Np = (size_t)s.Np;
    const unsigned int nblk = gridDim.x;
    const uint32_t stride = nblk * blockDim.x;
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur0 = (int)(t_prev & 1u);
    PKey K = Fp64::load_gkey(s, cur0);
    for (int d = tid; d < s.D; d += blockDim.x) Gsh[d] = s.G[(size_t)cur0 * s.D + d];
    __syncthreads();
    bool nan = false;
    int done = 0;
    for (int k = 0; k < iters; ++k) {
        const uint32_t t = t_prev + 1u + (uint32_t)k;
        PKey cand = key_none();
        for (uint32_t i = blockIdx.x * blockDim.x + tid; i < (uint32_t)s.N; i += stride) {
            const double f = Fp64::step_particle<FIT>(s, i, t, Gsh);   // Steps 2-3
            nan |= (f != f);
            if (f < s.pf[i]) {                                          // Step 4
                s.pf[i] = f;
                for (int d = 0; d < s.D; ++d) s.pb[(size_t)d * Np + i] = s.x[(size_t)d * Np + i];
                const PKey c = Fp64::key(f, i);
                if (key_less(c, K) && key_less(c, cand)) cand = c;
            }
        }
        const PKey mine = block_min_key(cand, red);
        PKey* slots = b.list + (size_t)(k & 1) * nblk;
        if (tid == 0) {
            slots[blockIdx.x].k = mine.k;
            slots[blockIdx.x].i = mine.i;
        }
        if (!grid_barrier(b, nblk, s.wait_limit_ns, s.status)) break;
        // Step 5: the same reduction in every block
        PKey m = K;
        for (unsigned int j = tid; j < nblk; j += blockDim.x) {
            PKey c;
            c.k = __ldcg(&slots[j].k);
            c.i = __ldcg(&slots[j].i);
            c.pad = 0u;
            if (key_less(c, m)) m = c;
        }
        const PKey nbest = block_min_key(m, red);
        if (key_less(nbest, K)) {
            K = nbest;
            for (int d = tid; d < s.D; d += blockDim.x) Gsh[d] = __ldcg(s.pb + (size_t)d * Np + nbest.i);
        }
        __syncthreads();
        done = k + 1;
    }
    if (__syncthreads_or(nan) && tid == 0) atomicOr(s.status, kStatusNaN);
    if (blockIdx.x == 0) {
        const uint32_t t_end = t_prev + (uint32_t)done;
        const int out = (int)(t_end & 1u);
        for (int d = tid; d < s.D; d += blockDim.x) s.G[(size_t)out * s.D + d] = Gsh[d];
        if (tid == 0) {
            Fp64::store_gkey(s, 0, K);
            Fp64::store_gkey(s, 1, K);
            *s.t_dev = t_end;
        }
    }
}

// ---------------------------------------------------------------------------
// Resident variant of the persistent FP64 swarm, for swarms of at most one
// particle per thread: x, v and pbest_pos stay in shared memory ([D][TB]) and
// pbest_fit in a register for all iterations of the launch, so an iteration
// touches global memory only for the Step-5 exchange. A block's candidate goes
// to its slot together with its position (index first, position after, as in
// Sec. 4.3); after the barrier every block reduces the same slots in the same
// order, and for D <= kResPos the position travels with the key in that one
// pass over the slots.
// ---------------------------------------------------------------------------
constexpr int kResPos = 4;
constexpr int kResMaxIters = 1 << 24;   // per launch: (k + 1) * blocks stays below 2^32

__device__ __forceinline__ unsigned int add_release_gpu(unsigned int* p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded grid barrier number k of a launch that started with the counter at
// zero: thread 0 of every block adds one arrival, and barrier k is complete
// once all blocks have arrived k + 1 times. One atomic per block, no reset and
// no generation word to read first. The arrival releases the block's writes
// (ordered before it by the block barrier) and the wait acquires the others'.
// A wait past the limit sets the timeout status and returns false.
__device__ bool grid_barrier_k(const PaperBufs& b, unsigned int nblocks, int k, long long limit_ns,
                               unsigned int* status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int target = (unsigned int)(k + 1) * nblocks;
        if (add_release_gpu(b.bar_count, 1u) + 1u < target) {
            const long long deadline = global_ns() + limit_ns;
            while (ld_acquire_gpu(b.bar_count) < target) {
                if (global_ns() > deadline) {
                    ok = 0;
                    atomicOr(status, kStatusTimeout);
                    break;
                }
            }
        } else {
            (void)ld_acquire_gpu(b.bar_count);   // the last arrival acquires too
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__host__ __device__ inline size_t res_slot_bytes(int D) { return (sizeof(PKey) + sizeof(double) * (size_t)D + 15) / 16 * 16; }

template <int FIT>
__global__ void __launch_bounds__(512) persist64r_kernel(const __grid_constant__ SwarmDev64 s,
                                                          const __grid_constant__ PaperBufs b, int iters) {
    extern __shared__ double sm64[];
    __shared__ PKey red[32];
    const int TB = (int)blockDim.x, D = s.D, tid = threadIdx.x;
    double* X = sm64;                       // [D][TB]
    double* V = X + (size_t)D * TB;
    double* PB = V + (size_t)D * TB;
    double* Gsh = PB + (size_t)D * TB;      // [D] the current gbest
    const unsigned int nblk = gridDim.x;
    const uint32_t i = blockIdx.x * (uint32_t)TB + (uint32_t)tid;
    const bool own = i < (uint32_t)s.N;
    const size_t Np = (size_t)s.Np;
    const size_t rec = res_slot_bytes(D);
    unsigned char* slots = reinterpret_cast<unsigned char*>(b.list);
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur0 = (int)(t_prev & 1u);
    PKey K = Fp64::load_gkey(s, cur0);
    for (int d = tid; d < D; d += TB) Gsh[d] = s.G[(size_t)cur0 * D + d];
    double pf = 0.0;
    if (own) {
        pf = s.pf[i];
        for (int d = 0; d < D; ++d) {
            const size_t g = (size_t)d * Np + i;
            X[d * TB + tid] = s.x[g];
            V[d * TB + tid] = s.v[g];
            PB[d * TB + tid] = s.pb[g];
        }
    }
    __syncthreads();
    bool nan = false;
    int done = 0;
    for (int k = 0; k < iters; ++k) {
        const uint32_t t = t_prev + 1u + (uint32_t)k;
        PKey cand = key_none();
        if (own) {   // Steps 2-4 of this thread's particle
            FitAcc64<FIT> acc;
            for (int d = 0; d < D; ++d) {
                const uint4 r = philox4x32_10(make_uint4((uint32_t)d, i, t, s.swarm), s.key0, s.key1);
                const int j = d * TB + tid;
                double x = X[j], v = V[j];
                move_one64(x, v, PB[j], Gsh[d], r, s);
                X[j] = x;
                V[j] = v;
                acc.add(d, x);
            }
            const double f = acc.finish();
            nan |= (f != f);
            if (f < pf) {
                pf = f;
                for (int d = 0; d < D; ++d) PB[d * TB + tid] = X[d * TB + tid];
                const PKey c = Fp64::key(f, i);
                if (key_less(c, K)) cand = c;
            }
        }
        const PKey best = block_min_key(cand, red);
        unsigned char* mine = slots + ((size_t)(k & 1) * nblk + blockIdx.x) * rec;
        if (best.i == kNoIdx) {
            if (tid == 0) *reinterpret_cast<PKey*>(mine) = key_none();
        } else if (best.i == i) {   // the candidate's own thread fills the slot
            double* pos = reinterpret_cast<double*>(mine + sizeof(PKey));
            for (int d = 0; d < D; ++d) pos[d] = PB[d * TB + tid];
            *reinterpret_cast<PKey*>(mine) = best;
        }
        if (!grid_barrier_k(b, nblk, k, s.wait_limit_ns, s.status)) break;
        // Step 5: the same reduction over the slots in every block
        PKey m = K;
        int mj = -1;
        double mpos[kResPos];
        for (unsigned int j = tid; j < nblk; j += TB) {
            const unsigned char* sl = slots + ((size_t)(k & 1) * nblk + j) * rec;
            const PKey* pk = reinterpret_cast<const PKey*>(sl);
            PKey c;
            c.k = __ldcg(&pk->k);
            c.i = __ldcg(&pk->i);
            c.pad = 0u;
            double q[kResPos];
            if (D <= kResPos) {
#pragma unroll
                for (int d = 0; d < kResPos; ++d)
                    q[d] = d < D ? __ldcg(reinterpret_cast<const double*>(sl + sizeof(PKey)) + d) : 0.0;
            }
            if (key_less(c, m)) {
                m = c;
                mj = (int)j;
#pragma unroll
                for (int d = 0; d < kResPos; ++d) mpos[d] = D <= kResPos ? q[d] : 0.0;
            }
        }
        const PKey nbest = block_min_key(m, red);
        if (key_less(nbest, K)) {
            // the thread that read the winning slot brings its position
            if (mj >= 0 && m.i == nbest.i && m.k == nbest.k) {
                if (D <= kResPos) {
#pragma unroll
                    for (int d = 0; d < kResPos; ++d)
                        if (d < D) Gsh[d] = mpos[d];
                } else {
                    const double* pos =
                        reinterpret_cast<const double*>(slots + ((size_t)(k & 1) * nblk + mj) * rec + sizeof(PKey));
                    for (int d = 0; d < D; ++d) Gsh[d] = __ldcg(pos + d);
                }
            }
            K = nbest;
        }
        __syncthreads();
        done = k + 1;
    }
    if (own) {
        s.pf[i] = pf;
        for (int d = 0; d < D; ++d) {
            const size_t g = (size_t)d * Np + i;
            s.x[g] = X[d * TB + tid];
            s.v[g] = V[d * TB + tid];
            s.pb[g] = PB[d * TB + tid];
        }
    }
    if (__syncthreads_or(nan) && tid == 0) atomicOr(s.status, kStatusNaN);
    if (blockIdx.x == 0) {
        const uint32_t t_end = t_prev + (uint32_t)done;
        const int out = (int)(t_end & 1u);
        for (int d = tid; d < D; d += TB) s.G[(size_t)out * D + d] = Gsh[d];
        if (tid == 0) {
            Fp64::store_gkey(s, 0, K);
            Fp64::store_gkey(s, 1, K);
            *s.t_dev = t_end;
        }
    }
}

#define CUPSO_DISPATCH_FIT32(fid, CALL)            \
    switch (fid) {                                 \
        case kSphere: { constexpr int F = kSphere; CALL; break; }         \
        case kRastrigin: { constexpr int F = kRastrigin; CALL; break; }   \
        case kAckley: { constexpr int F = kAckley; CALL; break; }         \
        case kRosenbrock: { constexpr int F = kRosenbrock; CALL; break; } \
        case kCubicMax: { constexpr int F = kCubicMax; CALL; break; }     \
        default: return cudaErrorInvalidValue;     \
    }

#define CUPSO_DISPATCH_FIT64(fid, CALL)            \
    switch (fid) {                                 \
        case kSphere: { constexpr int F = kSphere; CALL; break; }         \
        case kRosenbrock: { constexpr int F = kRosenbrock; CALL; break; } \
        case kCubicMax: { constexpr int F = kCubicMax; CALL; break; }     \
        default: return cudaErrorInvalidValue;     \
    }

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

size_t paper_bufs_bytes(int Np, int list_cap) {
    const size_t nb = (size_t)paper_blocks(Np);
    return al256(sizeof(PKey) * nb) + al256(sizeof(PKey) * (size_t)list_cap) + 256;
}

PaperBufs paper_bufs_at(void* base, int Np, int list_cap) {
    const size_t nb = (size_t)paper_blocks(Np);
    char* p = static_cast<char*>(base);
    PaperBufs b;
    b.aux = reinterpret_cast<PKey*>(p);
    p += al256(sizeof(PKey) * nb);
    b.list = reinterpret_cast<PKey*>(p);
    b.list_cap = (unsigned int)list_cap;
    p += al256(sizeof(PKey) * (size_t)list_cap);
    unsigned int* w = reinterpret_cast<unsigned int*>(p);
    b.lock = w;
    b.ticket = w + 1;
    b.list_n = w + 2;
    b.bar_count = w + 3;
    b.bar_gen = w + 4;
    return b;
}

cudaError_t launch_queue_step(const SwarmDev& s, const PaperBufs& b, int fid, bool lock, cudaStream_t st) {
    const int nb = paper_blocks(s.N);
    if (lock) {
        CUPSO_DISPATCH_FIT32(fid, return launch_pdl(paper_step_kernel<Fp32, F, kAggQueueLock>, dim3(nb),
                                                    dim3(kPaperBlock), 0, st, s, b));
    }
    cudaError_t e = cudaSuccess;
    CUPSO_DISPATCH_FIT32(fid, e = launch_pdl(paper_step_kernel<Fp32, F, kAggQueue>, dim3(nb), dim3(kPaperBlock), 0, st,
                                             s, b));
    if (e != cudaSuccess) return e;
    return launch_pdl(paper_finish_kernel<Fp32, kAggQueue, true>, dim3(1), dim3(1024), 0, st, s, b, nb);
}

bool fp64_fitness_supported(int fid) { return fid == kSphere || fid == kRosenbrock || fid == kCubicMax; }

cudaError_t launch_init64(const SwarmDev64& s, const PaperBufs& b, int fid, cudaStream_t st) {
    const int nb = paper_blocks(s.N);
    CUPSO_DISPATCH_FIT64(fid, (init64_kernel<F><<<nb, kPaperBlock, 0, st>>>(s, b)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    paper_finish_kernel<Fp64, kAggReduce, false><<<1, 1024, 0, st>>>(s, b, nb);
    return cudaGetLastError();
}

cudaError_t launch_recompute64(const SwarmDev64& s, const PaperBufs& b, cudaStream_t st) {
    const int nb = paper_blocks(s.N);
    pbest_min64_kernel<<<nb, kPaperBlock, 0, st>>>(s, b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    paper_finish_kernel<Fp64, kAggReduce, false><<<1, 1024, 0, st>>>(s, b, nb);
    return cudaGetLastError();
}

cudaError_t launch_step64(const SwarmDev64& s, const PaperBufs& b, int fid, int agg, int num_sms, cudaStream_t st) {
    const int nb = paper_blocks(s.N);
    if ((unsigned int)nb > b.list_cap) return cudaErrorInvalidConfiguration;
    if (agg == kAggSyncList && s.D >= kTileMinD && s.D <= kTileItems) {
        const int P = tile_particles(s.N, s.D, num_sms);
        const int tiles = (s.N + P - 1) / P;
        if ((unsigned int)tiles > b.list_cap) return cudaErrorInvalidConfiguration;
        const int threads = P * s.D >= 256 ? 256 : (P * s.D + 31) / 32 * 32;
        CUPSO_DISPATCH_FIT64(fid, return launch_pdl(sync64_tile_kernel<F>, dim3(tiles), dim3(threads), 0, st, s, b, P));
    }
    const dim3 g1(nb), b1(kPaperBlock), g2(1), b2(1024);
    cudaError_t e = cudaSuccess;
    switch (agg) {
        case kAggReduce:
            CUPSO_DISPATCH_FIT64(fid, e = launch_pdl(paper_step_kernel<Fp64, F, kAggReduce>, g1, b1, 0, st, s, b));
            if (e != cudaSuccess) return e;
            return launch_pdl(paper_finish_kernel<Fp64, kAggReduce, true>, g2, b2, 0, st, s, b, nb);
        case kAggReduceUnrolled:
            CUPSO_DISPATCH_FIT64(fid, e = launch_pdl(paper_step_kernel<Fp64, F, kAggReduceUnrolled>, g1, b1, 0, st, s, b));
            if (e != cudaSuccess) return e;
            return launch_pdl(paper_finish_kernel<Fp64, kAggReduceUnrolled, true>, g2, b2, 0, st, s, b, nb);
        case kAggQueue:
            CUPSO_DISPATCH_FIT64(fid, e = launch_pdl(paper_step_kernel<Fp64, F, kAggQueue>, g1, b1, 0, st, s, b));
            if (e != cudaSuccess) return e;
            return launch_pdl(paper_finish_kernel<Fp64, kAggQueue, true>, g2, b2, 0, st, s, b, nb);
        case kAggQueueLock:
            CUPSO_DISPATCH_FIT64(fid, return launch_pdl(paper_step_kernel<Fp64, F, kAggQueueLock>, g1, b1, 0, st, s, b));
        case kAggSyncList:
            CUPSO_DISPATCH_FIT64(fid, return launch_pdl(paper_step_kernel<Fp64, F, kAggSyncList>, g1, b1, 0, st, s, b));
        default:
            return cudaErrorInvalidValue;
    }
}

int persist64_grid(int fid, int N, int D, int num_sms) {
    int per_sm = 0;
    const size_t smem = sizeof(double) * (size_t)D;
    cudaError_t e = cudaErrorInvalidValue;
    switch (fid) {
        case kSphere: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist64_kernel<kSphere>, kPersistThreads, smem); break;
        case kRosenbrock: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist64_kernel<kRosenbrock>, kPersistThreads, smem); break;
        case kCubicMax: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist64_kernel<kCubicMax>, kPersistThreads, smem); break;
        default: break;
    }
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long long want = ((long long)N + kPersistThreads - 1) / kPersistThreads;
    const long long cap = (long long)per_sm * num_sms;
    return (int)(want < cap ? want : cap);
}

namespace {

const void* persist64r_fn(int fid) {
    switch (fid) {
        case kSphere: return (const void*)persist64r_kernel<kSphere>;
        case kRosenbrock: return (const void*)persist64r_kernel<kRosenbrock>;
        case kCubicMax: return (const void*)persist64r_kernel<kCubicMax>;
        default: return nullptr;
    }
}

// Threads per block of the resident variant (one particle each, at most one
// block per SM, block size from 128 doubling to 512), or 0 where it does not
// apply: too many particles, state over 48 KB per block, slots beyond the
// candidate list, or blocks that cannot all be resident.
int persist64r_block(int fid, int N, int D, int num_sms, unsigned int list_cap) {
    int tb = 128;
    while ((N + tb - 1) / tb > num_sms && tb < 512) tb *= 2;
    const int nblk = (N + tb - 1) / tb;
    if (nblk > num_sms) return 0;
    const size_t smem = sizeof(double) * (3 * (size_t)D * tb + (size_t)D);
    if (smem > 48 * 1024) return 0;
    if (2 * (size_t)nblk * res_slot_bytes(D) > sizeof(PKey) * (size_t)list_cap) return 0;
    const void* fn = persist64r_fn(fid);
    int per_sm = 0;
    if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, tb, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (long long)per_sm * num_sms >= nblk ? tb : 0;
}

}  // namespace

cudaError_t launch_persist64(const SwarmDev64& s, const PaperBufs& b, int fid, int iters, int num_sms,
                             cudaStream_t st) {
    if (s.D > 4096) return cudaErrorInvalidValue;
    if (const int tb = persist64r_block(fid, s.N, s.D, num_sms, b.list_cap)) {
        const int nblk = (s.N + tb - 1) / tb;
        const size_t smem = sizeof(double) * (3 * (size_t)s.D * tb + (size_t)s.D);
        for (int left = iters; left > 0;) {
            // the barrier counter starts every launch at zero
            cudaError_t me = cudaMemsetAsync(b.bar_count, 0, sizeof(unsigned int), st);
            if (me != cudaSuccess) return me;
            int iters_arg = left < kResMaxIters ? left : kResMaxIters;
            left -= iters_arg;
            SwarmDev64 s_arg = s;
            PaperBufs b_arg = b;
            void* args[] = {&s_arg, &b_arg, &iters_arg};
            cudaError_t e = cudaLaunchCooperativeKernel(persist64r_fn(fid), dim3(nblk), dim3(tb), args, smem, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const int grid = persist64_grid(fid, s.N, s.D, num_sms);
    if (2u * (unsigned)grid > b.list_cap) return cudaErrorInvalidConfiguration;
    // a barrier abandoned by a timed-out launch must not leave arrivals behind
    cudaError_t me = cudaMemsetAsync(b.bar_count, 0, sizeof(unsigned int), st);
    if (me != cudaSuccess) return me;
    const size_t smem = sizeof(double) * (size_t)s.D;
    int iters_arg = iters;
    SwarmDev64 s_arg = s;
    PaperBufs b_arg = b;
    void* args[] = {&s_arg, &b_arg, &iters_arg};
    switch (fid) {
        case kSphere:
            return cudaLaunchCooperativeKernel((const void*)persist64_kernel<kSphere>, dim3(grid), dim3(kPersistThreads),
                                               args, smem, st);
        case kRosenbrock:
            return cudaLaunchCooperativeKernel((const void*)persist64_kernel<kRosenbrock>, dim3(grid),
                                               dim3(kPersistThreads), args, smem, st);
        case kCubicMax:
            return cudaLaunchCooperativeKernel((const void*)persist64_kernel<kCubicMax>, dim3(grid),
                                               dim3(kPersistThreads), args, smem, st);
        default:
            return cudaErrorInvalidValue;
    }
}

namespace {

int max_optin_smem64() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return v;
}

int threads_for(int P, int D) {
    const long long work = (long long)P * D;
    int th = (int)((work + 31) / 32 * 32);
    return th < 32 ? 32 : (th > kOnchip64Threads ? kOnchip64Threads : th);
}

template <int FIT>
cudaError_t set_onchip64_attrs(size_t smem, int C) {
    cudaError_t e = cudaFuncSetAttribute(onchip64_kernel<FIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && C > 8)
        e = cudaFuncSetAttribute(onchip64_kernel<FIT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

cudaLaunchConfig_t onchip64_config(int C, int threads, size_t smem, cudaStream_t st, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

bool cluster64_schedulable(int N, int D, int C) {
    const Onchip64Layout L = onchip64_layout(N, D, C);
    if (set_onchip64_attrs<kSphere>(L.bytes, C) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = onchip64_config(C, threads_for(L.P, D), L.bytes, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, onchip64_kernel<kSphere>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

}  // namespace

// CTAs of the on-chip cluster for (N, D), or 0 if the swarm does not fit: the
// power of two that gives each CTA about 128 (particle, dimension) pairs (so
// the FP64 work of an iteration spreads over that many SMs), at least the
// smallest count whose shared memory fits, at most 16.
int onchip64_cluster(int N, int D) {
    const int limit = max_optin_smem64() - 1024;   // room for the static shared arrays
    if (limit <= 0) return 0;
    const long long pd = (long long)N * D;
    int C = 1;
    while (C < kMaxCluster64 && pd > 128ll * C && C < N) C *= 2;
    while (C <= kMaxCluster64 && onchip64_layout(N, D, C).bytes > (size_t)limit) C *= 2;
    if (C > kMaxCluster64) return 0;
    const int C_min = C;
    while (C >= 1 && !cluster64_schedulable(N, D, C)) C /= 2;
    if (C < 1 || onchip64_layout(N, D, C).bytes > (size_t)limit) return 0;
    (void)C_min;
    return C;
}

bool onchip64_fits(int N, int D) { return onchip64_cluster(N, D) > 0; }

cudaError_t launch_onchip64(const SwarmDev64& s, int fid, int iters, cudaStream_t st) {
    const int C = onchip64_cluster(s.N, s.D);
    if (C <= 0) return cudaErrorInvalidConfiguration;
    const Onchip64Layout L = onchip64_layout(s.N, s.D, C);
    const int threads = threads_for(L.P, s.D);
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = onchip64_config(C, threads, L.bytes, st, attr);
    switch (fid) {
        case kSphere: {
            cudaError_t e = set_onchip64_attrs<kSphere>(L.bytes, C);
            return e != cudaSuccess ? e : cudaLaunchKernelEx(&cfg, onchip64_kernel<kSphere>, s, iters);
        }
        case kRosenbrock: {
            cudaError_t e = set_onchip64_attrs<kRosenbrock>(L.bytes, C);
            return e != cudaSuccess ? e : cudaLaunchKernelEx(&cfg, onchip64_kernel<kRosenbrock>, s, iters);
        }
        case kCubicMax: {
            cudaError_t e = set_onchip64_attrs<kCubicMax>(L.bytes, C);
            return e != cudaSuccess ? e : cudaLaunchKernelEx(&cfg, onchip64_kernel<kCubicMax>, s, iters);
        }
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace cupso
