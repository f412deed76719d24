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
#include <cuda_runtime.h>

#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "paper_kernels.h"
#include "stream_common.cuh"

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

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// ---------------------------------------------------------------------------
// Double precision building blocks
// ---------------------------------------------------------------------------

// Two words -> (m + 1) 2^-53 with m = hi 2^21 + (lo >> 11), in (0, 1]. The
// double is assembled from integer parts: exponent from the leading bit of
// v = m + 1, the bits below it as the fraction (v <= 2^53, so it is exact).
__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
    const unsigned long long v = (((unsigned long long)hi << 21) | (unsigned long long)(lo >> 11)) + 1ull;
    const int lz = __clzll((long long)v);
    const unsigned long long frac = ((v << lz) << 1) >> 12;
    const unsigned long long e = (unsigned long long)(1033 - lz);
    return __longlong_as_double((long long)((e << 52) | frac));
}

__device__ __forceinline__ double clampd(double a, double lo, double hi) {
    if (a != a) return lo;
    return a < lo ? lo : (a > hi ? hi : a);
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

// Eq. 1 and Eq. 2 in binary64 with the clamps of Alg. 1 (same order as FP32).
__device__ __forceinline__ void move_one64(double& x, double& v, double pb, double g, double r1, double r2,
                                           const SwarmDev64& s) {
    const double cognitive = __dsub_rn(pb, x);
    const double social = __dsub_rn(g, x);
    double vel = __dmul_rn(s.w, v);
    vel = __fma_rn(__dmul_rn(s.c1, r1), cognitive, vel);
    vel = __fma_rn(__dmul_rn(s.c2, r2), social, vel);
    v = clampd(vel, -s.vmax, s.vmax);
    x = clampd(__dadd_rn(x, v), s.lo, s.hi);
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
            move_one64(x, v, s.pb[off], G[d], u53(r.x, r.y), u53(r.z, r.w), s);
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
        if (tid == 0 && k.i != kNoIdx) b.list[atomicAdd(b.list_n, 1u)] = k;
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
            const unsigned int n = __ldcg(b.list_n);
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
            const double x = clampd(__fma_rn(u53(r.x, r.y), span, s.lo), s.lo, s.hi);
            const double v = clampd(__fma_rn(u53(r.z, r.w), vspan, -s.vmax), -s.vmax, s.vmax);
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
// On-chip FP64 swarm: x, v, pbest_pos ([D][N]), pbest_fit and gbest stay in
// one CTA's shared memory for `iters` iterations; the kernel boundary of the
// paper's designs becomes a block barrier.
// ---------------------------------------------------------------------------
constexpr int kOnchip64Threads = 1024;

__host__ __device__ inline size_t onchip64_bytes(int N, int D) {
    return sizeof(double) * (3 * (size_t)N * (size_t)D + (size_t)N + (size_t)D) + sizeof(PKey) * 32;
}

template <int FIT>
__global__ void __launch_bounds__(kOnchip64Threads) onchip64_kernel(const __grid_constant__ SwarmDev64 s, int iters) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = s.N, D = s.D;
    const size_t ND = (size_t)N * (size_t)D;
    double* x = reinterpret_cast<double*>(smem);   // [D][N]
    double* v = x + ND;
    double* pb = v + ND;
    double* pf = pb + ND;                          // [N]
    double* G = pf + N;                            // [D]
    PKey* red = reinterpret_cast<PKey*>(G + D);    // [32]
    const size_t Np = (size_t)s.Np;
    const int tid = threadIdx.x;
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur0 = (int)(t_prev & 1u);

    for (size_t e = tid; e < ND; e += blockDim.x) {
        const size_t d = e / (size_t)N, p = e - d * (size_t)N;
        x[e] = s.x[d * Np + p];
        v[e] = s.v[d * Np + p];
        pb[e] = s.pb[d * Np + p];
    }
    for (int p = tid; p < N; p += blockDim.x) pf[p] = s.pf[p];
    for (int d = tid; d < D; d += blockDim.x) G[d] = s.G[(size_t)cur0 * D + d];
    PKey K = Fp64::load_gkey(s, cur0);
    __syncthreads();

    bool nan = false;
    for (int k = 0; k < iters; ++k) {
        const uint32_t t = t_prev + 1u + (uint32_t)k;
        // Step 2 for every (dimension, particle)
        for (size_t e = tid; e < ND; e += blockDim.x) {
            const uint32_t d = (uint32_t)(e / (size_t)N), p = (uint32_t)(e - (size_t)d * N);
            const uint4 r = philox4x32_10(make_uint4(d, p, t, s.swarm), s.key0, s.key1);
            double xx = x[e], vv = v[e];
            move_one64(xx, vv, pb[e], G[d], u53(r.x, r.y), u53(r.z, r.w), s);
            x[e] = xx;
            v[e] = vv;
        }
        __syncthreads();
        // Steps 3-4 per particle; the candidates of Step 5
        PKey cand = key_none();
        for (int p = tid; p < N; p += blockDim.x) {
            FitAcc64<FIT> acc;
            for (int d = 0; d < D; ++d) acc.add(d, x[(size_t)d * N + p]);
            const double f = acc.finish();
            nan |= (f != f);
            if (f < pf[p]) {
                pf[p] = f;
                for (int d = 0; d < D; ++d) pb[(size_t)d * N + p] = x[(size_t)d * N + p];
                const PKey c = Fp64::key(f, (uint32_t)p);
                if (key_less(c, cand)) cand = c;
            }
        }
        const PKey best = block_min_key(cand, red);   // barriers inside
        if (key_less(best, K)) {
            K = best;
            for (int d = tid; d < D; d += blockDim.x) G[d] = pb[(size_t)d * N + best.i];
        }
        __syncthreads();
    }
    for (size_t e = tid; e < ND; e += blockDim.x) {
        const size_t d = e / (size_t)N, p = e - d * (size_t)N;
        s.x[d * Np + p] = x[e];
        s.v[d * Np + p] = v[e];
        s.pb[d * Np + p] = pb[e];
    }
    for (int p = tid; p < N; p += blockDim.x) s.pf[p] = pf[p];
    const int out = (int)((t_prev + (uint32_t)iters) & 1u);
    for (int d = tid; d < D; d += blockDim.x) s.G[(size_t)out * D + d] = G[d];
    if (__syncthreads_or(nan) && tid == 0) atomicOr(s.status, kStatusNaN);
    if (tid == 0) {
        Fp64::store_gkey(s, 0, K);
        Fp64::store_gkey(s, 1, K);
        *s.t_dev = t_prev + (uint32_t)iters;
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

size_t paper_bufs_bytes(int Np) {
    const size_t nb = (size_t)paper_blocks(Np);
    return 2 * al256(sizeof(PKey) * nb) + 256;
}

PaperBufs paper_bufs_at(void* base, int Np) {
    const size_t nb = (size_t)paper_blocks(Np);
    char* p = static_cast<char*>(base);
    PaperBufs b;
    b.aux = reinterpret_cast<PKey*>(p);
    p += al256(sizeof(PKey) * nb);
    b.list = reinterpret_cast<PKey*>(p);
    p += al256(sizeof(PKey) * nb);
    unsigned int* w = reinterpret_cast<unsigned int*>(p);
    b.lock = w;
    b.ticket = w + 1;
    b.list_n = w + 2;
    return b;
}

cudaError_t launch_queue_step(const SwarmDev& s, const PaperBufs& b, int fid, bool lock, cudaStream_t st) {
    const int nb = paper_blocks(s.N);
    if (lock) {
        CUPSO_DISPATCH_FIT32(fid, (paper_step_kernel<Fp32, F, kAggQueueLock><<<nb, kPaperBlock, 0, st>>>(s, b)));
        return cudaGetLastError();
    }
    CUPSO_DISPATCH_FIT32(fid, (paper_step_kernel<Fp32, F, kAggQueue><<<nb, kPaperBlock, 0, st>>>(s, b)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    paper_finish_kernel<Fp32, kAggQueue, true><<<1, 1024, 0, st>>>(s, b, nb);
    return cudaGetLastError();
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

cudaError_t launch_step64(const SwarmDev64& s, const PaperBufs& b, int fid, int agg, cudaStream_t st) {
    const int nb = paper_blocks(s.N);
    switch (agg) {
        case kAggReduce:
            CUPSO_DISPATCH_FIT64(fid, (paper_step_kernel<Fp64, F, kAggReduce><<<nb, kPaperBlock, 0, st>>>(s, b)));
            break;
        case kAggReduceUnrolled:
            CUPSO_DISPATCH_FIT64(fid,
                                 (paper_step_kernel<Fp64, F, kAggReduceUnrolled><<<nb, kPaperBlock, 0, st>>>(s, b)));
            break;
        case kAggQueue:
            CUPSO_DISPATCH_FIT64(fid, (paper_step_kernel<Fp64, F, kAggQueue><<<nb, kPaperBlock, 0, st>>>(s, b)));
            break;
        case kAggQueueLock:
            CUPSO_DISPATCH_FIT64(fid, (paper_step_kernel<Fp64, F, kAggQueueLock><<<nb, kPaperBlock, 0, st>>>(s, b)));
            return cudaGetLastError();
        case kAggSyncList:
            CUPSO_DISPATCH_FIT64(fid, (paper_step_kernel<Fp64, F, kAggSyncList><<<nb, kPaperBlock, 0, st>>>(s, b)));
            return cudaGetLastError();
        default:
            return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (agg) {
        case kAggReduce: paper_finish_kernel<Fp64, kAggReduce, true><<<1, 1024, 0, st>>>(s, b, nb); break;
        case kAggReduceUnrolled: paper_finish_kernel<Fp64, kAggReduceUnrolled, true><<<1, 1024, 0, st>>>(s, b, nb); break;
        default: paper_finish_kernel<Fp64, kAggQueue, true><<<1, 1024, 0, st>>>(s, b, nb); break;
    }
    return cudaGetLastError();
}

bool onchip64_fits(int N, int D) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    return onchip64_bytes(N, D) <= (size_t)optin;
}

cudaError_t prepare_onchip64() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(onchip64_kernel<kSphere>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(onchip64_kernel<kRosenbrock>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(onchip64_kernel<kCubicMax>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    return e;
}

cudaError_t launch_onchip64(const SwarmDev64& s, int fid, int iters, cudaStream_t st) {
    const size_t smem = onchip64_bytes(s.N, s.D);
    const size_t work = (size_t)s.N * (size_t)s.D;
    int threads = (int)((work + 31) / 32 * 32);
    if (threads > kOnchip64Threads) threads = kOnchip64Threads;
    if (threads < 32) threads = 32;
    CUPSO_DISPATCH_FIT64(fid, (onchip64_kernel<F><<<1, threads, smem, st>>>(s, iters)));
    return cudaGetLastError();
}

}  // namespace cupso
