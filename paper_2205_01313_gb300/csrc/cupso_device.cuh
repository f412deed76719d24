// cupso_device.cuh -- device building blocks of the PSO iteration (sm_103a).
//
// Every floating-point step below is an explicit round-to-nearest intrinsic in
// a fixed order, so the synchronous path reproduces, bit for bit, the FP32
// reading of Eq. 1 (velocity), Eq. 2 (position) and Alg. 1 steps 3-5 (Sec. 2.1)
// that the CPU oracle computes. The file is compiled with -fmad=false as well.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cupso {

// ---------------------------------------------------------------------------
// Device state of one swarm. Positions, velocities and personal bests are
// dimension-major [D][Np] (structure of arrays, Sec. 4.1 and Fig. 2): the
// threads of a warp touch consecutive particles of one dimension, and each
// thread moves four particles with one 16-byte access.
// ---------------------------------------------------------------------------
struct SwarmDev {
    float* x;            // [D][Np] pos
    float* v;            // [D][Np] velocity
    float* pb;           // [D][Np] pbest_pos
    float* pf;           // [Np]    pbest_fit
    float* G;            // [2][D]  gbest_pos, double-buffered by iteration parity
    unsigned long long* gkey;   // [2] packed (order key of gbest_fit << 32 | index)
    unsigned int* ticket;       // last-CTA-done counter
    unsigned int* t_dev;        // iterations completed
    unsigned int* status;       // sticky error bits (kStatus*)
    unsigned long long* aux;    // tree baseline: one key per block of the first kernel
    unsigned int* work;         // pipelined step: next 128-particle unit to hand out
    unsigned int* bar;          // panel step over several iterations: grid-barrier counter
    // Lazy pbest (pipelined step): byte i is 1 when particle i improved in the
    // last iteration and its pbest_pos row has not been written yet; its
    // pbest_pos is then its pos. NULL or all-zero means pb is complete.
    unsigned char* pflag;       // [Np]
    // asynchronous variant: lock-protected gbest record read under a sequence lock
    float* Grec;                // [D]
    unsigned long long* claim;  // lowest key claimed so far (atomicMin target)
    unsigned long long* reckey; // key of the record in Grec
    unsigned int* lock;
    unsigned int* seq;
    int N, D, Np;
    float lo, hi, vmax, w, c1, c2;
    uint32_t key0, key1, swarm;
    long long wait_limit_ns;    // bound of every device-side wait
    // c1 * 2^-24 and c2 * 2^-24 (exact): c * r with r = (k + 1) 2^-24 is then
    // fma(cs, k, cs), one rounding of the same product. Valid when fast_cr.
    float c1s, c2s;
    int fast_cr;                // c1s, c2s exact (normal or zero)
    int fast_clamp;             // no bound is +-0: clampf_minmax == clampf
    // Philox round keys (key0 + r W0, key1 + r W1 for rounds r = 0..9), the same
    // for every draw of the swarm: kernels that take them from here (the
    // parameter space) skip the key additions of each round
    uint32_t rk0[10], rk1[10];
};

// One swarm of a batch (kernels_batch.cu): its state in the batch arena and
// its parameters. Same layouts as SwarmDev.
struct BatchSwarm {
    float *x, *v, *pb, *pf;
    unsigned char* pflag;
    float* G;                   // [2][D]
    unsigned long long* gkey;   // [2]
    unsigned int* done;         // units of this swarm finished in the current iteration
    unsigned int* status;
    int N, D, Np, fid;
    unsigned int nunits;        // Np / 128
    float lo, hi, vmax, w, c1, c2, c1s, c2s;
    uint32_t key0, key1, swarm;
    int fast;                   // fast_cr && fast_clamp
};

struct BatchDev {
    const BatchSwarm* swarms;
    const uint2* units;         // (swarm, unit) in hand-out order
    unsigned int nunits;
    unsigned int* work;         // [2] unit counters, alternating by iteration parity
    unsigned int* ticket;
    unsigned int* t_dev;
};

constexpr unsigned int kStatusNaN = 1u;
constexpr unsigned int kStatusTimeout = 2u;
constexpr unsigned int kStatusBadArg = 4u;

constexpr unsigned long long kKeyNone = ~0ull;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter-based, so the
// draw of (dimension pair, particle, iteration, swarm) needs no state.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += W0;
        k1 += W1;
    }
    return c;
}

// The same function with the round keys given (rk0[r] = k0 + r W0, rk1[r] =
// k1 + r W1 modulo 2^32): identical words.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t (&rk0)[10], const uint32_t (&rk1)[10]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ rk0[r], lo1, hi0 ^ c.w ^ rk1[r], lo0);
    }
    return c;
}

// Host side: the round keys of key (k0, k1).
inline void philox_round_keys(uint32_t k0, uint32_t k1, uint32_t (&rk0)[10], uint32_t (&rk1)[10]) {
    for (int r = 0; r < 10; ++r) {
        rk0[r] = k0 + (uint32_t)r * 0x9E3779B9u;
        rk1[r] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
}

// One 32-bit word -> ((w >> 8) + 1) * 2^-24 in (0, 1]. (w >> 8) converts
// exactly, and the fma adds 2^-24 exactly: the result is a multiple of 2^-24.
__device__ __forceinline__ float u01(uint32_t w) {
    return __fmaf_rn(__uint2float_rn(w >> 8), 0x1p-24f, 0x1p-24f);
}

// ---------------------------------------------------------------------------
// Own cos(2 pi x) and exp(y): range reduction + Taylor polynomial, constants
// rounded once to float32 (gen_constants.py prints them).
//   cos(2 pi a) = sum_j (-1)^j (2 pi)^(2j)/(2j)! a^(2j), j <= 7, 0 <= a <= 1/4
//   exp(r) = sum_k r^k/k!, k <= 8, after y = n ln2 + r (Cody and Waite)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float cos2pi_poly(float a) {
    const float z = __fmul_rn(a, a);
    float q = -0x1.b6e25p+0f;                 // c7
    q = __fmaf_rn(q, z, 0x1.f9d38ap+2f);      // c6
    q = __fmaf_rn(q, z, -0x1.a6d1f2p+4f);     // c5
    q = __fmaf_rn(q, z, 0x1.e1f506p+5f);      // c4
    q = __fmaf_rn(q, z, -0x1.55d3c8p+6f);     // c3
    q = __fmaf_rn(q, z, 0x1.03c1fp+6f);       // c2
    q = __fmaf_rn(q, z, -0x1.3bd3ccp+4f);     // c1
    q = __fmaf_rn(q, z, 0x1p+0f);             // c0
    return q;
}

__device__ __forceinline__ float cos2pi(float x) {
    // x - rint(x) is exact; |r| <= 1/2. cos is even; for a > 1/4 use
    // cos(2 pi a) = -cos(2 pi (1/2 - a)), and 1/2 - a is exact (Sterbenz).
    const float r = __fsub_rn(x, rintf(x));
    const float a = fabsf(r);
    if (a > 0.25f) return -cos2pi_poly(__fsub_rn(0.5f, a));
    return cos2pi_poly(a);
}

__device__ __forceinline__ float exp_own(float y) {
    if (y != y) return y;
    if (y > 88.8f) return __int_as_float(0x7f800000);
    if (y < -104.0f) return 0.0f;
    const float n = rintf(__fmul_rn(y, 0x1.715476p+0f));           // y * log2(e)
    float r = __fmaf_rn(-n, 0x1.62e4p-1f, y);                        // - n ln2_hi (exact product)
    r = __fmaf_rn(-n, 0x1.7f7d1cp-20f, r);                           // - n ln2_lo
    float q = 0x1.a01a02p-16f;                                       // 1/8!
    q = __fmaf_rn(q, r, 0x1.a01a02p-13f);                            // 1/7!
    q = __fmaf_rn(q, r, 0x1.6c16c2p-10f);                            // 1/6!
    q = __fmaf_rn(q, r, 0x1.111112p-7f);                             // 1/5!
    q = __fmaf_rn(q, r, 0x1.555556p-5f);                             // 1/4!
    q = __fmaf_rn(q, r, 0x1.555556p-3f);                             // 1/3!
    q = __fmaf_rn(q, r, 0x1p-1f);                                    // 1/2!
    q = __fmaf_rn(q, r, 0x1p+0f);                                    // 1/1!
    q = __fmaf_rn(q, r, 0x1p+0f);                                    // 1/0!
    // q * 2^n as two normal powers of two (n in [-150, 128] here).
    const int ni = (int)n;
    const int n1 = ni / 2;
    const int n2 = ni - n1;
    const float s1 = __int_as_float((n1 + 127) << 23);
    const float s2 = __int_as_float((n2 + 127) << 23);
    return __fmul_rn(__fmul_rn(q, s1), s2);
}

// ---------------------------------------------------------------------------
// Fitness functions (Step 3), accumulated dimension by dimension in order
// d = 0 .. D-1 from 0.0f. Lower is better; the paper's cubic (Eq. 3) is
// maximised there, so it is minimised here as its negation.
// ---------------------------------------------------------------------------
enum FitnessId : int { kSphere = 0, kRastrigin = 1, kAckley = 2, kRosenbrock = 3, kCubicMax = 4, kLsq = 5 };

template <int FIT>
struct FitAcc {
    float acc = 0.0f;  // sphere, Rastrigin, Rosenbrock, cubic
    float acc2 = 0.0f; // Ackley: sum of cos(2 pi x)
    float prev = 0.0f; // Rosenbrock: x_{d-1}

    // c = cos2pi(x); only Rastrigin and Ackley use it.
    static constexpr bool kNeedsCos = (FIT == kRastrigin || FIT == kAckley);

    __device__ __forceinline__ void add(int d, float x) {
        if constexpr (kNeedsCos) add_c(d, x, cos2pi(x));
        else add_c(d, x, 0.0f);
    }

    __device__ __forceinline__ void add_c(int d, float x, float c) {
        if constexpr (FIT == kSphere) {
            acc = __fmaf_rn(x, x, acc);
        } else if constexpr (FIT == kRastrigin) {
            const float ten_minus = __fmaf_rn(-10.0f, c, 10.0f);
            acc = __fadd_rn(acc, __fmaf_rn(x, x, ten_minus));
        } else if constexpr (FIT == kAckley) {
            acc = __fmaf_rn(x, x, acc);
            acc2 = __fadd_rn(acc2, c);
        } else if constexpr (FIT == kRosenbrock) {
            if (d > 0) {
                const float p = __fmaf_rn(-prev, prev, x);
                const float q = __fsub_rn(1.0f, prev);
                acc = __fadd_rn(acc, __fmaf_rn(__fmul_rn(100.0f, p), p, __fmul_rn(q, q)));
            }
            prev = x;
        } else if constexpr (FIT == kCubicMax) {
            const float h = __fmaf_rn(__fmaf_rn(__fsub_rn(x, 0.8f), x, -1000.0f), x, 8000.0f);
            acc = __fadd_rn(acc, h);
        }
        // kLsq: the least-squares fitness is a separate matrix product (kernels_lsq.cu)
    }

    __device__ __forceinline__ float finish(int D) const {
        if constexpr (FIT == kAckley) {
            const float fD = (float)D;
            const float m1 = __fdiv_rn(acc, fD);
            const float m2 = __fdiv_rn(acc2, fD);
            const float e1 = exp_own(__fmul_rn(-0.2f, __fsqrt_rn(m1)));
            const float part1 = __fsub_rn(20.0f, __fmul_rn(20.0f, e1));
            const float part2 = __fsub_rn(exp_own(1.0f), exp_own(m2));
            return __fadd_rn(part1, part2);
        } else if constexpr (FIT == kCubicMax) {
            return -acc;
        } else if constexpr (FIT == kLsq) {
            return __int_as_float(0x7f800000);   // evaluated later, by the matrix product
        } else {
            return acc;
        }
    }
};

// ---------------------------------------------------------------------------
// Ordering: an order-preserving 32-bit key of a fitness value (NaN last,
// -0 == +0) packed above the particle index. The minimum packed key is the
// lexicographic argmin over (pbest_fit, index): ties go to the lowest index.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t fit_key(float f) {
    if (f != f) return 0xFFFFFFFFu;
    uint32_t b = __float_as_uint(f);
    if ((b << 1) == 0u) b = 0u;  // -0 -> +0
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ unsigned long long pack_key(float f, uint32_t i) {
    return ((unsigned long long)fit_key(f) << 32) | (unsigned long long)i;
}

// Closed clamp to [lo, hi]; a NaN goes to the lower bound (IEEE maxNum).
// Written with comparisons, valid for any bounds.
__device__ __forceinline__ float clampf(float a, float lo, float hi) {
    if (a != a) return lo;
    return a < lo ? lo : (a > hi ? hi : a);
}

// The same clamp as two min/max instructions. Equal to clampf for every a
// when neither bound is +-0 (then no signed-zero tie can reach fmaxf/fminf).
__device__ __forceinline__ float clampf_minmax(float a, float lo, float hi) {
    return fminf(fmaxf(a, lo), hi);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, k, o);
        k = other < k ? other : k;
    }
    return k;
}

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace cupso
