// kernels_lsq.cu -- least-squares fitness f_i = ||A x_i - b||^2 of a whole swarm.
//
// For the dense fitness the swarm's Step 3 is a matrix product: with X the
// N x D matrix of positions, the residuals are R = X A^T - 1 b^T (N x M) and
// f_i = sum_m R_im^2. Three implementations:
//
//  * lsq_fp32_kernel: plain FP32 on the CUDA cores, every residual a chain of
//    fma over d in order and the squares summed over m in order -- the same
//    rounding as the oracle, so its trajectories match bit for bit.
//  * lsq_tc_kernel<false>: BF16 operands on the 5th-generation tensor cores
//    (tcgen05.mma, FP32 accumulation in tensor memory), operands staged by TMA
//    with 128-byte swizzle, and the epilogue (subtract b, square, sum over m)
//    fused onto the accumulator read-back.
//  * lsq_tc_kernel<true>: the same with FP8 e4m3 operands: A scaled per row,
//    X by one factor from the search bounds; the epilogue undoes the scales.
//
// The tensor-core kernel runs on pairs of SMs (clusters of two CTAs, MMAs of
// cta_group::2): a pair computes a tile of 256 particles x 256 residual rows,
// each CTA staging its own 128 particle rows and half of the 256 residual
// rows, so an SM takes in 32 KB of operands per 128-byte K step instead of
// the 48 KB a one-SM 128 x 256 tile needs, and the ring holds 6 stages.
// Warp-specialised: warp 0 of each CTA issues its TMA loads, warp 1 of the
// even CTA issues the MMAs (two accumulators alternating), warps 2-9 of both
// CTAs drain their half of the accumulator, two warps per TMEM lane quarter,
// each over 128 residual rows, in loads of 32 columns. Every mbarrier wait is
// bounded in time; on expiry the kernel records a timeout, frees its tensor
// memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "lsq_internal.h"
#include "tma_common.cuh"

namespace cupso {

namespace {

constexpr int BM = 128;          // particles per CTA (a pair's MMA M = 256)
constexpr int BN = 256;          // residual rows per tile (MMA N), 128 staged per CTA
constexpr int BNH = BN / 2;
constexpr int KB = 128;          // K bytes per stage: one 128-byte swizzle row
constexpr int STAGES = 6;
constexpr int kTcThreads = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int kEpiWarps = 8;
constexpr int X_BYTES = BM * KB; // 16 KB
constexpr int A_BYTES = BNH * KB; // 16 KB
constexpr int STAGE_BYTES = X_BYTES + A_BYTES;

// Address of the same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Tile copy into this CTA's shared memory, completing on an mbarrier that may
// sit in either CTA of the pair (cluster address).
// `policy` is an L2 cache policy (createpolicy).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, uint32_t cluster_bar,
                                            uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], "
        "[%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(cluster_bar), "l"(policy)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 bytes, 8-row atoms of 1024 bytes (stride byte offset), tile
// base 1024-byte aligned.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)(16u >> 4) << 16;            // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024u >> 4) << 32;          // stride byte offset: one 8-row atom
    d |= (uint64_t)1 << 46;                     // descriptor version of tcgen05
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulator, A and B K-major, M = 256 (the
// pair), N = 256. ab_fmt: BF16 = 1 for kind::f16, E4M3 = 0 for kind::f8f6f4.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t ab_fmt) {
    return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)((2 * BM) >> 4) << 24);
}

template <bool FP8>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (FP8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}
// Arrives on the barrier at this shared-memory offset in each CTA of `mask`
// once the MMAs issued so far are complete.
__device__ __forceinline__ void umma_commit(uint32_t bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            bar),
        "h"(mask)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane; the wait is in the
// same statement, so no register is read before the load has landed.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

}  // namespace

// Per-particle partial fitness over each block of 128 residual rows:
//   part[h][i] = sum over m in 128 h .. 128 h + 127 of (sum_d X[i,d] A[m,d] / scale_m + off[m])^2
// X: [Np][Kp] (K-major), A: [Mp][Kp], off: [Mp] (zero-padded rows contribute 0).
// With X the positions and off = -b this is ||A x - b||^2; with X the
// displacements x - c from a reference point c and off = A c - b (computed
// accurately elsewhere) it is the same function, ||A (x - c) + (A c - b)||^2,
// with the operand rounding scaled by |x - c| instead of |x|.
// Launched in clusters of two CTAs. Pair c (of gridDim.x / 2) takes tiles
// c, c + gridDim.x / 2, ... of the ceil(Np / 256) x (Mp / 256) tiles
// (residual-row tile fastest). CTA r of the pair stages particle rows
// 256 pb + 128 r .. + 127 and residual rows 256 mt + 128 r .. + 127; the MMA
// (issued by CTA 0) leaves particle row 128 r + lane of the tile, against all
// 256 residual rows, in lane `lane` of CTA r's tensor memory.
template <bool FP8>
__global__ void __launch_bounds__(kTcThreads, 1)
    lsq_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmA,
                  const float* __restrict__ off, const float* __restrict__ inv_scale, int Mp, int KT, int Np,
                  float* __restrict__ part, unsigned int* status, long long limit_ns) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base for the swizzled tiles (the same offset in both CTAs)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* base_ptr = smem_raw + (base - raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base_ptr + STAGES * STAGE_BYTES);
    // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2], drain; then the TMEM address slot.
    // full, tempty and drain are used in CTA 0 only; empty and tfull in both.
    const uint32_t bar0 = base + STAGES * STAGE_BYTES;
    auto full_bar = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (uint32_t)(STAGES + s); };
    auto tfull_bar = [&](int a) { return bar0 + 8u * (uint32_t)(2 * STAGES + a); };
    auto tempty_bar = [&](int a) { return bar0 + 8u * (uint32_t)(2 * STAGES + 2 + a); };
    const uint32_t drain_bar = bar0 + 8u * (uint32_t)(2 * STAGES + 4);
    volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars + 2 * STAGES + 5);
    __shared__ volatile int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t rank, pair, npairs;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(pair));
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(npairs));
    const int mtiles = Mp / BN;
    const int ntiles = ((Np + 2 * BM - 1) / (2 * BM)) * mtiles;
    const int nt = (int)pair < ntiles ? (ntiles - (int)pair + (int)npairs - 1) / (int)npairs : 0;
    // the jj-th tile of this pair: residual-row tile and 256-particle block
    auto tile_mt = [&](int jj) { return ((int)pair + jj * (int)npairs) % mtiles; };
    auto tile_pb = [&](int jj) { return ((int)pair + jj * (int)npairs) / mtiles; };

    if (threadIdx.x == 0) {
        prefetch_tensormap(&tmX);
        prefetch_tensormap(&tmA);
        s_fail = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull_bar(a), 1);
            mbar_init(tempty_bar(a), 2 * kEpiWarps);   // the epilogue warps of both CTAs
        }
        mbar_init(drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        // 512 columns in each CTA of the pair: two 128-lane x 256 FP32 accumulators
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void*)tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    cluster_sync();   // barriers of both CTAs initialised before any remote arrive
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int total = nt * KT;   // (tile, k-stage) steps
    int issued = 0;              // TMA stages issued (producer)
    const uint16_t both = 0x3;

    if (warp == 0) {
        if (lane == 0) {
            const int esz = FP8 ? 1 : 2;
            // A is the same in every launch and each tile of X is read by all
            // residual-row tiles: keep both in L2 ahead of the swarm state
            // that the move kernel streams between launches
            uint64_t keep;
            asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
            for (int step = 0; step < total; ++step) {
                const int s = step % STAGES, f = step / STAGES;
                if (f > 0 && !mbar_wait(empty_bar(s), (uint32_t)((f - 1) & 1), limit_ns)) {
                    atomicOr(status, kStatusTimeout);
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                const int jj = step / KT, kk = step % KT;
                // CTA 0's barrier counts the bytes of both CTAs' copies
                if (rank == 0) mbar_expect_tx(full_bar(s), (uint32_t)(2 * STAGE_BYTES));
                const uint32_t fb = cluster_addr(full_bar(s), 0);
                const uint32_t xs = base + (uint32_t)(s * STAGE_BYTES);
                tma_load_2d(xs, &tmX, kk * KB / esz, tile_pb(jj) * (2 * BM) + (int)rank * BM, fb, keep);
                tma_load_2d(xs + X_BYTES, &tmA, kk * KB / esz, tile_mt(jj) * BN + (int)rank * BNH, fb, keep);
                ++issued;
            }
            // CTA 0's barriers count both CTAs' copies: let the last ones land
            // (already consumed, so immediate, unless the pipeline stopped early)
            if (rank == 0)
                for (int step = issued - STAGES > 0 ? issued - STAGES : 0; step < issued; ++step)
                    mbar_wait(full_bar(step % STAGES), (uint32_t)((step / STAGES) & 1), limit_ns);
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            constexpr uint32_t idesc = make_idesc(FP8 ? 0u : 1u);
            constexpr uint32_t kstep_bytes = 32;   // 16 bf16 or 32 fp8 per MMA
            int step = 0;
            for (int jj = 0; jj < nt && !s_fail; ++jj) {
                const int a = jj & 1, u = jj >> 1;
                if (u > 0 && !mbar_wait(tempty_bar(a), (uint32_t)((u - 1) & 1), limit_ns)) {
                    atomicOr(status, kStatusTimeout);
                    s_fail = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(a * BN);
                for (int kk = 0; kk < KT; ++kk, ++step) {
                    const int s = step % STAGES, f = step / STAGES;
                    if (!mbar_wait(full_bar(s), (uint32_t)(f & 1), limit_ns)) {
                        atomicOr(status, kStatusTimeout);
                        s_fail = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t xs = base + (uint32_t)(s * STAGE_BYTES);
#pragma unroll
                    for (int k4 = 0; k4 < KB / (int)kstep_bytes; ++k4) {
                        const uint64_t ad = desc_sw128(xs + k4 * kstep_bytes);
                        const uint64_t bd = desc_sw128(xs + X_BYTES + k4 * kstep_bytes);
                        umma<FP8>(d_tmem, ad, bd, idesc, (kk > 0 || k4 > 0) ? 1u : 0u);
                    }
                    umma_commit(empty_bar(s), both);   // stage s is free in both CTAs once these are done
                }
                if (s_fail) break;
                umma_commit(tfull_bar(a), both);       // accumulator a holds tile jj in both CTAs
            }
            // every MMA issued has finished before tensor memory is released
            umma_commit(drain_bar, 0x1);
            if (!mbar_wait(drain_bar, 0u, limit_ns)) atomicOr(status, kStatusTimeout);
        }
        __syncwarp();
    } else {
        // epilogue: thread = one particle row of this CTA's half of the tile,
        // against residual rows 128 h .. 128 h + 127 of the tile
        const int q = warp & 3;                 // TMEM lane quarter this warp may access
        const int h = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        bool ok = true;
        for (int jj = 0; jj < nt; ++jj) {
            const int a = jj & 1, u = jj >> 1;
            const int mt = tile_mt(jj);
            const int i = tile_pb(jj) * (2 * BM) + (int)rank * BM + row;
            const size_t slot = (size_t)(2 * mt + h) * Np + i;
            // warp-uniform outcome: tcgen05.ld below needs the whole warp
            if (!__all_sync(0xFFFFFFFFu, mbar_wait(tfull_bar(a), (uint32_t)(u & 1), limit_ns))) {
                ok = false;
                if (i < Np) part[slot] = __int_as_float(0x7fc00000);
                break;
            }
            tc_fence_after();
            const int m0 = mt * BN + h * 128;
            float sum = 0.0f;
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * BN + h * 128);
#pragma unroll 1
            for (int c = 0; c < 128; c += 32) {
                // the offsets (and the FP8 scales) of these 32 rows, requested before the TMEM load
                float bb[32], sc[32];
#pragma unroll
                for (int e = 0; e < 32; e += 4) {
                    const float4 t = __ldg(reinterpret_cast<const float4*>(off + m0 + c + e));
                    bb[e] = t.x; bb[e + 1] = t.y; bb[e + 2] = t.z; bb[e + 3] = t.w;
                    if constexpr (FP8) {
                        const float4 z = __ldg(reinterpret_cast<const float4*>(inv_scale + m0 + c + e));
                        sc[e] = z.x; sc[e + 1] = z.y; sc[e + 2] = z.z; sc[e + 3] = z.w;
                    }
                }
                float v[32];
                tmem_ld32(taddr + (uint32_t)c, v);
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const float val = FP8 ? __fmul_rn(v[e], sc[e]) : v[e];
                    const float r = __fadd_rn(val, bb[e]);
                    sum = __fmaf_rn(r, r, sum);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(cluster_addr(tempty_bar(a), 0));
            if (i < Np) part[slot] = sum;
        }
        if (!ok) {
            if (lane == 0) atomicOr(status, kStatusTimeout);
            s_fail = 1;
        }
    }
    // CTA 0's MMAs read both CTAs' shared memory and the epilogues arrive on
    // CTA 0's barriers: neither CTA leaves or frees tensor memory before both
    // are done
    tc_fence_before();
    cluster_sync();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// Converts positions to the K-major tensor-core operand: dst[i][k] = src(i, k)
// rounded to BF16 (or x * scale to FP8 e4m3), zero for i >= N or k >= D.
// src(i, k) = src[i * si + k * sk]. One thread per 4 consecutive k of one row.
template <bool FP8>
__global__ void convert_operand_kernel(const float* __restrict__ src, size_t si, size_t sk, int N, int D, int Np,
                                       int Kp, float scale, void* __restrict__ dst) {
    const size_t groups = (size_t)Np * (size_t)(Kp / 4);
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / (size_t)(Kp / 4));
        const int k0 = (int)(g % (size_t)(Kp / 4)) * 4;
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = k0 + e;
            v[e] = (i < N && k < D) ? src[(size_t)i * si + (size_t)k * sk] : 0.0f;
        }
        if constexpr (FP8) {
            __nv_fp8x4_e4m3 q(make_float4(v[0] * scale, v[1] * scale, v[2] * scale, v[3] * scale));
            reinterpret_cast<__nv_fp8x4_e4m3*>(dst)[(size_t)i * (Kp / 4) + k0 / 4] = q;
        } else {
            __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
            __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
            __nv_bfloat162* d = reinterpret_cast<__nv_bfloat162*>(dst) + ((size_t)i * Kp + k0) / 2;
            d[0] = lo;
            d[1] = hi;
        }
    }
}

// The same conversion from the swarm's dimension-major layout src[k * ld + i]
// through a shared-memory tile: 64 dimensions x 64 particles per block, read
// along particles and written along dimensions (BF16 only).
__global__ void __launch_bounds__(256) convert_dimmajor_bf16_kernel(const float* __restrict__ src, size_t ld, int N,
                                                                    int D, int Np, int Kp,
                                                                    __nv_bfloat16* __restrict__ dst) {
    __shared__ float t[64][65];
    const int k0 = blockIdx.x * 64, i0 = blockIdx.y * 64;
    for (int e = threadIdx.x; e < 64 * 64; e += 256) {
        const int kk = e / 64, ii = e % 64;
        const int k = k0 + kk, i = i0 + ii;
        t[kk][ii] = (k < D && i < N) ? src[(size_t)k * ld + i] : 0.0f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {   // pairs of dimensions
        const int ii = e / 32, kp = (e % 32) * 2;
        const int i = i0 + ii, k = k0 + kp;
        if (i < Np && k < Kp)
            *reinterpret_cast<__nv_bfloat162*>(dst + (size_t)i * Kp + k) = __floats2bfloat162_rn(t[kp][ii], t[kp + 1][ii]);
    }
}

// Plain FP32 least-squares fitness with the oracle's rounding order. Block =
// 64 particles x all M, in tiles of 64 residual rows; thread (ty, tx) holds a
// 4 x 4 block of (particle, row) residuals, each a chain of fma over d in
// order; then 64 threads add the tile's squares to their particle's sum in
// row order. X(i, d) = x[d * ldx + i] (the swarm layout).
__global__ void __launch_bounds__(256) lsq_fp32_kernel(const float* __restrict__ x, int ldx, int N, int D,
                                                       const float* __restrict__ A, const float* __restrict__ b, int M,
                                                       float* __restrict__ f) {
    __shared__ __align__(16) float Xs[32][64 + 4];   // [d][particle]
    __shared__ __align__(16) float As[32][64 + 4];   // [d][row]
    __shared__ float Rs[64][64 + 1];   // [particle][row]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * 64;
    float acc_i = 0.0f;                // the running sum of particle i0 + threadIdx.x (threads < 64)
    for (int m0 = 0; m0 < M; m0 += 64) {
        float r[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int m = m0 + tx * 4 + c;
                r[a][c] = m < M ? -b[m] : 0.0f;
            }
        for (int d0 = 0; d0 < D; d0 += 32) {
            for (int e = threadIdx.x; e < 32 * 64; e += 256) {
                const int dd = e / 64, col = e % 64;
                const int d = d0 + dd;
                Xs[dd][col] = (d < D && i0 + col < N) ? x[(size_t)d * ldx + i0 + col] : 0.0f;
                As[dd][col] = (d < D && m0 + col < M) ? A[(size_t)(m0 + col) * D + d] : 0.0f;
            }
            __syncthreads();
            const int dn = min(32, D - d0);
            for (int dd = 0; dd < dn; ++dd) {
                // rows of 68 floats: every 4-float group is 16-byte aligned
                const float4 x4 = *reinterpret_cast<const float4*>(&Xs[dd][ty * 4]);
                const float4 a4 = *reinterpret_cast<const float4*>(&As[dd][tx * 4]);
                const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) r[a][c] = __fmaf_rn(av[c], xv[a], r[a][c]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) Rs[ty * 4 + a][tx * 4 + c] = r[a][c];
        __syncthreads();
        if (threadIdx.x < 64) {
            const int mn = min(64, M - m0);
            for (int c = 0; c < mn; ++c) acc_i = __fmaf_rn(Rs[threadIdx.x][c], Rs[threadIdx.x][c], acc_i);
        }
        __syncthreads();
    }
    if (threadIdx.x < 64 && i0 + threadIdx.x < N) f[i0 + threadIdx.x] = acc_i;
}

// FP64 least-squares fitness in the reference order, rounded once to FP32:
// per particle, acc = 0; for m ascending: r = -b_m, r = r + A_md x_d for d
// ascending (each product of two floats is exact in binary64, so the fma below
// rounds exactly as the separate product and sum would), acc = acc + r * r
// (square rounded, then added); f = acc rounded to float. Block = 64 particles
// x all M, in tiles of 32 residual rows; thread (ty, tx) holds the 4 x 2 block
// of (particle, row) residuals, each a chain over d in order; 64 threads then
// add the tile's squares to their particle's sum in row order.
__global__ void __launch_bounds__(256) lsq_fp64_kernel(const float* __restrict__ x, int ldx, int N, int D,
                                                       const float* __restrict__ A, const float* __restrict__ b, int M,
                                                       float* __restrict__ f) {
    __shared__ __align__(16) float Xs[32][64 + 4];   // [d][particle]
    __shared__ __align__(16) float As[32][32 + 4];   // [d][row]
    __shared__ double Rs[64][32 + 1];                 // [particle][row]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * 64;
    double acc_i = 0.0;                // the running sum of particle i0 + threadIdx.x (threads < 64)
    for (int m0 = 0; m0 < M; m0 += 32) {
        double r[4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int m = m0 + tx * 2 + c;
                r[a][c] = m < M ? -(double)b[m] : 0.0;
            }
        for (int d0 = 0; d0 < D; d0 += 32) {
            for (int e = threadIdx.x; e < 32 * 64; e += 256) {
                const int dd = e / 64, col = e % 64;
                const int d = d0 + dd;
                Xs[dd][col] = (d < D && i0 + col < N) ? x[(size_t)d * ldx + i0 + col] : 0.0f;
            }
            for (int e = threadIdx.x; e < 32 * 32; e += 256) {
                const int dd = e / 32, col = e % 32;
                const int d = d0 + dd;
                As[dd][col] = (d < D && m0 + col < M) ? A[(size_t)(m0 + col) * D + d] : 0.0f;
            }
            __syncthreads();
            const int dn = min(32, D - d0);
            for (int dd = 0; dd < dn; ++dd) {
                const float4 x4 = *reinterpret_cast<const float4*>(&Xs[dd][ty * 4]);
                const float2 a2 = *reinterpret_cast<const float2*>(&As[dd][tx * 2]);
                const double xv[4] = {(double)x4.x, (double)x4.y, (double)x4.z, (double)x4.w};
                const double av[2] = {(double)a2.x, (double)a2.y};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 2; ++c) r[a][c] = __fma_rn(av[c], xv[a], r[a][c]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 2; ++c) Rs[ty * 4 + a][tx * 2 + c] = r[a][c];
        __syncthreads();
        if (threadIdx.x < 64) {
            const int mn = min(32, M - m0);
            for (int c = 0; c < mn; ++c) {
                const double rc = Rs[threadIdx.x][c];
                acc_i = __dadd_rn(acc_i, __dmul_rn(rc, rc));
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 64 && i0 + threadIdx.x < N) f[i0 + threadIdx.x] = __double2float_rn(acc_i);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D map over a K-major [rows][Kp] operand, box = (128 bytes of K) x box_rows.
bool make_map(CUtensorMap* tm, void* ptr, bool fp8, int rows, int Kp, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const int esz = fp8 ? 1 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * esz};
    cuuint32_t box[2] = {(cuuint32_t)(KB / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(tm, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

size_t tc_smem() { return (size_t)STAGES * STAGE_BYTES + 1024 + 256; }

}  // namespace

bool lsq_tc_available() { return encode_fn() != nullptr; }

bool lsq_make_move_maps(unsigned char (*maps)[128], const float* x, const float* v, const float* pb, int Np, int D) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || Np % 64 != 0 || D < 1) return false;
    const float* arrays[3] = {x, v, pb};
    for (int a = 0; a < 3; ++a) {
        cuuint64_t dims[2] = {(cuuint64_t)Np, (cuuint64_t)D};
        cuuint64_t strides[1] = {(cuuint64_t)Np * sizeof(float)};
        cuuint32_t box[2] = {64, 64};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = fn(reinterpret_cast<CUtensorMap*>(maps[a]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        const_cast<float*>(arrays[a]), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

cudaError_t lsq_prepare() {
    cudaError_t e = cudaFuncSetAttribute(lsq_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(lsq_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem());
}

cudaError_t lsq_convert(const float* src, size_t si, size_t sk, int N, int D, int Np, int Kp, bool fp8, float scale,
                        void* dst, cudaStream_t st) {
    if (!fp8 && si == 1 && Kp % 64 == 0) {   // dimension-major source: tiled transpose
        convert_dimmajor_bf16_kernel<<<dim3(Kp / 64, (Np + 63) / 64), 256, 0, st>>>(
            src, sk, N, D, Np, Kp, reinterpret_cast<__nv_bfloat16*>(dst));
        return cudaGetLastError();
    }
    const size_t groups = (size_t)Np * (size_t)(Kp / 4);
    const int grid = (int)std::min<size_t>((groups + 255) / 256, 8192);
    if (fp8) convert_operand_kernel<true><<<grid, 256, 0, st>>>(src, si, sk, N, D, Np, Kp, scale, dst);
    else convert_operand_kernel<false><<<grid, 256, 0, st>>>(src, si, sk, N, D, Np, Kp, scale, dst);
    return cudaGetLastError();
}

bool lsq_tc_plan(LsqTcPlan* p, void* Xq, void* Aq, bool fp8, int Np, int Mp, int Kp) {
    p->fp8 = fp8;
    p->Np = Np;
    p->Mp = Mp;
    p->Kp = Kp;
    int dev = 0;
    p->num_sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || p->num_sms < 1)
        return false;
    if (!make_map(reinterpret_cast<CUtensorMap*>(p->tmX), Xq, fp8, Np, Kp, BM)) return false;
    if (!make_map(reinterpret_cast<CUtensorMap*>(p->tmA), Aq, fp8, Mp, Kp, BNH)) return false;
    // The persistent grid: as many CTA pairs as can be resident at once (a GPC
    // with an odd number of free SMs leaves one out), never more than SMs / 2.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * (p->num_sms / 2));
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = tc_smem();
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, fp8 ? (const void*)lsq_tc_kernel<true> : (const void*)lsq_tc_kernel<false>,
                                       &cfg) != cudaSuccess ||
        clusters < 1) {
        cudaGetLastError();
        return false;
    }
    p->num_sms = 2 * std::min(clusters, p->num_sms / 2);
    return true;
}

cudaError_t lsq_tc_launch(const LsqTcPlan& p, const float* off, const float* inv_scale, float* part,
                          unsigned int* status, long long limit_ns, cudaStream_t st) {
    const int ntiles = ((p.Np + 2 * BM - 1) / (2 * BM)) * (p.Mp / BN);
    const int pairs = std::max(1, std::min(ntiles, p.num_sms / 2));   // num_sms: the resident pairs x 2
    const int KT = p.Kp * (p.fp8 ? 1 : 2) / KB;
    const CUtensorMap& tx = *reinterpret_cast<const CUtensorMap*>(p.tmX);
    const CUtensorMap& ta = *reinterpret_cast<const CUtensorMap*>(p.tmA);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * pairs);
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = tc_smem();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (p.fp8)
        return cudaLaunchKernelEx(&cfg, lsq_tc_kernel<true>, tx, ta, off, inv_scale, p.Mp, KT, p.Np, part, status,
                                  limit_ns);
    return cudaLaunchKernelEx(&cfg, lsq_tc_kernel<false>, tx, ta, off, inv_scale, p.Mp, KT, p.Np, part, status,
                              limit_ns);
}

int lsq_tc_partials(const LsqTcPlan& p) { return p.Mp / 128; }

cudaError_t lsq_fp32_launch(const float* x, int ldx, int N, int D, const float* A, const float* b, int M, float* f,
                            cudaStream_t st) {
    lsq_fp32_kernel<<<(N + 63) / 64, 256, 0, st>>>(x, ldx, N, D, A, b, M, f);
    return cudaGetLastError();
}

cudaError_t lsq_fp64_launch(const float* x, int ldx, int N, int D, const float* A, const float* b, int M, float* f,
                            cudaStream_t st) {
    lsq_fp64_kernel<<<(N + 63) / 64, 256, 0, st>>>(x, ldx, N, D, A, b, M, f);
    return cudaGetLastError();
}

}  // namespace cupso
