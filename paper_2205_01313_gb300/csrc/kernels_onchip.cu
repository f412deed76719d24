// kernels_onchip.cu -- whole swarm resident in one thread-block cluster.
//
// For swarms whose state fits in the shared memory of a cluster (up to 16
// CTAs on GB300), the whole run of many iterations is one launch: x, v,
// pbest_pos and pbest_fit stay in shared memory (Sec. 4.3 keeps the hot data
// on chip), and the only exchange per iteration is the global best. Each CTA
// pushes its candidate -- the lowest improved key below the current gbest,
// with that particle's position (Sec. 4.3: index first, position after) --
// into a slot of every CTA of the cluster through distributed shared memory,
// then one cluster barrier replaces the paper's kernel boundary (Sec. 2.2).
// Every thread then reduces the same slots in the same order, so all hold the
// same gbest. pbest rows are copied lazily (in the next move), so an
// iteration takes three CTA barriers and the cluster barrier. The arithmetic
// is that of the streaming kernels: bit-identical synchronous PSO.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "stream_common.cuh"

namespace cg = cooperative_groups;

namespace cupso {

namespace {

constexpr int kOnchipThreads = 256;
constexpr int kMaxCluster = 16;

struct OnchipLayout {
    int P;            // particles per CTA (Np / cluster)
    int C;            // CTAs in the cluster
    size_t o_x, o_v, o_pb, o_aux, o_pf, o_imp, o_G, o_slots, bytes;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) / 16 * 16; }

__host__ __device__ inline OnchipLayout onchip_layout(int Np, int D, int C) {
    OnchipLayout L;
    L.C = C;
    L.P = Np / C;
    const size_t plane = sizeof(float) * (size_t)L.P * (size_t)D;
    size_t o = 0;
    L.o_x = o; o = al16(o + plane);
    L.o_v = o; o = al16(o + plane);
    L.o_pb = o; o = al16(o + plane);
    L.o_aux = o; o = al16(o + plane);                 // cos2pi(x') where the fitness needs it
    L.o_pf = o; o = al16(o + sizeof(float) * L.P);
    L.o_imp = o; o = al16(o + sizeof(int) * L.P);
    L.o_G = o; o = al16(o + sizeof(float) * D);
    // slots[2][C]: 8-byte key then D floats, padded to 16 bytes
    L.o_slots = o;
    const size_t slot = al16(8 + sizeof(float) * (size_t)D);
    o = al16(o + 2 * (size_t)C * slot);
    L.bytes = o;
    return L;
}

__device__ __forceinline__ size_t slot_bytes(int D) { return al16(8 + sizeof(float) * (size_t)D); }

template <int FIT, bool FAST>
__global__ void __launch_bounds__(kOnchipThreads) onchip_kernel(const __grid_constant__ SwarmDev s, int iters) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int D = s.D;
    const OnchipLayout L = onchip_layout(s.Np, D, C);
    const int P = L.P;
    float* x = reinterpret_cast<float*>(smem + L.o_x);     // [D][P]
    float* v = reinterpret_cast<float*>(smem + L.o_v);
    float* pb = reinterpret_cast<float*>(smem + L.o_pb);
    float* caux = reinterpret_cast<float*>(smem + L.o_aux);
    float* pf = reinterpret_cast<float*>(smem + L.o_pf);
    int* imp = reinterpret_cast<int*>(smem + L.o_imp);
    float* G = reinterpret_cast<float*>(smem + L.o_G);
    unsigned char* slots = smem + L.o_slots;
    const size_t sb = slot_bytes(D);
    __shared__ unsigned long long red[kOnchipThreads / 32];

    const uint32_t base = (uint32_t)rank * (uint32_t)P;   // first particle of this CTA
    const size_t Np = (size_t)s.Np;
    const uint32_t t_prev = __ldcg(s.t_dev);
    const int cur0 = (int)(t_prev & 1u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // Load the CTA's particles, gbest and its key. imp[p] marks a particle
    // whose pbest_pos row is still to be copied from its position (lazy
    // pbest: the copy happens in the next move, or at the end).
    for (int e = threadIdx.x; e < P * D; e += blockDim.x) {
        const int d = e / P, p = e - d * P;
        const size_t g = (size_t)d * Np + base + p;
        x[e] = s.x[g];
        v[e] = s.v[g];
        pb[e] = s.pb[g];
    }
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        pf[p] = s.pf[base + p];
        imp[p] = 0;
    }
    for (int d = threadIdx.x; d < D; d += blockDim.x) G[d] = s.G[(size_t)cur0 * D + d];
    // every thread keeps the gbest key; all of them compute the same one each iteration
    unsigned long long K = __ldcg(s.gkey + cur0);
    __syncthreads();

    const int npairs = (D + 1) / 2;
    // (pair, particle) items e = g2 * P + p, walked with a stride of the block
    // without a division per item
    const int g2_first = (int)threadIdx.x / P, p_first = (int)threadIdx.x - g2_first * P;
    const int g2_step = (int)blockDim.x / P, p_step = (int)blockDim.x - g2_step * P;
    bool nan = false;
    for (int k = 0; k < iters; ++k) {
        const uint32_t t = t_prev + 1u + (uint32_t)k;
        // Step 2 (Eq. 1, Eq. 2): one Philox call per (particle, dimension pair).
        int g2 = g2_first, p = p_first;
#pragma unroll 2
        for (; g2 < npairs;) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)g2, base + (uint32_t)p, t, s.swarm), s.key0, s.key1);
            const bool lazy = imp[p] != 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int d = 2 * g2 + h;
                if (d >= D) break;
                const int idx = d * P + p;
                float xx = x[idx], vv = v[idx];
                float pp = pb[idx];
                if (lazy) {
                    pp = xx;
                    pb[idx] = xx;
                }
                if constexpr (FAST)
                    move_one_fast(xx, vv, pp, G[d], hi24(word(r, 2 * h)), hi24(word(r, 2 * h + 1)), s);
                else
                    move_one(xx, vv, pp, G[d], u01(word(r, 2 * h)), u01(word(r, 2 * h + 1)), s);
                x[idx] = xx;
                v[idx] = vv;
                if constexpr (FitAcc<FIT>::kNeedsCos) caux[idx] = cos2pi(xx);
            }
            p += p_step;
            g2 += g2_step;
            if (p >= P) {
                p -= P;
                ++g2;
            }
        }
        __syncthreads();
        // Steps 3-4: fitness, sequential over d per particle; strict
        // improvement; the CTA's Step-5 candidate.
        unsigned long long cand = kKeyNone;
        for (int p = threadIdx.x; p < P; p += blockDim.x) {
            FitAcc<FIT> acc;
            for (int d = 0; d < D; ++d) acc.add_c(d, x[d * P + p], FitAcc<FIT>::kNeedsCos ? caux[d * P + p] : 0.0f);
            const float f = acc.finish(D);
            const uint32_t i = base + (uint32_t)p;
            int up = 0;
            if (i < (uint32_t)s.N) {
                nan |= (f != f);
                if (f < pf[p]) {
                    pf[p] = f;
                    up = 1;
                    const unsigned long long kk = pack_key(f, i);
                    if (kk < K && kk < cand) cand = kk;
                }
            }
            imp[p] = up;
        }
        cand = warp_min_u64(cand);
        if (lane == 0) red[warp] = cand;
        __syncthreads();
        // Warp 0 pushes the CTA's candidate into slot [k & 1][rank] of every
        // CTA of the cluster: key from lane r to CTA r, then the position.
        const int par = k & 1;
        const size_t my_slot = ((size_t)par * C + rank) * sb;
        if (warp == 0) {
            unsigned long long c2 = lane < (int)(blockDim.x >> 5) ? red[lane] : kKeyNone;
            c2 = warp_min_u64(c2);
            if (lane < C) {
                unsigned char* remote = cluster.map_shared_rank(slots, lane);
                *reinterpret_cast<unsigned long long*>(remote + my_slot) = c2;
            }
            if (c2 != kKeyNone) {
                const int pc = (int)((uint32_t)(c2 & 0xFFFFFFFFull) - base);
                for (int e = lane; e < C * D; e += 32) {
                    const int r = e / D, d = e - r * D;
                    unsigned char* remote = cluster.map_shared_rank(slots, r);
                    reinterpret_cast<float*>(remote + my_slot + 8)[d] = x[d * P + pc];
                }
            }
        }
        cluster.sync();
        // Step 5: every thread reduces the same slots in rank order.
        unsigned long long best = K;
        int win = -1;
        for (int r = 0; r < C; ++r) {
            const unsigned long long kk = *reinterpret_cast<const unsigned long long*>(slots + ((size_t)par * C + r) * sb);
            if (kk < best) {
                best = kk;
                win = r;
            }
        }
        if (win >= 0) {
            const float* row = reinterpret_cast<const float*>(slots + ((size_t)par * C + win) * sb + 8);
            for (int d = threadIdx.x; d < D; d += blockDim.x) G[d] = row[d];
        }
        K = best;
        __syncthreads();
    }

    // Write the state back so that every other mode and the host see it
    // (pending pbest rows included).
    for (int e = threadIdx.x; e < P * D; e += blockDim.x) {
        const int d = e / P, p = e - d * P;
        const size_t g = (size_t)d * Np + base + p;
        s.x[g] = x[e];
        s.v[g] = v[e];
        s.pb[g] = imp[p] ? x[e] : pb[e];
    }
    for (int p = threadIdx.x; p < P; p += blockDim.x) s.pf[base + p] = pf[p];
    if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(s.status, kStatusNaN);
    if (rank == 0) {
        const uint32_t t_end = t_prev + (uint32_t)iters;
        const int cur = (int)(t_end & 1u);
        for (int d = threadIdx.x; d < D; d += blockDim.x) s.G[(size_t)cur * D + d] = G[d];
        if (threadIdx.x == 0) {
            s.gkey[0] = K;
            s.gkey[1] = K;
            *s.t_dev = t_end;
        }
    }
    // No CTA may leave while others can still read its shared memory.
    cluster.sync();
}

int max_optin_smem() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return v;
}

// The cluster can be scheduled: the device reports room for at least one.
bool cluster_schedulable(int C, size_t smem) {
    auto kernel = onchip_kernel<kSphere, false>;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return false;
    if (C > 8 && cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    cfg.blockDim = dim3(kOnchipThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

}  // namespace

bool onchip_fits(int N, int D, int* cluster_out, int* per_cta_out) {
    const int Np = (N + kPad - 1) / kPad * kPad;
    const int limit = max_optin_smem() - 2048;   // room for the static shared arrays
    if (limit <= 0) return false;
    // Smallest cluster that fits, then grow towards ~64 particles per CTA for
    // parallelism; shrink again if the device cannot schedule that cluster.
    int C = 0;
    for (int c = 1; c <= kMaxCluster; c *= 2) {
        if (Np % c) break;
        if (onchip_layout(Np, D, c).bytes <= (size_t)limit) { C = c; break; }
    }
    if (C == 0) return false;
    const int C_min = C;
    while (C < kMaxCluster && Np / (2 * C) >= 64 && Np % (2 * C) == 0) C *= 2;
    while (C >= C_min && !cluster_schedulable(C, onchip_layout(Np, D, C).bytes)) C /= 2;
    if (C < C_min) return false;
    if (cluster_out) *cluster_out = C;
    if (per_cta_out) *per_cta_out = Np / C;
    return true;
}

namespace {
template <int FIT, bool FAST>
cudaError_t launch_onchip_t(const SwarmDev& s, int iters, cudaStream_t st) {
    int C = 0, P = 0;
    if (!onchip_fits(s.N, s.D, &C, &P)) return cudaErrorInvalidConfiguration;
    const OnchipLayout L = onchip_layout(s.Np, s.D, C);
    auto kernel = onchip_kernel<FIT, FAST>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
    if (e != cudaSuccess) return e;
    if (C > 8) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    cfg.blockDim = dim3(kOnchipThreads, 1, 1);
    cfg.dynamicSmemBytes = L.bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, s, iters);
}
}  // namespace

namespace {
template <bool FAST>
cudaError_t launch_onchip_f(const SwarmDev& s, int fid, int iters, cudaStream_t st) {
    switch (fid) {
        case kSphere: return launch_onchip_t<kSphere, FAST>(s, iters, st);
        case kRastrigin: return launch_onchip_t<kRastrigin, FAST>(s, iters, st);
        case kAckley: return launch_onchip_t<kAckley, FAST>(s, iters, st);
        case kRosenbrock: return launch_onchip_t<kRosenbrock, FAST>(s, iters, st);
        case kCubicMax: return launch_onchip_t<kCubicMax, FAST>(s, iters, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

cudaError_t launch_onchip(const SwarmDev& s, int fid, int iters, cudaStream_t st) {
    // the fast path (fused c r, min/max clamps) wherever it gives the same bits
    if (s.fast_cr && s.fast_clamp) return launch_onchip_f<true>(s, fid, iters, st);
    return launch_onchip_f<false>(s, fid, iters, st);
}

}  // namespace cupso
