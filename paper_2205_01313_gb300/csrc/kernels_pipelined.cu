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
//  * warps take units of 32 x PPT particles from a counter, so work is
//    balanced across SMs to within one unit instead of one 1024-particle
//    tile; PPT (particles per thread: 4, 2 or 1, loaded as float4, float2 or
//    float) is chosen so that even a smaller swarm has enough units to fill
//    the GPU.
#include <cuda_runtime.h>

#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "stream_common.cuh"

namespace cupso {

namespace {

template <int P> struct VT;
template <> struct VT<4> { using T = float4; };
template <> struct VT<2> { using T = float2; };
template <> struct VT<1> { using T = float; };

__device__ __forceinline__ float vget(const float4& v, int j) { return lane(v, j); }
__device__ __forceinline__ float vget(const float2& v, int j) { return j == 0 ? v.x : v.y; }
__device__ __forceinline__ float vget(const float& v, int) { return v; }
__device__ __forceinline__ void vset(float4& v, int j, float a) { set_lane(v, j, a); }
__device__ __forceinline__ void vset(float2& v, int j, float a) {
    if (j == 0) v.x = a; else v.y = a;
}
__device__ __forceinline__ void vset(float& v, int, float a) { v = a; }

template <int P>
__device__ __forceinline__ typename VT<P>::T ldv(const float* p) {
    return *reinterpret_cast<const typename VT<P>::T*>(p);
}
template <int P>
__device__ __forceinline__ void stv(float* p, const typename VT<P>::T& v) {
    *reinterpret_cast<typename VT<P>::T*>(p) = v;
}

template <int P>
__device__ __forceinline__ void cp_async_v(typename VT<P>::T* smem, const float* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (P == 4)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
    else if constexpr (P == 2)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
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
// rows 2g and 2g+1 of pos, v and pbest_pos, P floats per lane per row.
// Slot (stage, a, r) of this thread is my[(stage * 6 + 2 * a + r) * kBlock].
template <int P>
__device__ __forceinline__ void issue_step(const SwarmDev& s, typename VT<P>::T* my, uint32_t u, int g, int stage,
                                           uint32_t nunits, int lane_id) {
    if (u < nunits) {
        const size_t col = (size_t)u * (32 * P) + (size_t)lane_id * P;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int d = 2 * g + r;
            if (d < s.D) {
                const size_t off = (size_t)d * (size_t)s.Np + col;
                cp_async_v<P>(my + (stage * 6 + 0 + r) * kBlock, s.x + off);
                cp_async_v<P>(my + (stage * 6 + 2 + r) * kBlock, s.v + off);
                cp_async_v<P>(my + (stage * 6 + 4 + r) * kBlock, s.pb + off);
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
// explicit copy) and writes the pbest_pos row from it with full-width
// stores. The arithmetic is unchanged; only when pbest_pos is stored differs.
__device__ __forceinline__ uint32_t flag_bit(uint32_t fl, int j) { return (fl >> (8 * j)) & 1u; }

// The flags of particles i0 .. i0 + P - 1 (byte j = particle i0 + j).
template <int P>
__device__ __forceinline__ uint32_t load_flags(const SwarmDev& s, uint32_t i0) {
    if constexpr (P == 4) return __ldcg(reinterpret_cast<const unsigned int*>(s.pflag + i0));
    else if constexpr (P == 2) return (uint32_t)__ldcg(reinterpret_cast<const unsigned short*>(s.pflag + i0));
    else return (uint32_t)__ldcg(reinterpret_cast<const unsigned char*>(s.pflag + i0));
}
template <int P>
__device__ __forceinline__ void store_flags(const SwarmDev& s, uint32_t i0, uint32_t fl) {
    if constexpr (P == 4) *reinterpret_cast<unsigned int*>(s.pflag + i0) = fl;
    else if constexpr (P == 2) *reinterpret_cast<unsigned short*>(s.pflag + i0) = (unsigned short)fl;
    else *reinterpret_cast<unsigned char*>(s.pflag + i0) = (unsigned char)fl;
}

// Requires (D + 1) / 2 >= STAGES - 1 (the host falls back to the register
// kernel otherwise), Np a multiple of 128 and s.pflag set.
// FAST selects move_one_fast (requires s.fast_cr and s.fast_clamp).
template <int FIT, int STAGES, bool FAST, int P>
__global__ void __launch_bounds__(kBlock, (P == 4 ? 3 : (P == 2 ? 4 : 5)))
    sync_pipelined_kernel(const __grid_constant__ SwarmDev s) {
    using T = typename VT<P>::T;
    constexpr int kUnit = 32 * P;
    extern __shared__ float4 ring_raw[];  // [STAGES][6][kBlock] T, then gbest_pos [D]
    T* ring = reinterpret_cast<T*>(ring_raw);
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
    T* my = ring + threadIdx.x;

    uint32_t u_cur = fetch_unit(s, lane_id);
    uint32_t fl_cur = u_cur < nunits ? load_flags<P>(s, u_cur * kUnit + (uint32_t)lane_id * P) : 0u;
    uint32_t u_nxt = 0xFFFFFFFFu, fl_nxt = 0u;
#pragma unroll
    for (int j = 0; j < STAGES - 1; ++j) issue_step<P>(s, my, u_cur, j, j, nunits, lane_id);
    int ig = STAGES - 1;  // pair of the next issue, counted from the current unit
    int stage = 0;        // ring stage of the pair being computed

    unsigned long long best = kKeyNone;
    bool nan = false;
    while (u_cur < nunits) {
        const uint32_t i0 = u_cur * kUnit + (uint32_t)lane_id * P;
        FitAcc<FIT> acc[P];
        T PF{};
        for (int g = 0; g < npairs; ++g) {
            // keep STAGES-1 pairs in flight: issue the pair STAGES-1 ahead
            {
                int ws = stage + STAGES - 1;
                if (ws >= STAGES) ws -= STAGES;
                if (ig < npairs) {
                    issue_step<P>(s, my, u_cur, ig, ws, nunits, lane_id);
                } else {
                    if (u_nxt == 0xFFFFFFFFu) {
                        u_nxt = fetch_unit(s, lane_id);
                        if (u_nxt < nunits) fl_nxt = load_flags<P>(s, u_nxt * kUnit + (uint32_t)lane_id * P);
                    }
                    issue_step<P>(s, my, u_nxt, ig - npairs, ws, nunits, lane_id);
                }
                ++ig;
            }
            if (g == npairs - 1) PF = ldv<P>(s.pf + i0);  // needed after the last pair
            cp_wait<STAGES - 1>();  // this thread's copies of the current pair have landed
            uint4 rr[P];
#pragma unroll
            for (int j = 0; j < P; ++j)
                rr[j] = philox4x32_10(make_uint4((uint32_t)g, i0 + j, t, s.swarm), s.key0, s.key1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int d = 2 * g + h;
                if (h == 1 && d >= D) break;
                T X = my[(stage * 6 + 0 + h) * kBlock];
                T V = my[(stage * 6 + 2 + h) * kBlock];
                T Pb = my[(stage * 6 + 4 + h) * kBlock];
                const size_t off = (size_t)d * Np + i0;
                if (fl_cur) {
                    // pbest_pos of a flagged particle is its pos: use it and write it back
#pragma unroll
                    for (int j = 0; j < P; ++j)
                        if (flag_bit(fl_cur, j)) vset(Pb, j, vget(X, j));
                    stv<P>(s.pb + off, Pb);
                }
                const float gd = Gs[d];
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    float xj = vget(X, j), vj = vget(V, j);
                    if constexpr (FAST)
                        move_one_fast(xj, vj, vget(Pb, j), gd, hi24(word(rr[j], 2 * h)), hi24(word(rr[j], 2 * h + 1)),
                                      s);
                    else
                        move_one(xj, vj, vget(Pb, j), gd, u01(word(rr[j], 2 * h)), u01(word(rr[j], 2 * h + 1)), s);
                    vset(X, j, xj);
                    vset(V, j, vj);
                    acc[j].add(d, xj);
                }
                stv<P>(s.x + off, X);
                stv<P>(s.v + off, V);
            }
            if (++stage == STAGES) stage = 0;
        }
        // Step 4 (strict improvement; the new pbest_pos is pos, flagged) and Step 5.
        uint32_t fl_new = 0u;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const float f = acc[j].finish(D);
            const bool real = (i0 + j) < (uint32_t)s.N;
            nan |= real && (f != f);
            if (real && f < vget(PF, j)) {
                fl_new |= 1u << (8 * j);
                vset(PF, j, f);
                const unsigned long long k = pack_key(f, i0 + j);
                if (k < K && k < best) best = k;
            }
        }
        if (fl_new) stv<P>(s.pf + i0, PF);
        if (fl_new != fl_cur) store_flags<P>(s, i0, fl_new);
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

size_t smem_of(int stages, int ppt, int D) {
    return sizeof(float) * (size_t)ppt * (size_t)stages * 6 * kBlock + sizeof(float) * (size_t)D;
}

// The kernel instance for (fitness, ring depth, fast path, particles per thread).
template <int STAGES, bool FAST, int P>
const void* kernel_of_t(int fid) {
    switch (fid) {
        case kSphere: return (const void*)sync_pipelined_kernel<kSphere, STAGES, FAST, P>;
        case kRastrigin: return (const void*)sync_pipelined_kernel<kRastrigin, STAGES, FAST, P>;
        case kAckley: return (const void*)sync_pipelined_kernel<kAckley, STAGES, FAST, P>;
        case kRosenbrock: return (const void*)sync_pipelined_kernel<kRosenbrock, STAGES, FAST, P>;
        case kCubicMax: return (const void*)sync_pipelined_kernel<kCubicMax, STAGES, FAST, P>;
        default: return nullptr;
    }
}

template <int STAGES, int P>
const void* kernel_of_sp(bool fast, int fid) {
    return fast ? kernel_of_t<STAGES, true, P>(fid) : kernel_of_t<STAGES, false, P>(fid);
}

const void* kernel_of(int stages, bool fast, int fid, int ppt) {
    if (stages == 3) {
        if (ppt == 4) return kernel_of_sp<3, 4>(fast, fid);
        if (ppt == 2) return kernel_of_sp<3, 2>(fast, fid);
        return kernel_of_sp<3, 1>(fast, fid);
    }
    if (ppt == 4) return kernel_of_sp<4, 4>(fast, fid);
    if (ppt == 2) return kernel_of_sp<4, 2>(fast, fid);
    return kernel_of_sp<4, 1>(fast, fid);
}

}  // namespace

bool pipelined_supported(int stages, int D) {
    return (stages == 3 || stages == 4) && (D + 1) / 2 >= stages - 1 && D <= 8192;
}

cudaError_t prepare_pipelined(int D) {
    const int ppts[3] = {4, 2, 1};
    for (int stages = 3; stages <= 4; ++stages)
        for (int pi = 0; pi < 3; ++pi)
            for (int fast = 0; fast < 2; ++fast)
                for (int fid = kSphere; fid <= kCubicMax; ++fid) {
                    cudaError_t e = cudaFuncSetAttribute(kernel_of(stages, fast != 0, fid, ppts[pi]),
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)smem_of(stages, ppts[pi], D));
                    if (e != cudaSuccess) return e;
                }
    return cudaSuccess;
}

int pipelined_blocks_per_sm(int stages, int fid, int D, int ppt) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel_of(stages, true, fid, ppt), kBlock,
                                                      smem_of(stages, ppt, D)) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_materialize(const SwarmDev& s, int grid, cudaStream_t st) {
    if (!s.pflag) return cudaSuccess;
    materialize_kernel<<<grid, kBlock, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t launch_sync_pipelined(const SwarmDev& s, int fid, int stages, int ppt, int grid, cudaStream_t st) {
    if (!pipelined_supported(stages, s.D) || !s.pflag || (ppt != 1 && ppt != 2 && ppt != 4))
        return cudaErrorInvalidValue;
    const void* k = kernel_of(stages, s.fast_cr && s.fast_clamp, fid, ppt);
    if (!k) return cudaErrorInvalidValue;
    void* args[] = {const_cast<SwarmDev*>(&s)};
    return cudaLaunchKernel(k, dim3(grid), dim3(kBlock), args, smem_of(stages, ppt, s.D), st);
}

}  // namespace cupso
