// cupso_noalloc.cu -- one PSO iteration on caller-owned device memory, with
// no allocation at all.
//
// Who needs this: code that must not call cudaMalloc/cudaFree itself -- for
// example a host process whose device memory is owned by another allocator
// (a serving framework's caching pool, a memory budget enforced by an
// embedding application), where a private allocation would bypass that
// allocator's accounting or fail against its reservation. Such a caller keeps
// the swarm in its own device buffers and only needs the iteration.
//
// The iteration is the tree-reduction variant (first kernel: update, fitness,
// pbest and a block tree reduction into one key per block; second kernel:
// reduction of those keys and the gbest gather). Its working storage -- the
// per-block keys, the double-buffered gbest position, the iteration counter
// and status words -- lives in the file-scope device array below, of fixed
// size. Every GPU that loads the library holds that array until the process
// exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/cupso.h"
#include "cupso_device.cuh"
#include "cupso_internal.h"

namespace cupso {
namespace {

constexpr int kNoAllocMaxTiles = CUPSO_NOALLOC_MAX_N / kTile;   // one key per 1024-particle block
constexpr int kNoAllocMaxD = CUPSO_NOALLOC_MAX_D;

struct NoAllocScratch {
    unsigned long long gkey[2];
    unsigned int t_dev;
    unsigned int ticket;
    unsigned int status;
    unsigned int pad;
    unsigned long long aux[kNoAllocMaxTiles];
    float G[2 * kNoAllocMaxD];
};

// The scratch. Host code must not use this name as an address: it is only a
// host-side stand-in. The host obtains the device address with
// cudaGetSymbolAddress once per device (scratch_on_current_device below).
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Clears what must start fresh and loads the caller's gbest_pos as the gbest
// of iteration t-1.
__global__ void noalloc_prologue(NoAllocScratch* sc, const float* gbest_pos, int D, uint32_t t) {
    const uint32_t t_prev = t - 1u;
    const int cur = (int)(t_prev & 1u);
    for (int d = threadIdx.x; d < D; d += blockDim.x) sc->G[(size_t)cur * D + d] = gbest_pos[d];
    if (threadIdx.x == 0) {
        sc->t_dev = t_prev;
        sc->ticket = 0u;
        sc->status = 0u;
    }
}

// Writes the gbest of iteration t back to the caller's buffers.
__global__ void noalloc_epilogue(const NoAllocScratch* sc, float* gbest_pos, float* gbest_fit, int64_t* gbest_idx,
                                 unsigned int* status_out, int D, uint32_t t) {
    const int cur = (int)(t & 1u);
    for (int d = threadIdx.x; d < D; d += blockDim.x) gbest_pos[d] = sc->G[(size_t)cur * D + d];
    if (threadIdx.x == 0) {
        const unsigned long long key = sc->gkey[0];
        const uint32_t k = (uint32_t)(key >> 32);
        uint32_t bits = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
        if (k == 0xFFFFFFFFu) bits = 0x7FC00000u;   // NaN ranks last
        if (gbest_fit) *gbest_fit = __uint_as_float(bits);
        if (gbest_idx) *gbest_idx = (int64_t)(key & 0xFFFFFFFFull);
        if (status_out) *status_out = sc->status;
    }
}

// Device address of the scratch on the current device, looked up once per
// device with that device current. The address belongs to the module loaded
// into the device's current context: after cudaDeviceReset (or a primary
// context released and created again) the module is loaded anew and the
// symbol may move, so the cache also remembers the context it was taken in
// and looks the address up again when the current context differs.
constexpr int kMaxDevices = 64;
NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};
void* g_scratch_ctx[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// cuCtxGetCurrent through the runtime's driver entry point (no link to
// libcuda): the identity of the context whose module holds the scratch.
typedef int (*CtxGetCurrentFn)(void**);
CtxGetCurrentFn ctx_get_current_fn() {
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    });
    return fn;
}

int scratch_on_current_device(NoAllocScratch** out, char* err, size_t errlen) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        std::snprintf(err, errlen, "cudaGetDevice: %s", cudaGetErrorString(e));
        return CUPSO_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        std::snprintf(err, errlen, "device ordinal %d out of range", dev);
        return CUPSO_ERR_UNSUPPORTED;
    }
    CtxGetCurrentFn get_ctx = ctx_get_current_fn();
    void* ctx = nullptr;
    if (get_ctx) get_ctx(&ctx);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev] || !ctx || g_scratch_ctx[dev] != ctx) {
        // The lookup also makes the device's primary context current when no
        // context is yet, so the context is read again after it.
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            std::snprintf(err, errlen, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return CUPSO_ERR_CUDA;
        }
        ctx = nullptr;
        if (get_ctx) get_ctx(&ctx);
        g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_ptr[dev];
    return CUPSO_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int noalloc_step(int D, int N, const cupso_bounds* bounds, float w, float c1, float c2, int fitness_id,
                 uint64_t seed, uint32_t swarm_id, uint32_t t, float* pos, float* v, float* pbest_pos,
                 float* pbest_fit, int ld, float* gbest_pos, float* gbest_fit, int64_t* gbest_idx,
                 unsigned int* status_out, void* cuda_stream, char* err, size_t errlen) {
    if (D < 1 || N < 1 || !bounds) {
        std::snprintf(err, errlen, "D and N must be >= 1 and bounds non-NULL");
        return CUPSO_ERR_INVALID_ARG;
    }
    if (N > CUPSO_NOALLOC_MAX_N || D > CUPSO_NOALLOC_MAX_D) {
        std::snprintf(err, errlen, "no-allocation step supports N <= %d and D <= %d (got N=%d, D=%d)",
                      CUPSO_NOALLOC_MAX_N, CUPSO_NOALLOC_MAX_D, N, D);
        return CUPSO_ERR_INVALID_ARG;
    }
    if (ld < N || ld % kPad != 0) {
        std::snprintf(err, errlen, "ld must be a multiple of %d and >= N", kPad);
        return CUPSO_ERR_INVALID_ARG;
    }
    // Every column up to ld is moved and reduced: the first kernel runs one
    // block per kTile columns of the stride and each block writes one key into
    // the scratch, which holds kNoAllocMaxTiles of them. So the stride, not
    // only N, is bounded by the scratch.
    if (ld > CUPSO_NOALLOC_MAX_N) {
        std::snprintf(err, errlen, "no-allocation step supports ld <= %d (got ld=%d)", CUPSO_NOALLOC_MAX_N, ld);
        return CUPSO_ERR_INVALID_ARG;
    }
    if (!pos || !v || !pbest_pos || !pbest_fit || !gbest_pos || !aligned16(pos) || !aligned16(v) ||
        !aligned16(pbest_pos) || !aligned16(pbest_fit)) {
        std::snprintf(err, errlen, "state pointers must be non-NULL and 16-byte aligned");
        return CUPSO_ERR_INVALID_ARG;
    }
    if (t < 1u) {
        std::snprintf(err, errlen, "t (the iteration computed) must be >= 1");
        return CUPSO_ERR_INVALID_ARG;
    }
    if (!std::isfinite(bounds->min_pos) || !std::isfinite(bounds->max_pos) || !std::isfinite(bounds->max_v) ||
        !(bounds->min_pos < bounds->max_pos) || !(bounds->max_v > 0.0f) || !std::isfinite(w) ||
        !std::isfinite(c1) || !std::isfinite(c2) || fitness_id < CUPSO_SPHERE || fitness_id > CUPSO_CUBIC_MAX) {
        std::snprintf(err, errlen, "invalid bounds, coefficients or fitness_id");
        return CUPSO_ERR_INVALID_ARG;
    }
    NoAllocScratch* sc = nullptr;
    const int rc = scratch_on_current_device(&sc, err, errlen);
    if (rc != CUPSO_OK) return rc;

    SwarmDev s{};
    s.x = pos;
    s.v = v;
    s.pb = pbest_pos;
    s.pf = pbest_fit;
    s.G = sc->G;
    s.gkey = sc->gkey;
    s.ticket = &sc->ticket;
    s.t_dev = &sc->t_dev;
    s.status = &sc->status;
    s.aux = sc->aux;
    s.N = N;
    s.D = D;
    s.Np = ld;
    s.lo = bounds->min_pos;
    s.hi = bounds->max_pos;
    s.vmax = bounds->max_v;
    s.w = w;
    s.c1 = c1;
    s.c2 = c2;
    s.key0 = (uint32_t)(seed & 0xFFFFFFFFull);
    s.key1 = (uint32_t)(seed >> 32);
    philox_round_keys(s.key0, s.key1, s.rk0, s.rk1);
    s.swarm = swarm_id;
    s.wait_limit_ns = 2000000000ll;

    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    noalloc_prologue<<<1, 256, 0, st>>>(sc, gbest_pos, D, t);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_tree_step(s, fitness_id, false, st);
    if (e == cudaSuccess) {
        noalloc_epilogue<<<1, 256, 0, st>>>(sc, gbest_pos, gbest_fit, gbest_idx, status_out, D, t);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        std::snprintf(err, errlen, "launch: %s", cudaGetErrorString(e));
        return CUPSO_ERR_CUDA;
    }
    return CUPSO_OK;
}

}  // namespace
}  // namespace cupso

extern "C" CUPSO_API int cupso_tree_step_noalloc(int D, int N, const cupso_bounds* bounds, float w, float c1,
                                                 float c2, int fitness_id, uint64_t seed, uint32_t swarm_id,
                                                 uint32_t t, float* pos, float* v, float* pbest_pos,
                                                 float* pbest_fit, int ld, float* gbest_pos, float* gbest_fit,
                                                 int64_t* gbest_idx, unsigned int* status_out,
                                                 void* cuda_stream) {
    using namespace cupso;
    char err[256] = "";
    const size_t errlen = sizeof(err);
    int rc = noalloc_step(D, N, bounds, w, c1, c2, fitness_id, seed, swarm_id, t, pos, v, pbest_pos, pbest_fit,
                          ld, gbest_pos, gbest_fit, gbest_idx, status_out, cuda_stream, err, errlen);
    if (rc != CUPSO_OK) set_last_error(err);
    return rc;
}
