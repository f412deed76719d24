// cupso_api.cu -- the C ABI declared in include/cupso.h.
//
// Host-side control only (Sec. 2.2 splits PSO into host control and device
// work): argument checks, one device arena per swarm, stream and CUDA-graph
// management, and the launch of the kernels (kernels_*.cu). A handle holds
// either a single-precision swarm or a double-precision one (the paper's
// precision, kernels_paper.cu). Every step of the iteration runs on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/cupso.h"
#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "lsq_internal.h"
#include "paper_kernels.h"
#include "tiled_kernels.h"

using namespace cupso;

namespace {

thread_local char g_last_error[512] = "";

int fail(int code, const char* fmt, const char* detail = "") {
    std::snprintf(g_last_error, sizeof(g_last_error), fmt, detail);
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? CUPSO_ERR_OOM : CUPSO_ERR_CUDA;
}

#define CUPSO_CUDA(call, where)                      \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

void cupso::set_last_error(const char* msg) { std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

struct cupso_swarm {
    SwarmDev dev{};
    bool fp64 = false;              // a double-precision swarm: dev64 instead of dev
    SwarmDev64 dev64{};
    PaperBufs pbufs{};              // one-particle-per-thread designs (QUEUE, QUEUE_LOCK, FP64 modes)
    bool onchip64 = false;          // the FP64 swarm fits the on-chip kernel
    int N = 0, D = 0, Np = 0, fid = 0;
    uint64_t seed = 0;
    uint32_t swarm = 0;
    void* arena = nullptr;
    size_t arena_bytes = 0;
    cudaStream_t own = nullptr;     // the handle's non-blocking stream
    cudaStream_t stream = nullptr;  // where work is queued (own or the caller's)
    cudaStream_t capture = nullptr; // graphs are captured here, launched on `stream`
    int device = 0, num_sms = 1;
    int mode = CUPSO_MODE_AUTO;
    int graph_chunk = 16;
    cudaGraphExec_t graph = nullptr;
    int graph_mode = -1, graph_len = 0;
    uint32_t t_host = 0;
    int hold_lock = 0;
    int stall_barrier = 0;          // test hook: the multi-iteration panel launch waits for one CTA more
    int iters_per_launch = 0;       // panel SYNC step: iterations per launch, 0 = automatic
    int lsq_rescore = 0;            // CUPSO_OPT_LSQ_RESCORE: 0 float-float, 1 FP64
    int grid_override = 0;
    int onchip_cluster = 0;
    int sync_kernel = 0;            // CUPSO_SYNC_KERNEL_*
    int ppt_option = 0;             // particles per thread of the pipelined kernel, 0 = automatic
    bool pipelined_ok = false;      // shared-memory limit raised for the pipelined kernels
    bool panel_ok = false;          // the same for the panel kernels (D % 8 == 0)
    int panel = 0;                  // x, v, pb in the panel layout of this width (kernels_panel.cu), 0: dimension-major
    bool lazy_pending = false;      // the pipelined step may have left pbest rows unwritten
    // least-squares fitness (fitness_id CUPSO_LSQ), set by cupso_set_lsq
    struct Lsq {
        const float* A = nullptr;   // [M][D], borrowed
        const float* b = nullptr;   // [M], borrowed
        int M = 0, precision = 0;
        LsqTcState tc;              // BF16 / FP8 operands and plan
        void* buf = nullptr;        // f [Np] | cand [lists*16 + 16 + ticket] | partial [16 * chunks] | g64
        float* f = nullptr;
        unsigned long long* cand = nullptr;
        double* partial = nullptr;
        double* g64 = nullptr;
        unsigned int* flags = nullptr;   // [Np / 4]: improved this iteration (one byte per particle)
        int chunks = 32;                 // pieces of the FP64 rescoring per candidate (set with A)
        LsqGram gram;                    // A^T A etc. for the Gram-form rescoring when D <= M
        void* gram_buf = nullptr;
        bool time_fitness = false;       // CUPSO_OPT_TIME_FITNESS
        // the residual offsets of a new gbest are computed on a side stream while the
        // next move runs (fork and join events, also inside captured graphs)
        cudaStream_t side = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr;
        std::vector<cudaEvent_t> ev;     // pairs around the fitness phase
        double fitness_ms_sum = 0.0;
        int fitness_timed = 0;
    };
    Lsq* lsq = nullptr;
    // pinned host staging of the gbest reads (allocated on first use)
    void* pinned = nullptr;
    size_t pinned_bytes = 0;
    // result slots of cupso_gbest_post / _wait (allocated on first use): a
    // device record and a pinned host copy per slot, the copy stream, and per
    // slot the events of the snapshot and of its copy
    char* rec_dev = nullptr;
    char* rec_host = nullptr;
    cudaStream_t rec_stream = nullptr;
    cudaEvent_t rec_ev[2] = {nullptr, nullptr};
    cudaEvent_t rec_done[2] = {nullptr, nullptr};
    bool rec_posted[2] = {false, false};
};

namespace {

int resolved_mode(const cupso_swarm* h) {
    if (h->mode != CUPSO_MODE_AUTO) return h->mode;
    if (h->fp64) return h->onchip64 ? CUPSO_MODE_ONCHIP : CUPSO_MODE_SYNC;
    return h->onchip_cluster > 0 ? CUPSO_MODE_ONCHIP : CUPSO_MODE_SYNC;
}

// Particles per tile when the tiled SYNC kernel runs, else 0. AUTO takes it
// for D >= 8 up to the crossover measured on a GB300 against the pipelined
// kernel (which runs over d inside each thread and needs many particles per
// SM to hide its row latency): about 896 particles per SM, or 224 when the
// tiles are narrow (D > 64, so at most 32 particles per tile) and the fitness
// is cheap (no cos(2 pi x) to spread over the threads).
int sync_tile(const cupso_swarm* h) {
    if (h->fp64) return 0;
    if (h->sync_kernel == CUPSO_SYNC_KERNEL_TILED) return tiled_particles(h->N, h->D, h->num_sms);
    if (h->sync_kernel != CUPSO_SYNC_KERNEL_AUTO || h->D < 8) return 0;
    const bool has_cos = h->fid == CUPSO_RASTRIGIN || h->fid == CUPSO_ACKLEY;
    if (h->panel_ok && h->D % 8 == 0) {
        // against the panel kernel running each cupso_step call in one cooperative
        // launch (sweep on one GB300, N = 4096 .. 262144, D = 16 .. 256, Rosenbrock and
        // Rastrigin, steps of 96 iterations): the tiled kernel is the faster one only
        // below 2^17 particle-dimensions
        const long long pd = (long long)h->N * h->D;
        return pd < (1ll << 17) ? tiled_particles(h->N, h->D, h->num_sms) : 0;
    }
    const long long per_sm = (has_cos || h->D <= 64) ? 896 : 224;
    if ((long long)h->N > per_sm * h->num_sms) return 0;
    return tiled_particles(h->N, h->D, h->num_sms);
}

// Blocks of the tiled kernel: one wave of resident blocks (or the grid option).
int tiled_grid(const cupso_swarm* h, int P) {
    if (h->grid_override > 0) return h->grid_override;
    return h->num_sms * tiled_blocks_per_sm(h->fid, P, h->D);
}

// Ring depth of the pipelined SYNC kernel, or 0 for the register kernel.
int sync_stages(const cupso_swarm* h) {
    int want = 0;
    switch (h->sync_kernel) {
        case CUPSO_SYNC_KERNEL_REGISTER: return 0;
        case CUPSO_SYNC_KERNEL_PIPELINED3: want = 3; break;
        case CUPSO_SYNC_KERNEL_PIPELINED4: want = 4; break;
        default:  // deepest ring the dimension count allows
            if (h->pipelined_ok && pipelined_supported(4, h->D)) return 4;
            want = 3;
            break;
    }
    return (h->pipelined_ok && pipelined_supported(want, h->D)) ? want : 0;
}

// The panel SYNC kernel (the state in the panel layout) when it runs: its
// panel width and ring depth (5 panels where the panels allow, else 3); width
// 0 when the dimension-major kernels run. AUTO takes the panel kernel for
// D % 8 == 0 wherever the tiled kernel is not the faster one; 16-dimension
// panels for D >= 128 or up to 8192 particles, 8-dimension panels otherwise
// (Rosenbrock 2^20 x 64: a tie, 0.239 ms per iteration either way).
struct PanelCfg {
    int width = 0, stages = 0;
};
PanelCfg panel_cfg(const cupso_swarm* h) {
    PanelCfg c;
    if (h->fp64 || !h->panel_ok || h->fid == CUPSO_LSQ) return c;
    int widths[2] = {0, 0};
    switch (h->sync_kernel) {
        case CUPSO_SYNC_KERNEL_PANEL8: widths[0] = 8; break;
        case CUPSO_SYNC_KERNEL_PANEL16: widths[0] = 16; break;
        case CUPSO_SYNC_KERNEL_AUTO:
            if (sync_tile(h)) return c;
            // 16-dimension panels (units of 8 particles) for long particles (D >= 128)
            // and for swarms of up to 8192 particles, 8 otherwise (the same sweep; where
            // the other width wins, by at most 10 %, the units divide unevenly over
            // the warps)
            if (h->D % 16 == 0 && (h->D >= 128 || h->N <= 8192)) widths[0] = 16;
            widths[1] = 8;
            break;
        default: return c;
    }
    for (int w : widths) {
        if (!w) continue;
        for (int st : {5, 3})
            if (panel_supported(w, st, h->D)) {
                c.width = w;
                c.stages = st;
                return c;
            }
    }
    return c;
}

// Particles per thread of the pipelined kernel: 4 when the swarm has enough
// 128-particle units to keep every resident warp busy twice over, else fewer
// (more, smaller units).
int sync_ppt(const cupso_swarm* h) {
    if (h->ppt_option) return h->ppt_option;
    const long long resident_warps = (long long)h->num_sms * 16;
    if ((long long)h->Np >= 128ll * 2 * resident_warps) return 4;
    if ((long long)h->Np >= 64ll * resident_warps) return 2;
    return 1;
}

int sync_grid(const cupso_swarm* h) {
    const PanelCfg pc = panel_cfg(h);
    if (pc.width) {
        // persistent: warps pull units of 128 / width particles from a counter
        const int units = h->Np / (128 / pc.width);
        int g = h->grid_override > 0 ? h->grid_override
                                     : h->num_sms * panel_blocks_per_sm(pc.width, pc.stages, h->fid, h->D);
        const int useful = (units + kBlock / 32 - 1) / (kBlock / 32);
        return g < useful ? g : useful;
    }
    const int stages = sync_stages(h);
    if (stages) {
        // persistent: warps pull units of 32 * ppt particles from a counter
        const int ppt = sync_ppt(h);
        const int units = h->Np / (32 * ppt);
        const int per_sm = pipelined_blocks_per_sm(stages, h->fid, h->D, ppt);
        int g = h->grid_override > 0 ? h->grid_override : h->num_sms * per_sm;
        const int useful = (units + kBlock / 32 - 1) / (kBlock / 32);
        return g < useful ? g : useful;
    }
    const int ntiles = tiles_of(h->Np);
    int g = h->grid_override > 0 ? h->grid_override : h->num_sms * sync_blocks_per_sm(h->fid, h->D);
    return g < ntiles ? g : ntiles;
}

// Iterations per launch of the panel SYNC step: the option, else all of a
// cupso_step call up to kPanelMaxIters.
int panel_iters_per_launch(const cupso_swarm* h) {
    return h->iters_per_launch > 0 ? h->iters_per_launch : kPanelMaxIters;
}

// CTAs of a multi-iteration panel launch: the SYNC grid, at most what the SMs
// hold at once (a cooperative launch).
int panel_persist_grid(const cupso_swarm* h, const PanelCfg& pc) {
    const int resident = h->num_sms * panel_blocks_per_sm(pc.width, pc.stages, h->fid, h->D);
    return std::min(sync_grid(h), resident);
}

// ASYNC uses small CTAs when the swarm is small, so that it still spreads
// over many independently running CTAs.
int async_block(const cupso_swarm* h) {
    return (h->Np / kTile >= 2 * h->num_sms) ? kBlock : 32;
}

// Particles per tile of the tiled asynchronous kernel (0: the streaming one),
// by the crossover of the synchronous kernels: tiles where the tiled SYNC
// kernel is the faster one, else the streaming layout, which large swarms fill.
int async_tile(const cupso_swarm* h) {
    if (h->fp64 || h->D < 2) return 0;
    const bool has_cos = h->fid == CUPSO_RASTRIGIN || h->fid == CUPSO_ACKLEY;
    const long long per_sm = (has_cos || h->D <= 64) ? 896 : 224;
    if ((long long)h->N > per_sm * h->num_sms) return 0;
    return tiled_particles(h->N, h->D, h->num_sms);
}

int async_grid(const cupso_swarm* h) {
    if (const int P = async_tile(h)) {
        const int tiles = (h->N + P - 1) / P;
        const int g = h->grid_override > 0 ? h->grid_override : h->num_sms * async_tiled_blocks_per_sm(P, h->D);
        return g < tiles ? g : tiles;
    }
    const int tile = async_block(h) * kPerThread;
    const int ntiles = (h->Np + tile - 1) / tile;
    const int per_sm = async_blocks_per_sm(h->fid, h->D) * (kBlock / async_block(h));
    int g = h->grid_override > 0 ? h->grid_override : h->num_sms * per_sm;
    return g < ntiles ? g : ntiles;
}

void drop_graph(cupso_swarm* h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_mode = -1;
    h->graph_len = 0;
}

constexpr int kModeLsq = 100;   // internal: one least-squares iteration

// The tensor-core precisions: approximate fitness, FP64-verified gbest.
bool lsq_approx(int precision) { return precision == CUPSO_LSQ_BF16 || precision == CUPSO_LSQ_FP8; }

cudaError_t launch_lsq_iteration(cupso_swarm* h, cudaStream_t st) {
    cupso_swarm::Lsq& L = *h->lsq;
    const int grid = h->num_sms * 8;   // grid-stride over (particle group, dimension) items
    if (!lsq_approx(L.precision)) {
        cudaError_t e = lsq_launch_move(h->dev, grid, st);
        if (e == cudaSuccess)
            e = L.precision == CUPSO_LSQ_FP64 ? lsq_fp64_launch(h->dev.x, h->Np, h->N, h->D, L.A, L.b, L.M, L.f, st)
                                              : lsq_fp32_launch(h->dev.x, h->Np, h->N, h->D, L.A, L.b, L.M, L.f, st);
        if (e != cudaSuccess) return e;
        return lsq_launch_select_exact(h->dev, L.f, L.flags, grid, st);
    }
    // The residual offsets of the gbest this iteration moves towards (recomputed
    // only if the last acceptance moved it) run beside the move, which is
    // bound by HBM; the product, which adds them, waits for both. The move
    // writes the tensor-core operand too; the fitness is then the product alone.
    cudaError_t e = cudaEventRecord(L.fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(L.side, L.fork, 0);
    if (e == cudaSuccess) e = lsq_launch_offsets(h->dev, L.A, L.b, L.M, L.tc.roff, L.tc.roff_stale, h->num_sms, L.side);
    if (e == cudaSuccess) e = cudaEventRecord(L.join, L.side);
    if (e == cudaSuccess)
        e = lsq_launch_move_q(h->dev, L.tc.tmMove, L.tc.Xq, L.tc.Kp, L.tc.fp8, L.tc.sx, h->num_sms, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, L.join, 0);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (L.time_fitness) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
    }
    // the product leaves partial sums; the selection kernel adds them
    if (lsq_eval_tc_partials(&L.tc, st) != CUPSO_OK) return cudaErrorLaunchFailure;
    if (L.time_fitness) {
        cudaEventRecord(e1, st);
        L.ev.push_back(e0);
        L.ev.push_back(e1);
    }
    // offsets for the gbest this iteration accepts: at the start of the next one
    return lsq_launch_gbest_approx(h->dev, nullptr, L.tc.part, lsq_tc_partials(L.tc.plan), 0, true, L.A, L.b, L.M,
                                   L.cand, L.partial, L.chunks, L.g64, reinterpret_cast<unsigned int*>(h->dev.pflag),
                                   grid, L.gram, nullptr, L.tc.roff_stale, h->num_sms, st);
}

// gbest of an approximate-fitness swarm from scratch, with `fit` (device, [Np])
// as every particle's approximate fitness: the 16 lowest are rescored
// and the best becomes gbest (and the reference point of the tensor-core
// fitness, whose offsets are recomputed). t_dev ends at t.
cudaError_t lsq_reset_gbest(cupso_swarm* h, const float* fit, uint32_t t, cudaStream_t st) {
    cupso_swarm::Lsq& L = *h->lsq;
    const double inf = INFINITY;
    cudaError_t e = cudaMemcpyAsync(L.g64, &inf, sizeof(double), cudaMemcpyHostToDevice, st);
    // the accept kernel advances t: start one below and let it land on t
    if (e == cudaSuccess) e = lsq_launch_set_t(h->dev, t - 1u, st);
    if (e == cudaSuccess)
        e = lsq_launch_gbest_approx(h->dev, fit, nullptr, 0, 1, true, L.A, L.b, L.M, L.cand, L.partial, L.chunks,
                                    L.g64, reinterpret_cast<unsigned int*>(h->dev.pflag), h->num_sms * 8, L.gram,
                                    L.tc.roff, L.tc.roff_stale, h->num_sms, st);
    return e;
}

cudaError_t launch_one64(cupso_swarm* h, int mode, cudaStream_t st) {
    switch (mode) {
        case CUPSO_MODE_SYNC: return launch_step64(h->dev64, h->pbufs, h->fid, kAggSyncList, h->num_sms, st);
        case CUPSO_MODE_TREE: return launch_step64(h->dev64, h->pbufs, h->fid, kAggReduce, h->num_sms, st);
        case CUPSO_MODE_TREE_UNROLLED: return launch_step64(h->dev64, h->pbufs, h->fid, kAggReduceUnrolled, h->num_sms, st);
        case CUPSO_MODE_QUEUE: return launch_step64(h->dev64, h->pbufs, h->fid, kAggQueue, h->num_sms, st);
        case CUPSO_MODE_QUEUE_LOCK: return launch_step64(h->dev64, h->pbufs, h->fid, kAggQueueLock, h->num_sms, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_one(cupso_swarm* h, int mode, cudaStream_t st) {
    if (h->fp64) return launch_one64(h, mode, st);
    switch (mode) {
        case kModeLsq: return launch_lsq_iteration(h, st);
        case CUPSO_MODE_SYNC: {
            const PanelCfg pc = panel_cfg(h);
            if (pc.width) return launch_sync_panel(h->dev, h->fid, pc.width, pc.stages, sync_grid(h), 1, false, st);
            if (const int P = sync_tile(h))
                return launch_sync_tiled(h->dev, h->fid, P, tiled_grid(h, P), st);
            const int stages = sync_stages(h);
            if (stages) return launch_sync_pipelined(h->dev, h->fid, stages, sync_ppt(h), sync_grid(h), st);
            return launch_sync_step(h->dev, h->fid, sync_grid(h), st);
        }
        case CUPSO_MODE_TREE: return launch_tree_step(h->dev, h->fid, false, st);
        case CUPSO_MODE_TREE_UNROLLED: return launch_tree_step(h->dev, h->fid, true, st);
        case CUPSO_MODE_QUEUE: return launch_queue_step(h->dev, h->pbufs, h->fid, false, st);
        case CUPSO_MODE_QUEUE_LOCK: return launch_queue_step(h->dev, h->pbufs, h->fid, true, st);
        default: return cudaErrorInvalidValue;
    }
}

// Before any kernel that reads pbest_pos directly: write back the rows the
// pipelined step left pending.
int ensure_materialized(cupso_swarm* h) {
    if (h->fp64 || !h->lazy_pending) return CUPSO_OK;
    cudaError_t e;
    if (h->panel) {
        const int grid = std::max(1, std::min(h->num_sms * 8, (h->Np + kBlock - 1) / kBlock));
        e = launch_materialize_panel(h->dev, h->panel, grid, h->stream);
    } else {
        const int grid = std::max(1, std::min(h->num_sms * 8, (h->Np / 4 + kBlock - 1) / kBlock));
        e = launch_materialize(h->dev, grid, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "materialize launch");
    h->lazy_pending = false;
    return CUPSO_OK;
}

// Puts pos, v and pbest_pos in the layout the next kernel reads: the panel
// layout of width `want` (8 or 16) for the panel SYNC kernel, the
// dimension-major one (want 0) for every other kernel. Pending pbest rows are
// written back first; each array goes through a temporary copy (one array's
// size, freed again). Not for stream capture.
int ensure_layout(cupso_swarm* h, int want) {
    if (h->fp64 || h->panel == want) return CUPSO_OK;
    int rc = ensure_materialized(h);
    if (rc) return rc;
    drop_graph(h);
    const size_t bytes = sizeof(float) * (size_t)h->D * (size_t)h->Np;
    void* tmp = nullptr;
    CUPSO_CUDA(cudaMalloc(&tmp, bytes), "cudaMalloc (relayout)");
    float* arrays[3] = {h->dev.x, h->dev.v, h->dev.pb};
    const int grid = h->num_sms * 8;
    cudaError_t e = cudaSuccess;
    // at most two passes: out of the current panel width, into the wanted one
    const int passes[2][2] = {{h->panel, 0}, {want, 1}};
    for (const auto& ps : passes) {
        if (!ps[0]) continue;
        for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
            e = launch_relayout(arrays[a], static_cast<float*>(tmp), h->D, h->Np, ps[0], ps[1] != 0, grid, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(arrays[a], tmp, bytes, cudaMemcpyDeviceToDevice, h->stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "relayout");
    h->panel = want;
    return CUPSO_OK;
}

// A graph of `len` iterations. The kernels read the iteration counter from
// device memory, so one captured graph serves every later chunk.
int ensure_graph(cupso_swarm* h, int mode, int len) {
    if (h->graph && h->graph_mode == mode && h->graph_len == len) return CUPSO_OK;
    drop_graph(h);
    if (!h->capture) CUPSO_CUDA(cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking), "cudaStreamCreate");
    CUPSO_CUDA(cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < len && le == cudaSuccess; ++k) le = launch_one(h, mode, h->capture);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(h->capture, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(le, "kernel launch during capture");
    }
    if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        h->graph = nullptr;
        return cuda_fail(ie, "cudaGraphInstantiate");
    }
    h->graph_mode = mode;
    h->graph_len = len;
    return CUPSO_OK;
}

}  // namespace

int cupso::check_problem_args(int D, int N, const cupso_bounds* b, float w, float c1, float c2, int fid) {
    if (D < 1 || N < 1) return fail(CUPSO_ERR_INVALID_ARG, "D and N must be >= 1%s");
    if ((long long)N > (long long)0x7FFFFFFF - kPad) return fail(CUPSO_ERR_INVALID_ARG, "N too large%s");
    const long long Np = ((long long)N + kPad - 1) / kPad * kPad;
    if (Np * (long long)D >= (1ll << 31)) return fail(CUPSO_ERR_INVALID_ARG, "N * D must be < 2^31%s");
    if (!b) return fail(CUPSO_ERR_INVALID_ARG, "bounds is NULL%s");
    if (!std::isfinite(b->min_pos) || !std::isfinite(b->max_pos) || !std::isfinite(b->max_v))
        return fail(CUPSO_ERR_INVALID_ARG, "bounds must be finite%s");
    if (!(b->min_pos < b->max_pos)) return fail(CUPSO_ERR_INVALID_ARG, "min_pos must be < max_pos%s");
    if (!(b->max_v > 0.0f)) return fail(CUPSO_ERR_INVALID_ARG, "max_v must be > 0%s");
    if (!std::isfinite(w) || !std::isfinite(c1) || !std::isfinite(c2))
        return fail(CUPSO_ERR_INVALID_ARG, "w, c1, c2 must be finite%s");
    if (fid < CUPSO_SPHERE || fid > CUPSO_LSQ) return fail(CUPSO_ERR_INVALID_ARG, "unknown fitness_id%s");
    return CUPSO_OK;
}

namespace {

int create_swarm(int D, int N, const cupso_bounds* b, float w, float c1, float c2, int fid, uint64_t seed,
                 uint32_t swarm, cudaStream_t user_stream, cupso_handle* out) {
    if (!out) return fail(CUPSO_ERR_INVALID_ARG, "out is NULL%s");
    *out = nullptr;
    int rc = check_problem_args(D, N, b, w, c1, c2, fid);
    if (rc) return rc;
    cupso_swarm* h = new (std::nothrow) cupso_swarm();
    if (!h) return fail(CUPSO_ERR_OOM, "host allocation failed%s");
    h->N = N;
    h->D = D;
    h->Np = (N + kPad - 1) / kPad * kPad;
    h->fid = fid;
    h->seed = seed;
    h->swarm = swarm;
    auto bail = [&](int code) {
        cupso_destroy(h);
        return code;
    };
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaDeviceGetAttribute"));
    e = cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));
    h->stream = user_stream ? user_stream : h->own;

    // One arena: x, v, pb [D][Np]; pf [Np]; G [2][D]; Grec [D]; aux; words.
    const size_t A = 256;
    const size_t plane = sizeof(float) * (size_t)D * (size_t)h->Np;
    const size_t ntiles = (size_t)tiles_of(h->Np);
    size_t off = 0;
    const size_t o_x = off; off = align_up(off + plane, A);
    const size_t o_v = off; off = align_up(off + plane, A);
    const size_t o_pb = off; off = align_up(off + plane, A);
    const size_t o_pf = off; off = align_up(off + sizeof(float) * (size_t)h->Np, A);
    const size_t o_G = off; off = align_up(off + sizeof(float) * 2 * (size_t)D, A);
    const size_t o_Grec = off; off = align_up(off + sizeof(float) * (size_t)D, A);
    const size_t o_aux = off; off = align_up(off + sizeof(unsigned long long) * ntiles, A);
    const size_t o_flag = off; off = align_up(off + (size_t)h->Np, A);
    const size_t o_words = off; off = align_up(off + 128, A);
    const int list_cap = paper_blocks(h->Np);      // one candidate per block of the queue designs
    const size_t o_paper = off; off = align_up(off + paper_bufs_bytes(h->Np, list_cap), A);
    h->arena_bytes = off;
    e = cudaMalloc(&h->arena, h->arena_bytes);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    char* base = static_cast<char*>(h->arena);
    SwarmDev& s = h->dev;
    s.x = reinterpret_cast<float*>(base + o_x);
    s.v = reinterpret_cast<float*>(base + o_v);
    s.pb = reinterpret_cast<float*>(base + o_pb);
    s.pf = reinterpret_cast<float*>(base + o_pf);
    s.G = reinterpret_cast<float*>(base + o_G);
    s.Grec = reinterpret_cast<float*>(base + o_Grec);
    s.aux = reinterpret_cast<unsigned long long*>(base + o_aux);
    s.pflag = reinterpret_cast<unsigned char*>(base + o_flag);
    unsigned long long* w64 = reinterpret_cast<unsigned long long*>(base + o_words);
    s.gkey = w64;        // [2]
    s.claim = w64 + 2;
    s.reckey = w64 + 3;
    unsigned int* w32 = reinterpret_cast<unsigned int*>(w64 + 4);
    s.ticket = w32 + 0;
    s.t_dev = w32 + 1;
    s.status = w32 + 2;
    s.lock = w32 + 3;
    s.seq = w32 + 4;
    s.work = w32 + 5;
    s.bar = w32 + 6;
    s.N = N;
    s.D = D;
    s.Np = h->Np;
    s.lo = b->min_pos;
    s.hi = b->max_pos;
    s.vmax = b->max_v;
    s.w = w;
    s.c1 = c1;
    s.c2 = c2;
    s.key0 = (uint32_t)(seed & 0xFFFFFFFFull);
    s.key1 = (uint32_t)(seed >> 32);
    philox_round_keys(s.key0, s.key1, s.rk0, s.rk1);
    s.swarm = swarm;
    s.wait_limit_ns = 2000000000ll;
    h->pbufs = paper_bufs_at(base + o_paper, h->Np, list_cap);
    // c * 2^-24 is exact unless it would be subnormal; check by scaling back.
    s.c1s = std::ldexp(c1, -24);
    s.c2s = std::ldexp(c2, -24);
    s.fast_cr = (std::ldexp(s.c1s, 24) == c1 && std::ldexp(s.c2s, 24) == c2 &&
                 (c1 == 0.0f || std::fabs(s.c1s) >= FLT_MIN) && (c2 == 0.0f || std::fabs(s.c2s) >= FLT_MIN))
                    ? 1 : 0;
    s.fast_clamp = (b->min_pos != 0.0f && b->max_pos != 0.0f) ? 1 : 0;

    int cl = 0, per = 0;
    h->onchip_cluster = (fid != CUPSO_LSQ && onchip_fits(N, D, &cl, &per)) ? cl : 0;
    h->pipelined_ok = prepare_pipelined(D) == cudaSuccess;
    h->panel_ok = fid != CUPSO_LSQ && panel_supported(8, 3, D) && prepare_panel(D) == cudaSuccess;
    cudaGetLastError();

    e = cudaMemsetAsync(base + o_words, 0, 128, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.pflag, 0, (size_t)h->Np, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.gkey, 0xFF, 2 * sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_paper, 0, paper_bufs_bytes(h->Np, list_cap), h->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemsetAsync"));
    const int grid = std::min(tiles_of(h->Np), h->num_sms * 4);
    e = launch_init(s, fid, grid, h->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "init launch"));
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "init"));
    *out = h;
    return CUPSO_OK;
}

// k when c = 2^k exactly with |k| <= 512 (c r is then an exponent shift of a
// uniform in (2^-53, 1], which stays normal), else kNoExp.
int pow2_exponent(double c) {
    if (!(c > 0.0) || !std::isfinite(c)) return kNoExp;
    int e = 0;
    const double m = std::frexp(c, &e);   // c = m 2^e, m in [0.5, 1)
    if (m != 0.5) return kNoExp;
    const int k = e - 1;
    return (k >= -512 && k <= 512) ? k : kNoExp;
}

// A double-precision swarm: arena x, v, pb [D][Np], pf [Np], G [2][D]
// (binary64), gbest keys, counters, and the working storage of the
// one-particle-per-thread kernels.
int create_swarm64(int D, int N, const cupso_bounds_f64* b, double w, double c1, double c2, int fid, uint64_t seed,
                   cupso_handle* out) {
    if (!out) return fail(CUPSO_ERR_INVALID_ARG, "out is NULL%s");
    *out = nullptr;
    if (D < 1 || N < 1) return fail(CUPSO_ERR_INVALID_ARG, "D and N must be >= 1%s");
    if ((long long)N > (long long)0x7FFFFFFF - kPad) return fail(CUPSO_ERR_INVALID_ARG, "N too large%s");
    const long long Npl = ((long long)N + kPad - 1) / kPad * kPad;
    if (Npl * (long long)D >= (1ll << 31)) return fail(CUPSO_ERR_INVALID_ARG, "N * D must be < 2^31%s");
    if (!b) return fail(CUPSO_ERR_INVALID_ARG, "bounds is NULL%s");
    if (!std::isfinite(b->min_pos) || !std::isfinite(b->max_pos) || !std::isfinite(b->max_v))
        return fail(CUPSO_ERR_INVALID_ARG, "bounds must be finite%s");
    if (!(b->min_pos < b->max_pos)) return fail(CUPSO_ERR_INVALID_ARG, "min_pos must be < max_pos%s");
    if (!(b->max_v > 0.0)) return fail(CUPSO_ERR_INVALID_ARG, "max_v must be > 0%s");
    if (!std::isfinite(w) || !std::isfinite(c1) || !std::isfinite(c2))
        return fail(CUPSO_ERR_INVALID_ARG, "w, c1, c2 must be finite%s");
    if (fid < CUPSO_SPHERE || fid > CUPSO_LSQ) return fail(CUPSO_ERR_INVALID_ARG, "unknown fitness_id%s");
    if (!fp64_fitness_supported(fid))
        return fail(CUPSO_ERR_UNSUPPORTED, "double precision supports sphere, Rosenbrock and the cubic%s");
    cupso_swarm* h = new (std::nothrow) cupso_swarm();
    if (!h) return fail(CUPSO_ERR_OOM, "host allocation failed%s");
    h->fp64 = true;
    h->N = N;
    h->D = D;
    h->Np = (int)Npl;
    h->fid = fid;
    h->seed = seed;
    auto bail = [&](int code) {
        cupso_destroy(h);
        return code;
    };
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaDeviceGetAttribute"));
    e = cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));
    h->stream = h->own;

    const size_t A = 256;
    const size_t plane = sizeof(double) * (size_t)D * (size_t)h->Np;
    size_t off = 0;
    const size_t o_x = off; off = align_up(off + plane, A);
    const size_t o_v = off; off = align_up(off + plane, A);
    const size_t o_pb = off; off = align_up(off + plane, A);
    const size_t o_pf = off; off = align_up(off + sizeof(double) * (size_t)h->Np, A);
    const size_t o_G = off; off = align_up(off + sizeof(double) * 2 * (size_t)D, A);
    const size_t o_key = off; off = align_up(off + 2 * sizeof(PKey), A);
    const size_t o_words = off; off = align_up(off + 64, A);
    const int list_cap = h->Np;   // the tiled step may run up to one block per particle
    const size_t o_paper = off; off = align_up(off + paper_bufs_bytes(h->Np, list_cap), A);
    h->arena_bytes = off;
    e = cudaMalloc(&h->arena, h->arena_bytes);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    char* base = static_cast<char*>(h->arena);
    SwarmDev64& s = h->dev64;
    s.x = reinterpret_cast<double*>(base + o_x);
    s.v = reinterpret_cast<double*>(base + o_v);
    s.pb = reinterpret_cast<double*>(base + o_pb);
    s.pf = reinterpret_cast<double*>(base + o_pf);
    s.G = reinterpret_cast<double*>(base + o_G);
    s.gkey = reinterpret_cast<PKey*>(base + o_key);
    unsigned int* w32 = reinterpret_cast<unsigned int*>(base + o_words);
    s.t_dev = w32 + 0;
    s.status = w32 + 1;
    s.N = N;
    s.D = D;
    s.Np = h->Np;
    s.lo = b->min_pos;
    s.hi = b->max_pos;
    s.vmax = b->max_v;
    s.w = w;
    s.c1 = c1;
    s.c2 = c2;
    s.key0 = (uint32_t)(seed & 0xFFFFFFFFull);
    s.key1 = (uint32_t)(seed >> 32);
    s.swarm = 0u;
    s.wait_limit_ns = 2000000000ll;
    s.w_one = (w == 1.0) ? 1 : 0;
    s.c1_exp = pow2_exponent(c1);
    s.c2_exp = pow2_exponent(c2);
    s.k_lo = order_key64(b->min_pos);
    s.k_hi = order_key64(b->max_pos);
    s.k_vlo = order_key64(-b->max_v);
    s.k_vhi = order_key64(b->max_v);
    h->dev.wait_limit_ns = s.wait_limit_ns;
    h->dev.status = s.status;
    h->pbufs = paper_bufs_at(base + o_paper, h->Np, list_cap);
    h->onchip_cluster = onchip64_cluster(N, D);
    h->onchip64 = h->onchip_cluster > 0;
    cudaGetLastError();

    e = cudaMemsetAsync(base + o_words, 0, 64, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.gkey, 0xFF, 2 * sizeof(PKey), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_paper, 0, paper_bufs_bytes(h->Np, list_cap), h->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemsetAsync"));
    e = launch_init64(s, h->pbufs, fid, h->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "init launch"));
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "init"));
    *out = h;
    return CUPSO_OK;
}

// Pinned staging for small reads: async copies into pinned memory need no
// host-side staging and finish with one stream synchronisation.
int ensure_pinned(cupso_swarm* h, size_t bytes) {
    if (h->pinned_bytes >= bytes) return CUPSO_OK;
    if (h->pinned) cudaFreeHost(h->pinned);
    h->pinned = nullptr;
    h->pinned_bytes = 0;
    CUPSO_CUDA(cudaMallocHost(&h->pinned, bytes), "cudaMallocHost");
    h->pinned_bytes = bytes;
    return CUPSO_OK;
}

int status_code(unsigned st) {
    if (st & kStatusBadArg) return CUPSO_ERR_CUDA;   // a device-side bound check dropped work
    if (st & kStatusTimeout) return CUPSO_ERR_DEVICE_TIMEOUT;
    if (st & kStatusNaN) return CUPSO_ERR_NAN;
    return CUPSO_OK;
}

double key_to_fit64(unsigned long long key) {
    if (key == ~0ull) return NAN;
    const unsigned long long bits = (key >> 63) ? (key & 0x7FFFFFFFFFFFFFFFull) : ~key;
    double f;
    std::memcpy(&f, &bits, 8);
    return f;
}

float key_to_fit(unsigned long long key) {
    const uint32_t k = (uint32_t)(key >> 32);
    if (k == 0xFFFFFFFFu) return NAN;
    const uint32_t bits = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    float f;
    std::memcpy(&f, &bits, 4);
    return f;
}

}  // namespace

// One problem solved through its own handle: create, `iters` steps, gbest.
int cupso::solve_one_plain(const cupso_problem& p, int iters, cupso_result& r, cudaStream_t stream) {
    cupso_handle h = nullptr;
    int rc = create_swarm(p.D, p.N, &p.bounds, p.w, p.c1, p.c2, p.fitness_id, p.seed, p.swarm_id, stream, &h);
    if (rc == CUPSO_OK) rc = cupso_step(h, iters);
    if (rc == CUPSO_OK) rc = cupso_get_gbest(h, &r.fit, r.pos, &r.idx);
    r.status = rc;
    if (h) cupso_destroy(h);
    return rc;
}

void cupso::set_cuda_error(cudaError_t e, const char* where) { cuda_fail(e, where); }

namespace {

// Bytes of one result record: key at 0, status at 8, position from 32.
size_t rec_bytes(int D) { return (32 + sizeof(float) * (size_t)D + 255) / 256 * 256; }

// gbest of one parity -- its key, the sticky status and its position -- into
// a contiguous record.
__global__ void gbest_record_kernel(const unsigned long long* __restrict__ key, const unsigned* __restrict__ status,
                                    const float* __restrict__ G, int D, char* __restrict__ rec) {
    float* pos = reinterpret_cast<float*>(rec + 32);
    for (int d = threadIdx.x; d < D; d += blockDim.x) pos[d] = __ldcg(G + d);
    if (threadIdx.x == 0) {
        *reinterpret_cast<unsigned long long*>(rec) = __ldcg(key);
        *reinterpret_cast<unsigned*>(rec + 8) = __ldcg(status);
    }
}

int ensure_records(cupso_swarm* h) {
    if (h->rec_dev) return CUPSO_OK;
    const size_t bytes = 2 * rec_bytes(h->D);
    CUPSO_CUDA(cudaMalloc(&h->rec_dev, bytes), "cudaMalloc (gbest records)");
    CUPSO_CUDA(cudaMallocHost(&h->rec_host, bytes), "cudaMallocHost (gbest records)");
    CUPSO_CUDA(cudaStreamCreateWithFlags(&h->rec_stream, cudaStreamNonBlocking), "cudaStreamCreate");
    for (int k = 0; k < 2; ++k) {
        CUPSO_CUDA(cudaEventCreateWithFlags(&h->rec_ev[k], cudaEventDisableTiming), "cudaEventCreate");
        CUPSO_CUDA(cudaEventCreateWithFlags(&h->rec_done[k], cudaEventDisableTiming), "cudaEventCreate");
    }
    return CUPSO_OK;
}

}  // namespace

extern "C" {

int cupso_create(int D, int N, const cupso_bounds* bounds, float w, float c1, float c2, int fitness_id,
                 uint64_t seed, cupso_handle* out) {
    return create_swarm(D, N, bounds, w, c1, c2, fitness_id, seed, 0u, nullptr, out);
}

int cupso_set_stream(cupso_handle h, void* cuda_stream) {
    if (!h) return fail(CUPSO_ERR_INVALID_ARG, "handle is NULL%s");
    h->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : h->own;
    return CUPSO_OK;
}

int cupso_set_option(cupso_handle h, int key, long long value) {
    if (!h) return fail(CUPSO_ERR_INVALID_ARG, "handle is NULL%s");
    switch (key) {
        case CUPSO_OPT_MODE:
            if (value < CUPSO_MODE_AUTO || value > CUPSO_MODE_PERSISTENT)
                return fail(CUPSO_ERR_INVALID_ARG, "unknown mode%s");
            if (value == CUPSO_MODE_PERSISTENT && (!h->fp64 || h->D > 4096))
                return fail(CUPSO_ERR_UNSUPPORTED, "the persistent mode serves double-precision swarms with D <= 4096%s");
            if (h->fp64) {
                if (value == CUPSO_MODE_ASYNC)
                    return fail(CUPSO_ERR_UNSUPPORTED, "double-precision swarms have no ASYNC mode%s");
                if (value == CUPSO_MODE_ONCHIP && !h->onchip64)
                    return fail(CUPSO_ERR_UNSUPPORTED, "swarm does not fit in one CTA's shared memory%s");
                h->mode = (int)value;
                return CUPSO_OK;
            }
            if (h->fid == CUPSO_LSQ && value != CUPSO_MODE_AUTO && value != CUPSO_MODE_SYNC)
                return fail(CUPSO_ERR_UNSUPPORTED, "least-squares swarms run the synchronous iteration only%s");
            if (value == CUPSO_MODE_ONCHIP && h->onchip_cluster == 0)
                return fail(CUPSO_ERR_UNSUPPORTED, "swarm does not fit in one cluster's shared memory%s");
            h->mode = (int)value;
            return CUPSO_OK;
        case CUPSO_OPT_GRAPH_CHUNK:
            if (value < 0 || value > 4096) return fail(CUPSO_ERR_INVALID_ARG, "graph chunk out of range%s");
            h->graph_chunk = (int)value;
            drop_graph(h);
            return CUPSO_OK;
        case CUPSO_OPT_WAIT_LIMIT_NS:
            if (value < 1000 || value > 60000000000ll) return fail(CUPSO_ERR_INVALID_ARG, "wait limit out of range%s");
            h->dev.wait_limit_ns = value;
            h->dev64.wait_limit_ns = value;
            drop_graph(h);
            return CUPSO_OK;
        case CUPSO_OPT_CLEAR_STATUS:
            // with the status, the counters a wait that expired may have left behind
            CUPSO_CUDA(cudaMemsetAsync(h->dev.status, 0, sizeof(unsigned), h->stream), "cudaMemsetAsync");
            CUPSO_CUDA(cudaMemsetAsync(h->dev.ticket, 0, sizeof(unsigned), h->stream), "cudaMemsetAsync");
            CUPSO_CUDA(cudaMemsetAsync(h->dev.work, 0, 2 * sizeof(unsigned), h->stream), "cudaMemsetAsync");
            return CUPSO_OK;
        case CUPSO_OPT_GRID:
            if (value < 0 || value > (1 << 20)) return fail(CUPSO_ERR_INVALID_ARG, "grid out of range%s");
            h->grid_override = (int)value;
            drop_graph(h);
            return CUPSO_OK;
        case CUPSO_OPT_SYNC_KERNEL:
            if (value < CUPSO_SYNC_KERNEL_AUTO || value > CUPSO_SYNC_KERNEL_PANEL16)
                return fail(CUPSO_ERR_INVALID_ARG, "unknown sync kernel%s");
            h->sync_kernel = (int)value;
            drop_graph(h);
            return CUPSO_OK;
        case CUPSO_OPT_TIME_FITNESS:
            if (!h->lsq) return fail(CUPSO_ERR_INVALID_ARG, "timing applies to least-squares swarms after cupso_set_lsq%s");
            h->lsq->time_fitness = value != 0;
            drop_graph(h);
            return CUPSO_OK;
        case CUPSO_OPT_PARTICLES_PER_THREAD:
            if (value != 0 && value != 1 && value != 2 && value != 4)
                return fail(CUPSO_ERR_INVALID_ARG, "particles per thread must be 0 (automatic), 1, 2 or 4%s");
            h->ppt_option = (int)value;
            drop_graph(h);
            return CUPSO_OK;
        case CUPSO_OPT_ITERS_PER_LAUNCH:
            if (value < 0 || value > kPanelMaxIters)
                return fail(CUPSO_ERR_INVALID_ARG, "iterations per launch out of range%s");
            h->iters_per_launch = (int)value;
            return CUPSO_OK;
        case CUPSO_OPT_LSQ_RESCORE:
            if (value != 0 && value != 1) return fail(CUPSO_ERR_INVALID_ARG, "rescoring: 0 (float-float) or 1 (FP64)%s");
            h->lsq_rescore = (int)value;
            if (h->lsq) h->lsq->gram.ff = value == 0;
            drop_graph(h);
            return CUPSO_OK;
        case CUPSO_OPT_FAULT_HOLD_LOCK:
            h->hold_lock = value ? 1 : 0;
            return CUPSO_OK;
        case CUPSO_OPT_FAULT_STALL_BARRIER:
            h->stall_barrier = value ? 1 : 0;
            return CUPSO_OK;
        default:
            return fail(CUPSO_ERR_INVALID_ARG, "unknown option%s");
    }
}

int cupso_step(cupso_handle h, int iters) {
    if (!h) return fail(CUPSO_ERR_INVALID_ARG, "handle is NULL%s");
    if (iters < 0) return fail(CUPSO_ERR_INVALID_ARG, "iters must be >= 0%s");
    if (iters == 0) return CUPSO_OK;
    if ((uint64_t)h->t_host + (uint64_t)iters > 0xFFFFFFFFull)
        return fail(CUPSO_ERR_INVALID_ARG, "iteration counter would overflow%s");
    if (h->fid == CUPSO_LSQ) {
        if (!h->lsq) return fail(CUPSO_ERR_INVALID_ARG, "least-squares swarm: call cupso_set_lsq first%s");
        int left = iters;
        const int L = h->lsq->time_fitness ? 0 : h->graph_chunk;
        if (L > 1 && left >= L) {
            int rc = ensure_graph(h, kModeLsq, L);
            if (rc) return rc;
            while (left >= L) {
                cudaError_t e = cudaGraphLaunch(h->graph, h->stream);
                if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
                left -= L;
            }
        }
        for (; left > 0; --left) {
            cudaError_t e = launch_lsq_iteration(h, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "least-squares iteration");
        }
        // the tensor-core iteration leaves improved pbest rows to the next move
        if (lsq_approx(h->lsq->precision)) h->lazy_pending = true;
        h->t_host += (uint32_t)iters;
        return CUPSO_OK;
    }
    const int mode = resolved_mode(h);
    if (h->fp64 && mode == CUPSO_MODE_ONCHIP) {
        cudaError_t e = launch_onchip64(h->dev64, h->fid, iters, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "on-chip launch");
        h->t_host += (uint32_t)iters;
        return CUPSO_OK;
    }
    if (h->fp64 && mode == CUPSO_MODE_PERSISTENT) {
        cudaError_t e = launch_persist64(h->dev64, h->pbufs, h->fid, iters, h->num_sms, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "persistent launch");
        h->t_host += (uint32_t)iters;
        return CUPSO_OK;
    }
    const int panel = (!h->fp64 && mode == CUPSO_MODE_SYNC) ? panel_cfg(h).width : 0;
    {
        const int rc = ensure_layout(h, panel);
        if (rc) return rc;
    }
    const bool pipelined =
        panel != 0 || (!h->fp64 && mode == CUPSO_MODE_SYNC && sync_tile(h) == 0 && sync_stages(h) > 0);
    if (!pipelined) {
        const int rc = ensure_materialized(h);
        if (rc) return rc;
    }
    cudaError_t e = cudaSuccess;
    if (mode == CUPSO_MODE_ASYNC) {
        if (const int P = async_tile(h))
            e = launch_async_tiled(h->dev, h->fid, P, async_grid(h), h->t_host + 1u, iters, h->hold_lock, h->stream);
        else
            e = launch_async(h->dev, h->fid, async_grid(h), async_block(h), h->t_host + 1u, iters, h->hold_lock,
                             h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "async launch");
    } else if (mode == CUPSO_MODE_ONCHIP) {
        e = launch_onchip(h->dev, h->fid, iters, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "on-chip launch");
    } else {
        int left = iters;
        const int P = panel ? panel_iters_per_launch(h) : 1;
        if (P > 1 && left > 1) {
            // several iterations per cooperative launch, a grid barrier between them
            const PanelCfg pc = panel_cfg(h);
            const int grid = panel_persist_grid(h, pc);
            while (left > 1) {
                const int n = std::min(left, P);
                e = cudaMemsetAsync(h->dev.work, 0, 2 * sizeof(unsigned), h->stream);
                if (e == cudaSuccess)
                    e = launch_sync_panel(h->dev, h->fid, pc.width, pc.stages, grid, n, h->stall_barrier != 0,
                                          h->stream);
                if (e != cudaSuccess) return cuda_fail(e, "panel launch");
                left -= n;
            }
        }
        const int L = h->graph_chunk;
        if (L > 1 && left >= L) {
            int rc = ensure_graph(h, mode, L);
            if (rc) return rc;
            while (left >= L) {
                e = cudaGraphLaunch(h->graph, h->stream);
                if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
                left -= L;
            }
        }
        for (; left > 0; --left) {
            e = launch_one(h, mode, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "step launch");
        }
    }
    if (pipelined) h->lazy_pending = true;
    h->t_host += (uint32_t)iters;
    return CUPSO_OK;
}

int cupso_get_gbest(cupso_handle h, float* fit_out, float* pos_out, int64_t* idx_out) {
    if (!h) return fail(CUPSO_ERR_INVALID_ARG, "handle is NULL%s");
    if (h->fp64) return fail(CUPSO_ERR_UNSUPPORTED, "double-precision swarm: use the _fp64 functions%s");
    const int cur = (int)(h->t_host & 1u);
    int rc = ensure_pinned(h, 32 + sizeof(float) * (size_t)h->D);
    if (rc) return rc;
    char* pin = static_cast<char*>(h->pinned);
    CUPSO_CUDA(cudaMemcpyAsync(pin, h->dev.gkey + cur, 8, cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync");
    CUPSO_CUDA(cudaMemcpyAsync(pin + 8, h->dev.status, 4, cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync");
    if (pos_out)
        CUPSO_CUDA(cudaMemcpyAsync(pin + 32, h->dev.G + (size_t)cur * h->D, sizeof(float) * (size_t)h->D,
                                   cudaMemcpyDeviceToHost, h->stream),
                   "cudaMemcpyAsync");
    CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    unsigned long long key = 0;
    unsigned st = 0;
    std::memcpy(&key, pin, 8);
    std::memcpy(&st, pin + 8, 4);
    if (pos_out) std::memcpy(pos_out, pin + 32, sizeof(float) * (size_t)h->D);
    if (fit_out) *fit_out = key_to_fit(key);
    if (idx_out) *idx_out = (int64_t)(key & 0xFFFFFFFFull);
    rc = status_code(st);
    if (rc) fail(rc, "device status set: %s", cupso_status_string(rc));
    return rc;
}

int cupso_gbest_post(cupso_handle h, int slot) {
    if (!h) return fail(CUPSO_ERR_INVALID_ARG, "handle is NULL%s");
    if (h->fp64) return fail(CUPSO_ERR_UNSUPPORTED, "double-precision swarm: use the _fp64 functions%s");
    if (slot != 0 && slot != 1) return fail(CUPSO_ERR_INVALID_ARG, "slot must be 0 or 1%s");
    if (h->rec_posted[slot]) return fail(CUPSO_ERR_INVALID_ARG, "slot already holds a result; wait for it first%s");
    int rc = ensure_records(h);
    if (rc) return rc;
    const size_t rb = rec_bytes(h->D);
    char* dev = h->rec_dev + (size_t)slot * rb;
    const int cur = (int)(h->t_host & 1u);
    // the snapshot follows the queued steps on the handle's stream; the next
    // step cannot change what it copies (a step rewrites these words only
    // after the stream reaches it). Its copy to the host runs on the second
    // stream, beside the next steps.
    gbest_record_kernel<<<1, 256, 0, h->stream>>>(h->dev.gkey + cur, h->dev.status, h->dev.G + (size_t)cur * h->D,
                                                  h->D, dev);
    CUPSO_CUDA(cudaGetLastError(), "gbest record launch");
    CUPSO_CUDA(cudaEventRecord(h->rec_ev[slot], h->stream), "cudaEventRecord");
    CUPSO_CUDA(cudaStreamWaitEvent(h->rec_stream, h->rec_ev[slot], 0), "cudaStreamWaitEvent");
    CUPSO_CUDA(cudaMemcpyAsync(h->rec_host + (size_t)slot * rb, dev, rb, cudaMemcpyDeviceToHost, h->rec_stream),
               "cudaMemcpyAsync");
    CUPSO_CUDA(cudaEventRecord(h->rec_done[slot], h->rec_stream), "cudaEventRecord");
    h->rec_posted[slot] = true;
    return CUPSO_OK;
}

int cupso_gbest_wait(cupso_handle h, int slot, float* fit_out, float* pos_out, int64_t* idx_out) {
    if (!h) return fail(CUPSO_ERR_INVALID_ARG, "handle is NULL%s");
    if (slot != 0 && slot != 1) return fail(CUPSO_ERR_INVALID_ARG, "slot must be 0 or 1%s");
    if (!h->rec_posted[slot]) return fail(CUPSO_ERR_INVALID_ARG, "nothing posted to this slot%s");
    CUPSO_CUDA(cudaEventSynchronize(h->rec_done[slot]), "cudaEventSynchronize");
    h->rec_posted[slot] = false;
    const char* rec = h->rec_host + (size_t)slot * rec_bytes(h->D);
    unsigned long long key = 0;
    unsigned st = 0;
    std::memcpy(&key, rec, 8);
    std::memcpy(&st, rec + 8, 4);
    if (pos_out) std::memcpy(pos_out, rec + 32, sizeof(float) * (size_t)h->D);
    if (fit_out) *fit_out = key_to_fit(key);
    if (idx_out) *idx_out = (int64_t)(key & 0xFFFFFFFFull);
    const int rc = status_code(st);
    if (rc) fail(rc, "device status set: %s", cupso_status_string(rc));
    return rc;
}

int cupso_get_state(cupso_handle h, float* pos, float* v, float* pbest_pos, float* pbest_fit, uint32_t* t_out) {
    if (!h) return fail(CUPSO_ERR_INVALID_ARG, "handle is NULL%s");
    if (h->fp64) return fail(CUPSO_ERR_UNSUPPORTED, "double-precision swarm: use the _fp64 functions%s");
    const size_t N = (size_t)h->N, D = (size_t)h->D, Np = (size_t)h->Np;
    std::vector<float> stage;
    float* outs[3] = {pos, v, pbest_pos};
    const float* srcs[3] = {h->dev.x, h->dev.v, h->dev.pb};
    const int mrc = ensure_materialized(h);
    if (mrc) return mrc;
    CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    for (int a = 0; a < 3; ++a) {
        if (!outs[a]) continue;
        stage.resize(D * Np);
        CUPSO_CUDA(cudaMemcpy(stage.data(), srcs[a], sizeof(float) * D * Np, cudaMemcpyDeviceToHost), "cudaMemcpy");
        if (h->panel) {   // element (d, i) at ((d / W) Np + i) W + d % W
            const size_t W = (size_t)h->panel;
            for (size_t i = 0; i < N; ++i)
                for (size_t d = 0; d < D; ++d) outs[a][i * D + d] = stage[((d / W) * Np + i) * W + (d % W)];
        } else {
            for (size_t i = 0; i < N; ++i)
                for (size_t d = 0; d < D; ++d) outs[a][i * D + d] = stage[d * Np + i];
        }
    }
    if (pbest_fit)
        CUPSO_CUDA(cudaMemcpy(pbest_fit, h->dev.pf, sizeof(float) * N, cudaMemcpyDeviceToHost), "cudaMemcpy");
    if (t_out) *t_out = h->t_host;
    return CUPSO_OK;
}

int cupso_set_state(cupso_handle h, const float* pos, const float* v, const float* pbest_pos,
                    const float* pbest_fit, uint32_t t) {
    if (!h) return fail(CUPSO_ERR_INVALID_ARG, "handle is NULL%s");
    if (h->fp64) return fail(CUPSO_ERR_UNSUPPORTED, "double-precision swarm: use the _fp64 functions%s");
    if (!pos || !v || !pbest_pos || !pbest_fit) return fail(CUPSO_ERR_INVALID_ARG, "state array is NULL%s");
    const size_t N = (size_t)h->N, D = (size_t)h->D, Np = (size_t)h->Np;
    CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    std::vector<float> stage(D * Np, 0.0f);
    const float* ins[3] = {pos, v, pbest_pos};
    float* dsts[3] = {h->dev.x, h->dev.v, h->dev.pb};
    for (int a = 0; a < 3; ++a) {
        for (size_t i = 0; i < N; ++i)
            for (size_t d = 0; d < D; ++d) stage[d * Np + i] = ins[a][i * D + d];
        CUPSO_CUDA(cudaMemcpy(dsts[a], stage.data(), sizeof(float) * D * Np, cudaMemcpyHostToDevice), "cudaMemcpy");
    }
    std::vector<float> pf(Np, INFINITY);
    std::memcpy(pf.data(), pbest_fit, sizeof(float) * N);
    CUPSO_CUDA(cudaMemcpy(h->dev.pf, pf.data(), sizeof(float) * Np, cudaMemcpyHostToDevice), "cudaMemcpy");
    CUPSO_CUDA(cudaMemset(h->dev.pflag, 0, Np), "cudaMemset");
    h->lazy_pending = false;
    h->panel = 0;   // uploaded dimension-major
    if (h->lsq && lsq_approx(h->lsq->precision)) {
        // the given pbest_fit are approximate values: gbest only from the rescoring
        CUPSO_CUDA(lsq_reset_gbest(h, h->dev.pf, t, h->stream), "lsq gbest");
    } else {
        CUPSO_CUDA(launch_recompute(h->dev, t, h->stream), "recompute launch");
    }
    CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    h->t_host = t;
    return CUPSO_OK;
}

int cupso_set_lsq(cupso_handle h, const float* A_dev, const float* b_dev, int M, int precision) {
    if (!h) return fail(CUPSO_ERR_INVALID_ARG, "handle is NULL%s");
    if (h->fp64) return fail(CUPSO_ERR_UNSUPPORTED, "double-precision swarm: use the _fp64 functions%s");
    if (h->fid != CUPSO_LSQ) return fail(CUPSO_ERR_INVALID_ARG, "swarm was not created with CUPSO_LSQ%s");
    if (!A_dev || !b_dev || M < 1) return fail(CUPSO_ERR_INVALID_ARG, "A, b must be device arrays and M >= 1%s");
    if (precision < CUPSO_LSQ_FP32 || precision > CUPSO_LSQ_FP64) return fail(CUPSO_ERR_INVALID_ARG, "unknown precision%s");
    if (lsq_approx(precision) && !lsq_tc_available())
        return fail(CUPSO_ERR_UNSUPPORTED, "tensor-core least squares needs cuTensorMapEncodeTiled%s");
    int rc = ensure_materialized(h);
    if (rc) return rc;
    CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    drop_graph(h);
    if (h->lsq) {
        for (cudaEvent_t ev : h->lsq->ev) cudaEventDestroy(ev);
        if (h->lsq->fork) cudaEventDestroy(h->lsq->fork);
        if (h->lsq->join) cudaEventDestroy(h->lsq->join);
        if (h->lsq->side) cudaStreamDestroy(h->lsq->side);
        lsq_free_tc(&h->lsq->tc);
        if (h->lsq->buf) cudaFree(h->lsq->buf);
        if (h->lsq->gram_buf) cudaFree(h->lsq->gram_buf);
        delete h->lsq;
        h->lsq = nullptr;
    }
    auto* L = new (std::nothrow) cupso_swarm::Lsq();
    if (!L) return fail(CUPSO_ERR_OOM, "host allocation failed%s");
    h->lsq = L;
    L->A = A_dev;
    L->b = b_dev;
    L->M = M;
    L->precision = precision;
    const int nlists = lsq_cand_lists(h->Np);
    // FP64 rescoring in pieces of at most 8 row pairs of A^T A (one per warp of
    // a block), as many pieces as give every SM two of the 4 x pieces blocks
    {
        const int npairs = (h->D + 1) / 2;
        const int target = std::max(1, h->num_sms / 2);
        const int per = std::min(8, std::max(1, (npairs + target - 1) / target));
        L->chunks = std::max(32, (npairs + per - 1) / per);
    }
    // candidates: 16 per list, the merged 16, and the merging ticket; partial
    // sums: 16 per piece of the row-wise rescoring or tile of the float-float one
    const int npart = std::max(L->chunks, lsq_ff_tiles(h->D));
    const size_t bytes = align_up(sizeof(float) * h->Np, 256) + align_up(sizeof(unsigned long long) * (nlists * 16 + 17), 256) +
                         align_up(sizeof(double) * 16 * npart, 256) + align_up((size_t)h->Np, 256) + 256;
    cudaError_t e = cudaMalloc(&L->buf, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (lsq)");
    char* p = static_cast<char*>(L->buf);
    L->f = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * h->Np, 256);
    L->cand = reinterpret_cast<unsigned long long*>(p); p += align_up(sizeof(unsigned long long) * (nlists * 16 + 17), 256);
    L->partial = reinterpret_cast<double*>(p); p += align_up(sizeof(double) * 16 * npart, 256);
    L->flags = reinterpret_cast<unsigned int*>(p); p += align_up((size_t)h->Np, 256);
    L->g64 = reinterpret_cast<double*>(p);
    const double inf = INFINITY;
    CUPSO_CUDA(cudaMemcpyAsync(L->g64, &inf, sizeof(double), cudaMemcpyHostToDevice, h->stream), "cudaMemcpyAsync");
    CUPSO_CUDA(cudaMemsetAsync(L->f, 0, sizeof(float) * h->Np, h->stream), "cudaMemsetAsync");
    CUPSO_CUDA(cudaMemsetAsync(L->cand + (size_t)nlists * 16 + 16, 0, sizeof(unsigned long long), h->stream),
               "cudaMemsetAsync");
    if (lsq_approx(precision)) {
        CUPSO_CUDA(cudaStreamCreateWithFlags(&L->side, cudaStreamNonBlocking), "cudaStreamCreate");
        CUPSO_CUDA(cudaEventCreateWithFlags(&L->fork, cudaEventDisableTiming), "cudaEventCreate");
        CUPSO_CUDA(cudaEventCreateWithFlags(&L->join, cudaEventDisableTiming), "cudaEventCreate");
        // FP8 scale of the operand: displacements between two points of the box
        // are at most max_pos - min_pos in magnitude
        const float span = h->dev.hi - h->dev.lo;
        const float sx = std::isfinite(span) && span > 0.0f ? 448.0f / span : 1.0f;
        rc = lsq_setup_tc(&L->tc, A_dev, b_dev, M, h->D, h->Np, precision == CUPSO_LSQ_FP8, sx, h->stream);
        if (rc) return rc;
        if (!lsq_make_move_maps(L->tc.tmMove, h->dev.x, h->dev.v, h->dev.pb, h->Np, h->D))
            return fail(CUPSO_ERR_UNSUPPORTED, "tensor maps of the move could not be encoded%s");
        if (h->D <= M && h->D <= kGramMaxD) {
            // Gram data: A^T A, A^T b (device, FP64), A^T A again as binary32
            // pairs for the float-float rescoring, and b^T b (host, from b)
            const int ldf = (h->D + kFfTile - 1) / kFfTile * kFfTile;
            const size_t n64 = align_up(sizeof(double) * ((size_t)h->D * h->D + h->D), 256);
            CUPSO_CUDA(cudaMalloc(&L->gram_buf, n64 + sizeof(float2) * (size_t)ldf * ldf), "cudaMalloc (gram)");
            L->gram.Gm = static_cast<double*>(L->gram_buf);
            L->gram.cvec = L->gram.Gm + (size_t)h->D * h->D;
            L->gram.Gff = reinterpret_cast<float2*>(static_cast<char*>(L->gram_buf) + n64);
            L->gram.ldf = ldf;
            L->gram.ff = h->lsq_rescore == 0;
            CUPSO_CUDA(lsq_launch_gram(A_dev, b_dev, M, h->D, L->gram.Gm, L->gram.cvec, L->gram.Gff, ldf, h->stream),
                       "gram launch");
            std::vector<float> hb((size_t)M);
            CUPSO_CUDA(cudaMemcpyAsync(hb.data(), b_dev, sizeof(float) * M, cudaMemcpyDeviceToHost, h->stream),
                       "cudaMemcpyAsync");
            CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
            double bb = 0.0;
            for (float v : hb) bb = std::fma((double)v, (double)v, bb);
            L->gram.bb = bb;
        }
    }
    // Step 1 completes here: pbest_fit = f(pbest_pos), gbest from it.
    if (precision == CUPSO_LSQ_FP32 || precision == CUPSO_LSQ_FP64) {
        CUPSO_CUDA(precision == CUPSO_LSQ_FP32
                       ? lsq_fp32_launch(h->dev.pb, h->Np, h->N, h->D, A_dev, b_dev, M, L->f, h->stream)
                       : lsq_fp64_launch(h->dev.pb, h->Np, h->N, h->D, A_dev, b_dev, M, L->f, h->stream),
                   "lsq fitness");
        CUPSO_CUDA(lsq_launch_set_pf(h->dev, L->f, h->stream), "lsq pbest");
        CUPSO_CUDA(launch_recompute(h->dev, h->t_host, h->stream), "recompute launch");
    } else {
        // the positions' own fitness (reference point 0: offsets -b)
        rc = lsq_eval_tc(&L->tc, h->dev.pb, 1, (size_t)h->Np, h->N, L->f, h->stream);
        if (rc) return rc;
        CUPSO_CUDA(lsq_launch_set_pf(h->dev, L->f, h->stream), "lsq pbest");
        CUPSO_CUDA(lsq_reset_gbest(h, L->f, h->t_host, h->stream), "lsq gbest");
    }
    CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return CUPSO_OK;
}

int cupso_get_gbest_f64(cupso_handle h, double* fit_out) {
    if (!h || !fit_out) return fail(CUPSO_ERR_INVALID_ARG, "NULL argument%s");
    if (h->fid != CUPSO_LSQ || !h->lsq) return fail(CUPSO_ERR_INVALID_ARG, "not a least-squares swarm with A, b set%s");
    cupso_swarm::Lsq& L = *h->lsq;
    if (!lsq_approx(L.precision)) {
        // rescore the gbest particle's pbest_pos (== gbest_pos) in FP64
        const int rc = ensure_materialized(h);
        if (rc) return rc;
        const int cur = (int)(h->t_host & 1u);
        CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        unsigned long long key = 0;
        CUPSO_CUDA(cudaMemcpy(&key, h->dev.gkey + cur, sizeof(key), cudaMemcpyDeviceToHost), "cudaMemcpy");
        const double inf = INFINITY;
        CUPSO_CUDA(cudaMemcpy(L.g64, &inf, sizeof(double), cudaMemcpyHostToDevice), "cudaMemcpy");
        CUPSO_CUDA(lsq_rescore_one(h->dev, L.A, L.b, L.M, key, L.cand, L.partial, L.chunks, L.g64, h->stream),
                   "lsq rescore");
    }
    CUPSO_CUDA(cudaMemcpyAsync(fit_out, L.g64, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync");
    CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return CUPSO_OK;
}

int cupso_create_fp64(int D, int N, const cupso_bounds_f64* bounds, double w, double c1, double c2, int fitness_id,
                      uint64_t seed, cupso_handle* out) {
    return create_swarm64(D, N, bounds, w, c1, c2, fitness_id, seed, out);
}

int cupso_get_gbest_fp64(cupso_handle h, double* fit_out, double* pos_out, int64_t* idx_out) {
    if (!h) return fail(CUPSO_ERR_INVALID_ARG, "handle is NULL%s");
    if (!h->fp64) return fail(CUPSO_ERR_UNSUPPORTED, "not a double-precision swarm%s");
    const int cur = (int)(h->t_host & 1u);
    int rc = ensure_pinned(h, 32 + sizeof(double) * (size_t)h->D);
    if (rc) return rc;
    char* pin = static_cast<char*>(h->pinned);
    CUPSO_CUDA(cudaMemcpyAsync(pin, h->dev64.gkey + cur, sizeof(PKey), cudaMemcpyDeviceToHost, h->stream),
               "cudaMemcpyAsync");
    CUPSO_CUDA(cudaMemcpyAsync(pin + 16, h->dev64.status, 4, cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync");
    if (pos_out)
        CUPSO_CUDA(cudaMemcpyAsync(pin + 32, h->dev64.G + (size_t)cur * h->D, sizeof(double) * (size_t)h->D,
                                   cudaMemcpyDeviceToHost, h->stream),
                   "cudaMemcpyAsync");
    CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    PKey key{};
    unsigned st = 0;
    std::memcpy(&key, pin, sizeof(PKey));
    std::memcpy(&st, pin + 16, 4);
    if (pos_out) std::memcpy(pos_out, pin + 32, sizeof(double) * (size_t)h->D);
    if (fit_out) *fit_out = key_to_fit64(key.k);
    if (idx_out) *idx_out = (int64_t)key.i;
    rc = status_code(st);
    if (rc) fail(rc, "device status set: %s", cupso_status_string(rc));
    return rc;
}

int cupso_get_state_fp64(cupso_handle h, double* pos, double* v, double* pbest_pos, double* pbest_fit,
                         uint32_t* t_out) {
    if (!h) return fail(CUPSO_ERR_INVALID_ARG, "handle is NULL%s");
    if (!h->fp64) return fail(CUPSO_ERR_UNSUPPORTED, "not a double-precision swarm%s");
    const size_t N = (size_t)h->N, D = (size_t)h->D, Np = (size_t)h->Np;
    std::vector<double> stage;
    double* outs[3] = {pos, v, pbest_pos};
    const double* srcs[3] = {h->dev64.x, h->dev64.v, h->dev64.pb};
    CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    for (int a = 0; a < 3; ++a) {
        if (!outs[a]) continue;
        stage.resize(D * Np);
        CUPSO_CUDA(cudaMemcpy(stage.data(), srcs[a], sizeof(double) * D * Np, cudaMemcpyDeviceToHost), "cudaMemcpy");
        for (size_t i = 0; i < N; ++i)
            for (size_t d = 0; d < D; ++d) outs[a][i * D + d] = stage[d * Np + i];
    }
    if (pbest_fit)
        CUPSO_CUDA(cudaMemcpy(pbest_fit, h->dev64.pf, sizeof(double) * N, cudaMemcpyDeviceToHost), "cudaMemcpy");
    if (t_out) *t_out = h->t_host;
    return CUPSO_OK;
}

int cupso_set_state_fp64(cupso_handle h, const double* pos, const double* v, const double* pbest_pos,
                         const double* pbest_fit, uint32_t t) {
    if (!h) return fail(CUPSO_ERR_INVALID_ARG, "handle is NULL%s");
    if (!h->fp64) return fail(CUPSO_ERR_UNSUPPORTED, "not a double-precision swarm%s");
    if (!pos || !v || !pbest_pos || !pbest_fit) return fail(CUPSO_ERR_INVALID_ARG, "state array is NULL%s");
    const size_t N = (size_t)h->N, D = (size_t)h->D, Np = (size_t)h->Np;
    CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    std::vector<double> stage(D * Np, 0.0);
    const double* ins[3] = {pos, v, pbest_pos};
    double* dsts[3] = {h->dev64.x, h->dev64.v, h->dev64.pb};
    for (int a = 0; a < 3; ++a) {
        for (size_t i = 0; i < N; ++i)
            for (size_t d = 0; d < D; ++d) stage[d * Np + i] = ins[a][i * D + d];
        CUPSO_CUDA(cudaMemcpy(dsts[a], stage.data(), sizeof(double) * D * Np, cudaMemcpyHostToDevice), "cudaMemcpy");
    }
    std::vector<double> pf(Np, INFINITY);
    std::memcpy(pf.data(), pbest_fit, sizeof(double) * N);
    CUPSO_CUDA(cudaMemcpy(h->dev64.pf, pf.data(), sizeof(double) * Np, cudaMemcpyHostToDevice), "cudaMemcpy");
    CUPSO_CUDA(cudaMemcpy(h->dev64.t_dev, &t, sizeof(t), cudaMemcpyHostToDevice), "cudaMemcpy");
    CUPSO_CUDA(launch_recompute64(h->dev64, h->pbufs, h->stream), "recompute launch");
    CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    h->t_host = t;
    return CUPSO_OK;
}

int cupso_get_info(cupso_handle h, cupso_info* info) {
    if (!h || !info) return fail(CUPSO_ERR_INVALID_ARG, "NULL argument%s");
    info->N = h->N;
    info->D = h->D;
    info->Np = h->Np;
    info->mode = resolved_mode(h);
    info->t = h->t_host;
    if (h->fp64) {
        info->sync_grid = paper_blocks(h->N);
        info->async_grid = 0;
        info->onchip_cluster = h->onchip_cluster;
        info->sync_stages = 0;
        info->sync_ppt = 0;
        info->sync_tile = 0;
        info->sync_panel = 0;
        info->sync_iters_per_launch = 1;
    } else {
        const int tile = sync_tile(h);
        info->sync_grid = tile ? std::min(tiled_grid(h, tile), (h->N + tile - 1) / tile) : sync_grid(h);
        info->async_grid = async_grid(h);
        info->onchip_cluster = h->onchip_cluster;
        const PanelCfg pc = panel_cfg(h);
        info->sync_stages = pc.width ? pc.stages : (tile ? 0 : sync_stages(h));
        info->sync_ppt = pc.width ? 1 : ((!tile && sync_stages(h)) ? sync_ppt(h) : 0);
        info->sync_tile = pc.width ? 0 : tile;
        info->sync_panel = pc.width;
        info->sync_iters_per_launch = pc.width ? panel_iters_per_launch(h) : 1;
    }
    info->fitness_ms = 0.0f;
    info->fitness_timed = 0;
    if (h->lsq) {
        cupso_swarm::Lsq& L = *h->lsq;
        if (!L.ev.empty()) {
            CUPSO_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
            for (size_t k = 0; k + 1 < L.ev.size(); k += 2) {
                float ms = 0.0f;
                if (cudaEventElapsedTime(&ms, L.ev[k], L.ev[k + 1]) == cudaSuccess) {
                    L.fitness_ms_sum += ms;
                    ++L.fitness_timed;
                }
                cudaEventDestroy(L.ev[k]);
                cudaEventDestroy(L.ev[k + 1]);
            }
            L.ev.clear();
        }
        if (L.fitness_timed) {
            info->fitness_ms = (float)(L.fitness_ms_sum / L.fitness_timed);
            info->fitness_timed = L.fitness_timed;
        }
    }
    info->device_bytes = (uint64_t)h->arena_bytes;
    return CUPSO_OK;
}

int cupso_destroy(cupso_handle h) {
    if (!h) return CUPSO_OK;
    int rc = CUPSO_OK;
    if (h->stream) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    }
    drop_graph(h);
    if (h->lsq) {
        for (cudaEvent_t ev : h->lsq->ev) cudaEventDestroy(ev);
        if (h->lsq->fork) cudaEventDestroy(h->lsq->fork);
        if (h->lsq->join) cudaEventDestroy(h->lsq->join);
        if (h->lsq->side) cudaStreamDestroy(h->lsq->side);
        lsq_free_tc(&h->lsq->tc);
        if (h->lsq->buf) cudaFree(h->lsq->buf);
        if (h->lsq->gram_buf) cudaFree(h->lsq->gram_buf);
        delete h->lsq;
        h->lsq = nullptr;
    }
    if (h->rec_stream) {
        cudaError_t e = cudaStreamSynchronize(h->rec_stream);
        if (e != cudaSuccess && rc == CUPSO_OK) rc = cuda_fail(e, "cudaStreamSynchronize");
        cudaStreamDestroy(h->rec_stream);
    }
    for (int k = 0; k < 2; ++k) {
        if (h->rec_ev[k]) cudaEventDestroy(h->rec_ev[k]);
        if (h->rec_done[k]) cudaEventDestroy(h->rec_done[k]);
    }
    if (h->rec_dev) cudaFree(h->rec_dev);
    if (h->rec_host) cudaFreeHost(h->rec_host);
    if (h->arena) cudaFree(h->arena);
    if (h->pinned) cudaFreeHost(h->pinned);
    if (h->capture) cudaStreamDestroy(h->capture);
    if (h->own) cudaStreamDestroy(h->own);
    delete h;
    return rc;
}

const char* cupso_status_string(int status) {
    switch (status) {
        case CUPSO_OK: return "ok";
        case CUPSO_ERR_INVALID_ARG: return "invalid argument";
        case CUPSO_ERR_OOM: return "out of device memory";
        case CUPSO_ERR_CUDA: return "CUDA error";
        case CUPSO_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
        case CUPSO_ERR_NAN: return "fitness evaluated to NaN";
        case CUPSO_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

const char* cupso_last_error(void) { return g_last_error; }

}  // extern "C"
