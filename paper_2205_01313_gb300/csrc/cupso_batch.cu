// cupso_batch.cu -- cupso_solve_batch: many independent swarms at once.
//
// All swarms of a batch live in one device arena. One launch runs Step 1 of
// every swarm (batch_init_kernel), then every iteration is ONE launch of
// batch_step_kernel covering the units of all swarms (kernels_batch.cu); the
// `iters` launches are replayed from captured CUDA graphs. Two kernels can
// run the step: the streaming one (kernels_batch.cu: 128-particle units per
// warp, rows staged through a cp.async ring) and the tiled one
// (kernels_tiled.cu: tiles of P particles with all their dimensions per CTA,
// P chosen per swarm so that tiles cost about the same). The launch shape
// (kernel, ring depth, CTAs per SM) is chosen online: the first iterations of
// the real run are timed under each candidate shape and the fastest one runs
// the rest -- every shape computes the same bits, so tuning costs no extra
// work. Choices are remembered per batch shape for the life of the process.
//
// Swarms with fewer than three dimensions (too few dimension pairs for the
// ring's look-ahead) are solved one by one through their own handles.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/cupso.h"
#include "cupso_device.cuh"
#include "cupso_internal.h"
#include "tiled_kernels.h"

using namespace cupso;

namespace {

size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Shape {
    int stages;          // ring depth of the streaming kernel; 0: the tiled kernel
    int minb;            // register budget: CTAs per SM
    int blocks_per_sm;   // CTAs per SM launched
};

// Launch shapes remembered per batch signature.
std::mutex g_tune_mutex;
std::map<std::tuple<int, long long, int, int>, Shape> g_tuned;

struct BatchRun {
    cudaStream_t st = nullptr;
    BatchDev dev{};
    BatchTiles tiles{};
    int num_sms = 1;
    cudaGraphExec_t graph = nullptr;
    Shape graph_shape{0, 0, 0};
    int graph_len = 0;

    ~BatchRun() {
        if (graph) cudaGraphExecDestroy(graph);
    }

    cudaError_t launch(const Shape& sh) { return launch_on(sh, st); }

    cudaError_t launch_on(const Shape& sh, cudaStream_t s) {
        if (sh.stages == 0) return launch_batch_tiled(dev, tiles, num_sms * sh.blocks_per_sm, s);
        return launch_batch_step(dev, sh.stages, sh.minb, num_sms * sh.blocks_per_sm, s);
    }

    // `n` iterations with shape `sh`, through a captured graph of up to 32 launches.
    int run(const Shape& sh, int n) {
        const int L = std::min(n, 32);
        if (L >= 4 && (!graph || graph_len != L || graph_shape.stages != sh.stages || graph_shape.minb != sh.minb ||
                       graph_shape.blocks_per_sm != sh.blocks_per_sm)) {
            if (graph) cudaGraphExecDestroy(graph);
            graph = nullptr;
            cudaStream_t cap = nullptr;
            cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
            if (e != cudaSuccess) return set_cuda_error(e, "cudaStreamCreate"), CUPSO_ERR_CUDA;
            e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            cudaError_t le = cudaSuccess;
            for (int k = 0; k < L && e == cudaSuccess && le == cudaSuccess; ++k)
                le = launch_on(sh, cap);
            cudaGraph_t g = nullptr;
            cudaError_t ee = e == cudaSuccess ? cudaStreamEndCapture(cap, &g) : e;
            cudaStreamDestroy(cap);
            if (le != cudaSuccess || ee != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                set_cuda_error(le != cudaSuccess ? le : ee, "batch graph capture");
                return CUPSO_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                graph = nullptr;
                set_cuda_error(e, "cudaGraphInstantiate");
                return CUPSO_ERR_CUDA;
            }
            graph_len = L;
            graph_shape = sh;
        }
        int left = n;
        while (graph && left >= graph_len) {
            cudaError_t e = cudaGraphLaunch(graph, st);
            if (e != cudaSuccess) return set_cuda_error(e, "cudaGraphLaunch"), CUPSO_ERR_CUDA;
            left -= graph_len;
        }
        for (; left > 0; --left) {
            cudaError_t e = launch(sh);
            if (e != cudaSuccess) return set_cuda_error(e, "batch launch"), CUPSO_ERR_CUDA;
        }
        return CUPSO_OK;
    }
};

float key_fit(unsigned long long key) {
    const uint32_t k = (uint32_t)(key >> 32);
    if (k == 0xFFFFFFFFu) return NAN;
    const uint32_t bits = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    float f;
    std::memcpy(&f, &bits, 4);
    return f;
}

}  // namespace

extern "C" int cupso_solve_batch(int n_swarms, const cupso_problem* problems, int iters, cupso_result* results,
                                 void* cuda_stream) {
    if (n_swarms < 0 || iters < 0) {
        set_last_error("n_swarms and iters must be >= 0");
        return CUPSO_ERR_INVALID_ARG;
    }
    if (n_swarms > 0 && (!problems || !results)) {
        set_last_error("NULL problems/results");
        return CUPSO_ERR_INVALID_ARG;
    }
    for (int k = 0; k < n_swarms; ++k) {
        const cupso_problem& p = problems[k];
        const int rc = check_problem_args(p.D, p.N, &p.bounds, p.w, p.c1, p.c2, p.fitness_id);
        if (rc) return rc;
        if (p.fitness_id == CUPSO_LSQ) {
            // the least-squares fitness needs A and b (cupso_set_lsq); a problem record has neither
            set_last_error("the least-squares fitness is not available in a batch");
            return CUPSO_ERR_INVALID_ARG;
        }
    }
    if (n_swarms == 0) return CUPSO_OK;

    BatchRun run;
    cudaStream_t own = nullptr;
    if (cuda_stream) {
        run.st = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaStreamCreate"), CUPSO_ERR_CUDA;
        run.st = own;
    }
    int first = CUPSO_OK;
    auto note = [&](int rc) {
        if (rc != CUPSO_OK && first == CUPSO_OK) first = rc;
    };

    std::vector<int> batched;
    for (int k = 0; k < n_swarms; ++k) {
        if (problems[k].D >= 3) {
            batched.push_back(k);
        } else {
            note(solve_one_plain(problems[k], iters, results[k], run.st));
        }
    }
    const int nb = (int)batched.size();
    void* arena = nullptr;
    int rc = CUPSO_OK;
    do {
        if (nb == 0) break;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&run.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = prepare_batch();
        if (e != cudaSuccess) { set_cuda_error(e, "batch setup"); rc = CUPSO_ERR_CUDA; break; }

        // Arena: per-swarm planes, then gbest positions, keys, words, flags, descriptors, units, counters.
        const size_t A = 256;
        std::vector<size_t> o_state(nb), o_G(nb), o_flag(nb);
        std::vector<int> Np(nb);
        size_t off = 0, total_units = 0, sumG = 0, sumFlag = 0, total_tiles = 0;
        std::vector<int> tileP(nb);
        std::vector<unsigned> ntiles(nb);
        int minD = 1 << 30, maxD = 0;
        long long total_pd = 0;
        for (int j = 0; j < nb; ++j) {
            const cupso_problem& p = problems[batched[j]];
            Np[j] = (p.N + kPad - 1) / kPad * kPad;
            o_state[j] = off;
            off = up(off + sizeof(float) * ((size_t)3 * p.D * Np[j] + Np[j]), A);
            o_G[j] = sumG;
            sumG += 2 * (size_t)p.D;
            o_flag[j] = sumFlag;
            sumFlag += (size_t)Np[j];
            total_units += (size_t)Np[j] / 128;
            tileP[j] = batch_tile_particles(p.D);
            ntiles[j] = tileP[j] > 0 ? (unsigned)((p.N + tileP[j] - 1) / tileP[j]) : 0u;
            total_tiles += ntiles[j];
            minD = std::min(minD, p.D);
            maxD = std::max(maxD, p.D);
            total_pd += (long long)p.N * p.D;
        }
        const size_t o_Gall = off; off = up(off + sizeof(float) * sumG, A);
        const size_t o_keys = off; off = up(off + sizeof(unsigned long long) * 2 * nb, A);
        const size_t o_words = off; off = up(off + sizeof(unsigned int) * 4 * nb, A);
        const size_t o_flags = off; off = up(off + sumFlag, A);
        const size_t o_desc = off; off = up(off + sizeof(BatchSwarm) * nb, A);
        const size_t o_units = off; off = up(off + sizeof(uint2) * total_units, A);
        const size_t o_tunits = off; off = up(off + sizeof(uint2) * std::max<size_t>(total_tiles, 1), A);
        const size_t o_tileP = off; off = up(off + sizeof(int) * nb, A);
        const size_t o_ntiles = off; off = up(off + sizeof(unsigned) * nb, A);
        const size_t o_ctr = off; off = up(off + 64, A);
        e = cudaMalloc(&arena, off);
        if (e != cudaSuccess) { set_cuda_error(e, "cudaMalloc (batch arena)"); rc = e == cudaErrorMemoryAllocation ? CUPSO_ERR_OOM : CUPSO_ERR_CUDA; break; }
        char* base = static_cast<char*>(arena);
        float* Gall = reinterpret_cast<float*>(base + o_Gall);
        unsigned long long* keys = reinterpret_cast<unsigned long long*>(base + o_keys);
        unsigned int* words = reinterpret_cast<unsigned int*>(base + o_words);   // done, status, 2 spare
        unsigned char* flags = reinterpret_cast<unsigned char*>(base + o_flags);
        unsigned int* ctr = reinterpret_cast<unsigned int*>(base + o_ctr);       // work[2], ticket, t
        e = cudaMemsetAsync(keys, 0xFF, sizeof(unsigned long long) * 2 * nb, run.st);
        if (e == cudaSuccess) e = cudaMemsetAsync(base + o_words, 0, o_desc - o_words, run.st);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, 64, run.st);
        if (e != cudaSuccess) { set_cuda_error(e, "cudaMemsetAsync"); rc = CUPSO_ERR_CUDA; break; }

        // The descriptor of every swarm.
        std::vector<BatchSwarm> desc(nb);
        for (int j = 0; j < nb; ++j) {
            const cupso_problem& p = problems[batched[j]];
            float* st = reinterpret_cast<float*>(base + o_state[j]);
            const size_t plane = (size_t)p.D * Np[j];
            BatchSwarm& w = desc[j];
            w.x = st;
            w.v = st + plane;
            w.pb = st + 2 * plane;
            w.pf = st + 3 * plane;
            w.pflag = flags + o_flag[j];
            w.G = Gall + o_G[j];
            w.gkey = keys + 2 * j;
            w.done = words + 4 * j + 0;
            w.status = words + 4 * j + 1;
            w.N = p.N; w.D = p.D; w.Np = Np[j]; w.fid = p.fitness_id;
            w.nunits = (unsigned)(Np[j] / 128);
            w.lo = p.bounds.min_pos; w.hi = p.bounds.max_pos; w.vmax = p.bounds.max_v;
            w.w = p.w; w.c1 = p.c1; w.c2 = p.c2;
            w.c1s = std::ldexp(p.c1, -24);
            w.c2s = std::ldexp(p.c2, -24);
            const bool fast_cr = std::ldexp(w.c1s, 24) == p.c1 && std::ldexp(w.c2s, 24) == p.c2 &&
                                 (p.c1 == 0.0f || std::fabs(w.c1s) >= FLT_MIN) &&
                                 (p.c2 == 0.0f || std::fabs(w.c2s) >= FLT_MIN);
            w.fast = fast_cr && p.bounds.min_pos != 0.0f && p.bounds.max_pos != 0.0f;
            w.key0 = (uint32_t)(p.seed & 0xFFFFFFFFull);
            w.key1 = (uint32_t)(p.seed >> 32);
            w.swarm = p.swarm_id;
        }
        if (rc != CUPSO_OK) break;

        // Hand-out order: swarms that run the same code (fitness function and
        // arithmetic path) together, so that the warps of an SM share their
        // instructions; within such a class the units with the most dimensions
        // first, swarms of equal D interleaved. The smallest units come last
        // and fill the tail.
        std::vector<uint2> units;
        units.reserve(total_units);
        std::vector<int> order(nb);
        for (int j = 0; j < nb; ++j) order[j] = j;
        auto code_of = [&](int j) { return desc[j].fid * 2 + desc[j].fast; };
        auto same_group = [&](int a, int b) { return code_of(a) == code_of(b) && desc[a].D == desc[b].D; };
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            if (code_of(a) != code_of(b)) return code_of(a) < code_of(b);
            return desc[a].D > desc[b].D;
        });
        for (size_t pos = 0; pos < (size_t)nb;) {
            size_t endg = pos;
            while (endg < (size_t)nb && same_group(order[endg], order[pos])) ++endg;
            unsigned most = 0;
            for (size_t q = pos; q < endg; ++q) most = std::max(most, desc[order[q]].nunits);
            for (unsigned u = 0; u < most; ++u)
                for (size_t q = pos; q < endg; ++q)
                    if (u < desc[order[q]].nunits) units.push_back(make_uint2((unsigned)order[q], u));
            pos = endg;
        }
        e = cudaMemcpyAsync(base + o_desc, desc.data(), sizeof(BatchSwarm) * nb, cudaMemcpyHostToDevice, run.st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + o_units, units.data(), sizeof(uint2) * units.size(), cudaMemcpyHostToDevice,
                                run.st);
        if (e != cudaSuccess) { set_cuda_error(e, "cudaMemcpyAsync"); rc = CUPSO_ERR_CUDA; break; }
        run.dev.swarms = reinterpret_cast<const BatchSwarm*>(base + o_desc);
        run.dev.units = reinterpret_cast<const uint2*>(base + o_units);
        run.dev.nunits = (unsigned)units.size();
        run.dev.work = ctr;
        run.dev.ticket = ctr + 2;
        run.dev.t_dev = ctr + 3;

        // Step 1 of every swarm, one launch.
        e = launch_batch_init(run.dev, run.num_sms * 4, run.st);
        if (e != cudaSuccess) { set_cuda_error(e, "batch init launch"); rc = CUPSO_ERR_CUDA; break; }

        // The tiled kernel's units in the same order.
        const bool tiled_ok = maxD <= kTiledItems;
        if (tiled_ok) {
            std::vector<uint2> tunits;
            tunits.reserve(total_tiles);
            for (size_t pos = 0; pos < (size_t)nb;) {
                size_t endg = pos;
                while (endg < (size_t)nb && same_group(order[endg], order[pos])) ++endg;
                unsigned most = 0;
                for (size_t q = pos; q < endg; ++q) most = std::max(most, ntiles[order[q]]);
                for (unsigned u = 0; u < most; ++u)
                    for (size_t q = pos; q < endg; ++q)
                        if (u < ntiles[order[q]]) tunits.push_back(make_uint2((unsigned)order[q], u));
                pos = endg;
            }
            e = cudaMemcpyAsync(base + o_tunits, tunits.data(), sizeof(uint2) * tunits.size(), cudaMemcpyHostToDevice,
                                run.st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(base + o_tileP, tileP.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, run.st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(base + o_ntiles, ntiles.data(), sizeof(unsigned) * nb, cudaMemcpyHostToDevice,
                                    run.st);
            if (e != cudaSuccess) { set_cuda_error(e, "cudaMemcpyAsync"); rc = CUPSO_ERR_CUDA; break; }
            run.tiles.units = reinterpret_cast<const uint2*>(base + o_tunits);
            run.tiles.nunits = (unsigned)tunits.size();
            run.tiles.P = reinterpret_cast<const int*>(base + o_tileP);
            run.tiles.ntiles = reinterpret_cast<const unsigned*>(base + o_ntiles);
        }

        // Launch shapes to try: ring depth 4 needs three dimension pairs everywhere.
        std::vector<Shape> cand;
        if ((minD + 1) / 2 >= 3) cand.push_back(Shape{4, 2, batch_blocks_per_sm(4, 2)});
        cand.push_back(Shape{3, 2, batch_blocks_per_sm(3, 2)});
        cand.push_back(Shape{3, 3, batch_blocks_per_sm(3, 3)});
        if (tiled_ok) cand.push_back(Shape{0, 0, batch_tiled_blocks_per_sm()});
        const auto key = std::make_tuple(nb, total_pd, minD, maxD);
        Shape best = cand[0];
        bool known = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mutex);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) { best = it->second; known = true; }
        }
        // CUPSO_BATCH_KERNEL=tiled|streaming fixes the kernel instead of tuning
        // (for tests and measurements; both kernels give the same bits).
        if (const char* force = std::getenv("CUPSO_BATCH_KERNEL")) {
            const bool want_tiled = std::strcmp(force, "tiled") == 0;
            const bool want_stream = std::strcmp(force, "streaming") == 0;
            if (want_tiled && !tiled_ok) { set_last_error("CUPSO_BATCH_KERNEL=tiled: D too large"); rc = CUPSO_ERR_UNSUPPORTED; break; }
            if (want_tiled || want_stream) {
                for (const Shape& sh : cand)
                    if ((sh.stages == 0) == want_tiled) { best = sh; break; }
                known = true;
            }
        }
        int done_iters = 0;
        const int probe = 2;
        if (!known && iters >= (int)cand.size() * probe * 2) {
            float best_ms = 1e30f;
            cudaEvent_t ev0, ev1;
            cudaEventCreate(&ev0);
            cudaEventCreate(&ev1);
            for (const Shape& sh : cand) {
                cudaEventRecord(ev0, run.st);
                for (int k = 0; k < probe && rc == CUPSO_OK; ++k) {
                    e = run.launch(sh);
                    if (e != cudaSuccess) { set_cuda_error(e, "batch launch"); rc = CUPSO_ERR_CUDA; }
                }
                cudaEventRecord(ev1, run.st);
                cudaEventSynchronize(ev1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev0, ev1);
                if (rc == CUPSO_OK && ms < best_ms) { best_ms = ms; best = sh; }
                done_iters += probe;
            }
            cudaEventDestroy(ev0);
            cudaEventDestroy(ev1);
            if (rc == CUPSO_OK) {
                std::lock_guard<std::mutex> lk(g_tune_mutex);
                g_tuned[key] = best;
            }
        }
        if (rc != CUPSO_OK) break;
        rc = run.run(best, iters - done_iters);
        if (rc != CUPSO_OK) break;

        // Results: gbest key, position and status of every swarm.
        std::vector<unsigned long long> hkeys(2 * (size_t)nb);
        std::vector<float> hG(sumG);
        std::vector<unsigned int> hw(4 * (size_t)nb);
        e = cudaMemcpyAsync(hkeys.data(), keys, sizeof(unsigned long long) * 2 * nb, cudaMemcpyDeviceToHost, run.st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hG.data(), Gall, sizeof(float) * sumG, cudaMemcpyDeviceToHost, run.st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hw.data(), words, sizeof(unsigned) * 4 * nb, cudaMemcpyDeviceToHost, run.st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(run.st);
        if (e != cudaSuccess) { set_cuda_error(e, "batch results"); rc = CUPSO_ERR_CUDA; break; }
        const int cur = iters & 1;
        for (int j = 0; j < nb; ++j) {
            cupso_result& r = results[batched[j]];
            const unsigned long long k = hkeys[2 * j + cur];
            r.fit = key_fit(k);
            r.idx = (int64_t)(k & 0xFFFFFFFFull);
            if (r.pos) std::memcpy(r.pos, hG.data() + o_G[j] + (size_t)cur * desc[j].D, sizeof(float) * desc[j].D);
            r.status = (hw[4 * j + 1] & kStatusTimeout) ? CUPSO_ERR_DEVICE_TIMEOUT
                       : (hw[4 * j + 1] & kStatusNaN)   ? CUPSO_ERR_NAN
                                                        : CUPSO_OK;
            note(r.status);
        }
    } while (false);
    if (rc != CUPSO_OK) {
        for (int j = 0; j < nb; ++j) results[batched[j]].status = rc;
        note(rc);
    }
    if (arena) {
        cudaStreamSynchronize(run.st);
        cudaFree(arena);
    }
    if (own) cudaStreamDestroy(own);
    return first;
}
