"""Benchmark: particle-dimension updates per second of the fused PSO iteration.

Workload (default): Rosenbrock, N = 2^20 particles, D = 64, the synchronous
fused iteration (update + fitness + pbest + atomic gbest in one kernel), FP32.
One step = one PSO iteration over the whole swarm. The swarm state (805 MB)
is larger than L2 (129 MB), so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle (the
paper's serial Alg. 1 baseline, Sec. 5.1) on a bounded sample of the same
workload. Under torchrun with N > 1 every rank runs an independent replica of
the swarm (no collective on the data path; the barrier and the max-over-ranks
timing use torch.distributed).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2205_01313_gb300 import workloads  # noqa: E402

METRIC = "particle·dim updates/s per fused iter vs HBM roofline; batched & BF16 vs plain"
UNIT = "particle-dim updates/s"
DEFAULT_WORKLOAD = "rosenbrock_1048576x64"
FALLBACK_HBM_GBS = 6800.0
# Every file compiled into the benchmark's kernel (sync_panel_kernel): a
# stored traffic figure is only used while their hash is unchanged.
KERNEL_SOURCES = ["paper_2205_01313_gb300/csrc/kernels_panel.cu", "paper_2205_01313_gb300/csrc/stream_common.cuh",
                  "paper_2205_01313_gb300/csrc/cupso_device.cuh", "paper_2205_01313_gb300/csrc/cupso_internal.h"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_sync_panel_kernel.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(workloads.CONFIGS) + ["batch512", "lsq8192", "modes:sphere_1024x32",
                                                         "modes:rastrigin_65536x128", "paper:table2",
                                                         "paper:table3", "paper:table4"])
    ap.add_argument("--batch-swarms", type=int, default=512, help="batch512: number of swarms (a smaller batch for profiling)")
    ap.add_argument("--paper-rows", default="", help="paper:*: comma-separated particle counts to run (default: all rows)")
    ap.add_argument("--paper-modes", default="", help="paper:*: comma-separated modes (default: the table's designs and ours)")
    ap.add_argument("--paper-iters", type=int, default=0, help="paper:*: cap on the iterations per row (0: the table's)")
    ap.add_argument("--plain-sample", type=int, default=1,
                    help="batch512: time the per-swarm plain path on every k-th swarm and scale up")
    ap.add_argument("--mode", default="sync", choices=["sync", "tree", "tree_unrolled", "async", "onchip", "auto",
                                                       "queue", "queue_lock"])
    ap.add_argument("--sync-kernel", default="auto",
                    choices=["auto", "register", "pipelined3", "pipelined4", "panel8", "panel16"])
    ap.add_argument("--cpu-iters", type=int, default=4, help="oracle iterations in the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the batch and least-squares keys of the line")
    ap.add_argument("--lsq-launches", default="", choices=["", "bf16", "fp8", "fp32", "fp64", "bf16_rescore_fp64"],
                    help="lsq8192: only 6 + 20 iterations of one precision, one launch per kernel "
                         "(no graph), for a profiler's launch list; bf16_rescore_fp64: BF16 with the "
                         "FP64 Gram rescoring instead of the float-float one")
    return ap.parse_args()


# --------------------------------------------------------------------------- #
# distributed plumbing (replicas only)                                        #
# --------------------------------------------------------------------------- #

def dist_setup(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed / the slowest rank's time (weak scaling: each
    rank runs its own replica of the workload)."""
    return units_per_rank * world / seconds


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- #
# clocks (nvidia-smi sampled during the timed region)                          #
# --------------------------------------------------------------------------- #

class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.count(",") >= 9]
        self.file.close()
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[6 + k] and "Not" not in r[6 + k]})
        loaded = [x for x in sm if smax and x > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- #
# roofline inputs                                                              #
# --------------------------------------------------------------------------- #

def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(workload, first_iteration, iterations):
    """DRAM bytes per launch from the last ncu capture, if the kernel source is
    unchanged since and the capture took the same launch: the same first
    iteration and number of iterations as this run's timed launch."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_sha") != kernel_source_sha() or rec.get("workload") != workload:
        return None
    if rec.get("first_iteration") != first_iteration or rec.get("iterations") != iterations:
        return None
    return rec.get("dram_bytes_per_launch")


def workload_config(name, cfg, world):
    """The line's `config`, the same in both arms: the workload and its shape.
    What ran it (kernel, grid, launches) goes under `run`."""
    N, D = cfg["N"], cfg["D"]
    return {"workload": name, "fitness": workloads.FITNESS_NAMES[cfg["fitness_id"]], "N": N, "D": D,
            "step": "one PSO iteration over the whole swarm",
            "l2": "inputs larger than L2 (%.0f MB swarm state vs 129 MB L2), no flush" % (3 * 4 * N * D / 1e6),
            "parallelism": "replicas" if world > 1 else "single GPU"}


def kernel_name(info):
    if info["sync_tile"]:
        return "sync_tiled_kernel"
    if info.get("sync_panel"):
        return "sync_panel_kernel"
    return "sync_pipelined_kernel" if info["sync_stages"] else "sync_step_kernel"


def algorithmic_bytes(N, D, p=0.0):
    """Compulsory DRAM bytes of one fused iteration with a fraction p of the
    particles improving: read pos and v, write pos and v (16 B per
    particle-dimension); pbest_pos is read (4 B) for a particle that did not
    improve in the previous iteration, while for one that did it equals pos and
    is written instead (4 B): 20 B per particle-dimension either way; read
    pbest_fit (4 B per particle) and write it for the improvers (4 p B)."""
    return 20 * N * D + 4 * N + 4 * p * N


def bytes_with_pbest_rows(N, D, p):
    """The same with the pbest rows of the improvers counted on top of a full
    pbest_pos read (24 B per improving particle-dimension)."""
    return algorithmic_bytes(N, D, p) + 4 * p * N * D


def improvement_fractions(P, cfg, rank, iters):
    """Fraction of particles whose pbest improved in each of iterations 1..iters
    of the benchmark's swarm. The synchronous trajectory is deterministic, so a
    fresh swarm with the same seed replays exactly the iterations that were
    timed; pbest_fit is read back after each replayed iteration."""
    import ctypes as C
    import numpy as np
    N, D = cfg["N"], cfg["D"]
    sw = P.Swarm(D, N, cfg["bounds"], cfg["w"], cfg["c1"], cfg["c2"], cfg["fitness_id"], cfg["seed"] + rank,
                 mode="sync")
    pf = np.empty(N, np.float32)
    t = C.c_uint32()
    null = C.POINTER(C.c_float)()
    f32p = pf.ctypes.data_as(C.POINTER(C.c_float))
    P._check(P._lib.cupso_get_state(sw.h, null, null, null, f32p, C.byref(t)), "cupso_get_state")
    prev = pf.copy()
    fr = []
    for _ in range(iters):
        sw.step(1)
        P._check(P._lib.cupso_get_state(sw.h, null, null, null, f32p, C.byref(t)), "cupso_get_state")
        fr.append(float(np.count_nonzero(pf < prev)) / N)
        prev = pf.copy()
    sw.close()
    return fr


# --------------------------------------------------------------------------- #
# our arm                                                                      #
# --------------------------------------------------------------------------- #

def run_ours(a):
    import torch

    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    from paper_2205_01313_gb300 import build as B
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    barrier(world)
    from paper_2205_01313_gb300 import cupso as P

    cfg = workloads.config(a.workload)
    N, D, fid = cfg["N"], cfg["D"], cfg["fitness_id"]
    stream = torch.cuda.Stream()
    sw = P.Swarm(D, N, cfg["bounds"], cfg["w"], cfg["c1"], cfg["c2"], fid, cfg["seed"] + rank,
                 mode=a.mode, stream=stream.cuda_stream)
    sw.set_option(P.CUPSO_OPT_GRAPH_CHUNK, 0)   # no captured graphs: the kernels run as launched
    sw.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS[a.sync_kernel])
    info = sw.info()
    mode_used = {v: k for k, v in P.MODES.items()}[info["mode"]]
    if mode_used == "sync":
        if info["sync_tile"]:
            mode_used = "sync (tiled kernel, %d particles per tile)" % info["sync_tile"]
        else:
            mode_used = "sync (%s kernel)" % ("panels of %d dimensions, %d-stage ring" % (info["sync_panel"], info["sync_stages"])
                                              if info.get("sync_panel") else
                                              "pipelined, %d-stage ring" % info["sync_stages"]
                                              if info["sync_stages"] else "register")

    # W untimed iterations: W - 1 in one call (the timed region's launch form)
    # and one alone (the end-to-end loop's)
    if a.warmup > 1:
        sw.step(a.warmup - 1)
    sw.step(1)
    torch.cuda.synchronize()

    # The K timed iterations in one cupso_step call: on the panel layout one
    # cooperative launch runs them with a grid barrier between iterations (up
    # to sync_iters_per_launch per launch), otherwise one launch per iteration.
    K = a.steps
    ipl = min(K, info["sync_iters_per_launch"]) if mode_used.startswith("sync (panels") else 1
    launches = -(-K // ipl)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    sw.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    total_ms = e0.elapsed_time(e1)
    per_launch_ms = total_ms / launches
    total_ms = max_over_ranks(total_ms, world, device="cuda")

    # End to end through the public API: each step queues one iteration and
    # posts its result (gbest fitness, index, position, status) for copying to
    # host memory; the host reads it one step later (cupso_gbest_wait), while
    # the next iteration runs, and reads the last one before the clock stops.
    # The API takes no per-step input data. One read through each result slot
    # before the clock starts: their first use allocates them.
    for k in range(2):
        sw.gbest_post(k)
        sw.gbest_wait(k)
    barrier(world)
    t0 = time.perf_counter()
    for k in range(K):
        sw.step(1)
        sw.gbest_post(k & 1)
        if k:
            rc, fit, idx, pos = sw.gbest_wait((k - 1) & 1)
    rc, fit, idx, pos = sw.gbest_wait((K - 1) & 1)
    e2e_s = time.perf_counter() - t0
    barrier(world)
    clk = clocks.stop()
    e2e_s = max_over_ranks(e2e_s, world, device="cuda")
    rc, fit, idx, pos = sw.gbest()
    sw.close()

    work = float(N) * D * K * world
    value = whole_job_rate(float(N) * D * K, world, total_ms / 1e3)
    # the improvement fraction of exactly the timed iterations (W+1 .. W+K)
    fr = improvement_fractions(P, cfg, rank, a.warmup + K)
    p_timed = statistics.mean(fr[a.warmup:])
    bpl = algorithmic_bytes(N, D, p_timed) * ipl   # per launch of ipl iterations
    achieved = bpl / (per_launch_ms / 1e3) / 1e9
    peak, peak_src = hbm_peak()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": a.warmup,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": workload_config(a.workload, cfg, world),
        "run": {"mode": mode_used, "grid": info["sync_grid"],
                "timed": "the %d iterations in one cupso_step call: %d launch(es) of %d iteration(s)"
                         % (K, launches, ipl)},
        "e2e": {"value": work / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": (32 + 4 * D + 255) // 256 * 256,
                "api": "cupso_step(h, 1) + cupso_gbest_post(h, slot) per step, cupso_gbest_wait(h, slot, host "
                       "buffers) for each step's result one step later (the last before the clock stops)"},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": measured_traffic(a.workload, a.warmup + 1, ipl) if launches == 1 else None,
                     "kernel": kernel_name(info),
                     "algorithmic_bytes_per_launch": bpl,
                     "improved_fraction_timed": p_timed,
                     "improved_fraction_range": [min(fr[a.warmup:]), max(fr[a.warmup:])],
                     "iterations_per_launch": ipl,
                     "bytes_with_pbest_rows_per_launch": bytes_with_pbest_rows(N, D, p_timed) * ipl,
                     "frac_with_pbest_rows": bytes_with_pbest_rows(N, D, p_timed) * ipl / (per_launch_ms / 1e3) / 1e9
                                             / peak,
                     "launch_ms": per_launch_ms, "peak_source": peak_src},
        "clocks": clk,
        "result": {"gbest_fit": float(fit), "gbest_idx": idx, "status": rc},
    }
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, a.cpu_iters)
    if rank == 0 and world == 1 and not a.no_extras and a.workload == DEFAULT_WORKLOAD:
        # the metric's other two halves, timed in the same run: batched vs
        # per-swarm plain launches, and the BF16 (FP8) fitness vs the FP32 path
        # every 3rd swarm: the fitness functions cycle with the swarm index mod 4,
        # so a stride of 4 would time sphere swarms only (the cheapest)
        out["batch"] = batch_report(P, a, stream, plain_every=3)
        out["lsq"] = lsq_report(P, stream, quick=True)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(cfg, iters):
    """The oracle as it stands on the full swarm, init untimed: `iters`
    iterations on one thread (the paper's serial baseline, Sec. 5.1), then
    2 * iters more with Steps 2-4 on every host core the process may use
    (identical results: the particles of an iteration are independent)."""
    from oracle import oracle as O
    lo, hi, vmax = cfg["bounds"]
    s = O.Swarm(cfg["N"], cfg["D"], lo, hi, vmax, cfg["w"], cfg["c1"], cfg["c2"], cfg["fitness_id"], cfg["seed"])
    s.init()
    t0 = time.perf_counter()
    s.step_sync(iters)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    s.step_sync_threads(2 * iters, cores)
    dt_all = time.perf_counter() - t0
    return {"value": cfg["N"] * cfg["D"] * iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d iterations of the full %s swarm (N=%d, D=%d) after an untimed init; %.1f s"
                      % (iters, cfg["name"], cfg["N"], cfg["D"], dt),
            "host_cores_available": cores, "cpu_model": cpu_model(),
            "all_cores": {"value": cfg["N"] * cfg["D"] * 2 * iters / dt_all, "unit": UNIT, "cores": cores,
                          "kind": "oracle (Steps 2-4 over host threads, OpenMP)",
                          "sample": "the next %d iterations of the same swarm; %.1f s" % (2 * iters, dt_all)}}


# --------------------------------------------------------------------------- #
# reference arm: the CPU oracle                                                #
# --------------------------------------------------------------------------- #

REF_SAMPLE_N = 1 << 14


def run_reference(a):
    world, rank, _ = dist_setup("gloo")
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    from oracle import build as OB
    OB.build_oracle()
    from oracle import oracle as O
    cfg = workloads.config(a.workload)
    n = min(cfg["N"], REF_SAMPLE_N)
    lo, hi, vmax = cfg["bounds"]
    s = O.Swarm(n, cfg["D"], lo, hi, vmax, cfg["w"], cfg["c1"], cfg["c2"], cfg["fitness_id"], cfg["seed"]).init()
    for _ in range(a.warmup):
        s.step_sync(1)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        s.step_sync(1)
    dt = time.perf_counter() - t0
    value = n * cfg["D"] * a.steps / dt
    sample = ("each step: one synchronous iteration of the oracle over a %d-particle sub-swarm of %s "
              "(D=%d, same bounds, seed and parameters)" % (n, cfg["name"], cfg["D"]))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(a.workload, cfg, world),
        "run": {"mode": "oracle (serial synchronous PSO, Alg. 1)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------------------------- #
# batched solve: 512 uneven swarms, one launch per iteration for all of them   #
# --------------------------------------------------------------------------- #

BATCH_ITERS = 500


def batch_report(P, a, stream, plain_every=1):
    """512 independent swarms (N ~ U{64..8192}, D ~ U{8..256}, fitness cycling
    sphere/Rastrigin/Ackley/Rosenbrock), 500 iterations each, solved (1) by
    cupso_solve_batch and (2) plain: per swarm cupso_create, cupso_step(500)
    with one launch per iteration, cupso_get_gbest, cupso_destroy, on one stream -- timed on every
    `plain_every`-th swarm and scaled by particle-dimension updates. Both through
    the public API with host results. Correctness: swarms re-solved alone
    through the batch API must reproduce the batched results bit for bit."""
    import numpy as np
    import torch

    probs = workloads.batch_problems(n_swarms=a.batch_swarms)
    iters = BATCH_ITERS
    total_pd = sum(p["N"] * p["D"] for p in probs) * iters
    # warm-up: the same batch shape, a few iterations (builds graphs, tunes the launch shape)
    for _ in range(max(1, min(a.warmup, 3))):
        P.cupso_solve_batch(probs, 24, cuda_stream=stream.cuda_stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    rc, res = P.cupso_solve_batch(probs, iters, cuda_stream=stream.cuda_stream)
    batched_s = time.perf_counter() - t0
    sample = list(range(0, len(probs), max(1, plain_every)))
    t0 = time.perf_counter()
    for k in sample:
        p = probs[k]
        h = P.cupso_create(p["D"], p["N"], p["bounds"], p["w"], p["c1"], p["c2"], p["fitness_id"], p["seed"])
        P.cupso_set_stream(h, stream.cuda_stream)
        P.cupso_set_option(h, P.CUPSO_OPT_GRAPH_CHUNK, 0)       # one launch per iteration,
        P.cupso_set_option(h, P.CUPSO_OPT_ITERS_PER_LAUNCH, 1)  # also for a swarm in the panel layout
        # cupso_create draws with swarm id 0, so this trajectory differs from the batch's
        # (same work, other random streams); only its time is used here
        P.cupso_step(h, iters)
        P.cupso_get_gbest(h, p["D"])
        P.cupso_destroy(h)
    plain_sample_s = time.perf_counter() - t0
    clk = clocks.stop()
    sample_pd = sum(probs[k]["N"] * probs[k]["D"] for k in sample) * iters
    plain_s = plain_sample_s * total_pd / sample_pd
    mism = 0
    for k in sample[:8]:
        rc1, one = P.cupso_solve_batch([probs[k]], iters, cuda_stream=stream.cuda_stream)
        mism += int(one[0]["idx"] != res[k]["idx"] or not np.array_equal(one[0]["pos"], res[k]["pos"]))
    # The step kernel against HBM: compulsory bytes of one iteration of all
    # swarms (20 B per padded particle-dimension + 8 B per padded particle:
    # pbest_fit read and written) over the solve's time per iteration (set-up,
    # Step 1 and the host results included, so a lower bound).
    padded = [((p["N"] + 127) // 128 * 128, p["D"]) for p in probs]
    alg = sum(20 * n * d + 8 * n for n, d in padded)
    peak, src = hbm_peak()
    achieved = alg / (batched_s / iters) / 1e9
    return {
        "workload": "batch512", "swarms": len(probs), "iters": iters, "N": "U{64..8192}", "D": "U{8..256}",
        "fitness": "sphere/rastrigin/ackley/rosenbrock cycling", "particle_dims_per_iter": total_pd // iters,
        "batched": {"seconds": batched_s, "status": rc, "value": total_pd / batched_s, "unit": UNIT,
                    "api": "cupso_solve_batch (init + 500 iterations + host results)"},
        "plain": {"seconds": plain_s, "sampled_swarms": len(sample), "sampled_seconds": plain_sample_s,
                  "value": total_pd / plain_s, "unit": UNIT,
                  "api": "per swarm: cupso_create, cupso_step(500) one launch per iteration, cupso_get_gbest, "
                         "cupso_destroy; every %d-th swarm timed, scaled by particle-dimension updates"
                         % max(1, plain_every)},
        "batched_over_plain": plain_s / batched_s,
        "alone_vs_batched_mismatches": mism,
        "roofline": {"bound": "hbm", "kernel": "batch_step_kernel", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "algorithmic_bytes_per_iteration": alg, "peak_source": src},
        "clocks": clk,
    }


def run_batch(a):
    import torch

    torch.cuda.set_device(0)
    from paper_2205_01313_gb300 import build as B
    B.build()
    from paper_2205_01313_gb300 import cupso as P
    stream = torch.cuda.Stream()
    r = batch_report(P, a, stream, plain_every=a.plain_sample)
    out = {
        "metric": METRIC, "value": r["batched"]["value"], "unit": UNIT, "n_gpus": 1, "steps": r["iters"],
        "warmup": a.warmup, "ms_per_step": r["batched"]["seconds"] * 1e3 / r["iters"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {k: r[k] for k in ("workload", "swarms", "iters", "N", "D", "fitness", "particle_dims_per_iter")},
        "batched": r["batched"], "plain": r["plain"], "batched_over_plain": r["batched_over_plain"],
        "alone_vs_batched_mismatches": r["alone_vs_batched_mismatches"], "roofline": r["roofline"],
        "clocks": r["clocks"],
    }
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------- #
# least squares: fitness as a GEMM, FP32 CUDA cores vs BF16 / FP8 tensor cores #
# --------------------------------------------------------------------------- #

CONVERGE = {"N": 1024, "D": 64, "M": 512, "iters": 800}


def converging_problem(M, D, seed):
    """A least-squares problem PSO solves within the run: A ~ N(0, 1/M) (unit-norm
    columns), x* ~ U[-1, 1], b = A x* + N(0, 1e-6); returns A, b and the FP64
    minimum of ||A x - b||^2 (numpy lstsq)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((M, D)) / np.sqrt(M)).astype(np.float32)
    xs = rng.uniform(-1, 1, D).astype(np.float32)
    b = (A.astype(np.float64) @ xs + 1e-3 * rng.standard_normal(M)).astype(np.float32)
    x64, res, _, _ = np.linalg.lstsq(A.astype(np.float64), b.astype(np.float64), rcond=None)
    r = A.astype(np.float64) @ x64.astype(np.float32).astype(np.float64) - b.astype(np.float64)
    return A, b, float(r @ r)


def lsq_report(P, stream, quick):
    """The least-squares workload (||A x - b||^2, A 4096 x 1024 ~ N(0, 1/4096),
    N = 8192 particles in [-2, 2]^1024, max_v 0.4): milliseconds per iteration
    with BF16, FP8, FP32 and FP64 fitness, each timed with CUDA events over a
    run of iterations after 3 untimed ones; the tensor-core product alone against
    the measured BF16 peak; and the precision comparison in a regime PSO
    converges in (N = 1024, D = 64, M = 512, 800 iterations): each precision's
    final FP64 residual against the FP64-fitness run and the lstsq minimum, over
    seeds 1-2 (quick) or 1-5."""
    import numpy as np
    import torch

    cfg = workloads.lsq_config()
    N, D, M = cfg["N"], cfg["D"], cfg["M"]
    A, b, _ = workloads.lsq_problem(M, D, seed=cfg["seed"])
    dA, db = torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda()
    timed = {"bf16": 60, "fp8": 60, "fp32": 5, "fp64": 2} if quick else {"bf16": 300, "fp8": 300, "fp32": 20,
                                                                         "fp64": 3}
    # the BF16 iteration once more with the FP64 Gram rescoring (the default is float-float)
    timed["bf16_rescore_fp64"] = timed["bf16"]
    iters = {}
    for name, T in timed.items():
        prec = name.split("_")[0]
        with P.Swarm(D, N, cfg["bounds"], cfg["w"], cfg["c1"], cfg["c2"], P.CUPSO_LSQ, cfg["seed"],
                     stream=stream.cuda_stream) as s:
            s.set_option(P.CUPSO_OPT_LSQ_RESCORE, 1 if name.endswith("rescore_fp64") else 0)
            s.set_lsq(dA.data_ptr(), db.data_ptr(), M, prec)
            s.step(3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(T)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / T
            iters[name] = {"ms_per_iter": ms, "iters_timed": T, "pd_per_s": N * D / (ms / 1e3),
                           "gbest_residual_f64": s.gbest_f64()}
    # the product alone, CUDA events around each of 50 launches inside further iterations
    fit_ms = {}
    for prec in ("bf16", "fp8"):
        with P.Swarm(D, N, cfg["bounds"], cfg["w"], cfg["c1"], cfg["c2"], P.CUPSO_LSQ, cfg["seed"],
                     stream=stream.cuda_stream) as s:
            s.set_lsq(dA.data_ptr(), db.data_ptr(), M, prec)
            s.step(5)
            s.set_option(P.CUPSO_OPT_TIME_FITNESS, 1)
            s.step(50)
            fit_ms[prec] = s.info()["fitness_ms"]
    flops = 2.0 * N * M * D
    peak = 1875.6
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak = float(json.load(fh)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        pass
    # precision in a converging regime
    C = CONVERGE
    seeds = [1, 2] if quick else [1, 2, 3, 4, 5]
    conv = {prec: [] for prec in ("fp64", "bf16", "fp8", "fp32")}
    minima = []
    for sd in seeds:
        Ac, bc, fmin = converging_problem(C["M"], C["D"], sd)
        minima.append(fmin)
        dAc, dbc = torch.from_numpy(Ac).cuda(), torch.from_numpy(bc).cuda()
        for prec in conv:
            with P.Swarm(C["D"], C["N"], cfg["bounds"], cfg["w"], cfg["c1"], cfg["c2"], P.CUPSO_LSQ, sd,
                         stream=stream.cuda_stream) as s:
                s.set_lsq(dAc.data_ptr(), dbc.data_ptr(), C["M"], prec)
                s.step(C["iters"])
                conv[prec].append(s.gbest_f64())
    study = {"config": dict(C, seeds=seeds, bounds=cfg["bounds"]), "lstsq_minimum": minima}
    for prec, vals in conv.items():
        v = np.array(vals)
        study[prec] = {"final_residual_f64": vals,
                       "rel_excess_over_minimum_max": float(np.max((v - minima) / minima)),
                       "rel_gap_vs_fp64_run_max": float(np.max(np.abs(v - np.array(conv["fp64"])) /
                                                               np.array(conv["fp64"])))}
    bf, fp32 = iters["bf16"]["ms_per_iter"], iters["fp32"]["ms_per_iter"]
    return {
        "workload": "lsq8192", "N": N, "D": D, "M": M, "bounds": cfg["bounds"],
        "ms_per_iter": {k: v["ms_per_iter"] for k, v in iters.items()}, "runs": iters,
        "bf16_over_fp32": fp32 / bf, "fp8_over_fp32": fp32 / iters["fp8"]["ms_per_iter"],
        "rescoring": "Gram form, off-diagonal part in float-float (bf16_rescore_fp64: FP64 arithmetic)",
        "fitness_product_ms": fit_ms,
        "roofline": {"bound": "tensor", "kernel": "lsq_tc_kernel<bf16>", "achieved": flops / (fit_ms["bf16"] / 1e3) / 1e12,
                     "peak": peak, "unit": "TFLOP/s", "frac": flops / (fit_ms["bf16"] / 1e3) / 1e12 / peak,
                     "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops, burst)",
                     "fp8_achieved": flops / (fit_ms["fp8"] / 1e3) / 1e12},
        "converging_study": study,
    }


def cublas_fp8_tflops(n=8192, reps=20):
    """Dense FP8 e4m3 GEMM throughput of cuBLASLt (torch._scaled_mm, n x n x n,
    BF16 output), as context for the FP8 product's fraction; None where this
    PyTorch has no FP8 GEMM."""
    import torch
    try:
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.tensor(1.0, device="cuda")
        run = lambda: torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)  # noqa: E731
        for _ in range(3):
            run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        return 2.0 * n ** 3 / (e0.elapsed_time(e1) / reps / 1e3) / 1e12
    except (RuntimeError, AttributeError, TypeError):
        return None


def lsq_launches(P, stream, prec):
    """The least-squares workload in one precision: set-up, 6 iterations, then 20
    timed ones, each iteration's kernels launched directly (no captured graph),
    so that a profiler lists them one by one."""
    import torch
    cfg = workloads.lsq_config()
    N, D, M = cfg["N"], cfg["D"], cfg["M"]
    A, b, _ = workloads.lsq_problem(M, D, seed=cfg["seed"])
    dA, db = torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda()
    name, prec = prec, prec.split("_")[0]
    with P.Swarm(D, N, cfg["bounds"], cfg["w"], cfg["c1"], cfg["c2"], P.CUPSO_LSQ, cfg["seed"],
                 stream=stream.cuda_stream) as s:
        s.set_option(P.CUPSO_OPT_LSQ_RESCORE, 1 if name.endswith("rescore_fp64") else 0)
        s.set_lsq(dA.data_ptr(), db.data_ptr(), M, prec)
        s.set_option(P.CUPSO_OPT_GRAPH_CHUNK, 0)
        s.step(6)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(20)
        e1.record(stream)
        torch.cuda.synchronize()
        return {"workload": "lsq8192", "precision": name, "iters_timed": 20,
                "ms_per_iter": e0.elapsed_time(e1) / 20, "graph": "none (one launch per kernel)"}


def run_lsq(a):
    import torch

    torch.cuda.set_device(0)
    from paper_2205_01313_gb300 import build as B
    B.build()
    from paper_2205_01313_gb300 import cupso as P
    stream = torch.cuda.Stream()
    if a.lsq_launches:
        print(json.dumps(lsq_launches(P, stream, a.lsq_launches)), flush=True)
        return
    r = lsq_report(P, stream, quick=False)
    # FP8: the peak of the fraction is the measured BF16 peak times the nominal
    # FP8 / BF16 ratio (2); cuBLASLt's own FP8 GEMM, measured here, beside it
    fp8_peak = 2.0 * r["roofline"]["peak"]
    cub = cublas_fp8_tflops()
    r["roofline"].update({"fp8_peak": fp8_peak, "fp8_frac": r["roofline"]["fp8_achieved"] / fp8_peak,
                          "fp8_peak_source": "measured BF16 peak x 2 (nominal FP8 / BF16 ratio)",
                          "cublas_fp8_tflops_measured": cub,
                          "fp8_frac_of_cublas": r["roofline"]["fp8_achieved"] / cub if cub else None})
    out = {
        "metric": METRIC, "value": r["runs"]["bf16"]["pd_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": r["runs"]["bf16"]["iters_timed"], "warmup": 3, "ms_per_step": r["ms_per_iter"]["bf16"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 fitness GEMM (fp32 accumulate), f32 state", "data": "synthetic",
        "config": {"workload": "lsq8192", "N": r["N"], "D": r["D"], "M": r["M"], "bounds": r["bounds"]},
        "lsq": r, "roofline": r["roofline"],
    }
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------- #
# global-best aggregation compared: the paper's tree reduction vs atomics       #
# --------------------------------------------------------------------------- #

def run_modes(a, name):
    """One workload, every aggregation mode, the whole run (all iterations of the
    workload in one cupso_step call) timed with CUDA events from the same
    initial swarm: on-chip cluster (if the swarm fits), fused atomic SYNC, the
    tree-reduction baseline (two kernels per iteration) and its unrolled form,
    the paper's queue (Alg. 2) and queue-lock (Alg. 3) designs, and the
    asynchronous lock-protected mode."""
    import torch

    torch.cuda.set_device(0)
    from paper_2205_01313_gb300 import build as B
    B.build()
    from paper_2205_01313_gb300 import cupso as P

    cfg = workloads.config(name)
    N, D, T, fid = cfg["N"], cfg["D"], cfg["iters"], cfg["fitness_id"]
    stream = torch.cuda.Stream()
    modes = ["onchip", "sync", "tree", "tree_unrolled", "queue", "queue_lock", "async"]
    out_modes = {}
    for mode in modes:
        with P.Swarm(D, N, cfg["bounds"], cfg["w"], cfg["c1"], cfg["c2"], fid, cfg["seed"],
                     stream=stream.cuda_stream) as s:
            try:
                s.set_mode(mode)
            except P.CupsoError:
                continue   # on-chip: the swarm does not fit
            s.step(min(3, T))          # warm-up (compiles graphs, first launches)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(T)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            rc, fit, idx, _ = s.gbest()
            out_modes[mode] = {"seconds": ms / 1e3, "us_per_iter": ms * 1e3 / T,
                               "pd_per_s": N * D * T / (ms / 1e3), "final_gbest_fit": float(fit), "status": rc}
    base = out_modes.get("tree", {}).get("seconds")
    for m in out_modes:
        if base:
            out_modes[m]["speedup_vs_tree"] = base / out_modes[m]["seconds"]
    best = max(out_modes.values(), key=lambda v: v["pd_per_s"])
    out = {"metric": METRIC, "value": best["pd_per_s"], "unit": UNIT, "n_gpus": 1, "steps": T, "warmup": 3,
           "ms_per_step": best["us_per_iter"] / 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": name, "N": N, "D": D, "iters": T,
                      "fitness": workloads.FITNESS_NAMES[fid]},
           "modes": out_modes}
    print(json.dumps(out), flush=True)


def spec_iters(spec, N):
    """Iterations of the paper's row for N (Table 4 gives one per row)."""
    cols = dict(zip(spec["columns"], spec["rows"][N]))
    return int(cols.get("iters", spec.get("iters", 0)))


def run_paper(a, table):
    """The paper's own experiments in its precision (FP64): Eq. 3 maximised,
    w = 1, c1 = c2 = 2, the shapes of Table 2 (1D, N = 32..2048, 100,000
    iterations; the four GPU designs), Table 3 (queue lock, 1D, N up to
    131,072) or Table 4 (queue, 120D). Every design the table compares runs as
    the paper built it (one particle per thread), beside this library's own
    FP64 paths (the fused SYNC step and, where the swarm fits one CTA, the
    on-chip kernel). Each run is timed with CUDA events over exactly the
    table's iteration count after 3 warm-up iterations. The FP64 oracle is
    timed on a bounded prefix of iterations per row and scaled, as this host's
    serial baseline. The paper's published seconds (GTX 1080 Ti, Xeon
    E3-1275 v5) are printed beside them as context."""
    import torch

    torch.cuda.set_device(0)
    from paper_2205_01313_gb300 import build as B
    B.build()
    from paper_2205_01313_gb300 import cupso as P
    from oracle import oracle as O

    spec = {"table2": workloads.PAPER_TABLE2, "table3": workloads.PAPER_TABLE3,
            "table4": workloads.PAPER_TABLE4}[table]
    modes = {"table2": ["tree", "tree_unrolled", "queue", "queue_lock", "sync", "onchip", "persistent"],
             "table3": ["queue_lock", "sync", "onchip", "persistent"],
             "table4": ["queue", "sync", "onchip"]}[table]
    if a.paper_modes:
        modes = [m for m in a.paper_modes.split(",") if m]
    want_rows = {int(x) for x in a.paper_rows.split(",") if x}
    S = workloads.PAPER_SETTING
    D = spec["D"]
    stream = torch.cuda.Stream()
    rows = []
    cpu_total = 0.0
    for N, paper in spec["rows"].items():
        if want_rows and N not in want_rows:
            continue
        cols = dict(zip(spec["columns"], paper))
        T = int(cols.pop("iters", spec.get("iters", 0)))
        if a.paper_iters > 0:
            T = min(T, a.paper_iters)
        row = {"N": N, "D": D, "iters": T, "paper_seconds": cols, "seconds": {}, "final_gbest_fit": {}}
        for mode in modes:
            with P.Swarm(D, N, S["bounds"], S["w"], S["c1"], S["c2"], S["fitness_id"], S["seed"],
                         stream=stream.cuda_stream, dtype="f64") as s:
                try:
                    s.set_mode(mode)
                except P.CupsoError:
                    continue   # on-chip: the swarm does not fit one CTA
                s.step(3)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.step(T)
                e1.record(stream)
                torch.cuda.synchronize()
                row["seconds"][mode] = e0.elapsed_time(e1) / 1e3
                rc, fit, _, _ = s.gbest()
                row["final_gbest_fit"][mode] = fit if rc == P.CUPSO_OK else "status %d" % rc
        ours = {m: row["seconds"][m] for m in ("sync", "onchip", "persistent") if m in row["seconds"]} \
            or dict(row["seconds"])
        best_mode = min(ours, key=ours.get)
        row["ours_best"] = best_mode
        paper_best_gpu = min(v for k, v in cols.items() if k != "cpu")
        row["paper_best_gpu_over_ours"] = paper_best_gpu * (T / spec_iters(spec, N)) / ours[best_mode]
        # this host's serial FP64 baseline: a bounded prefix of the same run, scaled
        k = max(1, min(T, int(2e6 // (N * D))))
        o = O.Swarm64(N, D, *S["bounds"], S["w"], S["c1"], S["c2"], S["fitness_id"], S["seed"]).init()
        t0 = time.perf_counter()
        o.step_sync(k)
        dt = time.perf_counter() - t0
        cpu_total += dt
        row["cpu_oracle_seconds_scaled"] = dt * T / k
        row["cpu_oracle_sample_iters"] = k
        rows.append(row)
    last = rows[-1]
    best_s = last["seconds"][last["ours_best"]]
    out = {"metric": METRIC, "value": last["N"] * D * last["iters"] / best_s, "unit": UNIT, "n_gpus": 1,
           "steps": last["iters"], "warmup": 3, "ms_per_step": best_s * 1e3 / last["iters"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "paper:" + table, "fitness": "cubic_max (Eq. 3, maximised)", "w": S["w"],
                      "c1": S["c1"], "c2": S["c2"], "bounds": S["bounds"],
                      "value_is": "particle-dim updates/s of the fastest library mode on the largest row"},
           "paper_hardware": "GTX 1080 Ti (CUDA 11.2) and one Xeon E3-1275 v5 core, FP64",
           "cpu_oracle": {"cores": 1, "kind": "oracle (FP64)", "seconds_spent": cpu_total},
           "rows": rows}
    print(json.dumps(out), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch512":
        run_batch(a)
    elif a.workload == "lsq8192":
        run_lsq(a)
    elif a.workload.startswith("modes:"):
        run_modes(a, a.workload.split(":", 1)[1])
    elif a.workload.startswith("paper:"):
        run_paper(a, a.workload.split(":", 1)[1])
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
