"""Seeded synthetic workloads (parameters only; no PSO arithmetic here).

The paper uses no dataset: its fitness functions are analytic (Sec. 5.1,
Eq. 3). These are the five generated workloads this project measures; the
bounds and velocity limits follow the standard ranges of each test function,
with max_v = 0.1 (max_pos - min_pos) where no value is given. Both the
library's tests/benchmarks and the oracle read them from here.
"""
import numpy as np

W_STD, C_STD = 0.729, 1.49445   # inertia / acceleration constants used by every workload

BOUNDS = {
    0: (-100.0, 100.0, 20.0),        # sphere
    1: (-5.12, 5.12, 1.024),         # Rastrigin
    2: (-32.768, 32.768, 6.5536),    # Ackley
    3: (-30.0, 30.0, 6.0),           # Rosenbrock
    4: (-100.0, 100.0, 20.0),        # the paper's cubic, Eq. 3
}

# name: (fitness_id, N, D, iterations, seed)
CONFIGS = {
    "sphere_1024x32": (0, 1024, 32, 1000, 1),
    "rastrigin_65536x128": (1, 65536, 128, 2000, 1),
    "rosenbrock_1048576x64": (3, 1 << 20, 64, 1000, 1),
    # a quarter of the swarm above (201 MB of state, still larger than L2): the
    # case the detailed profiler captures run on
    "rosenbrock_262144x64": (3, 1 << 18, 64, 1000, 1),
    # the 2^20-particle swarm with half the dimensions (403 MB): same per-warp
    # work pattern as the 2^20 x 64 swarm at half the size, for detailed captures
    "rosenbrock_1048576x32": (3, 1 << 20, 32, 1000, 1),
}

FITNESS_NAMES = {0: "sphere", 1: "rastrigin", 2: "ackley", 3: "rosenbrock", 4: "cubic_max"}


def config(name):
    fid, N, D, T, seed = CONFIGS[name]
    lo, hi, vmax = BOUNDS[fid]
    return {"name": name, "fitness_id": fid, "N": N, "D": D, "iters": T, "seed": seed,
            "bounds": (lo, hi, vmax), "w": W_STD, "c1": C_STD, "c2": C_STD}


def batch_problems(n_swarms=512, seed=1, n_range=(64, 8192), d_range=(8, 256)):
    """Independent swarms of uneven size: N ~ U{64..8192}, D ~ U{8..256},
    fitness cycling sphere / Rastrigin / Ackley / Rosenbrock, seed_s = s + 1."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(n_range[0], n_range[1] + 1, n_swarms)
    Ds = rng.integers(d_range[0], d_range[1] + 1, n_swarms)
    out = []
    for s in range(n_swarms):
        fid = s % 4
        out.append({"D": int(Ds[s]), "N": int(Ns[s]), "bounds": BOUNDS[fid], "w": W_STD, "c1": C_STD,
                    "c2": C_STD, "fitness_id": fid, "seed": s + 1, "swarm_id": s})
    return out


def lsq_config():
    """The least-squares workload: N = 8192 particles in [-2, 2]^1024 (max_v
    0.4), A 4096 x 1024, 300 iterations."""
    return {"N": 8192, "D": 1024, "M": 4096, "iters": 300, "seed": 1, "bounds": (-2.0, 2.0, 0.4),
            "w": W_STD, "c1": C_STD, "c2": C_STD}


def lsq_problem(M, D, seed=1, noise_std=1e-3):
    """A ~ N(0, 1/4096) entries (unit-norm columns in expectation at M = 4096),
    x* ~ U[-1, 1], b = A x* + N(0, noise_std^2)."""
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((M, D)) / 64.0).astype(np.float32)
    xs = rng.uniform(-1.0, 1.0, D).astype(np.float32)
    b = (A.astype(np.float64) @ xs.astype(np.float64) + noise_std * rng.standard_normal(M)).astype(np.float32)
    return A, b, xs


# ---------------------------------------------------------------------------
# The paper's own experiments (Sec. 5.1): Eq. 3 maximised on [-100, 100] in
# FP64 with w = 1 and c1 = c2 = 2. max_v is not given; 0.1 (max - min) = 20 as
# for the other workloads. The published times (seconds, GTX 1080 Ti and a
# serial Xeon E3-1275 v5 run, FP64) are kept beside each shape as context.
# ---------------------------------------------------------------------------
PAPER_SETTING = {"fitness_id": 4, "bounds": (-100.0, 100.0, 20.0), "w": 1.0, "c1": 2.0, "c2": 2.0, "seed": 1}

# Table 2: 1D, 100,000 iterations; columns CPU, reduction, loop unrolling, queue, queue lock.
PAPER_TABLE2 = {
    "D": 1, "iters": 100000,
    "columns": ("cpu", "tree", "tree_unrolled", "queue", "queue_lock"),
    "rows": {32: (0.100, 0.413, 0.394, 0.368, 0.216), 64: (0.187, 0.419, 0.402, 0.368, 0.219),
             128: (0.385, 0.447, 0.408, 0.371, 0.220), 256: (0.825, 0.455, 0.419, 0.371, 0.222),
             512: (1.503, 0.467, 0.422, 0.391, 0.223), 1024: (3.042, 0.491, 0.439, 0.394, 0.227),
             2048: (6.277, 0.508, 0.451, 0.409, 0.230)},
}

# Table 3: queue lock vs CPU, 1D, 100,000 iterations.
PAPER_TABLE3 = {
    "D": 1, "iters": 100000,
    "columns": ("cpu", "queue_lock"),
    "rows": {128: (0.385, 0.220), 256: (0.825, 0.222), 512: (1.503, 0.223), 1024: (3.042, 0.227),
             2048: (6.277, 0.230), 4096: (12.410, 0.265), 8192: (23.850, 0.316), 16384: (47.355, 0.417),
             32768: (94.629, 0.643), 65536: (200.536, 1.026), 131072: (378.671, 2.759)},
}

# Table 4: queue vs CPU, 120D; (iterations, cpu, queue) per particle count.
PAPER_TABLE4 = {
    "D": 120,
    "columns": ("iters", "cpu", "queue"),
    "rows": {128: (5000, 2.392, 0.487), 256: (4000, 3.543, 0.384), 512: (3000, 5.305, 0.288),
             1024: (2000, 7.078, 0.225), 2048: (2000, 14.214, 0.255), 4096: (1500, 21.593, 0.220),
             8192: (1000, 29.494, 0.191), 16384: (1000, 59.125, 0.294), 32768: (1000, 128.349, 0.570),
             65536: (1000, 237.933, 1.169), 131072: (800, 379.820, 1.744)},
}
