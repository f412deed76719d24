"""Synchronous path vs the oracle, element by element (bit-exact).

Sizes span several 1024-particle tiles with a ragged tail (N = 3000 -> 3 tiles,
padded to 3072) and odd D (the last Philox call serves a single dimension).
Every synchronous mode -- fused atomic (SYNC), tree baseline (TREE and its
unrolled form), on-chip cluster (ONCHIP), the paper's queue design (QUEUE,
one particle per thread) -- must give the oracle's trajectory.
"""
import numpy as np
import pytest

from tests.gpu_common import W, C12, BOUNDS, assert_state_equal, load_cupso, oracle_swarm, same_bits, ulp_distance

pytestmark = pytest.mark.gpu

SYNC_MODES = ["sync", "sync_register", "sync_pipelined3", "sync_ppt1", "sync_ppt2", "sync_tiled", "tree",
              "tree_unrolled", "onchip", "queue"]


@pytest.fixture(scope="module")
def P():
    return load_cupso()


def gpu_swarm(P, fid, N, D, seed, mode, bounds=None, w=W, c1=C12, c2=C12):
    """mode: a cupso mode name, or sync_<kernel> for a given SYNC kernel."""
    s = P.Swarm(D, N, bounds or BOUNDS[fid], w, c1, c2, fid, seed)
    if mode.startswith("sync_ppt"):
        s.set_mode("sync")
        s.set_option(P.CUPSO_OPT_PARTICLES_PER_THREAD, int(mode[8:]))
    elif mode.startswith("sync_"):
        s.set_mode("sync")
        s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS[mode[5:]])
    else:
        s.set_mode(mode)
    return s


def test_sync_kernel_selection(P):
    with gpu_swarm(P, 3, 1 << 20, 15, 1, "sync") as s:
        assert s.info()["sync_ppt"] == 4           # a large swarm: 4 particles per thread
    with gpu_swarm(P, 3, 1 << 20, 16, 1, "sync_pipelined4") as s:
        assert s.info()["sync_ppt"] == 4 and s.info()["sync_panel"] == 0
    with gpu_swarm(P, 3, 5000, 7, 1, "sync") as s:
        assert s.info()["sync_ppt"] == 1           # a small one: more, smaller units
        assert s.info()["sync_stages"] == 4
        s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS["pipelined3"])
        assert s.info()["sync_stages"] == 3
        s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS["register"])
        assert s.info()["sync_stages"] == 0
    with gpu_swarm(P, 3, 5000, 4, 1, "sync") as s:   # two dimension pairs: only the 3-stage ring
        assert s.info()["sync_stages"] == 3
    with gpu_swarm(P, 3, 5000, 2, 1, "sync_pipelined4") as s:   # too few dimension pairs: register kernel
        assert s.info()["sync_stages"] == 0
    with gpu_swarm(P, 1, 20000, 15, 1, "sync") as s:            # few particles per SM, D % 8 != 0: tiled
        assert s.info()["sync_tile"] > 0 and s.info()["sync_stages"] == 0
    with gpu_swarm(P, 1, 4096, 16, 1, "sync") as s:             # below 2^17 particle-dimensions: tiled
        assert s.info()["sync_tile"] > 0 and s.info()["sync_panel"] == 0
    with gpu_swarm(P, 1, 65536, 128, 1, "sync") as s:           # 2^23 particle-dimensions: panels
        assert s.info()["sync_tile"] == 0 and s.info()["sync_panel"] == 16
    with gpu_swarm(P, 1, 65536, 120, 1, "sync") as s:           # D % 8 == 0, 120 / 16 not whole: 8-wide
        assert s.info()["sync_tile"] == 0 and s.info()["sync_panel"] == 8
    with gpu_swarm(P, 3, 65536, 127, 1, "sync") as s:           # D % 8 != 0, narrow tiles, no cos: from ~224 per SM
        assert s.info()["sync_tile"] == 0 and s.info()["sync_panel"] == 0
    with gpu_swarm(P, 3, 65536, 32, 1, "sync") as s:            # 2^21, D < 128, N > 8192: 8-wide panels
        assert s.info()["sync_tile"] == 0 and s.info()["sync_panel"] == 8
    with gpu_swarm(P, 3, 8192, 32, 1, "sync") as s:             # 2^18 with at most 8192 particles: 16-wide
        assert s.info()["sync_tile"] == 0 and s.info()["sync_panel"] == 16
    with gpu_swarm(P, 1, 32768, 256, 1, "sync") as s:           # D >= 128: 16-wide
        assert s.info()["sync_tile"] == 0 and s.info()["sync_panel"] == 16


@pytest.mark.parametrize("N,D", [(1, 1), (5, 3), (127, 2), (129, 5), (3000, 7), (1024, 32)])
@pytest.mark.parametrize("fid", [0, 1, 2, 3, 4])
def test_init_bit_exact(P, fid, N, D):
    with P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, 11) as s:
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = oracle_swarm(fid, N, D, 11).init()
    assert rc == P.CUPSO_OK
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and same_bits(pos, ref.gbest_pos)
    assert st["t"] == 0


@pytest.mark.parametrize("mode", SYNC_MODES)
@pytest.mark.parametrize("fid", [0, 1, 2, 3, 4])
def test_trajectory_bit_exact(P, fid, mode):
    N, D, T = 3000, 7, 40
    with gpu_swarm(P, fid, N, D, 3, mode) as s:
        s.step(1)
        s.step(16)     # one captured graph (chunk 16)
        s.step(23)     # graph + remainder
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = oracle_swarm(fid, N, D, 3).init().step_sync(T)
    assert rc == P.CUPSO_OK and st["t"] == T
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx, (idx, ref.gbest_idx)
    assert same_bits(fit, ref.gbest_fit) and same_bits(pos, ref.gbest_pos)


@pytest.mark.parametrize("mode", SYNC_MODES)
def test_single_step_from_shared_state(P, mode):
    """One step from a state the oracle provides (not one either side reached
    by itself): positions, velocities and pbests drawn at random."""
    rng = np.random.default_rng(5)
    fid, N, D = 3, 2500, 9
    lo, hi, vmax = BOUNDS[fid]
    pos = rng.uniform(lo, hi, (N, D)).astype(np.float32)
    v = rng.uniform(-vmax, vmax, (N, D)).astype(np.float32)
    pb = rng.uniform(lo, hi, (N, D)).astype(np.float32)
    ref = oracle_swarm(fid, N, D, 8)
    from oracle import oracle as O
    pf = np.array([O.fitness(fid, pb[i]) for i in range(N)], np.float32)
    ref.set_state(pos, v, pb, pf, 41)
    with gpu_swarm(P, fid, N, D, 8, mode) as s:
        s.set_state(pos, v, pb, pf, 41)
        rc, fit0, idx0, _ = s.gbest()
        assert idx0 == ref.gbest_idx and same_bits(fit0, ref.gbest_fit)
        s.step(1)
        st = s.state()
        rc, fit, idx, gpos = s.gbest()
    ref.step_sync(1)
    for name in ("pos", "v", "pbest_pos", "pbest_fit"):
        assert ulp_distance(st[name], getattr(ref, name)).max() <= 2, name
    assert_state_equal(st, ref)       # the bar is 2 ulp; the arithmetic is identical, so 0
    assert idx == ref.gbest_idx and st["t"] == 42


@pytest.mark.parametrize("fid", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("N,D", [(1, 1), (37, 2), (600, 9), (3000, 128), (200, 300), (33, 4096)])
def test_tiled_kernel_bit_exact(P, fid, N, D):
    """The tiled SYNC kernel over tile sizes from 1 to 32 particles (D up to
    4096), ragged last tiles and odd D."""
    T = 9
    with gpu_swarm(P, fid, N, D, 23, "sync_tiled") as s:
        assert s.info()["sync_tile"] > 0
        s.step(T)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = oracle_swarm(fid, N, D, 23).init().step_sync(T)
    assert rc == P.CUPSO_OK
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and same_bits(pos, ref.gbest_pos)


def test_modes_interchangeable_mid_run(P):
    fid, N, D = 1, 2048, 12
    with gpu_swarm(P, fid, N, D, 21, "sync") as s:
        s.step(7)
        s.set_mode("tree")
        s.step(5)
        s.set_mode("onchip")
        s.step(9)
        s.set_mode("tree_unrolled")
        s.step(3)
        s.set_mode("queue")
        s.step(4)
        s.set_mode("sync")
        s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS["tiled"])
        s.step(3)
        s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS["pipelined4"])
        s.step(2)
        st = s.state()
        _, fit, idx, pos = s.gbest()
    ref = oracle_swarm(fid, N, D, 21).init().step_sync(33)
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(pos, ref.gbest_pos)


@pytest.mark.parametrize("kernel", ["sync_register", "sync_pipelined3", "sync_pipelined4", "sync_ppt1", "sync_ppt2"])
@pytest.mark.parametrize("grid", [1, 2, 5])
@pytest.mark.parametrize("chunk", [0, 4])
def test_launch_shape_does_not_change_results(P, grid, chunk, kernel):
    fid, N, D, T = 2, 5000, 6, 12
    with gpu_swarm(P, fid, N, D, 4, kernel) as s:
        s.set_option(P.CUPSO_OPT_GRID, grid)
        s.set_option(P.CUPSO_OPT_GRAPH_CHUNK, chunk)
        s.step(T)
        st = s.state()
    ref = oracle_swarm(fid, N, D, 4).init().step_sync(T)
    assert_state_equal(st, ref)


def test_checkpoint_resume_bit_exact(P):
    fid, N, D = 3, 1500, 10
    with gpu_swarm(P, fid, N, D, 6, "sync") as a:
        a.step(10)
        ck = a.state()
        a.step(10)
        full = a.state()
    with gpu_swarm(P, fid, N, D, 6, "tree") as b:     # a fresh handle, another mode
        b.set_state(ck["pos"], ck["v"], ck["pbest_pos"], ck["pbest_fit"], ck["t"])
        b.step(10)
        resumed = b.state()
    for k in ("pos", "v", "pbest_pos", "pbest_fit"):
        assert same_bits(resumed[k], full[k]), k
    assert resumed["t"] == 20


@pytest.mark.parametrize("fid", [0, 1, 3])
@pytest.mark.parametrize("N,D", [(1, 3), (100, 5), (256, 8)])
def test_queue_lock_single_block_equals_sync(P, fid, N, D):
    """Alg. 3 with one block (N <= 256): nothing else can update gbest during
    the launch, so the result is the synchronous trajectory."""
    with gpu_swarm(P, fid, N, D, 6, "queue_lock") as s:
        s.step(1)
        s.step(16)
        s.step(13)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = oracle_swarm(fid, N, D, 6).init().step_sync(30)
    assert rc == P.CUPSO_OK
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and same_bits(pos, ref.gbest_pos)


@pytest.mark.parametrize("fid,N,D", [(1, 20000, 6), (3, 5000, 9), (4, 3000, 1)])
def test_queue_lock_invariants(P, fid, N, D):
    """Alg. 3 with many blocks: gbest is updated in place during the launch, so
    the trajectory depends on timing; after every launch gbest is still the
    lexicographic minimum over pbest, pbest never worsens, the state stays in
    its box, and every pbest_fit is the fitness of its pbest_pos."""
    from oracle import oracle as O
    lo, hi, vmax = BOUNDS[fid]
    with gpu_swarm(P, fid, N, D, 2, "queue_lock") as s:
        prev = s.state()
        for _ in range(4):
            s.step(10)
            st = s.state()
            rc, gfit, gidx, gpos = s.gbest()
            assert rc == P.CUPSO_OK
            assert np.all(np.abs(st["v"]) <= np.float32(vmax))
            assert np.all((st["pos"] >= np.float32(lo)) & (st["pos"] <= np.float32(hi)))
            assert np.all(st["pbest_fit"] <= prev["pbest_fit"])
            g = int(np.lexsort((np.arange(N), st["pbest_fit"]))[0])
            assert gidx == g and same_bits(gfit, st["pbest_fit"][g]) and same_bits(gpos, st["pbest_pos"][g])
            for i in np.random.default_rng(1).integers(0, N, 64):
                assert same_bits(O.fitness(fid, st["pbest_pos"][i]), st["pbest_fit"][i])
            prev = st


def test_gbest_ties_go_to_lowest_index(P):
    fid, N, D = 0, 300, 2
    pos = np.zeros((N, D), np.float32)
    pos[:, 0] = 1.0
    pf = np.full(N, 1.0, np.float32)
    pf[[17, 5, 250]] = 0.25
    pf[[9]] = -0.0
    pf[[4]] = 0.0
    with gpu_swarm(P, fid, N, D, 1, "sync") as s:
        s.set_state(pos, np.zeros_like(pos), pos, pf, 0)
        _, fit, idx, _ = s.gbest()
    assert idx == 4 and fit == 0.0


def test_nan_fitness_sets_status(P):
    """A NaN fitness (here inf - inf inside the cubic at +-1e30) sets the sticky
    status; the particle never becomes pbest or gbest."""
    fid, N, D = 4, 256, 2
    bounds = (-1e30, 1e30, 1.0)
    rng = np.random.default_rng(2)
    pos = rng.uniform(-1, 1, (N, D)).astype(np.float32)
    pos[77] = [1e30, -1e30]
    from oracle import oracle as O
    pf = np.array([O.fitness(fid, p) for p in pos], np.float32)
    assert np.isnan(pf[77])
    with gpu_swarm(P, fid, N, D, 1, "sync", bounds=bounds) as s:
        s.set_state(pos, np.zeros_like(pos), pos, pf, 0)
        s.step(1)
        rc, fit, idx, _ = s.gbest()
        st = s.state()
        assert rc == P.CUPSO_ERR_NAN
        assert idx != 77
        s.set_option(P.CUPSO_OPT_CLEAR_STATUS, 1)
        rc, _, _, _ = s.gbest()
        assert rc == P.CUPSO_OK
    ref = oracle_swarm(fid, N, D, 1, bounds=bounds)
    ref.set_state(pos, np.zeros_like(pos), pos, pf, 0)
    ref.step_sync(1)
    assert_state_equal(st, ref)


@pytest.mark.parametrize("case", ["zero_lower_bound", "zero_upper_bound", "tiny_c1"])
@pytest.mark.parametrize("mode", ["sync", "sync_register", "onchip"])
def test_trajectory_other_arithmetic_paths(P, case, mode):
    """Bounds at 0 (signed-zero ties possible: the min/max clamp is not used) and
    c1 so small that c1 * 2^-24 is subnormal (the fused c*r form is not used)."""
    fid, N, D, T = 0, 2000, 6, 30
    bounds, c1 = BOUNDS[0], C12
    if case == "zero_lower_bound":
        bounds = (0.0, 10.0, 2.0)
    elif case == "zero_upper_bound":
        bounds = (-10.0, 0.0, 2.0)
    else:
        c1 = 1e-38
    with gpu_swarm(P, fid, N, D, 5, mode, bounds=bounds, c1=c1) as s:
        s.step(T)
        st = s.state()
        _, fit, idx, pos = s.gbest()
    ref = oracle_swarm(fid, N, D, 5, bounds=bounds, c1=c1).init().step_sync(T)
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(pos, ref.gbest_pos)


def test_solve_batch_matches_single_swarms(P):
    probs = []
    for k, (fid, N, D) in enumerate([(0, 70, 8), (1, 1500, 13), (2, 333, 4), (3, 2100, 9), (4, 64, 1)]):
        probs.append(dict(D=D, N=N, bounds=BOUNDS[fid], w=W, c1=C12, c2=C12, fitness_id=fid, seed=k + 1,
                          swarm_id=k))
    rc, res = P.cupso_solve_batch(probs, 30)
    assert rc == P.CUPSO_OK
    for k, p in enumerate(probs):
        ref = oracle_swarm(p["fitness_id"], p["N"], p["D"], p["seed"], swarm=p["swarm_id"]).init().step_sync(30)
        assert res[k]["status"] == P.CUPSO_OK
        assert res[k]["idx"] == ref.gbest_idx
        assert same_bits(res[k]["fit"], ref.gbest_fit) and same_bits(res[k]["pos"], ref.gbest_pos)


def _mixed_batch(n, seed, n_range, d_range):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        fid = k % 5
        out.append(dict(D=int(rng.integers(*d_range)), N=int(rng.integers(*n_range)), bounds=BOUNDS[fid], w=W,
                        c1=C12, c2=C12, fitness_id=fid, seed=1000 + k, swarm_id=k))
    return out


@pytest.mark.parametrize("iters", [0, 1, 5, 30])
def test_batched_solve_matches_oracle(P, iters):
    """Uneven swarms with every fitness function in one batch; 0 iterations is
    Step 1 alone, 30 iterations run the launch-shape tuner on the real work
    first. Each swarm must equal its oracle run."""
    probs = _mixed_batch(24, 7, (64, 2500), (3, 40))
    probs[3]["D"] = 2              # too few dimension pairs: solved through its own handle
    probs[5]["D"] = 3              # the smallest batched dimension count
    rc, res = P.cupso_solve_batch(probs, iters)
    assert rc == P.CUPSO_OK
    for k, p in enumerate(probs):
        ref = oracle_swarm(p["fitness_id"], p["N"], p["D"], p["seed"], swarm=p["swarm_id"]).init().step_sync(iters)
        assert res[k]["status"] == P.CUPSO_OK
        assert res[k]["idx"] == ref.gbest_idx, k
        assert same_bits(res[k]["fit"], ref.gbest_fit) and same_bits(res[k]["pos"], ref.gbest_pos), k


@pytest.mark.parametrize("kernel", ["tiled", "streaming"])
def test_batched_solve_each_kernel_matches_oracle(P, kernel, monkeypatch):
    """Both batch kernels, fixed instead of tuned: every swarm equals its oracle
    run (tiles of 1 to 256 particles with D from 3 to 300)."""
    monkeypatch.setenv("CUPSO_BATCH_KERNEL", kernel)
    probs = _mixed_batch(20, 11, (40, 3000), (3, 300))
    rc, res = P.cupso_solve_batch(probs, 12)
    assert rc == P.CUPSO_OK
    for k, p in enumerate(probs):
        ref = oracle_swarm(p["fitness_id"], p["N"], p["D"], p["seed"], swarm=p["swarm_id"]).init().step_sync(12)
        assert res[k]["status"] == P.CUPSO_OK
        assert res[k]["idx"] == ref.gbest_idx, k
        assert same_bits(res[k]["fit"], ref.gbest_fit) and same_bits(res[k]["pos"], ref.gbest_pos), k


@pytest.mark.parametrize("kernel", ["tiled", "streaming"])
def test_batched_solve_general_path_matches_oracle(P, kernel, monkeypatch):
    """Swarms that cannot take the fast path (a bound at 0, so min/max clamps
    could meet a signed zero; c1 too small for the fused c*r) next to ones
    that can, every fitness function: each equals its oracle run."""
    monkeypatch.setenv("CUPSO_BATCH_KERNEL", kernel)
    probs = _mixed_batch(10, 17, (100, 1500), (4, 48))
    for k, p in enumerate(probs):
        if k % 3 == 0:
            p["bounds"] = (0.0, 10.0, 2.0)
        elif k % 3 == 1:
            p["c1"] = 1e-38
    rc, res = P.cupso_solve_batch(probs, 10)
    assert rc == P.CUPSO_OK
    for k, p in enumerate(probs):
        ref = oracle_swarm(p["fitness_id"], p["N"], p["D"], p["seed"], swarm=p["swarm_id"], bounds=p["bounds"],
                           c1=p["c1"]).init().step_sync(10)
        assert res[k]["status"] == P.CUPSO_OK
        assert res[k]["idx"] == ref.gbest_idx, k
        assert same_bits(res[k]["fit"], ref.gbest_fit) and same_bits(res[k]["pos"], ref.gbest_pos), k


def test_batched_solve_wide_swarm_matches_oracle(P, monkeypatch):
    """A swarm wider than any tile (D = 4500 > 4096 items) leaves only the
    streaming kernel to the tuner; next to small swarms it must still give
    every swarm's oracle result."""
    monkeypatch.delenv("CUPSO_BATCH_KERNEL", raising=False)
    probs = _mixed_batch(4, 21, (64, 300), (3, 20))
    probs.append(dict(D=4500, N=130, bounds=BOUNDS[3], w=W, c1=C12, c2=C12, fitness_id=3, seed=77, swarm_id=9))
    rc, res = P.cupso_solve_batch(probs, 20)
    assert rc == P.CUPSO_OK
    for k, p in enumerate(probs):
        ref = oracle_swarm(p["fitness_id"], p["N"], p["D"], p["seed"], swarm=p["swarm_id"]).init().step_sync(20)
        assert res[k]["idx"] == ref.gbest_idx, k
        assert same_bits(res[k]["fit"], ref.gbest_fit) and same_bits(res[k]["pos"], ref.gbest_pos), k


def test_batched_solve_nan_swarm_status(P):
    """A swarm whose fitness overflows to NaN (the cubic at +-1e30) gets the NaN
    status in its own result, the batch returns it as the first failure, the
    other swarms stay CUPSO_OK, and every swarm still equals its oracle run
    (NaN ranks last)."""
    probs = _mixed_batch(4, 23, (100, 600), (3, 12))
    probs.append(dict(D=2, N=300, bounds=(-1e30, 1e30, 1.0), w=W, c1=C12, c2=C12, fitness_id=4, seed=5,
                      swarm_id=40))
    rc, res = P.cupso_solve_batch(probs, 6)
    assert rc == P.CUPSO_ERR_NAN
    for k, p in enumerate(probs):
        ref = oracle_swarm(p["fitness_id"], p["N"], p["D"], p["seed"], swarm=p["swarm_id"],
                           bounds=p["bounds"]).init().step_sync(6)
        assert res[k]["status"] == (P.CUPSO_ERR_NAN if k == len(probs) - 1 else P.CUPSO_OK), k
        assert res[k]["idx"] == ref.gbest_idx, k
        assert same_bits(res[k]["pos"], ref.gbest_pos), k


def test_batched_kernels_interchange_with_lazy_pbest(P, monkeypatch):
    """The tuner may switch kernels between iterations of one solve; the
    streaming kernel leaves pbest rows pending (lazy write-back) and the tiled
    kernel must take them over. Forcing a long enough solve to tune covers
    the hand-over; the results must still be the oracle's."""
    monkeypatch.delenv("CUPSO_BATCH_KERNEL", raising=False)
    probs = _mixed_batch(12, 13, (100, 2000), (6, 64))
    rc, res = P.cupso_solve_batch(probs, 40)
    assert rc == P.CUPSO_OK
    for k, p in enumerate(probs):
        ref = oracle_swarm(p["fitness_id"], p["N"], p["D"], p["seed"], swarm=p["swarm_id"]).init().step_sync(40)
        assert res[k]["idx"] == ref.gbest_idx, k
        assert same_bits(res[k]["pos"], ref.gbest_pos), k


def test_batched_solve_repeatable(P):
    """A second identical batch reuses the remembered launch shape; same results."""
    probs = _mixed_batch(10, 9, (100, 1200), (5, 20))
    rc1, a = P.cupso_solve_batch(probs, 24)
    rc2, b = P.cupso_solve_batch(probs, 24)
    assert rc1 == rc2 == P.CUPSO_OK
    for x, y in zip(a, b):
        assert x["idx"] == y["idx"] and same_bits(x["pos"], y["pos"])


def test_onchip_selected_for_small_swarm(P):
    with P.Swarm(32, 1024, BOUNDS[0], W, C12, C12, 0, 1) as s:
        info = s.info()
        assert info["mode"] == P.CUPSO_MODE_ONCHIP and info["onchip_cluster"] >= 2
    with P.Swarm(64, 1 << 16, BOUNDS[3], W, C12, C12, 3, 1) as s:
        assert s.info()["mode"] == P.CUPSO_MODE_SYNC
        with pytest.raises(P.CupsoError):
            s.set_mode("onchip")


def test_sphere_1024x32_full_run_bit_exact(P):
    """The 1024-particle, 32-dimension, 1000-iteration sphere workload in full."""
    with P.Swarm(32, 1024, BOUNDS[0], W, C12, C12, 0, 1) as s:
        s.step(1000)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = oracle_swarm(0, 1024, 32, 1).init().step_sync(1000)
    assert rc == P.CUPSO_OK
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and float(fit) < 1e-4
