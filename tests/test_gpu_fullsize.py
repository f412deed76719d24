"""Full-size workloads in the launch configuration the benchmark times.

At 2^20 particles x 64 dimensions the oracle cannot replay whole iterations in
a test, so it checks sampled particles one by one (Steps 2-4 from the state
before the step, with that step's gbest), and properties that hold at any size
check the rest: gbest is the lowest-index argmin of pbest_fit over all
particles, gbest_pos is that particle's pbest_pos, bounds hold everywhere.
"""
import numpy as np
import pytest

from tests.gpu_common import W, C12, BOUNDS, load_cupso, oracle_swarm, same_bits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return load_cupso()


def _check_step(P, s, fid, N, D, seed, samples):
    before = s.state()
    _, _, gidx, gpos = s.gbest()
    s.step(1)
    after = s.state()
    rc, fit, idx, pos = s.gbest()
    assert rc == P.CUPSO_OK and after["t"] == before["t"] + 1
    ref = oracle_swarm(fid, N, D, seed)
    t = after["t"]
    for i in samples:
        x, v, pb, pf, _ = ref.move_one(t, int(i), before["pos"][i], before["v"][i], before["pbest_pos"][i],
                                       before["pbest_fit"][i], gpos)
        assert same_bits(after["pos"][i], x), i
        assert same_bits(after["v"][i], v), i
        assert same_bits(after["pbest_pos"][i], pb), i
        assert same_bits(after["pbest_fit"][i], pf), i
    lo, hi, vmax = BOUNDS[fid]
    assert np.all((after["pos"] >= np.float32(lo)) & (after["pos"] <= np.float32(hi)))
    assert np.all(np.abs(after["v"]) <= np.float32(vmax))
    assert np.all(after["pbest_fit"] <= before["pbest_fit"])
    g = int(np.lexsort((np.arange(N), after["pbest_fit"]))[0])
    assert idx == g and same_bits(fit, after["pbest_fit"][g]) and same_bits(pos, after["pbest_pos"][g])


@pytest.mark.parametrize("mode", ["sync", "sync_register", "tree"])
def test_rosenbrock_2p20_x64_sampled(P, mode):
    """The benchmark's launch configuration is the default SYNC kernel, one launch per step."""
    fid, N, D, seed = 3, 1 << 20, 64, 1
    rng = np.random.default_rng(1)
    samples = np.concatenate([[0, 1, 1023, 1024, N - 1], rng.integers(0, N, 250)])
    with P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, seed, mode=mode.split("_")[0]) as s:
        s.set_option(P.CUPSO_OPT_GRAPH_CHUNK, 0)
        if mode == "sync_register":
            s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS["register"])
        s.step(3)
        _check_step(P, s, fid, N, D, seed, samples)


def test_rastrigin_65536x128_sampled(P):
    fid, N, D, seed = 1, 65536, 128, 1
    rng = np.random.default_rng(2)
    samples = np.concatenate([[0, N - 1], rng.integers(0, N, 200)])
    with P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, seed, mode="sync") as s:
        s.step(2)
        _check_step(P, s, fid, N, D, seed, samples)


def test_batch512_full_solve_sampled(P):
    """The benchmark's 512-swarm batch, 500 iterations, in the launch configuration
    it times (tuned kernel, graph-captured iterations): the swarms small enough
    for the oracle to replay whole (about 3 million particle-dimension updates
    each) must equal their oracle runs bit for bit, and every swarm's result
    must be a valid gbest (finite, within its bounds)."""
    from paper_2205_01313_gb300 import workloads as Wl
    probs = Wl.batch_problems(512)
    iters = 500
    rc, res = P.cupso_solve_batch(probs, iters)
    assert rc == P.CUPSO_OK
    for p, r in zip(probs, res):
        lo, hi, _ = p["bounds"]
        assert r["status"] == P.CUPSO_OK and np.isfinite(r["fit"])
        assert 0 <= r["idx"] < p["N"]
        assert np.all((r["pos"] >= np.float32(lo)) & (r["pos"] <= np.float32(hi)))
    small = sorted(range(len(probs)), key=lambda k: probs[k]["N"] * probs[k]["D"])[:6]
    for k in small:
        p = probs[k]
        ref = oracle_swarm(p["fitness_id"], p["N"], p["D"], p["seed"], swarm=p["swarm_id"],
                           bounds=p["bounds"]).init().step_sync(iters)
        assert res[k]["idx"] == ref.gbest_idx, k
        assert same_bits(res[k]["fit"], ref.gbest_fit) and same_bits(res[k]["pos"], ref.gbest_pos), k


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_lsq_8192x1024_full_size(P, precision):
    """The benchmark's least-squares swarm (N = 8192, D = 1024, M = 4096) in the
    launch configuration it times (graph-captured iterations): gbest's FP64
    fitness never increases and equals the oracle's ||A g - b||^2; sampled
    improvers of the last iteration hold the oracle's displacement-form fitness
    of their new position around that iteration's gbest; every position stays
    within the bounds."""
    import torch
    from oracle import oracle as O
    from paper_2205_01313_gb300 import workloads as Wl
    from tests.test_gpu_lsq import _check_improvers_displacement
    cfg = Wl.lsq_config()
    N, D, M = cfg["N"], cfg["D"], cfg["M"]
    A, b, _ = Wl.lsq_problem(M, D, seed=cfg["seed"])
    dA, db = torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda()
    lo, hi, vmax = cfg["bounds"]
    with P.Swarm(D, N, cfg["bounds"], cfg["w"], cfg["c1"], cfg["c2"], P.CUPSO_LSQ, cfg["seed"]) as s:
        s.set_lsq(dA.data_ptr(), db.data_ptr(), M, precision)
        prev = s.gbest_f64()
        for _ in range(2):
            s.step(16)
            g64 = s.gbest_f64()
            rc, fit, idx, pos = s.gbest()
            assert rc == P.CUPSO_OK and g64 <= prev
            exact = O.lsq_f64(A, b, pos)
            assert abs(g64 - exact) <= 1e-9 * exact
            prev = g64
        before = s.state()
        g = s.gbest()[3]
        s.step(1)
        st = s.state()
    assert np.all((st["pos"] >= np.float32(lo)) & (st["pos"] <= np.float32(hi)))
    assert np.all(np.abs(st["v"]) <= np.float32(vmax))
    assert (hi - lo) == 4.0      # the FP8 displacement scale of the tests, 448 / 4
    _check_improvers_displacement(A, b, before, g, st, precision, sample=24)


@pytest.mark.parametrize("mode", ["onchip", "sync", "tree"])
def test_sphere_1024x32_full_run(P, mode):
    """The sphere workload whole: 1024 particles x 32 dimensions, 1000 iterations
    in one cupso_step call (on-chip: a single launch of the cluster kernel); the
    final state equals the oracle's full run bit for bit."""
    from tests.gpu_common import assert_state_equal
    fid, N, D, T, seed = 0, 1024, 32, 1000, 1
    with P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, seed, mode=mode) as s:
        s.step(T)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = oracle_swarm(fid, N, D, seed).init().step_sync(T)
    assert rc == P.CUPSO_OK and st["t"] == T
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and same_bits(pos, ref.gbest_pos)


def test_rastrigin_65536x128_async_invariants(P):
    """ASYNC at the benchmark's Rastrigin size (persistent CTAs, no grid barrier):
    after each run, gbest is the lowest-index argmin of pbest_fit and equals its
    pbest_pos, sampled pbest_fit equal the oracle's fitness of their pbest_pos,
    pbest_fit never increases, and every position and velocity is in bounds."""
    from oracle import oracle as O
    fid, N, D, seed = 1, 65536, 128, 1
    lo, hi, vmax = BOUNDS[fid]
    rng = np.random.default_rng(4)
    sample = rng.choice(N, 100, replace=False)
    with P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, seed, mode="async") as s:
        prev = s.state()
        for _ in range(2):
            s.step(100)
            st = s.state()
            rc, fit, idx, pos = s.gbest()
            assert rc == P.CUPSO_OK
            assert np.all(st["pbest_fit"] <= prev["pbest_fit"])
            g = int(np.lexsort((np.arange(N), st["pbest_fit"]))[0])
            assert idx == g and same_bits(fit, st["pbest_fit"][g]) and same_bits(pos, st["pbest_pos"][g])
            for i in sample:
                assert same_bits(np.float32(O.fitness(fid, st["pbest_pos"][i])), st["pbest_fit"][i]), i
            assert np.all((st["pos"] >= np.float32(lo)) & (st["pos"] <= np.float32(hi)))
            assert np.all(np.abs(st["v"]) <= np.float32(vmax))
            prev = st


def test_paper_cubic_131072x120_fp64_sampled(P):
    """The paper's largest 120D shape in its own precision (Eq. 3 maximised,
    w = 1, c1 = c2 = 2, FP64; the tiled FP64 SYNC step): one step checked on
    sampled particles against the FP64 oracle's single-particle step from the
    state before it, gbest by brute force over all pbest."""
    from oracle import oracle as O
    fid, N, D, seed = 4, 131072, 120, 1
    lo, hi, vmax = -100.0, 100.0, 20.0
    with P.Swarm(D, N, (lo, hi, vmax), 1.0, 2.0, 2.0, fid, seed, mode="sync", dtype="f64") as s:
        s.step(3)
        before = s.state()
        _, _, _, gpos = s.gbest()
        s.step(1)
        after = s.state()
        rc, fit, idx, pos = s.gbest()
    assert rc == P.CUPSO_OK and after["t"] == before["t"] + 1
    ref = O.Swarm64(N, D, lo, hi, vmax, 1.0, 2.0, 2.0, fid, seed)
    rng = np.random.default_rng(5)
    for i in np.concatenate([[0, N - 1], rng.integers(0, N, 60)]):
        x, v, pb, pf, _ = ref.move_one(after["t"], int(i), before["pos"][i], before["v"][i], before["pbest_pos"][i],
                                       before["pbest_fit"][i], gpos)
        for got, want in ((after["pos"][i], x), (after["v"][i], v), (after["pbest_pos"][i], pb)):
            assert np.array_equal(np.asarray(got, np.float64).view(np.uint64), np.asarray(want, np.float64).view(np.uint64)), i
        assert np.float64(after["pbest_fit"][i]).view(np.uint64) == np.float64(pf).view(np.uint64), i
    assert np.all((after["pos"] >= lo) & (after["pos"] <= hi)) and np.all(np.abs(after["v"]) <= vmax)
    g = int(np.lexsort((np.arange(N), after["pbest_fit"]))[0])
    assert idx == g and fit == after["pbest_fit"][g] and np.array_equal(pos, after["pbest_pos"][g])
