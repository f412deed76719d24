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
