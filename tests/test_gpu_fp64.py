"""Double-precision swarms (the paper's precision) vs the FP64 oracle, bit-exact.

Every synchronous mode -- the fused one-launch step (SYNC), the paper's
reduction (TREE), unrolled reduction (TREE_UNROLLED) and queue (QUEUE)
designs with one particle per thread, and the on-chip kernel (ONCHIP) --
must give the oracle's trajectory bit for bit. The queue-lock design (Alg. 3)
equals it with one block and keeps the invariants with many. Sizes span
several 256-particle blocks with a ragged tail.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_common import load_cupso

pytestmark = pytest.mark.gpu

PAPER = dict(bounds=(-100.0, 100.0, 20.0), w=1.0, c=2.0)          # Sec. 5.1: Eq. 3, w = 1, c1 = c2 = 2
BOUNDS = {0: (-100.0, 100.0, 20.0), 3: (-30.0, 30.0, 6.0), 4: (-100.0, 100.0, 20.0)}
W, C12 = 0.729, 1.49445
STREAM_MODES = ["sync", "tree", "tree_unrolled", "queue", "persistent"]


@pytest.fixture(scope="module")
def P():
    return load_cupso()


def gpu64(P, fid, N, D, seed, mode=None, bounds=None, w=W, c1=C12, c2=C12):
    return P.Swarm(D, N, bounds or BOUNDS[fid], w, c1, c2, fid, seed, mode=mode, dtype="f64")


def ora64(fid, N, D, seed, bounds=None, w=W, c1=C12, c2=C12):
    lo, hi, vmax = bounds or BOUNDS[fid]
    return O.Swarm64(N, D, lo, hi, vmax, w, c1, c2, fid, seed)


def same64(a, b):
    a = np.ascontiguousarray(a, np.float64).view(np.uint64)
    b = np.ascontiguousarray(b, np.float64).view(np.uint64)
    return a.shape == b.shape and np.array_equal(a, b)


def assert_state64(st, ref):
    for name in ("pos", "v", "pbest_pos", "pbest_fit"):
        got, want = st[name], getattr(ref, name)
        if not same64(got, want):
            diff = np.argwhere(got.view(np.uint64) != want.view(np.uint64))
            k = tuple(diff[0])
            raise AssertionError("%s differs at %d places, first %s: gpu %r oracle %r"
                                 % (name, len(diff), k, got[k], want[k]))


@pytest.mark.parametrize("N,D", [(1, 1), (5, 3), (300, 1), (3000, 7), (513, 120)])
@pytest.mark.parametrize("fid", [0, 3, 4])
def test_init_bit_exact_fp64(P, fid, N, D):
    with gpu64(P, fid, N, D, 13) as s:
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = ora64(fid, N, D, 13).init()
    assert rc == P.CUPSO_OK and st["t"] == 0
    assert_state64(st, ref)
    assert idx == ref.gbest_idx and same64(fit, ref.gbest_fit) and same64(pos, ref.gbest_pos)


@pytest.mark.parametrize("mode", STREAM_MODES)
@pytest.mark.parametrize("fid", [0, 3, 4])
def test_trajectory_bit_exact_fp64(P, fid, mode):
    N, D, T = 3000, 5, 30
    with gpu64(P, fid, N, D, 4, mode) as s:
        s.step(1)
        s.step(16)      # one captured graph
        s.step(13)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = ora64(fid, N, D, 4).init().step_sync(T)
    assert rc == P.CUPSO_OK and st["t"] == T
    assert_state64(st, ref)
    assert idx == ref.gbest_idx and same64(fit, ref.gbest_fit) and same64(pos, ref.gbest_pos)


@pytest.mark.parametrize("mode", STREAM_MODES + ["onchip"])
@pytest.mark.parametrize("N,D", [(700, 4), (2048, 1), (40, 120)])
def test_trajectory_bit_exact_fp64_small(P, mode, N, D):
    fid, T = 4, 25
    with gpu64(P, fid, N, D, 8, mode, **_paper_kw()) as s:
        s.step(T)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = ora64(fid, N, D, 8, **_paper_kw()).init().step_sync(T)
    assert rc == P.CUPSO_OK
    assert_state64(st, ref)
    assert idx == ref.gbest_idx and same64(pos, ref.gbest_pos)


def _paper_kw():
    return dict(bounds=PAPER["bounds"], w=PAPER["w"], c1=PAPER["c"], c2=PAPER["c"])


@pytest.mark.parametrize("fid,N,D", [(4, 3000, 16), (3, 777, 33), (0, 5000, 120), (3, 129, 64), (4, 40, 2048),
                                     (0, 9, 2100)])
def test_sync_many_dimensions_bit_exact_fp64(P, fid, N, D):
    """D >= 16: the tiled SYNC kernel (a particle's dimensions spread over
    threads, the ordered sum by one thread); D > 2048 falls back to one
    particle per thread."""
    T = 12
    with gpu64(P, fid, N, D, 12, "sync") as s:
        s.step(T)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = ora64(fid, N, D, 12).init().step_sync(T)
    assert rc == P.CUPSO_OK
    assert_state64(st, ref)
    assert idx == ref.gbest_idx and same64(fit, ref.gbest_fit) and same64(pos, ref.gbest_pos)


@pytest.mark.parametrize("fid,N,D,C", [(4, 5, 3, 1), (4, 300, 1, 4), (3, 2048, 1, 16), (0, 100, 20, 16),
                                       (3, 511, 7, 16), (4, 17, 9, 2)])
def test_onchip_cluster_bit_exact_fp64(P, fid, N, D, C):
    """The on-chip kernel over clusters of 1 to 16 CTAs (some CTAs of a
    cluster may hold no particle)."""
    T = 40
    with gpu64(P, fid, N, D, 14, "onchip") as s:
        assert s.info()["onchip_cluster"] == C
        s.step(1)
        s.step(T - 1)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = ora64(fid, N, D, 14).init().step_sync(T)
    assert rc == P.CUPSO_OK
    assert_state64(st, ref)
    assert idx == ref.gbest_idx and same64(fit, ref.gbest_fit) and same64(pos, ref.gbest_pos)


@pytest.mark.parametrize("N,D", [(1, 2), (200, 3), (256, 1)])
def test_queue_lock_single_block_equals_sync_fp64(P, N, D):
    fid = 3
    with gpu64(P, fid, N, D, 6, "queue_lock") as s:
        s.step(20)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = ora64(fid, N, D, 6).init().step_sync(20)
    assert_state64(st, ref)
    assert idx == ref.gbest_idx and same64(pos, ref.gbest_pos)


@pytest.mark.parametrize("fid,N,D", [(3, 6000, 4), (4, 4096, 1)])
def test_queue_lock_invariants_fp64(P, fid, N, D):
    lo, hi, vmax = BOUNDS[fid]
    with gpu64(P, fid, N, D, 3, "queue_lock") as s:
        prev = s.state()
        for _ in range(3):
            s.step(10)
            st = s.state()
            rc, gfit, gidx, gpos = s.gbest()
            assert rc == P.CUPSO_OK
            assert np.all(np.abs(st["v"]) <= vmax) and np.all((st["pos"] >= lo) & (st["pos"] <= hi))
            assert np.all(st["pbest_fit"] <= prev["pbest_fit"])
            g = int(np.lexsort((np.arange(N), st["pbest_fit"]))[0])
            assert gidx == g and same64(gfit, st["pbest_fit"][g]) and same64(gpos, st["pbest_pos"][g])
            for i in np.random.default_rng(2).integers(0, N, 64):
                assert same64(O.fitness_d(fid, st["pbest_pos"][i]), st["pbest_fit"][i])
            prev = st


@pytest.mark.parametrize("mode", STREAM_MODES + ["onchip"])
def test_single_step_from_shared_state_fp64(P, mode):
    rng = np.random.default_rng(7)
    fid, N, D = 3, 900, 6
    lo, hi, vmax = BOUNDS[fid]
    pos = rng.uniform(lo, hi, (N, D))
    v = rng.uniform(-vmax, vmax, (N, D))
    pb = rng.uniform(lo, hi, (N, D))
    pf = np.array([O.fitness_d(fid, pb[i]) for i in range(N)])
    ref = ora64(fid, N, D, 9).set_state(pos, v, pb, pf, 77)
    with gpu64(P, fid, N, D, 9, mode) as s:
        s.set_state(pos, v, pb, pf, 77)
        _, fit0, idx0, _ = s.gbest()
        assert idx0 == ref.gbest_idx and same64(fit0, ref.gbest_fit)
        s.step(1)
        st = s.state()
        _, fit, idx, gpos = s.gbest()
    ref.step_sync(1)
    assert_state64(st, ref)
    assert idx == ref.gbest_idx and same64(gpos, ref.gbest_pos) and st["t"] == 78


def test_modes_interchangeable_mid_run_fp64(P):
    fid, N, D = 0, 1500, 3
    with gpu64(P, fid, N, D, 5, "sync") as s:
        assert s.info()["onchip_cluster"] == 16
        for mode, k in (("sync", 3), ("tree", 4), ("onchip", 5), ("queue", 2), ("tree_unrolled", 3), ("sync", 2)):
            s.set_mode(mode)
            s.step(k)
        st = s.state()
        _, fit, idx, pos = s.gbest()
    ref = ora64(fid, N, D, 5).init().step_sync(19)
    assert_state64(st, ref)
    assert idx == ref.gbest_idx and same64(pos, ref.gbest_pos)


def test_ties_go_to_lowest_index_fp64(P):
    fid, N, D = 0, 600, 2
    pos = np.ones((N, D))
    pf = np.full(N, 2.0)
    pf[[400, 33, 599]] = 0.5
    pf[301] = -0.0
    pf[302] = 0.0
    with gpu64(P, fid, N, D, 1, "sync") as s:
        s.set_state(pos, np.zeros_like(pos), pos, pf, 3)
        _, fit, idx, _ = s.gbest()
    assert idx == 301 and fit == 0.0


@pytest.mark.parametrize("mode", ["onchip", "sync", "queue", "tree"])
def test_paper_workload_reaches_the_maximiser(P, mode):
    """Eq. 3 maximised on [-100, 100] with w = 1, c1 = c2 = 2 (Sec. 5.1), 1D and
    N = 2048 as in Table 2: gbest reaches x = 100 exactly and is the lowest
    index among the particles whose pbest is there."""
    N, D, T = 2048, 1, 300
    with gpu64(P, 4, N, D, 1, mode, **_paper_kw()) as s:
        s.step(T)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    assert rc == P.CUPSO_OK
    assert fit == -900000.0 and pos[0] == 100.0
    assert idx == int(np.flatnonzero(st["pbest_pos"][:, 0] == 100.0)[0])


@pytest.mark.parametrize("N,D", [(1, 1), (129, 3), (8192, 1), (20000, 2), (300000, 1)])
def test_persistent_bit_exact_fp64(P, N, D):
    """The cooperative persistent kernel: all iterations of a cupso_step call in
    one launch, a grid barrier per iteration (N = 300000 makes threads loop
    over several particles)."""
    fid, T = 4, 15
    with gpu64(P, fid, N, D, 21, "persistent", **_paper_kw()) as s:
        s.step(7)
        s.step(T - 7)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = ora64(fid, N, D, 21, **_paper_kw()).init().step_sync(T)
    assert rc == P.CUPSO_OK
    assert_state64(st, ref)
    assert idx == ref.gbest_idx and same64(fit, ref.gbest_fit) and same64(pos, ref.gbest_pos)


@pytest.mark.parametrize("fid", [0, 3, 4])
@pytest.mark.parametrize("N,D", [(500, 7), (6000, 2), (60000, 1)])
def test_persistent_resident_bit_exact_fp64(P, fid, N, D):
    """Swarms of at most one particle per thread keep their state in shared
    memory for the whole launch; candidates travel with their positions (read
    with the key for D <= 4, after the reduction above that). N = 6000 has more
    blocks (94) than threads per block (64), so a reducing thread reads several
    slots; N = 60000 takes blocks of 512 threads."""
    T = 12
    with gpu64(P, fid, N, D, 29, "persistent") as s:
        s.step(5)
        s.step(T - 5)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = ora64(fid, N, D, 29).init().step_sync(T)
    assert rc == P.CUPSO_OK
    assert_state64(st, ref)
    assert idx == ref.gbest_idx and same64(fit, ref.gbest_fit) and same64(pos, ref.gbest_pos)


@pytest.mark.parametrize("N", [1, 127, 1000, 8192])
def test_persistent_restart_from_earlier_iteration(P, N):
    """The persistent kernel across launches: a run that goes back to an
    earlier iteration count (set_state) and one that switches to another mode
    and back must still follow the oracle (one dimension, the paper's 1D
    shapes)."""
    fid = 4
    kw = _paper_kw()
    with gpu64(P, fid, N, 1, 31, "persistent", **kw) as s:
        s.step(6)
        st = s.state()
        s.set_state(st["pos"], st["v"], st["pbest_pos"], st["pbest_fit"], 4)   # iterations 5, 6 again
        s.step(3)
        s.set_mode("sync")
        s.step(2)
        s.set_mode("persistent")
        s.step(4)
        st2 = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = ora64(fid, N, 1, 31, **kw).init().step_sync(6)
    ref.set_state(ref.pos.copy(), ref.v.copy(), ref.pbest_pos.copy(), ref.pbest_fit.copy(), 4)
    ref.step_sync(9)
    assert rc == P.CUPSO_OK and st2["t"] == 13
    assert_state64(st2, ref)
    assert idx == ref.gbest_idx and same64(fit, ref.gbest_fit) and same64(pos, ref.gbest_pos)


def test_fp64_handle_rejections(P):
    with gpu64(P, 0, 300, 2, 1) as s:
        assert s.info()["mode"] == P.CUPSO_MODE_ONCHIP            # AUTO: the swarm fits one CTA
        with pytest.raises(P.CupsoError) as e:
            s.set_mode("async")
        assert e.value.code == P.CUPSO_ERR_UNSUPPORTED
        L = P.lib()
        import ctypes as C
        f = C.c_float()
        assert L.cupso_get_gbest(s.h, C.byref(f), None, None) == P.CUPSO_ERR_UNSUPPORTED
        assert L.cupso_get_state(s.h, None, None, None, None, None) == P.CUPSO_ERR_UNSUPPORTED
    with gpu64(P, 0, 20000, 64, 1) as big:
        assert big.info()["mode"] == P.CUPSO_MODE_SYNC
        with pytest.raises(P.CupsoError) as e:
            big.set_mode("onchip")
        assert e.value.code == P.CUPSO_ERR_UNSUPPORTED
    with P.Swarm(2, 300, (-1.0, 1.0, 0.5), W, C12, C12, 0, 1) as s32:
        with pytest.raises(P.CupsoError) as e:
            s32.set_mode("persistent")
        assert e.value.code == P.CUPSO_ERR_UNSUPPORTED
        import ctypes as C
        d = C.c_double()
        assert P.lib().cupso_get_gbest_fp64(s32.h, C.byref(d), None, None) == P.CUPSO_ERR_UNSUPPORTED
