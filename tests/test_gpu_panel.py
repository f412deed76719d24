"""The SYNC step on the panel layout (state in panels of 8 or 16 dimensions) against
the oracle, bit for bit: whole trajectories with captured graphs and a ragged
particle count, a single step from an oracle-provided state, switches between
the panel kernel and kernels on the dimension-major layout in the middle of a
run (the state is converted between them), and checkpoint/resume through
cupso_get_state / cupso_set_state while the state is in panels."""
import time

import numpy as np
import pytest

from tests.gpu_common import W, C12, BOUNDS, assert_state_equal, load_cupso, oracle_swarm, same_bits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return load_cupso()


def _panel_swarm(P, fid, N, D, seed, kernel):
    s = P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, seed)
    s.set_mode("sync")
    s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS[kernel])
    return s


def test_panel_selection(P):
    """AUTO on a large swarm: 16-dimension panels for D >= 128, 8 below (the deepest
    ring the panels allow, 5, else 3); none for D % 8 != 0 or a single panel.
    Smaller swarms: 16-dimension panels up to 8192 particles, the tiled kernel
    below 2^17 particle-dimensions."""
    want = {64: (8, 5), 32: (8, 5), 48: (8, 5), 16: (8, 3), 24: (8, 3), 40: (8, 5), 128: (16, 5), 12: (0, None),
            8: (0, None)}
    for D, (width, stages) in want.items():
        with P.Swarm(D, 1 << 20, BOUNDS[3], W, C12, C12, 3, 1, mode="sync") as s:
            i = s.info()
            assert i["sync_panel"] == width, D
            if width:
                assert i["sync_stages"] == stages and i["sync_ppt"] == 1, D
    for N, D, fid, width, tile in [(131072, 64, 3, 8, False), (65536, 128, 1, 16, False), (65536, 64, 1, 8, False),
                                   (65536, 32, 3, 8, False), (262144, 32, 3, 8, False), (8192, 128, 3, 16, False),
                                   (32768, 128, 3, 16, False), (16384, 64, 1, 8, False), (8192, 32, 3, 16, False),
                                   (4096, 16, 1, 0, True), (2048, 32, 3, 0, True)]:
        with P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, 1, mode="sync") as s:
            i = s.info()
            assert i["sync_panel"] == width and (i["sync_tile"] > 0) == tile, (N, D, fid)
    with P.Swarm(64, 1 << 20, BOUNDS[3], W, C12, C12, 3, 1, mode="sync") as s:
        s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS["panel16"])
        assert s.info()["sync_panel"] == 16 and s.info()["sync_stages"] == 5
    with P.Swarm(32, 1 << 20, BOUNDS[3], W, C12, C12, 3, 1, mode="sync") as s:
        s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS["panel16"])
        assert s.info()["sync_panel"] == 16 and s.info()["sync_stages"] == 3
        s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS["pipelined4"])
        assert s.info()["sync_panel"] == 0 and s.info()["sync_ppt"] == 4


@pytest.mark.parametrize("kernel,D", [("panel8", 16), ("panel8", 40), ("panel16", 32), ("panel16", 64),
                                      ("panel16", 48)])
@pytest.mark.parametrize("fid", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("ipl", [1, 5, 0])
def test_panel_trajectory_bit_exact(P, fid, kernel, D, ipl):
    """ipl 1: one launch per iteration (a captured graph of 16, then single
    launches); 5: cooperative launches of up to 5 iterations with a grid
    barrier between them; 0 (default): one launch per cupso_step call."""
    N, T = 3000, 40            # 94 units of 32 particles, the last one ragged; padded to 3072
    with _panel_swarm(P, fid, N, D, 3, kernel) as s:
        s.set_option(P.CUPSO_OPT_ITERS_PER_LAUNCH, ipl)
        assert s.info()["sync_panel"] == int(kernel[5:])
        assert s.info()["sync_iters_per_launch"] == (ipl or 4096)
        s.step(1)
        s.step(16)
        s.step(23)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = oracle_swarm(fid, N, D, 3).init().step_sync(T)
    assert rc == P.CUPSO_OK and st["t"] == T
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and same_bits(pos, ref.gbest_pos)


@pytest.mark.parametrize("kernel", ["panel8", "panel16"])
def test_panel_single_step_from_shared_state(P, kernel):
    rng = np.random.default_rng(5)
    fid, N, D = 3, 2500, 32
    lo, hi, vmax = BOUNDS[fid]
    pos = rng.uniform(lo, hi, (N, D)).astype(np.float32)
    v = rng.uniform(-vmax, vmax, (N, D)).astype(np.float32)
    pb = rng.uniform(lo, hi, (N, D)).astype(np.float32)
    from oracle import oracle as O
    pf = np.array([O.fitness(fid, pb[i]) for i in range(N)], np.float32)
    ref = oracle_swarm(fid, N, D, 8)
    ref.set_state(pos, v, pb, pf, 41)
    with _panel_swarm(P, fid, N, D, 8, kernel) as s:
        s.set_state(pos, v, pb, pf, 41)
        s.step(1)
        st = s.state()
        rc, fit, idx, gpos = s.gbest()
    ref.step_sync(1)
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and same_bits(gpos, ref.gbest_pos)


def test_panel_mode_switches_mid_run(P):
    """Panel and dimension-major kernels alternate (the state is converted, with
    pbest rows pending across the switches): the oracle's trajectory."""
    fid, N, D = 1, 4100, 64
    plan = [("sync", "panel16", 3), ("sync", "panel8", 2), ("tree", None, 2), ("sync", "panel8", 4),
            ("sync", "pipelined3", 2), ("sync", "panel16", 17), ("queue", None, 1), ("sync", "register", 1),
            ("sync", "panel8", 2)]
    total = 0
    with P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, 6) as s:
        for mode, kernel, n in plan:
            s.set_mode(mode)
            if kernel:
                s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS[kernel])
            s.step(n)
            total += n
            if mode == "tree":
                s.state()          # a state read while the layout is dimension-major
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = oracle_swarm(fid, N, D, 6).init().step_sync(total)
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and same_bits(pos, ref.gbest_pos)


def test_panel_checkpoint_resume(P):
    """cupso_get_state while the state is in panels (rows pending), cupso_set_state
    into a new handle, continue on the panel kernel: the oracle's trajectory."""
    fid, N, D = 3, 5000, 32
    with _panel_swarm(P, fid, N, D, 9, "panel16") as s:
        s.step(7)
        ck = s.state()
    with _panel_swarm(P, fid, N, D, 9, "panel16") as s2:
        s2.set_state(ck["pos"], ck["v"], ck["pbest_pos"], ck["pbest_fit"], ck["t"])
        s2.step(9)
        st = s2.state()
        rc, fit, idx, pos = s2.gbest()
    ref = oracle_swarm(fid, N, D, 9).init().step_sync(16)
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and same_bits(pos, ref.gbest_pos)


@pytest.mark.parametrize("kernel,D", [("panel8", 16), ("panel16", 32)])
@pytest.mark.parametrize("N", [1, 17, 130])
@pytest.mark.parametrize("fid", [0, 3])
def test_panel_tiny_and_ragged_swarms(P, fid, N, D, kernel):
    """Swarms smaller than one warp unit or one 128-particle pad: padded
    particles move but never win; trajectories bit-exact with the oracle."""
    with _panel_swarm(P, fid, N, D, 5, kernel) as s:
        assert s.info()["sync_panel"] == int(kernel[5:])
        s.step(12)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = oracle_swarm(fid, N, D, 5).init().step_sync(12)
    assert rc == P.CUPSO_OK
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and same_bits(pos, ref.gbest_pos)


@pytest.mark.parametrize("kernel", ["panel8", "panel16"])
@pytest.mark.parametrize("T", [1, 3])
def test_panel_nan_fitness_sets_status(P, kernel, T):
    """A NaN fitness (inf - inf inside the cubic at +-1e30) sets the sticky status;
    the particle never becomes pbest or gbest; the steps are the oracle's (three
    iterations: one cooperative launch)."""
    fid, N, D = 4, 300, 16
    bounds = (-1e30, 1e30, 1.0)
    rng = np.random.default_rng(2)
    pos = rng.uniform(-1, 1, (N, D)).astype(np.float32)
    pos[77, :2] = [1e30, -1e30]
    from oracle import oracle as O
    pf = np.array([O.fitness(fid, p) for p in pos], np.float32)
    assert np.isnan(pf[77])
    with P.Swarm(D, N, bounds, W, C12, C12, fid, 1) as s:
        s.set_mode("sync")
        s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS[kernel])
        s.set_state(pos, np.zeros_like(pos), pos, pf, 0)
        s.step(T)
        rc, fit, idx, _ = s.gbest()
        st = s.state()
        assert rc == P.CUPSO_ERR_NAN and idx != 77
    ref = oracle_swarm(fid, N, D, 1, bounds=bounds)
    ref.set_state(pos, np.zeros_like(pos), pos, pf, 0)
    ref.step_sync(T)
    assert_state_equal(st, ref)


@pytest.mark.parametrize("ipl", [2, 3, 0])
def test_panel_multi_iteration_launch_shapes(P, ipl):
    """Cooperative launches of several iterations on grids of every kind: more
    warps than units (each warp's own first unit is all there is), a CTA count
    asked for above what the SMs hold (the launch is clamped to it), and odd
    step lengths that leave single launches behind: the oracle's trajectory."""
    cases = [(3, 130, 16, "panel8", 0), (1, 2000, 32, "panel16", 0), (3, 20000, 24, "panel8", 1 << 16),
             (2, 9000, 48, "panel16", 3)]
    for fid, N, D, kernel, grid in cases:
        with _panel_swarm(P, fid, N, D, 11, kernel) as s:
            s.set_option(P.CUPSO_OPT_ITERS_PER_LAUNCH, ipl)
            if grid:
                s.set_option(P.CUPSO_OPT_GRID, grid)
            for n in (7, 1, 4, 3):
                s.step(n)
            st = s.state()
            rc, fit, idx, pos = s.gbest()
        ref = oracle_swarm(fid, N, D, 11).init().step_sync(15)
        assert rc == P.CUPSO_OK, (fid, N, D)
        assert_state_equal(st, ref)
        assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and same_bits(pos, ref.gbest_pos)


def test_panel_launch_forms_agree_at_scale(P):
    """Rastrigin 65536 x 128 (16-dimension panels), 60 iterations in one
    cupso_step call: one cooperative launch and one launch per iteration give
    the same state, bit for bit."""
    fid, N, D = 1, 65536, 128
    out = []
    for ipl in (0, 1):
        with P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, 2, mode="sync") as s:
            s.set_option(P.CUPSO_OPT_ITERS_PER_LAUNCH, ipl)
            assert s.info()["sync_panel"] == 16
            s.step(60)
            rc, fit, idx, pos = s.gbest()
            assert rc == P.CUPSO_OK
            out.append((s.state(), idx, fit, pos))
    (a, ia, fa, pa), (b, ib, fb, pb) = out
    for k in ("pos", "v", "pbest_pos", "pbest_fit"):
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k
    assert ia == ib and same_bits(fa, fb) and same_bits(pa, pb)


def test_panel_barrier_wait_expires_and_reports(P):
    """A multi-iteration launch whose barrier waits for one CTA more than it has:
    every wait ends at the limit, the step reports CUPSO_ERR_DEVICE_TIMEOUT, and
    the context stays usable (status cleared, the swarm steps again, and a new
    swarm still follows the oracle)."""
    fid, N, D = 3, 20000, 32
    with _panel_swarm(P, fid, N, D, 7, "panel8") as s:
        s.set_option(P.CUPSO_OPT_WAIT_LIMIT_NS, 50_000_000)      # 50 ms
        s.set_option(P.CUPSO_OPT_FAULT_STALL_BARRIER, 1)
        t0 = time.time()
        s.step(3)
        rc, _, _, _ = s.gbest()
        assert rc == P.CUPSO_ERR_DEVICE_TIMEOUT
        assert time.time() - t0 < 30
        s.set_option(P.CUPSO_OPT_FAULT_STALL_BARRIER, 0)
        s.set_option(P.CUPSO_OPT_CLEAR_STATUS, 1)
        s.step(4)
        rc, _, _, _ = s.gbest()
        assert rc == P.CUPSO_OK
    with _panel_swarm(P, fid, 3000, 16, 5, "panel8") as s2:
        s2.step(9)
        st = s2.state()
    assert_state_equal(st, oracle_swarm(fid, 3000, 16, 5).init().step_sync(9))


@pytest.mark.parametrize("kernel,D", [("panel8", 64), ("pipelined4", 37)])
def test_gbest_result_slots_match_blocking_reads(P, kernel, D):
    """cupso_gbest_post / cupso_gbest_wait, a step ahead as a pipelined loop
    uses them: every result equals what cupso_get_gbest gives at that step (a
    twin swarm stepped and read in lock step), and the misuse of a slot is
    refused on the host."""
    fid, N, T = 3, 5000, 9
    with _panel_swarm(P, fid, N, D, 4, kernel) as s, _panel_swarm(P, fid, N, D, 4, kernel) as twin:
        want = []
        for k in range(T):
            twin.step(1)
            want.append(twin.gbest())
        got = []
        for k in range(T):
            s.step(1)
            s.gbest_post(k & 1)
            if k > 0:
                got.append(s.gbest_wait((k - 1) & 1))
        got.append(s.gbest_wait((T - 1) & 1))
        for (rc, fit, idx, pos), (rc2, fit2, idx2, pos2) in zip(got, want):
            assert rc == rc2 == P.CUPSO_OK and idx == idx2
            assert same_bits(fit, fit2) and same_bits(pos, pos2)
        with pytest.raises(P.CupsoError):
            s.gbest_wait(0)                  # nothing posted
        s.gbest_post(0)
        with pytest.raises(P.CupsoError):
            s.gbest_post(0)                  # still holds a result
        assert s.gbest_wait(0)[0] == P.CUPSO_OK


def test_gbest_result_slot_carries_the_status(P):
    """A NaN fitness reaches the reader through a result slot as through
    cupso_get_gbest."""
    fid, N, D = 4, 300, 16
    bounds = (-1e30, 1e30, 1.0)
    rng = np.random.default_rng(2)
    pos = rng.uniform(-1, 1, (N, D)).astype(np.float32)
    pos[77, :2] = [1e30, -1e30]
    from oracle import oracle as O
    pf = np.array([O.fitness(fid, p) for p in pos], np.float32)
    with P.Swarm(D, N, bounds, W, C12, C12, fid, 1) as s:
        s.set_mode("sync")
        s.set_state(pos, np.zeros_like(pos), pos, pf, 0)
        s.step(2)
        s.gbest_post(1)
        rc, fit, idx, _ = s.gbest_wait(1)
        assert rc == P.CUPSO_ERR_NAN and idx != 77
