"""Asynchronous path (Sec. 3.2 / Alg. 3 without a grid barrier).

Its trajectory depends on timing, so it is checked by invariants, by the one
case where it must equal the synchronous path (a single CTA), and by reaching
the known optimum to 1e-4 on workloads where PSO does. Its bounded waits are
tested by holding the lock from the start: every wait must expire, set the
timeout status and leave the GPU usable.
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_common import W, C12, BOUNDS, assert_state_equal, load_cupso, oracle_swarm, same_bits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return load_cupso()


@pytest.mark.parametrize("fid,D", [(0, 5), (1, 5), (3, 5), (4, 1), (1, 1)])
def test_async_single_cta_equals_sync(P, fid, D):
    """D = 1 runs the streaming asynchronous kernel, D >= 2 the tiled one."""
    N, T = 700, 30
    with P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, 9, mode="async") as s:
        s.set_option(P.CUPSO_OPT_GRID, 1)
        s.step(T)
        st = s.state()
        rc, fit, idx, pos = s.gbest()
    ref = oracle_swarm(fid, N, D, 9).init().step_sync(T)
    assert rc == P.CUPSO_OK
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(pos, ref.gbest_pos)


@pytest.mark.parametrize("fid,N,D", [(1, 20000, 16), (3, 70000, 8), (2, 4096, 30), (4, 50000, 1)])
def test_async_invariants(P, fid, N, D):
    lo, hi, vmax = BOUNDS[fid]
    with P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, 2, mode="async") as s:
        assert s.info()["async_grid"] > 1
        prev = s.state()
        prev_g = s.gbest()[1]
        for _ in range(4):
            s.step(15)
            st = s.state()
            rc, gfit, gidx, gpos = s.gbest()
            assert rc == P.CUPSO_OK
            assert np.all(np.abs(st["v"]) <= np.float32(vmax))
            assert np.all((st["pos"] >= np.float32(lo)) & (st["pos"] <= np.float32(hi)))
            assert np.all(st["pbest_fit"] <= prev["pbest_fit"])          # pbest never worsens
            assert gfit <= prev_g                                         # gbest never worsens
            g = int(np.lexsort((np.arange(N), st["pbest_fit"]))[0])
            assert gidx == g and same_bits(gfit, st["pbest_fit"][g])      # gbest = min over pbest
            assert same_bits(gpos, st["pbest_pos"][g])
            for i in np.random.default_rng(0).integers(0, N, 64):         # pbest_fit = F(pbest_pos)
                assert same_bits(O.fitness(fid, st["pbest_pos"][i]), st["pbest_fit"][i])
            prev, prev_g = st, gfit


@pytest.mark.parametrize("fid,N,D,T", [(0, 1024, 32, 1000), (1, 1024, 4, 1000), (2, 1024, 8, 1000),
                                       (3, 1024, 4, 1000)])
def test_async_reaches_known_optimum(P, fid, N, D, T):
    with P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, 1, mode="async") as s:
        assert s.info()["async_grid"] > 1
        s.step(T)
        rc, fit, idx, pos = s.gbest()
    assert rc == P.CUPSO_OK
    assert float(fit) <= 1e-4, fit
    opt = 1.0 if fid == 3 else 0.0
    assert np.max(np.abs(pos - opt)) < (5e-2 if fid == 3 else 1e-2)


def test_async_lock_wait_expires_and_reports(P):
    N, D = 20000, 8
    with P.Swarm(D, N, BOUNDS[1], W, C12, C12, 1, 3, mode="async") as s:
        s.set_option(P.CUPSO_OPT_WAIT_LIMIT_NS, 50_000_000)      # 50 ms
        s.set_option(P.CUPSO_OPT_FAULT_HOLD_LOCK, 1)
        t0 = time.time()
        s.step(200)
        rc, _, _, _ = s.gbest()
        assert rc == P.CUPSO_ERR_DEVICE_TIMEOUT
        assert time.time() - t0 < 30
        # The context is still usable: clear, release the hook, run again.
        s.set_option(P.CUPSO_OPT_FAULT_HOLD_LOCK, 0)
        s.set_option(P.CUPSO_OPT_CLEAR_STATUS, 1)
        s.step(5)
        rc, _, _, _ = s.gbest()
        assert rc == P.CUPSO_OK
    # and a fresh synchronous swarm still matches the oracle
    with P.Swarm(3, 200, BOUNDS[0], W, C12, C12, 0, 5, mode="sync") as s2:
        s2.step(5)
        st = s2.state()
    assert_state_equal(st, oracle_swarm(0, 200, 3, 5).init().step_sync(5))


def test_async_after_pipelined_sync_steps(P):
    """The pipelined SYNC step leaves pbest rows pending (lazy pbest); the next
    kernel that reads pbest_pos directly must see them written back."""
    fid, N, D = 3, 3000, 9
    with P.Swarm(D, N, BOUNDS[fid], W, C12, C12, fid, 4, mode="sync") as s:
        s.set_option(P.CUPSO_OPT_SYNC_KERNEL, P.SYNC_KERNELS["pipelined4"])
        assert s.info()["sync_stages"] > 0
        s.step(6)
        s.set_mode("async")
        s.set_option(P.CUPSO_OPT_GRID, 1)
        s.step(5)
        st = s.state()
        _, fit, idx, pos = s.gbest()
    ref = oracle_swarm(fid, N, D, 4).init().step_sync(11)
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(pos, ref.gbest_pos)
