"""Least-squares fitness ||A x - b||^2 of many positions: the plain FP32 path
against the oracle (bit for bit), the BF16 and FP8 tensor-core paths against
the FP64 value within bounds derived from the operand rounding."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_common import load_cupso

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return load_cupso()


def _problem(M, D, N, seed=0):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((M, D)) / 64.0).astype(np.float32)      # N(0, 1/4096)
    xs = rng.uniform(-1, 1, D).astype(np.float32)
    b = (A.astype(np.float64) @ xs + 1e-3 * rng.standard_normal(M)).astype(np.float32)
    X = rng.uniform(-2, 2, (N, D)).astype(np.float32)
    return A, b, X


def _eval(P, A, b, X, precision):
    import torch
    dA, db, dX = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (A, b, X))
    f = torch.full((X.shape[0],), float("nan"), dtype=torch.float32, device="cuda")
    P.cupso_lsq_eval(dA.data_ptr(), db.data_ptr(), A.shape[0], A.shape[1], dX.data_ptr(), X.shape[0], precision,
                     f.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return f.cpu().numpy()


def _round_bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("M,D,N", [(40, 7, 30), (300, 65, 257), (513, 130, 129)])
def test_lsq_fp32_bit_exact(P, M, D, N):
    A, b, X = _problem(M, D, N)
    f = _eval(P, A, b, X, P.CUPSO_LSQ_FP32)
    ref = np.array([O.lsq_f32(A, b, X[i]) for i in range(N)], np.float32)
    np.testing.assert_array_equal(f.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("M,D,N", [(256, 64, 128), (700, 200, 1000), (4096, 1024, 512), (1300, 96, 1100)])
def test_lsq_bf16_tensor_cores(P, M, D, N):
    """f~ from BF16 operands equals the FP64 fitness of the BF16-rounded operands up
    to FP32 accumulation error, and the FP64 fitness of the exact operands within
    the bound the operand rounding implies."""
    A, b, X = _problem(M, D, N, seed=M)
    f = _eval(P, A, b, X, P.CUPSO_LSQ_BF16).astype(np.float64)
    Ab, Xb = _round_bf16(A), _round_bf16(X)
    Rb = Xb @ Ab.T - b.astype(np.float64)[None, :]
    f_rounded = np.sum(Rb * Rb, axis=1)
    np.testing.assert_allclose(f, f_rounded, rtol=2e-5, atol=1e-6)
    R = X.astype(np.float64) @ A.astype(np.float64).T - b.astype(np.float64)[None, :]
    f64 = np.sum(R * R, axis=1)
    dR = np.abs(Xb @ Ab.T - X.astype(np.float64) @ A.astype(np.float64).T)
    bound = np.sum(2 * np.abs(R) * dR + dR * dR, axis=1) * 1.01 + 1e-5 * f64
    assert np.all(np.abs(f - f64) <= bound)
    assert np.median(np.abs(f - f64) / f64) < 5e-3


@pytest.mark.parametrize("M,D,N", [(256, 128, 128), (700, 300, 1000), (1300, 96, 1100)])
def test_lsq_fp8_tensor_cores(P, M, D, N):
    A, b, X = _problem(M, D, N, seed=M + 1)
    f = _eval(P, A, b, X, P.CUPSO_LSQ_FP8).astype(np.float64)
    R = X.astype(np.float64) @ A.astype(np.float64).T - b.astype(np.float64)[None, :]
    f64 = np.sum(R * R, axis=1)
    # e4m3 keeps 3 mantissa bits: relative rounding 2^-4 per operand (scaled to use the range)
    dR = np.abs(X.astype(np.float64)) @ np.abs(A.astype(np.float64)).T * (2 * 2.0 ** -4 + 2.0 ** -8)
    bound = np.sum(2 * np.abs(R) * dR + dR * dR, axis=1) + 1e-5 * f64
    assert np.all(np.abs(f - f64) <= bound)
    assert np.median(np.abs(f - f64) / f64) < 5e-2


# --------------------------------------------------------------------------- #
# Swarms with the least-squares fitness                                        #
# --------------------------------------------------------------------------- #

LSQ_BOUNDS = (-2.0, 2.0, 0.4)
W, C12 = 0.729, 1.49445


def _lsq_swarm(P, A, b, N, seed, precision):
    import torch
    dA = torch.from_numpy(A).cuda()
    db = torch.from_numpy(b).cuda()
    s = P.Swarm(A.shape[1], N, LSQ_BOUNDS, W, C12, C12, P.CUPSO_LSQ, seed)
    s.set_lsq(dA.data_ptr(), db.data_ptr(), A.shape[0], precision)
    s._keep = (dA, db)        # the library borrows A and b
    return s


def test_lsq_swarm_needs_set_lsq(P):
    with P.Swarm(8, 100, LSQ_BOUNDS, W, C12, C12, P.CUPSO_LSQ, 1) as s:
        with pytest.raises(P.CupsoError):
            s.step(1)


@pytest.mark.parametrize("N,D,M", [(300, 24, 100), (1100, 9, 40)])
def test_lsq_fp32_swarm_bit_exact(P, N, D, M):
    from tests.gpu_common import assert_state_equal, same_bits
    A, b, _ = _problem(M, D, 1, seed=N)
    with _lsq_swarm(P, A, b, N, 3, "fp32") as s:
        st0 = s.state()
        s.step(1)
        s.step(17)        # a captured graph of 16 + 1
        st = s.state()
        _, fit, idx, pos = s.gbest()
        g64 = s.gbest_f64()
    ref = O.Swarm(N, D, *LSQ_BOUNDS, W, C12, C12, O.LSQ, 3, lsq=(A, b)).init()
    np.testing.assert_array_equal(st0["pbest_fit"], ref.pbest_fit)
    ref.step_sync(18)
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and same_bits(pos, ref.gbest_pos)
    assert abs(g64 - O.lsq_f64(A, b, pos)) <= 1e-12 * g64


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("N,D,M", [(2000, 96, 640), (1000, 200, 120)])
def test_lsq_approx_swarm_gbest_is_fp64_verified(P, precision, N, D, M):
    """pbest follows the approximate fitness; gbest only moves to FP64-verified
    improvements: its FP64 fitness never increases and equals ||A g - b||^2.
    D <= M rescores in the Gram form (A^T A), D > M row by row."""
    A, b, _ = _problem(M, D, 1, seed=11)
    with _lsq_swarm(P, A, b, N, 5, precision) as s:
        prev64 = s.gbest_f64()
        prev = s.state()
        for _ in range(6):
            s.step(3)
            rc, fit, idx, pos = s.gbest()
            g64 = s.gbest_f64()
            st = s.state()
            assert rc == P.CUPSO_OK
            assert g64 <= prev64
            exact = float(np.sum((A.astype(np.float64) @ pos.astype(np.float64) - b.astype(np.float64)) ** 2))
            assert abs(g64 - exact) <= 1e-9 * exact
            assert np.float32(g64) == fit
            np.testing.assert_array_equal(st["pbest_pos"][idx], pos)
            assert np.all(st["pbest_fit"] <= prev["pbest_fit"])
            assert np.all(np.abs(st["v"]) <= np.float32(0.4))
            prev64, prev = g64, st


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_lsq_swarm_operand_matches_standalone_eval(P, precision):
    """The swarm's move kernel writes the tensor-core operand itself; the fitness
    that follows must be what cupso_lsq_eval computes from the same positions:
    every particle whose pbest improved in a step holds exactly that value.
    D = 200 leaves a ragged last dimension tile, N = 1500 a ragged particle block."""
    N, D, M = 1500, 200, 300
    A, b, _ = _problem(M, D, 1, seed=5)
    with _lsq_swarm(P, A, b, N, 7, precision) as s:
        s.step(2)
        before = s.state()
        s.step(1)
        st = s.state()
    improved = st["pbest_fit"] < before["pbest_fit"]
    assert improved.sum() > 10
    X = st["pos"]
    if precision == "fp8":
        # cupso_lsq_eval scales X by 448 / max|X|; a row at the bound gives the swarm's scale, 448 / 2
        X = np.vstack([X, np.full((1, D), 2.0, np.float32)])
    f = _eval(P, A, b, X, P.CUPSO_LSQ_BF16 if precision == "bf16" else P.CUPSO_LSQ_FP8)[:N]
    np.testing.assert_array_equal(st["pbest_fit"][improved].view(np.uint32), f[improved].view(np.uint32))


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_lsq_swarm_lazy_pbest_consistent(P, precision):
    """The tensor-core iteration leaves improved particles' pbest rows to be
    written back by the next move (or before the state is read). With state
    reads in the middle of the run, every particle's pbest_fit must still be
    the approximate fitness of its pbest_pos, bit for bit."""
    N, D, M = 700, 72, 200
    A, b, _ = _problem(M, D, 1, seed=9)
    with _lsq_swarm(P, A, b, N, 3, precision) as s:
        s.step(3)
        s.state()            # writes the pending rows back in the middle of the run
        s.step(20)           # a captured graph of 16, then single launches
        st = s.state()
    X = st["pbest_pos"]
    if precision == "fp8":
        X = np.vstack([X, np.full((1, D), 2.0, np.float32)])   # the swarm's FP8 scale, 448 / 2
    f = _eval(P, A, b, X, P.CUPSO_LSQ_BF16 if precision == "bf16" else P.CUPSO_LSQ_FP8)[:N]
    np.testing.assert_array_equal(st["pbest_fit"].view(np.uint32), f.view(np.uint32))
