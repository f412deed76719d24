"""Least-squares fitness ||A x - b||^2 on the GPU against the oracle.

- Plain FP32 and FP64 fitness: bit for bit (ora_lsq_f32, ora_lsq_f64).
- BF16 / FP8 tensor-core fitness: against the oracle's value of the same
  rounded operands (ora_lsq_disp, FP64) up to the FP32 accumulation, and
  against the FP64 fitness (ora_lsq_f64) within the operand-rounding bound.
- Swarms: the FP32 and FP64 trajectories bit-exact with the oracle's; the
  tensor-core swarms' fitness is the displacement form around gbest; their
  gbest is accepted only on FP64-verified values, per iteration the best of the
  rescored candidates and within 1e-3 of the FP64 best of all improvers; in a
  converging regime their final residual is within 1e-3 of the FP64-fitness
  run and of the closed-form least-squares minimum.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_common import load_cupso

pytestmark = pytest.mark.gpu

# relative tolerance of a tensor-core fitness against the oracle's FP64 value of
# the same rounded operands: the FP32 accumulation of up to 4096 x 1024 products
RTOL_ACC = {"bf16": 2e-5, "fp8": 1e-4}


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


def _rounding_bound(A, b, X, G, unit):
    """|f~ - f| bound when every operand of A (X - G) carries a relative rounding
    of at most `unit` (and the offsets one binary32 rounding): per row the
    residual moves by at most dR, so the square by 2 |R| dR + dR^2."""
    A64 = A.astype(np.float64)
    R = X.astype(np.float64) @ A64.T - b.astype(np.float64)[None, :]
    dR = np.abs(X.astype(np.float64) - G.astype(np.float64)) @ np.abs(A64).T * (2 * unit + unit * unit) \
        + (np.abs(G.astype(np.float64)) @ np.abs(A64).T + np.abs(b)) * 2.0 ** -24 + 1e-12
    return np.sum(2 * np.abs(R) * dR + dR * dR, axis=1)


@pytest.mark.parametrize("M,D,N", [(40, 7, 30), (300, 65, 257), (513, 130, 129)])
def test_lsq_fp32_bit_exact(P, M, D, N):
    A, b, X = _problem(M, D, N)
    f = _eval(P, A, b, X, P.CUPSO_LSQ_FP32)
    ref = np.array([O.lsq_f32(A, b, X[i]) for i in range(N)], np.float32)
    np.testing.assert_array_equal(f.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("M,D,N", [(40, 7, 30), (300, 65, 257), (513, 130, 129), (33, 1, 70)])
def test_lsq_fp64_bit_exact(P, M, D, N):
    A, b, X = _problem(M, D, N, seed=D)
    f = _eval(P, A, b, X, P.CUPSO_LSQ_FP64)
    ref = np.array([np.float32(O.lsq_f64(A, b, X[i])) for i in range(N)], np.float32)
    np.testing.assert_array_equal(f.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
@pytest.mark.parametrize("M,D,N", [(256, 64, 128), (700, 200, 1000), (4096, 1024, 96), (1300, 96, 1100)])
def test_lsq_tensor_cores_standalone(P, fmt, M, D, N):
    """cupso_lsq_eval on the positions themselves (reference point 0): equal to the
    oracle's FP64 value of the same rounded operands up to the FP32 accumulation,
    and within the operand-rounding bound of the FP64 fitness."""
    A, b, X = _problem(M, D, N, seed=M + (fmt == "fp8"))
    prec = P.CUPSO_LSQ_BF16 if fmt == "bf16" else P.CUPSO_LSQ_FP8
    f = _eval(P, A, b, X, prec).astype(np.float64)
    sx = np.float32(448.0) / np.float32(np.abs(X).max())      # the standalone FP8 scale of X
    zero = np.zeros(D, np.float32)
    f_disp = np.array([O.lsq_disp(A, b, X[i], zero, fmt, sx) for i in range(N)])
    np.testing.assert_allclose(f, f_disp, rtol=RTOL_ACC[fmt], atol=1e-7)
    f64 = np.array([O.lsq_f64(A, b, X[i]) for i in range(N)])
    unit = 2.0 ** -8 if fmt == "bf16" else 2.0 ** -3
    bound = _rounding_bound(A, b, X, np.zeros_like(X), unit) * 1.01 + RTOL_ACC[fmt] * f64
    assert np.all(np.abs(f - f64) <= bound)


# --------------------------------------------------------------------------- #
# Swarms with the least-squares fitness                                        #
# --------------------------------------------------------------------------- #

LSQ_BOUNDS = (-2.0, 2.0, 0.4)
W, C12 = 0.729, 1.49445
SX = np.float32(448.0) / np.float32(4.0)        # FP8 scale of a displacement within [-2, 2]


RESCORE = {"ff": 0, "fp64": 1}      # CUPSO_OPT_LSQ_RESCORE: float-float or FP64 Gram form


def _lsq_swarm(P, A, b, N, seed, precision, rescore="ff"):
    import torch
    dA = torch.from_numpy(A).cuda()
    db = torch.from_numpy(b).cuda()
    s = P.Swarm(A.shape[1], N, LSQ_BOUNDS, W, C12, C12, P.CUPSO_LSQ, seed)
    s.set_option(P.CUPSO_OPT_LSQ_RESCORE, RESCORE[rescore])
    s.set_lsq(dA.data_ptr(), db.data_ptr(), A.shape[0], precision)
    s._keep = (dA, db)        # the library borrows A and b
    return s


def test_lsq_swarm_needs_set_lsq(P):
    with P.Swarm(8, 100, LSQ_BOUNDS, W, C12, C12, P.CUPSO_LSQ, 1) as s:
        with pytest.raises(P.CupsoError):
            s.step(1)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("N,D,M", [(300, 24, 100), (1100, 9, 40)])
def test_lsq_exact_swarm_bit_exact(P, precision, N, D, M):
    """FP32 fitness (ora_lsq_f32) and FP64 fitness rounded to float (the oracle's
    FP64-fitness swarm): whole trajectories bit for bit, with a captured graph."""
    from tests.gpu_common import assert_state_equal, same_bits
    A, b, _ = _problem(M, D, 1, seed=N)
    with _lsq_swarm(P, A, b, N, 3, precision) as s:
        st0 = s.state()
        s.step(1)
        s.step(17)        # a captured graph of 16 + 1
        st = s.state()
        _, fit, idx, pos = s.gbest()
        g64 = s.gbest_f64()
    ref = O.Swarm(N, D, *LSQ_BOUNDS, W, C12, C12, O.LSQ, 3, lsq=(A, b), lsq_fp64=precision == "fp64").init()
    np.testing.assert_array_equal(st0["pbest_fit"], ref.pbest_fit)
    ref.step_sync(18)
    assert_state_equal(st, ref)
    assert idx == ref.gbest_idx and same_bits(fit, ref.gbest_fit) and same_bits(pos, ref.gbest_pos)
    assert abs(g64 - O.lsq_f64(A, b, pos)) <= 1e-12 * g64


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("N,D,M,rescore", [(2000, 96, 640, "ff"), (2000, 96, 640, "fp64"), (1000, 200, 120, "ff"),
                                           (300, 1600, 1664, "ff"), (300, 1600, 1664, "fp64")])
def test_lsq_approx_swarm_gbest_is_fp64_verified(P, precision, N, D, M, rescore):
    """pbest follows the approximate fitness; gbest only moves to verified
    improvements: its rescored fitness never increases and equals the oracle's
    FP64 ||A g - b||^2. D <= M rescores in the Gram form (A^T A; float-float or
    FP64 arithmetic), D > M row by row in FP64; D = 1600 holds 50 KB of
    candidates in shared memory in the FP64 Gram kernel, past the default 48 KB
    limit, and leaves a ragged last tile of 64 in the float-float one."""
    A, b, _ = _problem(M, D, 1, seed=11)
    with _lsq_swarm(P, A, b, N, 5, precision, rescore) as s:
        prev64 = s.gbest_f64()
        prev = s.state()
        for _ in range(6):
            s.step(3)
            rc, fit, idx, pos = s.gbest()
            g64 = s.gbest_f64()
            st = s.state()
            assert rc == P.CUPSO_OK
            assert g64 <= prev64
            exact = O.lsq_f64(A, b, pos)
            assert abs(g64 - exact) <= 1e-9 * exact
            assert np.float32(g64) == fit
            np.testing.assert_array_equal(st["pbest_pos"][idx], pos)
            assert np.all(st["pbest_fit"] <= prev["pbest_fit"])
            assert np.all(np.abs(st["v"]) <= np.float32(0.4))
            prev64, prev = g64, st


def _check_improvers_displacement(A, b, before, g, st, fmt, sample=None):
    """Every particle whose pbest improved in the step from `before` to `st` holds
    the approximate fitness of its new position around the step's reference
    point g (the gbest it moved towards): the oracle's displacement form, up to
    the FP32 accumulation; and within the rounding bound of the FP64 fitness."""
    improved = np.nonzero(st["pbest_fit"] < before["pbest_fit"])[0]
    assert improved.size > 0
    if sample is not None and improved.size > sample:
        improved = np.random.default_rng(0).choice(improved, sample, replace=False)
    X = st["pos"][improved]
    np.testing.assert_array_equal(st["pbest_pos"][improved], X)
    got = st["pbest_fit"][improved].astype(np.float64)
    ref = np.array([O.lsq_disp(A, b, x, g, fmt, SX) for x in X])
    np.testing.assert_allclose(got, ref, rtol=RTOL_ACC[fmt], atol=1e-7)
    f64 = np.array([O.lsq_f64(A, b, x) for x in X])
    unit = 2.0 ** -8 if fmt == "bf16" else 2.0 ** -3
    bound = _rounding_bound(A, b, X, np.broadcast_to(g, X.shape), unit) * 1.01 + RTOL_ACC[fmt] * f64
    assert np.all(np.abs(got - f64) <= bound)
    return improved.size


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_lsq_swarm_fitness_is_the_displacement_form(P, precision):
    """The move kernel writes each particle's displacement from gbest as the
    tensor-core operand and the product adds the offsets A g - b: the fitness of
    every improver equals the oracle's displacement form. D = 200 leaves a
    ragged last dimension tile, N = 1500 a ragged particle block."""
    N, D, M = 1500, 200, 300
    A, b, _ = _problem(M, D, 1, seed=5)
    with _lsq_swarm(P, A, b, N, 7, precision) as s:
        s.step(2)
        before = s.state()
        g = s.gbest()[3]
        s.step(1)
        st = s.state()
    assert _check_improvers_displacement(A, b, before, g, st, precision) > 10


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_lsq_swarm_lazy_pbest_consistent(P, precision):
    """The tensor-core iteration leaves improved particles' pbest rows to be
    written back by the next move (or before the state is read). Writing them
    back at other times must not change the trajectory: a swarm whose state is
    read after every iteration (so no row stays pending) and one run in a
    captured graph with a state read in the middle end bit for bit equal."""
    from tests.gpu_common import same_bits
    N, D, M = 700, 72, 200
    A, b, _ = _problem(M, D, 1, seed=9)
    with _lsq_swarm(P, A, b, N, 3, precision) as s:
        s.step(3)
        s.state()            # writes the pending rows back in the middle of the run
        s.step(20)           # a captured graph of 16, then single launches
        lazy = s.state()
        g_lazy = s.gbest()
    with _lsq_swarm(P, A, b, N, 3, precision) as s:
        for _ in range(22):
            s.step(1)
            s.state()
        before = s.state()
        g = s.gbest()[3]
        s.step(1)
        eager = s.state()
        g_eager = s.gbest()
    for k in ("pos", "v", "pbest_pos", "pbest_fit"):
        assert same_bits(lazy[k], eager[k]), k
    assert g_lazy[2] == g_eager[2] and same_bits(g_lazy[3], g_eager[3])
    _check_improvers_displacement(A, b, before, g, eager, precision)


@pytest.mark.parametrize("precision,rescore,N,D,M,iters", [("bf16", "ff", 600, 48, 200, 30), ("fp8", "ff", 600, 48, 200, 30),
                                                            ("bf16", "fp64", 600, 48, 200, 30),
                                                            ("bf16", "ff", 12000, 64, 256, 8)])
def test_lsq_acceptance_per_iteration(P, precision, rescore, N, D, M, iters):
    """Each iteration, against the oracle's FP64 fitness of every improver: the
    16 improvers with the lowest approximate keys are the rescored candidates;
    gbest's new FP64 value is the lowest of theirs when that beats the old one
    (else unchanged), and it is within 1e-3 relative of the FP64 best over all
    improvers and the old gbest. How often the true FP64 best lies outside the
    16 is counted and reported. N = 12000 makes 376 candidate lists of 32
    particles, more than one warp merges: the selection over all their keys."""
    A, b, _ = _problem(M, D, 1, seed=17)
    misses = checked = 0
    worst = 0.0
    with _lsq_swarm(P, A, b, N, 11, precision, rescore) as s:
        prev = s.state()
        g64_prev = s.gbest_f64()
        for _ in range(iters):
            s.step(1)
            st = s.state()
            g64 = s.gbest_f64()
            _, fit, idx, pos = s.gbest()
            imp = np.nonzero(st["pbest_fit"] < prev["pbest_fit"])[0]
            if imp.size:
                f_imp = np.array([O.lsq_f64(A, b, st["pos"][i]) for i in imp])
                keys = [(O.fit_key(st["pbest_fit"][i]), i) for i in imp]
                order = sorted(range(imp.size), key=lambda k: keys[k])[:16]
                top_f = f_imp[order]
                best_top = float(top_f.min())
                if best_top < g64_prev:
                    assert abs(g64 - best_top) <= 1e-9 * best_top
                    assert idx == imp[order[int(np.argmin(top_f))]]
                else:
                    assert g64 == g64_prev
                true_best = min(float(f_imp.min()), g64_prev)
                assert g64 <= true_best * (1 + 1e-3), (g64, true_best)
                worst = max(worst, g64 / true_best - 1.0)
                misses += int(f_imp.min() < best_top)
                checked += 1
            else:
                assert g64 == g64_prev
            assert abs(g64 - O.lsq_f64(A, b, pos)) <= 1e-9 * g64
            prev, g64_prev = st, g64
    assert checked >= (2 * iters) // 3
    print("\n%s: %d iterations checked, true FP64 best outside the 16 candidates in %d, worst gap %.2e"
          % (precision, checked, misses, worst))


@pytest.mark.parametrize("N,D,M,iters", [(2000, 96, 640, 40), (1500, 200, 300, 30), (1024, 1024, 4096, 12)])
def test_lsq_rescore_ff_matches_fp64(P, N, D, M, iters):
    """The float-float rescoring against the FP64 one on the same swarm: every
    iteration both accept the same particle (so the trajectories stay equal
    bit for bit), their values agree to 1e-12 relative, and both equal the
    oracle's FP64 residual sum of gbest_pos to 1e-11 relative. D = 200 leaves a
    ragged last tile (zero-padded Gram pairs); D = 1024 is 136 tiles."""
    from tests.gpu_common import same_bits
    A, b, _ = _problem(M, D, 1, seed=D + 3)
    with _lsq_swarm(P, A, b, N, 13, "bf16", "ff") as s1, _lsq_swarm(P, A, b, N, 13, "bf16", "fp64") as s2:
        moved = 0
        g_prev = s1.gbest_f64()
        assert abs(g_prev - s2.gbest_f64()) <= 1e-12 * g_prev
        for _ in range(iters):
            s1.step(1)
            s2.step(1)
            _, fit1, idx1, pos1 = s1.gbest()
            _, fit2, idx2, pos2 = s2.gbest()
            g1, g2 = s1.gbest_f64(), s2.gbest_f64()
            assert idx1 == idx2 and same_bits(pos1, pos2)
            assert abs(g1 - g2) <= 1e-12 * g2, (g1, g2)
            exact = O.lsq_f64(A, b, pos1)
            assert abs(g1 - exact) <= 1e-11 * exact and abs(g2 - exact) <= 1e-11 * exact
            moved += int(g1 < g_prev)
            g_prev = g1
        st1, st2 = s1.state(), s2.state()
    for k in ("pos", "v", "pbest_pos", "pbest_fit"):
        assert same_bits(st1[k], st2[k]), k
    assert moved >= 3


def _converging_problem(M, D, seed):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((M, D)) / np.sqrt(M)).astype(np.float32)
    xs = rng.uniform(-1, 1, D).astype(np.float32)
    b = (A.astype(np.float64) @ xs + 1e-3 * rng.standard_normal(M)).astype(np.float32)
    x64, res, _, _ = np.linalg.lstsq(A.astype(np.float64), b.astype(np.float64), rcond=None)
    return A, b, float(O.lsq_f64(A, b, x64.astype(np.float32)))


@pytest.mark.parametrize("seed", [1, 2])
def test_lsq_converging_regime(P, seed):
    """A problem PSO solves (N = 1024, D = 64, M = 512, 800 iterations): the
    FP64-fitness run (bit-exact with the oracle's FP64-fitness swarm on small
    cases) reaches the least-squares minimum to 1e-6; the BF16 and FP8 runs'
    final FP64 residuals are within 1e-3 relative of both that run's and the
    minimum. The FP32 run is reported beside them."""
    N, D, M, T = 1024, 64, 512, 800
    A, b, fmin = _converging_problem(M, D, seed)
    final = {}
    for prec in ("fp64", "bf16", "fp8", "fp32"):
        with _lsq_swarm(P, A, b, N, seed, prec) as s:
            s.step(T)
            final[prec] = s.gbest_f64()
    rel = {k: (v - fmin) / fmin for k, v in final.items()}
    print("\nseed %d, lstsq minimum %.6e: relative excess %s" % (seed, fmin, {k: "%.2e" % v for k, v in rel.items()}))
    assert -1e-9 <= rel["fp64"] <= 1e-6
    for prec in ("bf16", "fp8"):
        assert rel[prec] <= 1e-3, prec
        assert abs(final[prec] - final["fp64"]) <= 1e-3 * final["fp64"], prec


def test_lsq_rescore_option_switch(P):
    """CUPSO_OPT_LSQ_RESCORE takes 0 or 1 (anything else is refused), before or
    after cupso_set_lsq; switched between iterations (the captured graphs are
    rebuilt), every accepted gbest still equals the oracle's FP64 residual sum
    of gbest_pos, and the trajectory equals a swarm that rescored in FP64 all
    along (both rescorings accept the same particles here)."""
    from tests.gpu_common import same_bits
    N, D, M = 1500, 96, 400
    A, b, _ = _problem(M, D, 1, seed=31)
    with _lsq_swarm(P, A, b, N, 9, "bf16", "ff") as s1, _lsq_swarm(P, A, b, N, 9, "bf16", "fp64") as s2:
        for bad in (2, -1):
            with pytest.raises(P.CupsoError):
                s1.set_option(P.CUPSO_OPT_LSQ_RESCORE, bad)
        for k in range(4):
            s1.set_option(P.CUPSO_OPT_LSQ_RESCORE, k & 1)
            s1.step(17)           # a captured graph of 16 and one more
            s2.step(17)
            _, fit, idx, pos = s1.gbest()
            g64 = s1.gbest_f64()
            exact = O.lsq_f64(A, b, pos)
            assert abs(g64 - exact) <= 1e-9 * exact
        st1, st2 = s1.state(), s2.state()
    for key in ("pos", "v", "pbest_pos", "pbest_fit"):
        assert same_bits(st1[key], st2[key]), key
