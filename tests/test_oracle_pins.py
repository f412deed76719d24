"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test fixes one part of the oracle to something the paper, a published
definition or plain mathematics determines: published Philox known answers,
exact polynomial coefficients, known optima, FP64 textbook formulas, a swarm
stepped by hand (Eq. 1, Eq. 2, Alg. 1), closed forms and invariants.
"""
import math

import mpmath
import numpy as np
import pytest

from oracle import oracle as O
from tests import golden_io

F32 = np.float32


# --------------------------------------------------------------------------- #
# Philox4x32-10 and the uniform mapping (Sec. 4.4: r1, r2 uniform)             #
# --------------------------------------------------------------------------- #

def test_philox_known_answers():
    kat = golden_io.philox_kat()
    assert len(kat) == 3
    for ctr, key, expect in kat:
        assert O.philox4x32_10(ctr, key) == expect


def test_u01_closed_form():
    assert O.u01(0) == F32(2.0 ** -24)
    assert O.u01(0xFF) == F32(2.0 ** -24)          # low 8 bits are dropped
    assert O.u01(0x100) == F32(2.0 ** -23)
    assert O.u01(0xFFFFFFFF) == F32(1.0)           # (0, 1]: 1 is reachable, 0 is not
    rng = np.random.default_rng(5)
    for w in rng.integers(0, 2 ** 32, 200, dtype=np.uint64):
        assert O.u01(int(w)) == F32(((int(w) >> 8) + 1) * 2.0 ** -24)


def test_draw_word_mapping():
    """r1, r2 of (t, i, d) are words 2*(d&1) and 2*(d&1)+1 of Philox((d>>1, i, t, swarm), seed)."""
    seed = 0x0123456789ABCDEF
    s = O.Swarm(7, 5, -1, 1, 0.5, 0.7, 1.5, 1.5, O.SPHERE, seed, swarm=3)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for (t, i, d) in [(0, 0, 0), (1, 6, 4), (17, 3, 1), (2 ** 31 + 5, 2, 3)]:
        words = O.philox4x32_10([d >> 1, i, t, 3], key)
        r1, r2 = s.draw_r(t, i, d)
        assert r1 == O.u01(words[2 * (d & 1)])
        assert r2 == O.u01(words[2 * (d & 1) + 1])


def test_uniform_chi_square():
    key = [1, 0]
    counts = np.zeros(64, np.int64)
    for c in range(4096):
        for w in O.philox4x32_10([c, 7, 1, 0], key):
            counts[min(int(float(O.u01(w)) * 64), 63)] += 1
    n = counts.sum()
    chi2 = float(((counts - n / 64) ** 2 / (n / 64)).sum())
    assert chi2 < 120.0          # 63 degrees of freedom; p ~ 1e-5 bound


# --------------------------------------------------------------------------- #
# Own cos(2 pi x) and exp(y)                                                   #
# --------------------------------------------------------------------------- #

def _is_nearest_f32(val_f32, exact):
    """val_f32 is a float32 nearest to the mpmath number `exact`."""
    v = F32(val_f32)
    up = np.nextafter(v, F32(np.inf), dtype=np.float32)
    dn = np.nextafter(v, F32(-np.inf), dtype=np.float32)
    e = abs(mpmath.mpf(float(v)) - exact)
    return e <= abs(mpmath.mpf(float(up)) - exact) and e <= abs(mpmath.mpf(float(dn)) - exact)


def test_cos2pi_coefficients_are_rounded_taylor():
    mpmath.mp.dps = 50
    c = O.cos2pi_coeffs()
    for j in range(8):
        exact = (-1) ** j * (2 * mpmath.pi) ** (2 * j) / mpmath.factorial(2 * j)
        assert _is_nearest_f32(c[j], exact), j


def test_exp_constants():
    mpmath.mp.dps = 50
    c, log2e, hi, lo = O.exp_coeffs()
    for k in range(9):
        assert _is_nearest_f32(c[k], 1 / mpmath.factorial(k)), k
    assert _is_nearest_f32(log2e, 1 / mpmath.log(2))
    # ln2_hi carries at most 16 significant bits, so n * ln2_hi is exact for |n| < 256.
    m, e = math.frexp(float(hi))
    assert (m * 2 ** 16).is_integer()
    assert _is_nearest_f32(lo, mpmath.log(2) - mpmath.mpf(float(hi)))
    assert abs(mpmath.mpf(float(hi)) + mpmath.mpf(float(lo)) - mpmath.log(2)) < 2 ** -40


def test_cos2pi_special_points_exact():
    for k in range(-20, 21):
        assert O.cos2pi(k) == 1.0
        assert O.cos2pi(k + 0.5) == -1.0
        assert O.cos2pi(k + 0.25) == 0.0
        assert O.cos2pi(k - 0.25) == 0.0
    assert O.cos2pi(2.0 ** 23 + 1) == 1.0
    assert O.cos2pi(-0.0) == 1.0


def test_cos2pi_accuracy_vs_fp64():
    mpmath.mp.dps = 30
    rng = np.random.default_rng(11)
    xs = rng.uniform(-33, 33, 3000).astype(np.float32)
    worst = 0.0
    for x in xs:
        exact = float(mpmath.cos(2 * mpmath.pi * mpmath.mpf(float(x))))
        worst = max(worst, abs(float(O.cos2pi(x)) - exact))
    assert worst < 2.5e-7, worst


def test_exp_accuracy_vs_fp64():
    rng = np.random.default_rng(12)
    ys = np.concatenate([rng.uniform(-12, 3, 3000), rng.uniform(-100, 80, 300)]).astype(np.float32)
    for y in ys:
        exact = math.exp(float(y))
        got = float(O.exp(y))
        # 3e-7 relative in the normal range; one subnormal unit below 2^-126
        assert abs(got - exact) <= max(3e-7 * exact, 2.0 ** -149), (y, got, exact)
    assert O.exp(0.0) == 1.0 and O.exp(-0.0) == 1.0
    assert O.exp(200.0) == np.inf and O.exp(-200.0) == 0.0


# --------------------------------------------------------------------------- #
# Fitness functions (Step 3): optima and FP64 textbook formulas                #
# --------------------------------------------------------------------------- #

def _fp64(fid, x):
    x = np.asarray(x, np.float64)
    D = x.size
    if fid == O.SPHERE:
        return float(np.sum(x * x))
    if fid == O.RASTRIGIN:
        return float(10 * D + np.sum(x * x - 10 * np.cos(2 * np.pi * x)))
    if fid == O.ACKLEY:
        return float(-20 * np.exp(-0.2 * np.sqrt(np.mean(x * x))) - np.exp(np.mean(np.cos(2 * np.pi * x)))
                     + 20 + np.e)
    if fid == O.ROSENBROCK:
        return float(np.sum(100 * (x[1:] - x[:-1] ** 2) ** 2 + (1 - x[:-1]) ** 2))
    if fid == O.CUBIC_MAX:   # Eq. 3, maximised -> minimise the negation
        return float(-np.sum(x ** 3 - 0.8 * x ** 2 - 1000 * x + 8000))
    raise ValueError(fid)


@pytest.mark.parametrize("D", [1, 2, 7, 32, 128])
def test_known_optima_exact(D):
    assert O.fitness(O.SPHERE, np.zeros(D)) == 0.0
    assert O.fitness(O.RASTRIGIN, np.zeros(D)) == 0.0
    assert O.fitness(O.ACKLEY, np.zeros(D)) == 0.0
    assert O.fitness(O.ROSENBROCK, np.ones(D)) == 0.0


def test_cubic_boundary_optimum():
    # Eq. 3 on [-100, 100]: f'(x) = 3x^2 - 1.6x - 1000 has roots near 18.526 and -17.993;
    # the maximum over the box is at x = 100, f = 900000 per dimension.
    for D in (1, 3, 120):
        got = O.fitness(O.CUBIC_MAX, np.full(D, 100.0))
        assert abs(float(got) + 900000.0 * D) <= 1e-6 * 900000.0 * D
    grid = np.linspace(-100, 100, 20001).astype(np.float32)
    vals = [float(O.fitness(O.CUBIC_MAX, np.array([g]))) for g in grid[::50]]
    assert min(vals) == float(O.fitness(O.CUBIC_MAX, np.array([100.0])))
    # interior local maximum of f at x ~ -17.993 (local minimum of -f), f ~ 19908.8
    xs = np.linspace(-19, -17, 2001).astype(np.float32)
    vals = np.array([float(O.fitness(O.CUBIC_MAX, np.array([x]))) for x in xs])
    # f'' = -109.6 there, so f moves by < 1 float32 ulp (0.002) within 0.006 of the peak
    assert abs(float(xs[np.argmin(vals)]) + 17.993) < 1e-2
    assert abs(-vals.min() - 19908.8) < 0.5


@pytest.mark.parametrize("fid,lo,hi", [(O.SPHERE, -100, 100), (O.RASTRIGIN, -5.12, 5.12),
                                       (O.ACKLEY, -32.768, 32.768), (O.ROSENBROCK, -30, 30),
                                       (O.CUBIC_MAX, -100, 100)])
@pytest.mark.parametrize("D", [2, 33, 128])
def test_fitness_vs_fp64(fid, lo, hi, D):
    rng = np.random.default_rng(fid * 1000 + D)
    for _ in range(40):
        x = rng.uniform(lo, hi, D).astype(np.float32)
        got = float(O.fitness(fid, x))
        ref = _fp64(fid, x)
        # relative to the sum of |terms| (the cubic's terms cancel; the others are >= 0)
        scale = abs(ref)
        if fid == O.CUBIC_MAX:
            x64 = x.astype(np.float64)
            scale = float(np.sum(np.abs(x64 ** 3 - 0.8 * x64 ** 2 - 1000 * x64 + 8000)))
        assert abs(got - ref) <= 1e-5 * scale + 1e-5, (fid, got, ref)


def test_fit_key_order():
    rng = np.random.default_rng(3)
    vals = list(rng.standard_normal(300).astype(np.float32) * F32(1e3))
    vals += [F32(0.0), F32(-0.0), F32(np.inf), F32(-np.inf), F32(1e-45), F32(-1e-45)]
    keyed = sorted(vals, key=O.fit_key)
    assert all(keyed[k] <= keyed[k + 1] for k in range(len(keyed) - 1))
    assert O.fit_key(-0.0) == O.fit_key(0.0)
    assert O.fit_key(np.nan) == 0xFFFFFFFF
    assert O.fit_key(np.inf) < O.fit_key(np.nan)


# --------------------------------------------------------------------------- #
# The whole step: hand-stepped swarm, closed forms, invariants                  #
# --------------------------------------------------------------------------- #

def _hand_swarm(g):
    p = g["param"]
    s = O.Swarm(4, 2, p["min_pos"], p["max_pos"], p["max_v"], p["w"], p["c1"], p["c2"], O.SPHERE, 1)
    s.set_state(g["init"]["pos"].reshape(4, 2), g["init"]["v"].reshape(4, 2),
                g["init"]["pbest_pos"].reshape(4, 2), g["init"]["pbest_fit"], 0)
    return s


def _check_against(s, ref):
    np.testing.assert_array_equal(s.pos.ravel(), ref["pos"])
    np.testing.assert_array_equal(s.v.ravel(), ref["v"])
    np.testing.assert_array_equal(s.pbest_pos.ravel(), ref["pbest_pos"])
    np.testing.assert_array_equal(s.pbest_fit, ref["pbest_fit"])
    assert s.gbest_idx == int(ref["gbest_idx"][0])
    assert s.gbest_fit == ref["gbest_fit"][0]
    np.testing.assert_array_equal(s.gbest_pos, ref["gbest_pos"])


def test_hand_step_sync():
    g = golden_io.hand_step()
    s = _hand_swarm(g)
    assert s.gbest_idx == 0 and s.gbest_fit == F32(1.25)
    s.step_sync(1, g["r"][1])
    _check_against(s, g["sync1"])
    s.step_sync(1, g["r"][2])
    _check_against(s, g["sync2"])
    assert s.t == 2


def test_hand_step_two_iterations_at_once():
    g = golden_io.hand_step()
    s = _hand_swarm(g)
    s.step_sync(2, np.concatenate([g["r"][1], g["r"][2]]))
    _check_against(s, g["sync2"])


def test_hand_step_serial_differs():
    g = golden_io.hand_step()
    s = _hand_swarm(g)
    s.step_serial(1, g["r"][1])
    _check_against(s, g["serial1"])


def _swarm(N, D, fid, lo, hi, vmax, w=0.729, c1=1.49445, c2=1.49445, seed=1):
    return O.Swarm(N, D, lo, hi, vmax, w, c1, c2, fid, seed).init()


def test_init_closed_form():
    N, D, lo, hi, vmax = 37, 9, -5.12, 5.12, 1.024
    s = _swarm(N, D, O.RASTRIGIN, lo, hi, vmax)
    span = np.float64(F32(F32(hi) - F32(lo)))
    vspan = np.float64(F32(2) * F32(vmax))
    key = [1, 0]
    for i in range(N):
        for d in range(D):
            words = O.philox4x32_10([d >> 1, i, 0, 0], key)
            ux, uv = O.u01(words[2 * (d & 1)]), O.u01(words[2 * (d & 1) + 1])
            # u * span + lo is exact in float64 here; one rounding to float32 = fmaf
            assert s.pos[i, d] == F32(np.float64(ux) * span + np.float64(F32(lo)))
            assert s.v[i, d] == F32(np.float64(uv) * vspan - np.float64(F32(vmax)))
    assert np.all((s.pos > F32(lo)) & (s.pos <= F32(hi)))
    assert np.all((s.v > -F32(vmax)) & (s.v <= F32(vmax)))
    np.testing.assert_array_equal(s.pbest_pos, s.pos)
    for i in range(N):
        assert s.pbest_fit[i] == O.fitness(O.RASTRIGIN, s.pos[i])
    g = int(np.lexsort((np.arange(N), s.pbest_fit))[0])
    assert s.gbest_idx == g


def test_r_override_equals_philox_draws():
    N, D, T = 11, 5, 3
    a = _swarm(N, D, O.ROSENBROCK, -30, 30, 6)
    b = _swarm(N, D, O.ROSENBROCK, -30, 30, 6)
    r = np.zeros((T, N, D, 2), np.float32)
    for k in range(T):
        for i in range(N):
            for d in range(D):
                r[k, i, d] = a.draw_r(k + 1, i, d)
    a.step_sync(T)
    b.step_sync(T, r)
    np.testing.assert_array_equal(a.pos, b.pos)
    np.testing.assert_array_equal(a.pbest_pos, b.pbest_pos)
    assert a.gbest_idx == b.gbest_idx


def test_inertia_only_closed_form():
    """c1 = c2 = 0, w = 1/2: v_t = v_0 / 2^t exactly; pos_t = clip(pos_0 + v_0 (1 - 2^-t)).

    v keeps its sign, so a particle that reaches a wall stays clamped there."""
    N, D, T = 6, 4, 12
    s = O.Swarm(N, D, -1000, 1000, 20, 0.5, 0.0, 0.0, O.SPHERE, 9).init()
    v0, x0 = s.v.astype(np.float64), s.pos.astype(np.float64)
    for t in range(1, T + 1):
        s.step_sync(1)
        np.testing.assert_array_equal(s.v, (v0 * 0.5 ** t).astype(np.float32))
        np.testing.assert_allclose(s.pos, np.clip(x0 + v0 * (1 - 0.5 ** t), -1000, 1000), rtol=0, atol=1e-4 * t)


def test_frozen_swarm():
    """w = c1 = c2 = 0: velocities vanish, positions and bests stay where they are."""
    s = O.Swarm(9, 3, -5, 5, 1, 0.0, 0.0, 0.0, O.ACKLEY, 4).init()
    x0, pf0, g0 = s.pos.copy(), s.pbest_fit.copy(), s.gbest_idx
    s.step_sync(5)
    assert np.all(s.v == 0)
    np.testing.assert_array_equal(s.pos, x0)
    np.testing.assert_array_equal(s.pbest_fit, pf0)
    assert s.gbest_idx == g0


def test_nan_is_clamped_to_lower_bound():
    """Clamp reading: a NaN velocity or position goes to the lower bound (IEEE maxNum)."""
    s = O.Swarm(3, 2, -4, 6, 2, 0.5, 1, 1, O.SPHERE, 1)
    pos = np.array([[np.nan, 1.0], [0.5, 0.5], [2.0, -1.0]], np.float32)
    pf = np.array([O.fitness(O.SPHERE, p) for p in pos], np.float32)
    s.set_state(pos, np.zeros_like(pos), pos, pf, 0)
    s.step_sync(1, np.full((1, 3, 2, 2), 0.5, np.float32))
    assert s.v[0, 0] == np.float32(-2.0)       # NaN velocity -> -max_v
    assert s.pos[0, 0] == np.float32(-4.0)     # NaN position -> min_pos
    assert np.all(np.isfinite(s.pos))


def test_gbest_ties_lowest_index():
    N, D = 6, 2
    s = O.Swarm(N, D, -10, 10, 1, 0.5, 1, 1, O.SPHERE, 1)
    pos = np.array([[3, 4], [0, 1], [1, 0], [-1, 0], [0, -1], [5, 5]], np.float32)
    s.set_state(pos, np.zeros_like(pos), pos, np.array([25, 1, 1, 1, 1, 50], np.float32), 0)
    assert s.gbest_idx == 1
    pf = np.array([np.nan, 2, -0.0, 0.0, 7, np.nan], np.float32)
    s.set_state(pos, np.zeros_like(pos), pos, pf, 0)
    assert s.gbest_idx == 2          # -0 and +0 tie; the lower index wins; NaN ranks last
    s.set_state(pos, np.zeros_like(pos), pos, np.full(N, np.nan, np.float32), 0)
    assert s.gbest_idx == 0


@pytest.mark.parametrize("fid,lo,hi,vmax", [(O.SPHERE, -100, 100, 20), (O.RASTRIGIN, -5.12, 5.12, 1.024),
                                            (O.ACKLEY, -32.768, 32.768, 6.5536),
                                            (O.ROSENBROCK, -30, 30, 6), (O.CUBIC_MAX, -100, 100, 20)])
def test_invariants(fid, lo, hi, vmax):
    N, D, T = 64, 6, 40
    s = _swarm(N, D, fid, lo, hi, vmax, seed=fid + 17)
    prev_pf, prev_g = s.pbest_fit.copy(), s.gbest_fit
    for _ in range(T):
        s.step_sync(1)
        assert np.all(np.abs(s.v) <= F32(vmax))
        assert np.all((s.pos >= F32(lo)) & (s.pos <= F32(hi)))
        assert np.all(s.pbest_fit <= prev_pf)
        assert s.gbest_fit <= prev_g
        g = int(np.lexsort((np.arange(N), s.pbest_fit))[0])
        assert s.gbest_idx == g and s.gbest_fit == s.pbest_fit[g]
        np.testing.assert_array_equal(s.gbest_pos, s.pbest_pos[g])
        prev_pf, prev_g = s.pbest_fit.copy(), s.gbest_fit
    for i in range(N):
        ref = _fp64(fid, s.pbest_pos[i])
        assert abs(float(s.pbest_fit[i]) - ref) <= 1e-5 * abs(ref) + 1e-4


def test_sphere_converges():
    s = _swarm(256, 8, O.SPHERE, -100, 100, 20)
    s.step_sync(400)
    assert float(s.gbest_fit) < 1e-4
    assert np.max(np.abs(s.gbest_pos)) < 1e-2


def test_rejects_invalid_params():
    with pytest.raises(ValueError):
        O.Swarm(0, 3, -1, 1, 1, 0.5, 1, 1, O.SPHERE, 1).init()
    with pytest.raises(ValueError):
        O.Swarm(4, 3, 1, -1, 1, 0.5, 1, 1, O.SPHERE, 1).init()
    with pytest.raises(ValueError):
        O.Swarm(4, 3, -1, 1, 0, 0.5, 1, 1, O.SPHERE, 1).init()


# --------------------------------------------------------------------------- #
# Least squares ||A x - b||^2 (the dense fitness of the precision study)       #
# --------------------------------------------------------------------------- #

def _lsq_problem(M, D, seed=0, noise=1e-3):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((M, D)) / np.sqrt(M)).astype(np.float32)
    xs = rng.uniform(-1, 1, D).astype(np.float32)
    b = (A.astype(np.float64) @ xs + noise * rng.standard_normal(M)).astype(np.float32)
    return A, b, xs


def test_lsq_fp64_minimum_is_the_lstsq_solution():
    """The FP64 fitness at numpy's least-squares solution is the closed-form minimum
    (the residual norm lstsq reports), and no perturbation goes below it."""
    A, b, _ = _lsq_problem(96, 12)
    x64, res, rank, _ = np.linalg.lstsq(A.astype(np.float64), b.astype(np.float64), rcond=None)
    xf = x64.astype(np.float32)
    fmin = O.lsq_f64(A, b, xf)
    assert abs(fmin - float(res[0])) <= 1e-6 * float(res[0]) + 1e-9   # float32 rounding of x only
    rng = np.random.default_rng(1)
    for _ in range(20):
        assert O.lsq_f64(A, b, (x64 + 1e-2 * rng.standard_normal(12)).astype(np.float32)) > fmin


def test_lsq_f32_within_rounding_of_f64():
    A, b, xs = _lsq_problem(300, 40, seed=3)
    rng = np.random.default_rng(4)
    for _ in range(10):
        x = rng.uniform(-2, 2, 40).astype(np.float32)
        f64 = O.lsq_f64(A, b, x)
        f32 = float(O.lsq_f32(A, b, x))
        assert abs(f32 - f64) <= 1e-5 * f64
    assert O.lsq_f64(A, b, xs) < 1e-3 * 300       # b = A x* + noise: f(x*) ~ M sigma^2


def test_lsq_swarm_steps_follow_the_swarm_rules():
    A, b, _ = _lsq_problem(64, 6, seed=5)
    s = O.Swarm(40, 6, -2, 2, 0.4, 0.729, 1.49445, 1.49445, O.LSQ, 2, lsq=(A, b)).init()
    prev = s.pbest_fit.copy()
    for _ in range(15):
        s.step_sync(1)
        assert np.all(s.pbest_fit <= prev)
        prev = s.pbest_fit.copy()
    for i in range(40):
        assert s.pbest_fit[i] == O.lsq_f32(A, b, s.pbest_pos[i])
    assert s.gbest_idx == int(np.lexsort((np.arange(40), s.pbest_fit))[0])


def test_lsq_f64_is_the_exact_residual_sum():
    """ora_lsq_f64 against the exact rational value of sum_m (sum_d A_md x_d - b_m)^2
    (every float32 input is an exact rational): within the binary64 rounding of
    its M (D + 2) operations. A dropped term, a sign error on b or a transposed
    A would be off by far more."""
    from fractions import Fraction as Fr
    rng = np.random.default_rng(21)
    for M, D in [(7, 3), (5, 11), (13, 1)]:
        A = rng.standard_normal((M, D)).astype(np.float32)
        b = rng.standard_normal(M).astype(np.float32)
        x = rng.uniform(-2, 2, D).astype(np.float32)
        exact = Fr(0)
        for m in range(M):
            r = -Fr(float(b[m])) + sum(Fr(float(A[m, d])) * Fr(float(x[d])) for d in range(D))
            exact += r * r
        got = O.lsq_f64(A, b, x)
        assert abs(Fr(got) - exact) <= Fr(M * (D + 3)) * Fr(2) ** -52 * (exact + 1), (M, D)


def test_lsq_fp64_fitness_swarm():
    """The FP64-fitness swarm (the reference run of the precision study): every
    pbest_fit is the FP64 fitness of its pbest_pos rounded once to float32, the
    gbest is the lowest-index argmin, pbest_fit never increases, and on a small
    convex problem the swarm reaches the closed-form least-squares minimum to
    1e-6 relative."""
    A, b, _ = _lsq_problem(64, 6, seed=5)
    s = O.Swarm(40, 6, -2, 2, 0.4, 0.729, 1.49445, 1.49445, O.LSQ, 2, lsq=(A, b), lsq_fp64=True).init()
    for i in range(40):
        assert s.pbest_fit[i] == np.float32(O.lsq_f64(A, b, s.pbest_pos[i]))
    prev = s.pbest_fit.copy()
    for _ in range(20):
        s.step_sync(1)
        assert np.all(s.pbest_fit <= prev)
        prev = s.pbest_fit.copy()
    for i in range(40):
        assert s.pbest_fit[i] == np.float32(O.lsq_f64(A, b, s.pbest_pos[i]))
    assert s.gbest_idx == int(np.lexsort((np.arange(40), s.pbest_fit))[0])
    s.step_sync(600)
    x64, res, _, _ = np.linalg.lstsq(A.astype(np.float64), b.astype(np.float64), rcond=None)
    fmin = float(res[0])
    g = O.lsq_f64(A, b, s.gbest_pos)
    assert fmin <= g * (1 + 1e-12) and g <= fmin * (1 + 1e-6), (g, fmin)


# --------------------------------------------------------------------------- #
# Operand roundings and the displacement form of the tensor-core fitness      #
# --------------------------------------------------------------------------- #

def _special_floats():
    rng = np.random.default_rng(31)
    v = np.concatenate([rng.standard_normal(20000).astype(np.float32) * np.float32(10.0) ** rng.integers(-12, 12, 20000),
                        np.array([0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -1.5, 3e38, 1e-40,
                                  2 ** -126, 2 ** -133], np.float32)]).astype(np.float32)
    return v


def test_round_bf16_closed_forms_and_torch():
    """Ties go to the even neighbour (1 + 2^-8 -> 1; 1 + 3 2^-8 -> 1 + 2^-6), and every
    value agrees bit for bit with torch's float32 -> bfloat16 conversion."""
    torch = pytest.importorskip("torch")
    r = O.round_bf16(np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, 255.5, 3.4e38], np.float32))
    assert r[0] == 1.0 and r[1] == 1 + 2 ** -6 and r[2] == 1 + 2 ** -7 and r[3] == 256.0 and np.isinf(r[4])
    v = _special_floats()
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(O.round_bf16(v).view(np.uint32), ref.view(np.uint32))


def test_round_e4m3_closed_forms_and_torch():
    """The format's grid: largest 448, smallest subnormal 2^-9, ties to even
    (2^-10 -> 0, 3 2^-10 -> 2^-8, 1 + 2^-4 -> 1, 1 + 3 2^-4 -> 1.25), saturation
    above 448; in range, bit for bit what torch's float8_e4m3fn conversion gives."""
    torch = pytest.importorskip("torch")
    cases = {448.0: 448.0, 500.0: 448.0, -1e6: -448.0, 2.0 ** -9: 2.0 ** -9, 2.0 ** -10: 0.0,
             3 * 2.0 ** -10: 2.0 ** -8, 1 + 2.0 ** -4: 1.0, 1 + 3 * 2.0 ** -4: 1.25, 0.1: 0.1015625}
    got = O.round_e4m3(np.array(list(cases), np.float32))
    np.testing.assert_array_equal(got, np.array(list(cases.values()), np.float32))
    v = _special_floats()
    v = v[np.abs(v) <= 448.0]
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    np.testing.assert_array_equal(O.round_e4m3(v), ref)


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_lsq_disp_is_the_fitness_up_to_operand_rounding(fmt):
    """The displacement form is the same function: its distance from the FP64
    fitness stays within the bound the operand rounding implies, and that bound
    (hence the error) scales with |x - g|, which is the point of the form: 100x
    closer to the reference point, about 100x smaller error. With g = x the
    displacement is zero and only the offsets' float rounding is left."""
    A, b, _ = _lsq_problem(200, 24, seed=8)
    rng = np.random.default_rng(9)
    g = rng.uniform(-2, 2, 24).astype(np.float32)
    sx = np.float32(448.0 / 4.0)
    unit = 2 ** -8 if fmt == "bf16" else 2 ** -3     # relative rounding of one operand (with margin)
    errs = []
    for eps in (1.0, 1e-2):
        x = (g + eps * rng.uniform(-1, 1, 24)).astype(np.float32)
        f = O.lsq_f64(A, b, x)
        fd = O.lsq_disp(A, b, x, g, fmt, sx)
        R = A.astype(np.float64) @ x.astype(np.float64) - b
        dR = np.abs(A.astype(np.float64)) @ np.abs((x - g).astype(np.float64)) * 2 * unit \
            + np.abs(R) * 2 ** -23 + 1e-12
        bound = float(np.sum(2 * np.abs(R) * dR + dR * dR))
        assert abs(fd - f) <= bound, (eps, fd, f, bound)
        errs.append(abs(fd - f))
    assert errs[1] < errs[0] / 20 + 1e-9
    f0 = O.lsq_disp(A, b, g, g, fmt, sx)
    R = A.astype(np.float64) @ g.astype(np.float64) - b
    assert abs(f0 - O.lsq_f64(A, b, g)) <= float(np.sum(2 * np.abs(R) * np.abs(R) * 2 ** -24)) * 1.01 + 1e-15


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_lsq_disp_exact_on_representable_operands(fmt):
    """Closed form: when A (each row holding 448, so the FP8 row scale is 1),
    the displacements x - g and A g - b are exact in the format (sx = 1), the
    displacement form rounds nothing, and must equal the exact rational value
    of sum_m (A_m x - b_m)^2 -- a dropped term, a sign error on the offset or a
    wrong scale would not."""
    from fractions import Fraction as Fr
    A = np.array([[448, 1, -2, 0.5], [3, 448, 0.25, -1], [-448, 2, 1, 1.5], [0.5, -3, 448, 2],
                  [1, 1, 1, -448]], np.float32)
    g = np.array([1, -2, 0.5, 0.25], np.float32)
    x = (g + np.array([0.5, -1, 2, -0.125], np.float32)).astype(np.float32)
    b = np.array([3, -7, 5, 11, -2], np.float32)
    exact = sum((sum(Fr(float(A[m, d])) * Fr(float(x[d])) for d in range(4)) - Fr(float(b[m]))) ** 2
                for m in range(5))
    assert O.lsq_disp(A, b, x, g, fmt, 1.0) == float(exact)
    assert O.lsq_f64(A, b, x) == float(exact)


@pytest.mark.parametrize("fid", [1, 3])
def test_threaded_sync_step_is_the_serial_one(fid):
    """The all-cores baseline (Steps 2-4 over host threads, Step 5 serial) gives the
    single-threaded oracle's state bit for bit, for any thread count."""
    lo, hi, vmax = {1: (-5.12, 5.12, 1.024), 3: (-30.0, 30.0, 6.0)}[fid]
    a = O.Swarm(3001, 9, lo, hi, vmax, 0.729, 1.49445, 1.49445, fid, 4).init().step_sync(6)
    for threads in (1, 3, 8):
        b = O.Swarm(3001, 9, lo, hi, vmax, 0.729, 1.49445, 1.49445, fid, 4).init().step_sync_threads(6, threads)
        for k in ("pos", "v", "pbest_pos", "pbest_fit", "gbest_pos"):
            np.testing.assert_array_equal(getattr(a, k).view(np.uint32), getattr(b, k).view(np.uint32))
        assert a.gbest_idx == b.gbest_idx and a.t == b.t
