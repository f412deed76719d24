"""Pins of the double-precision oracle (the paper's own precision, Sec. 5.1).

The paper runs its PSO in FP64 on the cubic of Eq. 3 with w = 1, c1 = c2 = 2.
The double-precision oracle follows the same steps as the FP32 one; these
tests tie it to facts outside itself: the closed form of the 53-bit uniform,
the KAT-pinned Philox words it must use, textbook FP64 formulas, the exact
(rational) value of Eq. 1 and Eq. 2, the inertia-only closed form, the known
maximiser of Eq. 3 on its box, and the invariants of Alg. 1.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

EPS = 2.0 ** -53


# --------------------------------------------------------------------------- #
# 53-bit uniforms (Sec. 4.4: r1, r2 uniform in cuRAND's (0, 1] range)          #
# --------------------------------------------------------------------------- #

def test_u53_closed_form():
    assert O.u53(0, 0) == 2.0 ** -53                     # 0 is not reachable
    assert O.u53(0, 0x7FF) == 2.0 ** -53                 # low 11 bits of lo are dropped
    assert O.u53(0, 0x800) == 2.0 * 2.0 ** -53
    assert O.u53(1, 0) == (2 ** 21 + 1) * 2.0 ** -53     # hi supplies the top 32 bits
    assert O.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0          # 1 is reachable
    rng = np.random.default_rng(3)
    for hi, lo in rng.integers(0, 2 ** 32, (300, 2), dtype=np.uint64):
        m = (int(hi) << 21) | (int(lo) >> 11)
        assert O.u53(int(hi), int(lo)) == (m + 1) / 2.0 ** 53


def test_draws_use_one_philox_call_per_dimension():
    """Counter (d, i, t, swarm), key = seed; r1 from words 0,1, r2 from 2,3."""
    seed, swarm = 0x0123456789ABCDEF, 7
    s = O.Swarm64(10, 5, -1, 1, 0.5, 1, 2, 2, O.SPHERE, seed, swarm)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for t, i, d in [(0, 0, 0), (1, 3, 4), (99, 9, 2), (2 ** 31, 1, 1)]:
        w = O.philox4x32_10((d, i, t, swarm), key)
        assert s.draw_r(t, i, d) == (O.u53(w[0], w[1]), O.u53(w[2], w[3]))


def test_u53_moments():
    s = O.Swarm64(1, 1, -1, 1, 0.5, 1, 2, 2, O.SPHERE, 11)
    r = np.array([s.draw_r(1, i, d) for i in range(400) for d in range(5)]).ravel()
    assert abs(r.mean() - 0.5) < 0.02
    assert abs(r.var() - 1.0 / 12.0) < 0.01
    assert r.min() > 0.0 and r.max() <= 1.0


# --------------------------------------------------------------------------- #
# Fitness (Step 3) in FP64                                                     #
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("D", [1, 2, 7, 120])
def test_known_optima_exact_fp64(D):
    assert O.fitness_d(O.SPHERE, np.zeros(D)) == 0.0
    assert O.fitness_d(O.ROSENBROCK, np.ones(D)) == 0.0
    # Eq. 3 on [-100, 100]: x^3 - 0.8 x^2 - 1000 x + 8000 is largest at the wall
    # x = 100 (900000); minimised as -f.
    assert O.fitness_d(O.CUBIC_MAX, np.full(D, 100.0)) == -900000.0 * D
    assert O.fitness_d(O.CUBIC_MAX, np.full(D, -100.0)) == 900000.0 * D


def test_cubic_maximiser_on_the_box():
    """Brute force over a fine grid of [-100, 100]: the maximum of Eq. 3 is at 100."""
    xs = np.linspace(-100.0, 100.0, 20001)
    f = np.array([-O.fitness_d(O.CUBIC_MAX, np.array([x])) for x in xs])
    assert xs[np.argmax(f)] == 100.0
    # the interior stationary points 0.8/3 +- sqrt(0.64/9 + 1000/3) are not maxima on the box
    xm = 0.8 / 3 - np.sqrt(0.64 / 9 + 1000 / 3)
    assert -O.fitness_d(O.CUBIC_MAX, np.array([xm])) < 900000.0


@pytest.mark.parametrize("fid", [O.SPHERE, O.ROSENBROCK, O.CUBIC_MAX])
def test_fitness_fp64_vs_textbook(fid):
    rng = np.random.default_rng(fid + 40)
    for D in (1, 3, 64, 120):
        for _ in range(20):
            x = rng.uniform(-100, 100, D)
            if fid == O.SPHERE:
                terms = x * x
                ref = np.sum(terms)
            elif fid == O.ROSENBROCK:
                terms = np.concatenate([100.0 * (x[1:] - x[:-1] ** 2) ** 2, (1.0 - x[:-1]) ** 2])
                ref = np.sum(terms)
            else:
                terms = np.concatenate([x ** 3, 0.8 * x ** 2, 1000.0 * x, np.full(D, 8000.0)])
                ref = -np.sum(x ** 3 - 0.8 * x ** 2 - 1000.0 * x + 8000.0)
            got = O.fitness_d(fid, x)
            assert abs(got - ref) <= 1e-13 * np.sum(np.abs(terms)) + 1e-300


def test_fit_key_d_order():
    rng = np.random.default_rng(8)
    vals = np.concatenate([rng.standard_normal(200) * 10.0 ** rng.integers(-300, 300, 200),
                           [0.0, -0.0, np.inf, -np.inf, 5e-324, -5e-324]])
    keys = [O.fit_key_d(v) for v in vals]
    order = np.argsort(vals, kind="stable")
    assert all(keys[order[k]] <= keys[order[k + 1]] for k in range(len(vals) - 1))
    assert O.fit_key_d(0.0) == O.fit_key_d(-0.0)
    assert O.fit_key_d(float("nan")) == 2 ** 64 - 1
    assert O.fit_key_d(np.inf) < O.fit_key_d(float("nan"))


# --------------------------------------------------------------------------- #
# Steps 1-5                                                                    #
# --------------------------------------------------------------------------- #

def test_init_closed_form_fp64():
    s = O.Swarm64(37, 4, -100, 100, 20, 1, 2, 2, O.CUBIC_MAX, 5, 3).init()
    key = (5, 0)
    for i in (0, 17, 36):
        for d in range(4):
            w = O.philox4x32_10((d, i, 0, 3), key)
            x = Fraction(O.u53(w[0], w[1])) * 200 - 100       # exact; one rounding in the oracle
            v = Fraction(O.u53(w[2], w[3])) * 40 - 20
            assert s.pos[i, d] == float(x)
            assert s.v[i, d] == float(v)
    assert np.all(s.pbest_pos == s.pos)
    assert s.gbest_idx == int(np.lexsort((np.arange(37), s.pbest_fit))[0])


def _exact_step(s, t, i, pos, v, pb, g):
    """Eq. 1 and Eq. 2 with their clamps in exact rational arithmetic."""
    p = s.p
    out_x, out_v, mag = [], [], []
    for d in range(s.D):
        r1, r2 = s.draw_r(t, i, d)
        w, c1, c2 = Fraction(p.w), Fraction(p.c1), Fraction(p.c2)
        X, V, PB, G = (Fraction(float(a)) for a in (pos[d], v[d], pb[d], g[d]))
        terms = [w * V, c1 * Fraction(r1) * (PB - X), c2 * Fraction(r2) * (G - X)]
        vel = sum(terms)
        vmax = Fraction(p.max_v)
        vel = min(max(vel, -vmax), vmax)
        x = min(max(X + vel, Fraction(p.min_pos)), Fraction(p.max_pos))
        out_x.append(x)
        out_v.append(vel)
        mag.append(float(sum(abs(a) for a in terms)) + abs(float(X)))
    return out_x, out_v, mag


@pytest.mark.parametrize("fid,lo,hi,vmax,w,c1,c2", [(O.CUBIC_MAX, -100, 100, 20, 1.0, 2.0, 2.0),
                                                     (O.SPHERE, -5, 5, 1, 0.729, 0.5, 2.5),
                                                     (O.ROSENBROCK, -30, 30, 6, 0.729, 2.25, 0.75)])
def test_single_step_equals_exact_eq1_eq2(fid, lo, hi, vmax, w, c1, c2):
    """From a state with nonzero cognitive and social terms, each coordinate of
    the oracle's step is the exact rational value of Eq. 1/2 up to the
    rounding of its six operations."""
    N, D = 6, 5
    s = O.Swarm64(N, D, lo, hi, vmax, w, c1, c2, fid, 21).init()
    s.step_sync(3)
    st = {k: getattr(s, k).copy() for k in ("pos", "v", "pbest_pos")}
    g = s.gbest_pos.copy()
    t = s.t + 1
    s.step_sync(1)
    for i in range(N):
        ex, ev, mag = _exact_step(s, t, i, st["pos"][i], st["v"][i], st["pbest_pos"][i], g)
        for d in range(D):
            tol = 8 * EPS * mag[d]
            assert abs(s.v[i, d] - float(ev[d])) <= tol
            assert abs(s.pos[i, d] - float(ex[d])) <= tol + 2 * EPS * abs(float(ex[d]))
    # Step 4: pbest is the position where the fitness is lowest so far
    for i in range(N):
        assert s.pbest_fit[i] == O.fitness_d(fid, s.pbest_pos[i])


def test_inertia_only_closed_form_fp64():
    """c1 = c2 = 0, w = 1/2: v_t = v_0 / 2^t exactly and x_t = x_{t-1} + v_t."""
    s = O.Swarm64(9, 3, -1e6, 1e6, 20, 0.5, 0.0, 0.0, O.SPHERE, 2).init()
    v0, x = s.v.copy(), s.pos.copy()
    for t in range(1, 30):
        s.step_sync(1)
        assert np.array_equal(s.v, v0 * 0.5 ** t)
        x = x + v0 * 0.5 ** t
        assert np.array_equal(s.pos, x)


def test_lone_particle_only_has_inertia():
    """N = 1: pbest = gbest = pos after init, so Eq. 1 reduces to w v."""
    s = O.Swarm64(1, 4, -100, 100, 20, 0.75, 2, 2, O.SPHERE, 4).init()
    v0, x0 = s.v.copy(), s.pos.copy()
    s.step_sync(1)
    assert np.array_equal(s.v, v0 * 0.75)
    assert np.array_equal(s.pos, np.clip(x0 + v0 * 0.75, -100, 100))


@pytest.mark.parametrize("fid,lo,hi,vmax", [(O.CUBIC_MAX, -100, 100, 20), (O.SPHERE, -100, 100, 20),
                                            (O.ROSENBROCK, -30, 30, 6)])
def test_invariants_fp64(fid, lo, hi, vmax):
    N, D = 50, 6
    s = O.Swarm64(N, D, lo, hi, vmax, 0.729, 1.49445, 1.49445, fid, 9).init()
    prev_pf, prev_g = s.pbest_fit.copy(), s.gbest_fit
    for _ in range(15):
        s.step_sync(1)
        assert np.all(s.pbest_fit <= prev_pf)
        assert s.gbest_fit <= prev_g
        assert np.all(np.abs(s.v) <= vmax) and np.all((s.pos >= lo) & (s.pos <= hi))
        g = int(np.lexsort((np.arange(N), s.pbest_fit))[0])
        assert s.gbest_idx == g and np.array_equal(s.gbest_pos, s.pbest_pos[g])
        for i in range(N):
            assert s.pbest_fit[i] == O.fitness_d(fid, s.pbest_pos[i])
        prev_pf, prev_g = s.pbest_fit.copy(), s.gbest_fit


@pytest.mark.parametrize("D", [1, 3])
def test_paper_workload_reaches_the_wall(D):
    """The paper's setting (Eq. 3 maximised on [-100, 100], w = 1, c1 = c2 = 2):
    the swarm reaches the maximiser x = 100 exactly (clamped at the wall), and
    among the particles whose pbest sits there, gbest is the lowest index."""
    N = 256
    s = O.Swarm64(N, D, -100, 100, 20, 1.0, 2.0, 2.0, O.CUBIC_MAX, 1).init()
    s.step_sync(300)
    assert s.gbest_fit == -900000.0 * D
    assert np.all(s.gbest_pos == 100.0)
    at_wall = np.flatnonzero(np.all(s.pbest_pos == 100.0, axis=1))
    assert s.gbest_idx == at_wall[0]


def test_rejects_unsupported_fitness_fp64():
    for fid in (O.RASTRIGIN, O.ACKLEY, O.LSQ):
        with pytest.raises(ValueError):
            O.Swarm64(4, 2, -1, 1, 1, 1, 2, 2, fid, 1).init()
