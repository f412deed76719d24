"""Python view of the CPU oracle (ctypes over oracle/_build/libcupso_oracle.so).

TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the benchmark's
CPU-baseline leg. The library never imports this module.

State arrays are particle-major numpy float32 arrays, shape (N, D).
"""
import ctypes as C
import os

import numpy as np

from .build import build_oracle

SPHERE, RASTRIGIN, ACKLEY, ROSENBROCK, CUBIC_MAX, LSQ = 0, 1, 2, 3, 4, 5

_lib = None


class _Params(C.Structure):
    _fields_ = [("N", C.c_int), ("D", C.c_int),
                ("min_pos", C.c_float), ("max_pos", C.c_float), ("max_v", C.c_float),
                ("w", C.c_float), ("c1", C.c_float), ("c2", C.c_float),
                ("fitness", C.c_int), ("seed", C.c_uint64), ("swarm", C.c_uint32),
                ("lsq_A", C.c_void_p), ("lsq_b", C.c_void_p), ("lsq_M", C.c_int), ("lsq_fp64", C.c_int)]


class _State(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("v", C.c_void_p), ("pbest_pos", C.c_void_p),
                ("pbest_fit", C.c_void_p), ("fit", C.c_void_p), ("gbest_pos", C.c_void_p),
                ("gbest_fit", C.c_float), ("gbest_idx", C.c_int64), ("t", C.c_uint32)]


class _ParamsD(C.Structure):
    _fields_ = [("N", C.c_int), ("D", C.c_int),
                ("min_pos", C.c_double), ("max_pos", C.c_double), ("max_v", C.c_double),
                ("w", C.c_double), ("c1", C.c_double), ("c2", C.c_double),
                ("fitness", C.c_int), ("seed", C.c_uint64), ("swarm", C.c_uint32)]


class _StateD(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("v", C.c_void_p), ("pbest_pos", C.c_void_p),
                ("pbest_fit", C.c_void_p), ("fit", C.c_void_p), ("gbest_pos", C.c_void_p),
                ("gbest_fit", C.c_double), ("gbest_idx", C.c_int64), ("t", C.c_uint32)]


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = C.CDLL(path)
        f32p = C.POINTER(C.c_float)
        L.ora_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.ora_u01.argtypes = [C.c_uint32]
        L.ora_u01.restype = C.c_float
        L.ora_draw_r.argtypes = [C.POINTER(_Params), C.c_uint32, C.c_int, C.c_int, f32p, f32p]
        L.ora_cos2pi.argtypes = [C.c_float]
        L.ora_cos2pi.restype = C.c_float
        L.ora_exp.argtypes = [C.c_float]
        L.ora_exp.restype = C.c_float
        L.ora_cos2pi_coeffs.argtypes = [f32p]
        L.ora_exp_coeffs.argtypes = [f32p, f32p, f32p, f32p]
        L.ora_fitness.argtypes = [C.c_int, f32p, C.c_int]
        L.ora_fitness.restype = C.c_float
        L.ora_fit_key.argtypes = [C.c_float]
        L.ora_fit_key.restype = C.c_uint32
        for name in ("ora_init",):
            getattr(L, name).argtypes = [C.POINTER(_Params), C.POINTER(_State)]
            getattr(L, name).restype = C.c_int
        for name in ("ora_step_sync", "ora_step_serial"):
            getattr(L, name).argtypes = [C.POINTER(_Params), C.POINTER(_State), C.c_int, f32p]
            getattr(L, name).restype = C.c_int
        L.ora_step_sync_threads.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.c_int, C.c_int]
        L.ora_step_sync_threads.restype = C.c_int
        L.ora_move_one.argtypes = [C.POINTER(_Params), C.c_uint32, C.c_int, f32p, f32p, f32p, f32p, f32p, f32p]
        L.ora_move_one.restype = C.c_float
        L.ora_lsq_f32.argtypes = [f32p, f32p, C.c_int, C.c_int, f32p]
        L.ora_lsq_f32.restype = C.c_float
        L.ora_lsq_f64.argtypes = [f32p, f32p, C.c_int, C.c_int, f32p]
        L.ora_lsq_f64.restype = C.c_double
        L.ora_round_bf16_n.argtypes = [f32p, f32p, C.c_size_t]
        L.ora_round_e4m3_n.argtypes = [f32p, f32p, C.c_size_t]
        L.ora_lsq_disp.argtypes = [f32p, f32p, C.c_int, C.c_int, f32p, f32p, C.c_int, C.c_float]
        L.ora_lsq_disp.restype = C.c_double
        L.ora_argmin_pbest.argtypes = [C.POINTER(_Params), C.POINTER(_State)]
        L.ora_argmin_pbest.restype = C.c_int64
        f64p = C.POINTER(C.c_double)
        L.ora_u53.argtypes = [C.c_uint32, C.c_uint32]
        L.ora_u53.restype = C.c_double
        L.ora_draw_r_d.argtypes = [C.POINTER(_ParamsD), C.c_uint32, C.c_int, C.c_int, f64p, f64p]
        L.ora_fitness_d.argtypes = [C.c_int, f64p, C.c_int]
        L.ora_fitness_d.restype = C.c_double
        L.ora_fit_key_d.argtypes = [C.c_double]
        L.ora_fit_key_d.restype = C.c_uint64
        L.ora_init_d.argtypes = [C.POINTER(_ParamsD), C.POINTER(_StateD)]
        L.ora_init_d.restype = C.c_int
        L.ora_step_sync_d.argtypes = [C.POINTER(_ParamsD), C.POINTER(_StateD), C.c_int]
        L.ora_step_sync_d.restype = C.c_int
        L.ora_argmin_pbest_d.argtypes = [C.POINTER(_ParamsD), C.POINTER(_StateD)]
        L.ora_argmin_pbest_d.restype = C.c_int64
        L.ora_move_one_d.argtypes = [C.POINTER(_ParamsD), C.c_uint32, C.c_int, f64p, f64p, f64p, f64p, f64p]
        L.ora_move_one_d.restype = C.c_double
        _lib = L
    return _lib


def _f32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().ora_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def u01(w):
    return np.float32(lib().ora_u01(int(w) & 0xFFFFFFFF))


def cos2pi(x):
    return np.float32(lib().ora_cos2pi(float(np.float32(x))))


def exp(y):
    return np.float32(lib().ora_exp(float(np.float32(y))))


def cos2pi_coeffs():
    out = np.zeros(8, np.float32)
    lib().ora_cos2pi_coeffs(_f32p(out))
    return out


def exp_coeffs():
    out = np.zeros(9, np.float32)
    a, b, c = C.c_float(), C.c_float(), C.c_float()
    lib().ora_exp_coeffs(_f32p(out), C.byref(a), C.byref(b), C.byref(c))
    return out, np.float32(a.value), np.float32(b.value), np.float32(c.value)


def fitness(fid, x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    return np.float32(lib().ora_fitness(int(fid), _f32p(x), int(x.shape[-1])))


def lsq_f32(A, b, x):
    A = np.ascontiguousarray(A, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    return np.float32(lib().ora_lsq_f32(_f32p(A), _f32p(b), A.shape[0], A.shape[1], _f32p(x)))


def lsq_f64(A, b, x):
    A = np.ascontiguousarray(A, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    return float(lib().ora_lsq_f64(_f32p(A), _f32p(b), A.shape[0], A.shape[1], _f32p(x)))


def round_bf16(a):
    """Elementwise round-to-nearest-even to bfloat16 (as float32 values)."""
    a = np.ascontiguousarray(a, np.float32)
    out = np.empty_like(a)
    lib().ora_round_bf16_n(_f32p(a), _f32p(out), a.size)
    return out


def round_e4m3(a):
    """Elementwise round-to-nearest-even to FP8 e4m3, saturated to +-448 (as float32 values)."""
    a = np.ascontiguousarray(a, np.float32)
    out = np.empty_like(a)
    lib().ora_round_e4m3_n(_f32p(a), _f32p(out), a.size)
    return out


LSQ_FMT = {"bf16": 1, "fp8": 2}


def lsq_disp(A, b, x, g, fmt, sx=1.0):
    """||A (x - g) + (A g - b)||^2 on the operands the tensor-core modes round
    (fmt "bf16" or "fp8"; sx: the FP8 scale of the displacement), in FP64."""
    A = np.ascontiguousarray(A, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    g = np.ascontiguousarray(g, np.float32)
    return float(lib().ora_lsq_disp(_f32p(A), _f32p(b), A.shape[0], A.shape[1], _f32p(x), _f32p(g),
                                    LSQ_FMT[fmt], float(np.float32(sx))))


def fit_key(f):
    return int(lib().ora_fit_key(float(np.float32(f))))


class Swarm:
    """One swarm as the oracle holds it. Fields mirror Table 1 of the paper."""

    def __init__(self, N, D, min_pos, max_pos, max_v, w, c1, c2, fitness, seed, swarm=0, lsq=None, lsq_fp64=False):
        """lsq = (A [M][D] float32, b [M] float32) for the least-squares fitness;
        lsq_fp64: that fitness in binary64 (ora_lsq_f64's order), rounded to
        float32, instead of the binary32 order of ora_lsq_f32."""
        self.p = _Params(int(N), int(D), float(np.float32(min_pos)), float(np.float32(max_pos)),
                         float(np.float32(max_v)), float(np.float32(w)), float(np.float32(c1)),
                         float(np.float32(c2)), int(fitness), int(seed), int(swarm), None, None, 0,
                         1 if lsq_fp64 else 0)
        if lsq is not None:
            self._A = np.ascontiguousarray(lsq[0], np.float32)
            self._b = np.ascontiguousarray(lsq[1], np.float32)
            assert self._A.shape == (self._b.size, int(D))
            self.p.lsq_A = self._A.ctypes.data
            self.p.lsq_b = self._b.ctypes.data
            self.p.lsq_M = int(self._b.size)
        self.N, self.D = int(N), int(D)
        self.pos = np.zeros((N, D), np.float32)
        self.v = np.zeros((N, D), np.float32)
        self.pbest_pos = np.zeros((N, D), np.float32)
        self.pbest_fit = np.zeros(N, np.float32)
        self.fit = np.zeros(N, np.float32)
        self.gbest_pos = np.zeros(D, np.float32)
        self.s = _State()
        self._bind()

    def _bind(self):
        s = self.s
        s.pos = self.pos.ctypes.data
        s.v = self.v.ctypes.data
        s.pbest_pos = self.pbest_pos.ctypes.data
        s.pbest_fit = self.pbest_fit.ctypes.data
        s.fit = self.fit.ctypes.data
        s.gbest_pos = self.gbest_pos.ctypes.data

    @property
    def t(self):
        return int(self.s.t)

    @property
    def gbest_fit(self):
        return np.float32(self.s.gbest_fit)

    @property
    def gbest_idx(self):
        return int(self.s.gbest_idx)

    def init(self):
        rc = lib().ora_init(C.byref(self.p), C.byref(self.s))
        if rc != 0:
            raise ValueError("oracle: invalid parameters")
        return self

    def set_state(self, pos, v, pbest_pos, pbest_fit, t):
        """Load a state; gbest is recomputed from pbest (Step 5)."""
        self.pos[...] = pos
        self.v[...] = v
        self.pbest_pos[...] = pbest_pos
        self.pbest_fit[...] = pbest_fit
        self.s.t = int(t)
        g = int(lib().ora_argmin_pbest(C.byref(self.p), C.byref(self.s)))
        self.s.gbest_idx = g
        self.s.gbest_fit = float(self.pbest_fit[g])
        self.gbest_pos[...] = self.pbest_pos[g]
        return self

    def _r(self, r_override, iters):
        if r_override is None:
            return None
        r = np.ascontiguousarray(r_override, dtype=np.float32)
        assert r.size == iters * self.N * self.D * 2
        return r

    def step_sync(self, iters=1, r_override=None):
        r = self._r(r_override, iters)
        rc = lib().ora_step_sync(C.byref(self.p), C.byref(self.s), int(iters),
                                 _f32p(r) if r is not None else None)
        if rc != 0:
            raise ValueError("oracle: invalid parameters")
        return self

    def step_sync_threads(self, iters, threads):
        """step_sync with Steps 2-4 on `threads` host threads (identical result)."""
        if lib().ora_step_sync_threads(C.byref(self.p), C.byref(self.s), int(iters), int(threads)) != 0:
            raise ValueError("oracle: invalid parameters")
        return self

    def step_serial(self, iters=1, r_override=None):
        r = self._r(r_override, iters)
        rc = lib().ora_step_serial(C.byref(self.p), C.byref(self.s), int(iters),
                                   _f32p(r) if r is not None else None)
        if rc != 0:
            raise ValueError("oracle: invalid parameters")
        return self

    def draw_r(self, t, i, d):
        r1, r2 = C.c_float(), C.c_float()
        lib().ora_draw_r(C.byref(self.p), int(t), int(i), int(d), C.byref(r1), C.byref(r2))
        return np.float32(r1.value), np.float32(r2.value)

    def move_one(self, t, i, pos, v, pbest_pos, pbest_fit, gbest_pos):
        """Steps 2-4 for one particle (global index i) at iteration t, on copies.
        Returns (pos, v, pbest_pos, pbest_fit, fit)."""
        pos = np.array(pos, np.float32)
        v = np.array(v, np.float32)
        pb = np.array(pbest_pos, np.float32)
        pf = np.array([pbest_fit], np.float32)
        g = np.ascontiguousarray(gbest_pos, np.float32)
        f = lib().ora_move_one(C.byref(self.p), int(t), int(i), _f32p(pos), _f32p(v), _f32p(pb), _f32p(pf),
                               _f32p(g), None)
        return pos, v, pb, np.float32(pf[0]), np.float32(f)

    def argmin_pbest(self):
        return int(lib().ora_argmin_pbest(C.byref(self.p), C.byref(self.s)))


# ---------------------------------------------------------------------------
# Double precision (the paper's precision): sphere, Rosenbrock, cubic.
# ---------------------------------------------------------------------------

def _f64p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def u53(hi, lo):
    return float(lib().ora_u53(int(hi) & 0xFFFFFFFF, int(lo) & 0xFFFFFFFF))


def fitness_d(fid, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().ora_fitness_d(int(fid), _f64p(x), int(x.shape[-1])))


def fit_key_d(f):
    return int(lib().ora_fit_key_d(float(f)))


class Swarm64:
    """A double-precision swarm as the oracle holds it (state arrays float64, (N, D))."""

    def __init__(self, N, D, min_pos, max_pos, max_v, w, c1, c2, fitness, seed, swarm=0):
        self.p = _ParamsD(int(N), int(D), float(min_pos), float(max_pos), float(max_v), float(w), float(c1),
                          float(c2), int(fitness), int(seed), int(swarm))
        self.N, self.D = int(N), int(D)
        self.pos = np.zeros((N, D), np.float64)
        self.v = np.zeros((N, D), np.float64)
        self.pbest_pos = np.zeros((N, D), np.float64)
        self.pbest_fit = np.zeros(N, np.float64)
        self.fit = np.zeros(N, np.float64)
        self.gbest_pos = np.zeros(D, np.float64)
        self.s = _StateD()
        s = self.s
        s.pos, s.v, s.pbest_pos = self.pos.ctypes.data, self.v.ctypes.data, self.pbest_pos.ctypes.data
        s.pbest_fit, s.fit, s.gbest_pos = self.pbest_fit.ctypes.data, self.fit.ctypes.data, self.gbest_pos.ctypes.data

    @property
    def t(self):
        return int(self.s.t)

    @property
    def gbest_fit(self):
        return float(self.s.gbest_fit)

    @property
    def gbest_idx(self):
        return int(self.s.gbest_idx)

    def init(self):
        if lib().ora_init_d(C.byref(self.p), C.byref(self.s)) != 0:
            raise ValueError("oracle: invalid parameters")
        return self

    def set_state(self, pos, v, pbest_pos, pbest_fit, t):
        self.pos[...] = pos
        self.v[...] = v
        self.pbest_pos[...] = pbest_pos
        self.pbest_fit[...] = pbest_fit
        self.s.t = int(t)
        g = int(lib().ora_argmin_pbest_d(C.byref(self.p), C.byref(self.s)))
        self.s.gbest_idx = g
        self.s.gbest_fit = float(self.pbest_fit[g])
        self.gbest_pos[...] = self.pbest_pos[g]
        return self

    def step_sync(self, iters=1):
        if lib().ora_step_sync_d(C.byref(self.p), C.byref(self.s), int(iters)) != 0:
            raise ValueError("oracle: invalid parameters")
        return self

    def draw_r(self, t, i, d):
        r1, r2 = C.c_double(), C.c_double()
        lib().ora_draw_r_d(C.byref(self.p), int(t), int(i), int(d), C.byref(r1), C.byref(r2))
        return r1.value, r2.value

    def move_one(self, t, i, pos, v, pbest_pos, pbest_fit, gbest_pos):
        """Steps 2-4 for one particle at iteration t, on copies: (pos, v, pbest_pos, pbest_fit, fit)."""
        pos = np.array(pos, np.float64)
        v = np.array(v, np.float64)
        pb = np.array(pbest_pos, np.float64)
        pf = np.array([pbest_fit], np.float64)
        g = np.ascontiguousarray(gbest_pos, np.float64)
        f = lib().ora_move_one_d(C.byref(self.p), int(t), int(i), _f64p(pos), _f64p(v), _f64p(pb), _f64p(pf),
                                 _f64p(g))
        return pos, v, pb, float(pf[0]), float(f)

    def argmin_pbest(self):
        return int(lib().ora_argmin_pbest_d(C.byref(self.p), C.byref(self.s)))
