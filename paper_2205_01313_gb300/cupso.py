"""Python binding of libcupso.so (include/cupso.h), argument marshalling only.

Every function keeps the C name and forwards to the library; the swarm lives
in device memory owned by the library, and every step of the iteration runs
in its CUDA kernels. There is no CPU fallback: if the library is missing or
cannot load, importing this module raises.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcupso.so")

CUPSO_SPHERE, CUPSO_RASTRIGIN, CUPSO_ACKLEY, CUPSO_ROSENBROCK, CUPSO_CUBIC_MAX = 0, 1, 2, 3, 4
FITNESS = {"sphere": 0, "rastrigin": 1, "ackley": 2, "rosenbrock": 3, "cubic_max": 4, "lsq": 5}

CUPSO_OK = 0
CUPSO_ERR_INVALID_ARG = -1
CUPSO_ERR_OOM = -2
CUPSO_ERR_CUDA = -3
CUPSO_ERR_DEVICE_TIMEOUT = -4
CUPSO_ERR_NAN = -5
CUPSO_ERR_UNSUPPORTED = -6

(CUPSO_MODE_AUTO, CUPSO_MODE_SYNC, CUPSO_MODE_TREE, CUPSO_MODE_TREE_UNROLLED, CUPSO_MODE_ASYNC, CUPSO_MODE_ONCHIP,
 CUPSO_MODE_QUEUE, CUPSO_MODE_QUEUE_LOCK, CUPSO_MODE_PERSISTENT) = range(9)
MODES = {"auto": 0, "sync": 1, "tree": 2, "tree_unrolled": 3, "async": 4, "onchip": 5, "queue": 6, "queue_lock": 7,
         "persistent": 8}

CUPSO_OPT_MODE = 1
CUPSO_OPT_GRAPH_CHUNK = 2
CUPSO_OPT_WAIT_LIMIT_NS = 3
CUPSO_OPT_CLEAR_STATUS = 4
CUPSO_OPT_GRID = 5
CUPSO_OPT_SYNC_KERNEL = 6
CUPSO_OPT_TIME_FITNESS = 7
CUPSO_OPT_PARTICLES_PER_THREAD = 8
CUPSO_OPT_ITERS_PER_LAUNCH = 9
CUPSO_OPT_LSQ_RESCORE = 10
SYNC_KERNELS = {"auto": 0, "register": 1, "pipelined3": 2, "pipelined4": 3, "tiled": 4, "panel8": 5, "panel16": 6}
CUPSO_OPT_FAULT_HOLD_LOCK = 100
CUPSO_OPT_FAULT_STALL_BARRIER = 101

# The names the library must export (every function of include/cupso.h).
ABI_FUNCTIONS = ("cupso_create", "cupso_set_stream", "cupso_set_option", "cupso_step", "cupso_get_gbest",
                 "cupso_get_state", "cupso_set_state", "cupso_get_info", "cupso_solve_batch", "cupso_destroy",
                 "cupso_status_string", "cupso_last_error", "cupso_tree_step_noalloc", "cupso_lsq_eval",
                 "cupso_set_lsq", "cupso_get_gbest_f64", "cupso_create_fp64", "cupso_get_gbest_fp64",
                 "cupso_get_state_fp64", "cupso_set_state_fp64", "cupso_gbest_post", "cupso_gbest_wait")

CUPSO_LSQ = 5
CUPSO_LSQ_FP32, CUPSO_LSQ_BF16, CUPSO_LSQ_FP8, CUPSO_LSQ_FP64 = 0, 1, 2, 3
LSQ_PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2, "fp64": 3}

CUPSO_NOALLOC_MAX_N = 4194304
CUPSO_NOALLOC_MAX_D = 1024


class cupso_bounds(C.Structure):
    _fields_ = [("min_pos", C.c_float), ("max_pos", C.c_float), ("max_v", C.c_float)]


class cupso_bounds_f64(C.Structure):
    _fields_ = [("min_pos", C.c_double), ("max_pos", C.c_double), ("max_v", C.c_double)]


class cupso_info(C.Structure):
    _fields_ = [("N", C.c_int), ("D", C.c_int), ("Np", C.c_int), ("mode", C.c_int), ("t", C.c_uint32),
                ("sync_grid", C.c_int), ("async_grid", C.c_int), ("onchip_cluster", C.c_int),
                ("sync_stages", C.c_int), ("sync_ppt", C.c_int), ("sync_tile", C.c_int), ("fitness_ms", C.c_float),
                ("fitness_timed", C.c_int),
                ("device_bytes", C.c_uint64), ("sync_panel", C.c_int), ("sync_iters_per_launch", C.c_int)]


class cupso_problem(C.Structure):
    _fields_ = [("D", C.c_int), ("N", C.c_int), ("bounds", cupso_bounds), ("w", C.c_float), ("c1", C.c_float),
                ("c2", C.c_float), ("fitness_id", C.c_int), ("seed", C.c_uint64), ("swarm_id", C.c_uint32)]


class cupso_result(C.Structure):
    _fields_ = [("fit", C.c_float), ("idx", C.c_int64), ("pos", C.POINTER(C.c_float)), ("status", C.c_int)]


class CupsoError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s (%d): %s" % (where, status_string(code), code, last_error()))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libcupso.so is not built (%s); build it with paper_2205_01313_gb300.build.build()"
                          % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    h = C.c_void_p
    f32p = C.POINTER(C.c_float)
    L.cupso_create.argtypes = [C.c_int, C.c_int, C.POINTER(cupso_bounds), C.c_float, C.c_float, C.c_float,
                               C.c_int, C.c_uint64, C.POINTER(h)]
    L.cupso_set_stream.argtypes = [h, C.c_void_p]
    L.cupso_set_option.argtypes = [h, C.c_int, C.c_longlong]
    L.cupso_step.argtypes = [h, C.c_int]
    L.cupso_get_gbest.argtypes = [h, f32p, f32p, C.POINTER(C.c_int64)]
    L.cupso_gbest_post.argtypes = [h, C.c_int]
    L.cupso_gbest_wait.argtypes = [h, C.c_int, f32p, f32p, C.POINTER(C.c_int64)]
    L.cupso_get_state.argtypes = [h, f32p, f32p, f32p, f32p, C.POINTER(C.c_uint32)]
    L.cupso_set_state.argtypes = [h, f32p, f32p, f32p, f32p, C.c_uint32]
    L.cupso_get_info.argtypes = [h, C.POINTER(cupso_info)]
    L.cupso_solve_batch.argtypes = [C.c_int, C.POINTER(cupso_problem), C.c_int, C.POINTER(cupso_result),
                                    C.c_void_p]
    L.cupso_tree_step_noalloc.argtypes = [C.c_int, C.c_int, C.POINTER(cupso_bounds), C.c_float, C.c_float,
                                          C.c_float, C.c_int, C.c_uint64, C.c_uint32, C.c_uint32, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p]
    L.cupso_lsq_eval.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                 C.c_void_p, C.c_void_p]
    L.cupso_set_lsq.argtypes = [h, C.c_void_p, C.c_void_p, C.c_int, C.c_int]
    L.cupso_get_gbest_f64.argtypes = [h, C.POINTER(C.c_double)]
    f64p = C.POINTER(C.c_double)
    L.cupso_create_fp64.argtypes = [C.c_int, C.c_int, C.POINTER(cupso_bounds_f64), C.c_double, C.c_double,
                                    C.c_double, C.c_int, C.c_uint64, C.POINTER(h)]
    L.cupso_get_gbest_fp64.argtypes = [h, f64p, f64p, C.POINTER(C.c_int64)]
    L.cupso_get_state_fp64.argtypes = [h, f64p, f64p, f64p, f64p, C.POINTER(C.c_uint32)]
    L.cupso_set_state_fp64.argtypes = [h, f64p, f64p, f64p, f64p, C.c_uint32]
    L.cupso_destroy.argtypes = [h]
    L.cupso_status_string.argtypes = [C.c_int]
    L.cupso_status_string.restype = C.c_char_p
    L.cupso_last_error.argtypes = []
    L.cupso_last_error.restype = C.c_char_p
    for name in ABI_FUNCTIONS:
        if name not in ("cupso_status_string", "cupso_last_error"):
            getattr(L, name).restype = C.c_int
    return L


_lib = _load()


def lib():
    return _lib


def status_string(code):
    return _lib.cupso_status_string(int(code)).decode()


def last_error():
    return _lib.cupso_last_error().decode()


def _check(rc, where):
    if rc != CUPSO_OK:
        raise CupsoError(rc, where)


def _f32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_float)) if a is not None else None


def _bounds(b):
    if isinstance(b, cupso_bounds):
        return b
    lo, hi, vmax = b
    return cupso_bounds(float(lo), float(hi), float(vmax))


def cupso_create(D, N, bounds, w, c1, c2, fitness_id, seed):
    """Create a swarm and initialise it on the device; returns the handle."""
    h = C.c_void_p()
    b = _bounds(bounds)
    _check(_lib.cupso_create(int(D), int(N), C.byref(b), float(w), float(c1), float(c2), int(fitness_id),
                             int(seed) & 0xFFFFFFFFFFFFFFFF, C.byref(h)), "cupso_create")
    return h


def cupso_set_stream(h, cuda_stream):
    """cuda_stream: an integer cudaStream_t (e.g. torch.cuda.Stream.cuda_stream) or None/0."""
    _check(_lib.cupso_set_stream(h, C.c_void_p(int(cuda_stream) if cuda_stream else None)), "cupso_set_stream")


def cupso_set_option(h, key, value):
    _check(_lib.cupso_set_option(h, int(key), int(value)), "cupso_set_option")


def cupso_step(h, iters):
    _check(_lib.cupso_step(h, int(iters)), "cupso_step")


def cupso_get_gbest(h, D, pos_out=None):
    """Returns (status, fit, idx, pos). status is CUPSO_OK or the sticky device
    status (CUPSO_ERR_DEVICE_TIMEOUT / CUPSO_ERR_NAN); other errors raise."""
    pos = pos_out if pos_out is not None else np.empty(int(D), np.float32)
    fit = C.c_float()
    idx = C.c_int64()
    rc = _lib.cupso_get_gbest(h, C.byref(fit), _f32p(pos), C.byref(idx))
    if rc not in (CUPSO_OK, CUPSO_ERR_DEVICE_TIMEOUT, CUPSO_ERR_NAN):
        raise CupsoError(rc, "cupso_get_gbest")
    return rc, np.float32(fit.value), int(idx.value), pos


def cupso_gbest_post(h, slot):
    """Queues a copy of the current gbest into result slot 0 or 1; does not wait."""
    _check(_lib.cupso_gbest_post(h, int(slot)), "cupso_gbest_post")


def cupso_gbest_wait(h, D, slot, pos_out=None):
    """Waits for result slot `slot`; returns (status, fit, idx, pos) as cupso_get_gbest."""
    pos = pos_out if pos_out is not None else np.empty(int(D), np.float32)
    fit = C.c_float()
    idx = C.c_int64()
    rc = _lib.cupso_gbest_wait(h, int(slot), C.byref(fit), _f32p(pos), C.byref(idx))
    if rc not in (CUPSO_OK, CUPSO_ERR_DEVICE_TIMEOUT, CUPSO_ERR_NAN):
        raise CupsoError(rc, "cupso_gbest_wait")
    return rc, np.float32(fit.value), int(idx.value), pos


def cupso_get_state(h, N, D):
    pos = np.empty((N, D), np.float32)
    v = np.empty((N, D), np.float32)
    pb = np.empty((N, D), np.float32)
    pf = np.empty(N, np.float32)
    t = C.c_uint32()
    _check(_lib.cupso_get_state(h, _f32p(pos), _f32p(v), _f32p(pb), _f32p(pf), C.byref(t)), "cupso_get_state")
    return {"pos": pos, "v": v, "pbest_pos": pb, "pbest_fit": pf, "t": int(t.value)}


def cupso_set_state(h, pos, v, pbest_pos, pbest_fit, t):
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (pos, v, pbest_pos, pbest_fit)]
    _check(_lib.cupso_set_state(h, *[_f32p(a) for a in arrs], int(t)), "cupso_set_state")


def cupso_get_info(h):
    info = cupso_info()
    _check(_lib.cupso_get_info(h, C.byref(info)), "cupso_get_info")
    return {k: getattr(info, k) for k, _ in cupso_info._fields_}


def cupso_solve_batch(problems, iters, cuda_stream=None, want_pos=True):
    """problems: sequence of dicts with keys D, N, bounds, w, c1, c2, fitness_id,
    seed, swarm_id. Returns (status, list of dicts fit/idx/pos/status)."""
    n = len(problems)
    P = (cupso_problem * max(n, 1))()
    R = (cupso_result * max(n, 1))()
    keep = []
    for k, p in enumerate(problems):
        P[k] = cupso_problem(int(p["D"]), int(p["N"]), _bounds(p["bounds"]), float(p["w"]), float(p["c1"]),
                             float(p["c2"]), int(p["fitness_id"]), int(p["seed"]) & 0xFFFFFFFFFFFFFFFF,
                             int(p.get("swarm_id", 0)))
        pos = np.empty(int(p["D"]), np.float32) if want_pos else None
        keep.append(pos)
        R[k].pos = _f32p(pos) if pos is not None else None
    rc = _lib.cupso_solve_batch(n, P, int(iters), R, C.c_void_p(int(cuda_stream) if cuda_stream else None))
    if rc == CUPSO_ERR_INVALID_ARG:
        raise CupsoError(rc, "cupso_solve_batch")
    out = [{"fit": np.float32(R[k].fit), "idx": int(R[k].idx), "pos": keep[k], "status": int(R[k].status)}
           for k in range(n)]
    return rc, out


def cupso_tree_step_noalloc(D, N, bounds, w, c1, c2, fitness_id, seed, swarm_id, t, pos, v, pbest_pos, pbest_fit,
                            ld, gbest_pos, gbest_fit=0, gbest_idx=0, status_out=0, cuda_stream=0):
    """One iteration on caller-owned device buffers; every buffer argument is a
    device address (int), e.g. torch.Tensor.data_ptr(). Allocates nothing."""
    b = _bounds(bounds)
    _check(_lib.cupso_tree_step_noalloc(int(D), int(N), C.byref(b), float(w), float(c1), float(c2),
                                        int(fitness_id), int(seed) & 0xFFFFFFFFFFFFFFFF, int(swarm_id), int(t),
                                        pos, v, pbest_pos, pbest_fit, int(ld), gbest_pos, gbest_fit or None,
                                        gbest_idx or None, status_out or None, cuda_stream or None),
           "cupso_tree_step_noalloc")


def cupso_lsq_eval(A_dev, b_dev, M, D, X_dev, N, precision, f_out_dev, cuda_stream=0):
    """f_out[i] = ||A x_i - b||^2; every buffer argument is a device address (int)."""
    _check(_lib.cupso_lsq_eval(A_dev, b_dev, int(M), int(D), X_dev, int(N), int(precision), f_out_dev,
                               cuda_stream or None), "cupso_lsq_eval")


def cupso_set_lsq(h, A_dev, b_dev, M, precision):
    """A_dev, b_dev: device addresses (int) of A [M][D] and b [M], float32, borrowed."""
    _check(_lib.cupso_set_lsq(h, A_dev, b_dev, int(M), int(precision)), "cupso_set_lsq")


def cupso_get_gbest_f64(h):
    v = C.c_double()
    _check(_lib.cupso_get_gbest_f64(h, C.byref(v)), "cupso_get_gbest_f64")
    return float(v.value)


def _f64p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def cupso_create_fp64(D, N, bounds, w, c1, c2, fitness_id, seed):
    """Create a double-precision swarm and initialise it on the device."""
    h = C.c_void_p()
    lo, hi, vmax = bounds
    b = cupso_bounds_f64(float(lo), float(hi), float(vmax))
    _check(_lib.cupso_create_fp64(int(D), int(N), C.byref(b), float(w), float(c1), float(c2), int(fitness_id),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, C.byref(h)), "cupso_create_fp64")
    return h


def cupso_get_gbest_fp64(h, D, pos_out=None):
    """Returns (status, fit, idx, pos) of a double-precision swarm (as cupso_get_gbest)."""
    pos = pos_out if pos_out is not None else np.empty(int(D), np.float64)
    fit = C.c_double()
    idx = C.c_int64()
    rc = _lib.cupso_get_gbest_fp64(h, C.byref(fit), _f64p(pos), C.byref(idx))
    if rc not in (CUPSO_OK, CUPSO_ERR_DEVICE_TIMEOUT, CUPSO_ERR_NAN):
        raise CupsoError(rc, "cupso_get_gbest_fp64")
    return rc, float(fit.value), int(idx.value), pos


def cupso_get_state_fp64(h, N, D):
    pos, v, pb = (np.empty((N, D), np.float64) for _ in range(3))
    pf = np.empty(N, np.float64)
    t = C.c_uint32()
    _check(_lib.cupso_get_state_fp64(h, _f64p(pos), _f64p(v), _f64p(pb), _f64p(pf), C.byref(t)),
           "cupso_get_state_fp64")
    return {"pos": pos, "v": v, "pbest_pos": pb, "pbest_fit": pf, "t": int(t.value)}


def cupso_set_state_fp64(h, pos, v, pbest_pos, pbest_fit, t):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (pos, v, pbest_pos, pbest_fit)]
    _check(_lib.cupso_set_state_fp64(h, *[_f64p(a) for a in arrs], int(t)), "cupso_set_state_fp64")


def cupso_destroy(h):
    if h is not None and h.value:
        _check(_lib.cupso_destroy(h), "cupso_destroy")
        h.value = None


class Swarm:
    """Owning wrapper of one handle (marshalling only)."""

    def __init__(self, D, N, bounds, w, c1, c2, fitness, seed, mode=None, stream=None, dtype="f32"):
        """dtype "f32" (cupso_create) or "f64" (cupso_create_fp64, the paper's precision)."""
        fid = FITNESS[fitness] if isinstance(fitness, str) else int(fitness)
        self.D, self.N = int(D), int(N)
        self.fp64 = dtype == "f64"
        if dtype not in ("f32", "f64"):
            raise ValueError("dtype must be 'f32' or 'f64'")
        self.h = (cupso_create_fp64 if self.fp64 else cupso_create)(D, N, bounds, w, c1, c2, fid, seed)
        if stream is not None:
            cupso_set_stream(self.h, stream)
        if mode is not None:
            self.set_mode(mode)

    def set_mode(self, mode):
        cupso_set_option(self.h, CUPSO_OPT_MODE, MODES[mode] if isinstance(mode, str) else int(mode))

    def set_option(self, key, value):
        cupso_set_option(self.h, key, value)

    def set_stream(self, stream):
        cupso_set_stream(self.h, stream)

    def step(self, iters=1):
        cupso_step(self.h, iters)

    def gbest(self):
        if self.fp64:
            return cupso_get_gbest_fp64(self.h, self.D)
        return cupso_get_gbest(self.h, self.D)

    def gbest_post(self, slot):
        cupso_gbest_post(self.h, slot)

    def gbest_wait(self, slot, pos_out=None):
        return cupso_gbest_wait(self.h, self.D, slot, pos_out)

    def state(self):
        if self.fp64:
            return cupso_get_state_fp64(self.h, self.N, self.D)
        return cupso_get_state(self.h, self.N, self.D)

    def set_state(self, pos, v, pbest_pos, pbest_fit, t):
        if self.fp64:
            cupso_set_state_fp64(self.h, pos, v, pbest_pos, pbest_fit, t)
        else:
            cupso_set_state(self.h, pos, v, pbest_pos, pbest_fit, t)

    def info(self):
        return cupso_get_info(self.h)

    def set_lsq(self, A_dev, b_dev, M, precision):
        cupso_set_lsq(self.h, A_dev, b_dev, M, LSQ_PRECISIONS[precision] if isinstance(precision, str) else precision)

    def gbest_f64(self):
        return cupso_get_gbest_f64(self.h)

    def close(self):
        cupso_destroy(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None and self.h.value:
                _lib.cupso_destroy(self.h)
                self.h.value = None
        except Exception:
            pass
