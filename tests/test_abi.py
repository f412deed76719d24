"""The C-ABI library: builds, loads and exports every declared symbol; host-side
argument checks; constants of the device code vs the oracle's. No GPU needed:
nothing here launches a kernel (invalid arguments are rejected before any CUDA
call)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cupso.h")
DEVICE_CUH = os.path.join(ROOT, "paper_2205_01313_gb300", "csrc", "cupso_device.cuh")


@pytest.fixture(scope="module")
def P():
    from paper_2205_01313_gb300 import build as B
    B.build()
    from paper_2205_01313_gb300 import cupso
    return cupso


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"CUPSO_API\s+(?:int|const char\*)\s+(cupso_\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cupso_create", "cupso_step", "cupso_get_gbest", "cupso_solve_batch", "cupso_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(P):
    lib = C.CDLL(P.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(P.ABI_FUNCTIONS) == declared_functions()


def _header_enum(prefix):
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(%s\w*)\s*=\s*(-?\d+)" % prefix, txt)}


def test_binding_constants_match_the_header(P):
    """Every option, mode, SYNC kernel and return code the header defines has
    the same value in the Python binding."""
    for prefix in ("CUPSO_OPT_", "CUPSO_MODE_", "CUPSO_ERR_", "CUPSO_OK"):
        for name, value in _header_enum(prefix).items():
            assert getattr(P, name) == value, name
    kernels = _header_enum("CUPSO_SYNC_KERNEL_")
    assert {k: kernels["CUPSO_SYNC_KERNEL_" + k.upper()] for k in P.SYNC_KERNELS} == P.SYNC_KERNELS
    assert len(P.SYNC_KERNELS) == len(kernels)


def test_info_struct_matches_the_header(P):
    """cupso_info's fields, in order, as the binding lays them out."""
    txt = open(HEADER).read()
    body = re.search(r"typedef struct \{((?:(?!typedef).)*?)\} cupso_info;", txt, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            names += [n.strip() for n in decl.split(None, 1)[1].split(",")]
    assert [f[0] for f in P.cupso_info._fields_] == names


def test_status_strings(P):
    assert P.status_string(0) == "ok"
    assert "timed out" in P.status_string(P.CUPSO_ERR_DEVICE_TIMEOUT)
    assert P.status_string(12345) == "unknown status"


@pytest.mark.parametrize("args", [
    dict(D=0, N=10), dict(D=3, N=0), dict(D=3, N=10, bounds=(1.0, -1.0, 1.0)),
    dict(D=3, N=10, bounds=(-1.0, 1.0, 0.0)), dict(D=3, N=10, bounds=(-1.0, float("inf"), 1.0)),
    dict(D=3, N=10, fid=9), dict(D=3, N=10, w=float("nan")), dict(D=1 << 16, N=1 << 16),
])
def test_invalid_arguments_rejected_on_host(P, args):
    D, N = args["D"], args["N"]
    b = P.cupso_bounds(*args.get("bounds", (-1.0, 1.0, 0.5)))
    h = C.c_void_p(1234)
    rc = P.lib().cupso_create(D, N, C.byref(b), args.get("w", 0.7), 1.5, 1.5, args.get("fid", 0), 1, C.byref(h))
    assert rc == P.CUPSO_ERR_INVALID_ARG
    assert h.value is None
    assert P.last_error() != ""


def test_result_slots_reject_a_null_handle(P):
    """The asynchronous gbest reads check their handle on the host."""
    lib = P.lib()
    f, i = C.c_float(), C.c_int64()
    assert lib.cupso_gbest_post(None, 0) == P.CUPSO_ERR_INVALID_ARG
    assert lib.cupso_gbest_wait(None, 0, C.byref(f), None, C.byref(i)) == P.CUPSO_ERR_INVALID_ARG


@pytest.mark.parametrize("args,code", [
    (dict(D=0, N=10), "INVALID_ARG"), (dict(D=3, N=10, bounds=(1.0, -1.0, 1.0)), "INVALID_ARG"),
    (dict(D=3, N=10, bounds=(-1.0, 1.0, -2.0)), "INVALID_ARG"), (dict(D=3, N=10, fid=9), "INVALID_ARG"),
    (dict(D=3, N=10, w=float("inf")), "INVALID_ARG"),
    (dict(D=3, N=10, fid=1), "UNSUPPORTED"), (dict(D=3, N=10, fid=2), "UNSUPPORTED"), (dict(D=3, N=10, fid=5), "UNSUPPORTED"),
])
def test_fp64_invalid_arguments_rejected_on_host(P, args, code):
    b = P.cupso_bounds_f64(*args.get("bounds", (-1.0, 1.0, 0.5)))
    h = C.c_void_p(1234)
    rc = P.lib().cupso_create_fp64(args["D"], args["N"], C.byref(b), args.get("w", 1.0), 2.0, 2.0,
                                   args.get("fid", 4), 1, C.byref(h))
    assert rc == getattr(P, "CUPSO_ERR_" + code)
    assert h.value is None


def test_null_handle_calls_rejected(P):
    L = P.lib()
    assert L.cupso_step(None, 1) == P.CUPSO_ERR_INVALID_ARG
    assert L.cupso_set_option(None, P.CUPSO_OPT_MODE, 1) == P.CUPSO_ERR_INVALID_ARG
    assert L.cupso_get_gbest(None, None, None, None) == P.CUPSO_ERR_INVALID_ARG
    assert L.cupso_get_gbest_fp64(None, None, None, None) == P.CUPSO_ERR_INVALID_ARG
    assert L.cupso_get_state_fp64(None, None, None, None, None, None) == P.CUPSO_ERR_INVALID_ARG
    assert L.cupso_destroy(None) == P.CUPSO_OK
    with pytest.raises(P.CupsoError) as e:
        P.cupso_solve_batch([dict(D=0, N=4, bounds=(-1, 1, 1), w=0.5, c1=1, c2=1, fitness_id=0, seed=1)], 3)
    assert e.value.code == P.CUPSO_ERR_INVALID_ARG
    with pytest.raises(P.CupsoError) as e:   # least squares needs A and b: no batch form
        P.cupso_solve_batch([dict(D=4, N=64, bounds=(-1, 1, 1), w=0.5, c1=1, c2=1, fitness_id=P.CUPSO_LSQ, seed=1)], 3)
    assert e.value.code == P.CUPSO_ERR_INVALID_ARG


def _cuh_floats(pattern):
    txt = open(DEVICE_CUH).read()
    return [np.float32(float.fromhex(h)) for h in re.findall(pattern, txt)]


def test_device_constants_equal_oracle_constants():
    """The literals hard-coded in the device code and the oracle's run-time
    constants are two independent roundings of the same real numbers."""
    body = open(DEVICE_CUH).read()
    cos_block = body[body.index("float cos2pi_poly"):body.index("__device__ __forceinline__ float cos2pi(")]
    lits = [np.float32(float.fromhex(h)) for h in re.findall(r"(-?0x[0-9a-f.]+p[+-]\d+)f", cos_block)]
    assert lits == list(O.cos2pi_coeffs()[::-1])  # written c7 .. c0
    exp_block = body[body.index("float exp_own"):body.index("// Fitness functions")]
    lits = [np.float32(float.fromhex(h)) for h in re.findall(r"(-?0x[0-9a-f.]+p[+-]\d+)f", exp_block)]
    c, log2e, hi, lo = O.exp_coeffs()
    assert lits[0] == log2e and lits[1] == hi and lits[2] == lo
    assert lits[3:] == list(c[::-1])
