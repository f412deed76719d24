"""Helpers shared by the GPU tests: build/load the library, run the oracle."""
import numpy as np
import pytest

from oracle import oracle as O

W, C12 = 0.729, 1.49445
BOUNDS = {0: (-100.0, 100.0, 20.0), 1: (-5.12, 5.12, 1.024), 2: (-32.768, 32.768, 6.5536),
          3: (-30.0, 30.0, 6.0), 4: (-100.0, 100.0, 20.0)}


def load_cupso():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2205_01313_gb300 import build as B
    B.build()
    from paper_2205_01313_gb300 import cupso
    torch.cuda.set_device(0)
    return cupso


def oracle_swarm(fid, N, D, seed, swarm=0, bounds=None, w=W, c1=C12, c2=C12):
    lo, hi, vmax = bounds or BOUNDS[fid]
    return O.Swarm(N, D, lo, hi, vmax, w, c1, c2, fid, seed, swarm=swarm)


def same_bits(a, b):
    """Element-wise identical float32 values (NaN == NaN, -0 != +0)."""
    a = np.ascontiguousarray(a, np.float32).view(np.uint32)
    b = np.ascontiguousarray(b, np.float32).view(np.uint32)
    return a.shape == b.shape and np.array_equal(a, b)


def assert_state_equal(st, ref):
    for name, refarr in (("pos", ref.pos), ("v", ref.v), ("pbest_pos", ref.pbest_pos), ("pbest_fit", ref.pbest_fit)):
        got = st[name]
        if not same_bits(got, refarr):
            diff = np.argwhere(got.view(np.uint32) != refarr.view(np.uint32))
            k = tuple(diff[0])
            raise AssertionError("%s differs at %d places, first %s: gpu %r oracle %r"
                                 % (name, len(diff), k, got[k], refarr[k]))


def ulp_distance(a, b):
    a = np.ascontiguousarray(a, np.float32).view(np.int32).astype(np.int64)
    b = np.ascontiguousarray(b, np.float32).view(np.int32).astype(np.int64)
    a = np.where(a < 0, -(a & 0x7FFFFFFF), a)
    b = np.where(b < 0, -(b & 0x7FFFFFFF), b)
    return np.abs(a - b)
