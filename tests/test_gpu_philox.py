"""Philox4x32-10 on the GPU: the library's device function, cuRAND's
Philox4_32_10 (a library, independent of this project) and the CPU oracle give
the same words for the same (counter, key)."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_common import load_cupso

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    load_cupso()
    out = str(tmp_path_factory.mktemp("philox") / "philox_check.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", os.path.join(HERE, "cuda", "philox_check.cu"), "-o", out], check=True)
    L = C.CDLL(out)
    L.philox_check.argtypes = [C.c_void_p, C.c_int, C.c_uint, C.c_uint, C.c_void_p, C.c_void_p]
    L.philox_check.restype = C.c_int
    return L


def test_device_philox_equals_curand_and_oracle(checker):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, (4096, 4), dtype=np.uint64).astype(np.uint32)
    # cuRAND reaches counter (c0, c1) through a 64-bit offset of 4 (c0 + 2^32 c1) words,
    # so c1 must stay below 2^30 (the library's c1 is a particle index).
    ctr[:, 1] &= 0x3FFFFFFF
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF, 0x3FFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF], [5, 17, 3, 0], [1, 2, 0xFFFFFFFF, 7]]
    for key in [(1, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0x89ABCDEF, 0x01234567)]:
        own = np.zeros_like(ctr)
        ref = np.zeros_like(ctr)
        assert checker.philox_check(ctr.ctypes.data, len(ctr), key[0], key[1], own.ctypes.data, ref.ctypes.data) == 0
        np.testing.assert_array_equal(own, ref)
        for k in range(0, len(ctr), 97):
            assert O.philox4x32_10(ctr[k], key) == [int(x) for x in own[k]]
