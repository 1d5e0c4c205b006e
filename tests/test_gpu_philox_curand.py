"""The library's device Philox4x32-10 against cuRAND's Philox4_32_10
generator, a third-party implementation called through its documented
device API (needs a GPU and nvcc; the helper is compiled into a temporary
directory)."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import gpu_util as G
from paper_2606_09356_b300 import build as _build
from paper_2606_09356_b300 import soma

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_device_philox_matches_curand():
    G.lib()
    rng = np.random.default_rng(31)
    n = 4096
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    ctr[2] = [0xFFFFFFFF, 0xFFFFFFFF, 5, 0]  # carries across words 0-1 stay inside them
    with tempfile.TemporaryDirectory() as td:
        so = os.path.join(td, "libcurand_ref.so")
        subprocess.check_call([_build.NVCC] + _build.ARCH + ["-O2", "-shared", "-Xcompiler", "-fPIC", "-o", so,
                                                             os.path.join(HERE, "curand_philox_ref.cu")])
        L = ctypes.CDLL(so)
        L.curand_philox_words.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
        ref = np.zeros((n, 4), np.uint32)
        assert L.curand_philox_words(ctr.ctypes.data, key.ctypes.data, ref.ctypes.data, n) == 0
    got = soma.soma_philox4x32(ctr, key)
    bad = np.nonzero((got != ref).any(axis=1))[0]
    assert not len(bad), f"{len(bad)} of {n} counters differ from cuRAND (first {bad[:5]})"
