"""The library's stable radix sort (the sort of the chain reorder) against
numpy's stable argsort, bit for bit: sizes around its 1,024-item tiles,
ragged sizes, heavily repeated keys (stability), several key widths."""
import numpy as np
import pytest

import gpu_util as G
from paper_2606_09356_b300 import soma

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


@pytest.mark.parametrize("n", [1, 2, 31, 1023, 1024, 1025, 4095, 4097, 8192 + 511, 100003, (1 << 20) + 7])
@pytest.mark.parametrize("end_bit,distinct", [(46, None), (64, None), (40, 50), (8, None)])
def test_sort_matches_numpy_stable_argsort(n, end_bit, distinct):
    rng = np.random.default_rng(n * 131 + end_bit)
    if distinct:  # few distinct keys: the order among equals must be the input order
        keys = rng.choice(rng.integers(0, 2**63, size=distinct, dtype=np.uint64), size=n)
    else:
        keys = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n,
                                                                                          dtype=np.uint64)
    vals = rng.permutation(n).astype(np.uint32)
    mask = np.uint64((1 << end_bit) - 1) if end_bit < 64 else np.uint64(2**64 - 1)
    order = np.argsort(keys & mask, kind="stable")
    ko, vo = soma.soma_sort_pairs(keys, vals, end_bit)
    assert np.array_equal(ko, keys[order]) and np.array_equal(vo, vals[order])


def test_sort_arguments():
    k = np.arange(4, dtype=np.uint64)
    v = np.arange(4, dtype=np.uint32)
    for bad in (0, 65):
        with pytest.raises(soma.SomaError) as e:
            soma.soma_sort_pairs(k, v, bad)
        assert e.value.code == soma.SOMA_EINVAL
    ko, vo = soma.soma_sort_pairs(k[:0], v[:0], 8)
    assert ko.size == 0 and vo.size == 0
