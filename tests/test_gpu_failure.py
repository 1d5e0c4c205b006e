"""Failure detection without a GPU fault (needs a GPU): the bounded-wait
failure path of the move kernels reports SOMA_ETIMEOUT and leaves the
context usable; an allocator that runs dry makes soma_create fail cleanly
with SOMA_ENOMEM and every block it handed out comes back."""
import ctypes
import time

import numpy as np
import pytest
import torch

import gpu_util as G
from paper_2606_09356_b300 import soma, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


def test_bounded_wait_gives_up_and_the_context_survives():
    t0 = time.perf_counter()
    assert soma.soma_selfcheck_timeout(0, 100_000_000) == soma.SOMA_ETIMEOUT  # ~0.05 s of SM clock
    assert time.perf_counter() - t0 < 30.0
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    with soma.Handle(s, device=0) as h:
        h.mc_steps(3)
        h.sync()
        assert h.observables()["step"] == 3


def test_selfcheck_rejects_out_of_range_limits():
    assert soma.soma_selfcheck_timeout(0, 10) == soma.SOMA_EINVAL


class DryAllocator:
    """Device memory from torch's caching allocator; fails after `budget` blocks."""

    def __init__(self, budget):
        self.budget = budget
        self.live = {}
        self.alloc = soma._ALLOC(self._alloc)
        self.free = soma._FREE(self._free)

    def _alloc(self, nbytes, ctx):
        if len(self.live) >= self.budget:
            return None
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, ctx):
        self.live.pop(ptr, None)


@pytest.mark.parametrize("budget", [0, 3, 12])
def test_allocator_running_dry_fails_cleanly(budget):
    lib = G.lib()
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    d = (soma.soma_system_desc * 1)(s.desc())
    o = soma.soma_options_default()
    o.device = 0
    dry = DryAllocator(budget)
    o.alloc, o.free = dry.alloc, dry.free
    h = ctypes.c_void_p()
    assert lib.soma_create(d, 1, ctypes.byref(o), ctypes.byref(h)) == soma.SOMA_ENOMEM
    assert not h.value
    assert not dry.live  # everything handed out was returned


def test_allocator_with_enough_memory_runs_and_returns_everything():
    lib = G.lib()
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    d = (soma.soma_system_desc * 1)(s.desc())
    o = soma.soma_options_default()
    o.device = 0
    pool = DryAllocator(10_000)
    o.alloc, o.free = pool.alloc, pool.free
    h = ctypes.c_void_p()
    assert lib.soma_create(d, 1, ctypes.byref(o), ctypes.byref(h)) == soma.SOMA_OK
    assert pool.live
    assert lib.soma_mc_steps(h, 5, None) == soma.SOMA_OK
    assert lib.soma_sync(h, None) == soma.SOMA_OK
    counts = np.zeros((2, s.n_cells), np.uint32)
    assert lib.soma_get_density(h, 0, counts.ctypes.data_as(ctypes.c_void_p), counts.size, soma.SOMA_HOST) == 0
    assert counts.sum() == s.n_beads
    lib.soma_destroy(h)
    assert not pool.live
