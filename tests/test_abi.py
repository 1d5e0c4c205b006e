"""The C-ABI library builds, loads and exports every entry point declared in
include/soma.h; struct layouts agree between C and the binding; argument
validation answers without touching a GPU.  CPU only."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2606_09356_b300 import build as _build
from paper_2606_09356_b300 import soma

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "soma.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s+(soma_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return soma.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} declared in soma.h but not exported"
    assert set(names) == set(soma.EXPORTS), "binding export list differs from the header"


def test_exported_symbols_are_c_linkage(lib):
    out = subprocess.check_output(["nm", "-D", "--defined-only", soma.LIBRARY]).decode()
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for n in declared_functions():
        assert n in syms


def test_struct_layouts_match_c():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "soma.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(soma_system_desc), sizeof(soma_options), sizeof(soma_obs),
         sizeof(soma_info), offsetof(soma_system_desc, box), offsetof(soma_system_desc, seed),
         offsetof(soma_options, alloc), offsetof(soma_options, move_warps));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "s.c")
        exe = os.path.join(td, "s")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", exe, c])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    exp = [ctypes.sizeof(soma.soma_system_desc), ctypes.sizeof(soma.soma_options), ctypes.sizeof(soma.soma_obs),
           ctypes.sizeof(soma.soma_info), soma.soma_system_desc.box.offset, soma.soma_system_desc.seed.offset,
           soma.soma_options.alloc.offset, soma.soma_options.move_warps.offset]
    assert got == exp


def test_strerror_and_defaults(lib):
    assert soma.soma_strerror(0) == "ok"
    assert "invalid" in soma.soma_strerror(soma.SOMA_EINVAL)
    o = soma.soma_options_default()
    assert o.device == -1 and o.graph_steps > 0 and o.hist_mode == soma.SOMA_HIST_AUTO


@pytest.mark.parametrize("bad", [
    dict(n_poly=0), dict(N=0), dict(n_A=33), dict(n_A=-1), dict(grid=(0, 4, 4)), dict(box=(0.0, 4.0, 4.0)),
    dict(box=(1.0, 4.0, 4.0)),          # shorter than two bond tails
    dict(N=1, n_A=1, A=0.0),            # no default proposal without bonds
    dict(A=5.0),                        # proposal wider than the box
    dict(chiN=float("nan")),
    dict(move=2),                       # unknown move kind
    dict(wall_z=2),                     # unknown z boundary
    dict(move=1, A=0.2),                # smart: drift A^2 (N-1)/2 above 1/2
    dict(move=1, N=1, n_A=1, A=0.7, box=(4.5, 4.5, 4.5)),  # smart: Gaussian tail wider than half the box
    dict(n_poly=(2**31 - 64) // 32 + 1),  # one chain past 2^31 - 65 beads
    dict(grid=(1024, 1024, 512)),         # 2^29 cells: past the cell limit
])
def test_create_rejects_bad_descriptors_without_gpu(lib, bad):
    kw = dict(n_poly=8, N=32, n_A=16, box=(4.0, 4.0, 4.0), grid=(4, 4, 4), chiN=1.0, kappaN=1.0)
    kw.update(bad)
    d = soma.System(**kw).desc()
    arr = (soma.soma_system_desc * 1)(d)
    h = ctypes.c_void_p()
    assert lib.soma_create(arr, 1, None, ctypes.byref(h)) == soma.SOMA_EINVAL
    assert not h.value


def test_create_rejects_more_than_2_32_chains_in_one_handle_without_gpu(lib):
    """Each system is within its own limits, but the chain reorder numbers
    the chains of all systems of a handle in 32 bits."""
    n = 2**31 - 65
    ds = [soma.System(n_poly=n, N=1, n_A=1, box=(4.0, 4.0, 4.0), grid=(4, 4, 4), chiN=0.0, kappaN=1.0, A=0.1,
                      system_id=i).desc() for i in range(3)]
    h = ctypes.c_void_p()
    assert lib.soma_create((soma.soma_system_desc * 3)(*ds), 3, None, ctypes.byref(h)) == soma.SOMA_EINVAL
    assert not h.value


@pytest.mark.parametrize("kw,opts", [
    (dict(N=80, n_A=40, move=1), None),                          # smart moves: register path only
    (dict(N=32, n_A=16, move=1), dict(precision=1)),             # smart moves: FP32 form only
    (dict(N=32, n_A=16, wall_z=1), dict(precision=1)),           # walls: FP32 form only
])
def test_create_rejects_unsupported_smart_moves_without_gpu(lib, kw, opts):
    d = soma.System(n_poly=8, box=(4.0, 4.0, 4.0), grid=(4, 4, 4), chiN=1.0, kappaN=1.0, **kw).desc()
    arr = (soma.soma_system_desc * 1)(d)
    o = soma.soma_options_default()
    for k, v in (opts or {}).items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    assert lib.soma_create(arr, 1, ctypes.byref(o), ctypes.byref(h)) == soma.SOMA_ENOTSUP
    assert not h.value


def test_null_arguments(lib):
    assert lib.soma_create(None, 1, None, None) == soma.SOMA_EINVAL
    assert lib.soma_mc_steps(None, 1, None) == soma.SOMA_EINVAL
    assert lib.soma_observables(None, 0, None) == soma.SOMA_EINVAL
    lib.soma_destroy(None)
    assert lib.soma_philox4x32(None, None, None, 0) == soma.SOMA_OK
    # every handle call rejects a NULL handle before touching the device
    assert lib.soma_set_conversion(None, 0, 1, 0.0, 0.0, None) == soma.SOMA_EINVAL
    assert lib.soma_get_conversions(None, 0, None) == soma.SOMA_EINVAL
    assert lib.soma_get_chain_types(None, 0, None, 0) == soma.SOMA_EINVAL
    assert lib.soma_set_chain_types(None, 0, None, 0) == soma.SOMA_EINVAL
    assert lib.soma_copy_accepted(None, 0, None, None) == soma.SOMA_EINVAL
    assert lib.soma_set_umbrella(None, 0, None, 0, 0.0, 0) == soma.SOMA_EINVAL
    assert lib.soma_place(None, 0, None, 0, 0) == soma.SOMA_EINVAL


def test_noalloc_binding_checks_buffers_before_the_c_call(lib, monkeypatch):
    # A wrongly typed, short or host-side S (or pos) is refused in the binding,
    # before the C call could write or read past it on the device.
    import numpy as np
    import torch

    def no_c_call():
        raise AssertionError("the C call was reached")

    monkeypatch.setattr(soma, "load_library", no_c_call)
    m = np.ones((5, 3), np.int32)
    pos = torch.zeros((64, 3), dtype=torch.float32)
    cases = [
        (pos, torch.zeros(5, dtype=torch.float32), "S"),       # FP32 instead of FP64
        (pos, torch.zeros(4, dtype=torch.float64), "S"),       # shorter than nq
        (pos[:32], torch.zeros(5, dtype=torch.float64), "pos"),  # fewer than 3 n_beads floats
        (pos.t(), torch.zeros(5, dtype=torch.float64), "pos"),   # not contiguous
        (pos, torch.zeros(5, dtype=torch.float64), "CUDA"),    # host tensors on a CPU machine
    ]
    for p, S, what in cases:
        with pytest.raises(ValueError, match=what):
            soma.soma_structure_factor_noalloc(p, 64, 32, 16, (4.0, 4.0, 4.0), m, S)
    with pytest.raises(ValueError, match="box"):
        soma.soma_structure_factor_noalloc(pos, 64, 32, 16, (4.0, 4.0), m, torch.zeros(5, dtype=torch.float64))
