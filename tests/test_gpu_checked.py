"""The checked build (libsoma_debug.so, -DSOMA_DEBUG: device bounds checks on
every final cell, position and image counter of the move kernel) runs the
same shapes as the product library, at each block shape of the move kernel
(8, 12 and 24 consumer warps per CTA), with no check firing and
bit-identical results (needs a GPU).  Each library runs in its own
process."""
import json
import os
import subprocess
import sys

import pytest

from paper_2606_09356_b300 import build as _build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r'''
import hashlib, json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2606_09356_b300 import soma, workloads
soma.load_library(LIB)
shapes = [
    dict(workloads.system_kwargs("melt_512x32")),
    dict(workloads.system_kwargs("melt_512x32"), move=soma.SOMA_MOVE_SMART),
    dict(n_poly=37, N=7, n_A=3, box=(4.0, 4.5, 5.0), grid=(16, 18, 20), chiN=15.0, kappaN=40.0, seed=7),
    dict(n_poly=40, N=80, n_A=30, box=(2.0, 2.0, 2.0), grid=(8, 8, 8), chiN=25.0, kappaN=50.0, seed=7),
    dict(n_poly=200, N=1, n_A=1, box=(2.0, 2.0, 2.0), grid=(4, 4, 4), chiN=5.0, kappaN=10.0, A=0.25),
    dict(workloads.system_kwargs("melt_512x32"), move=soma.SOMA_MOVE_SMART, wall_z=1),
]
out = []
for kw, warps in [(kw, w) for kw in shapes for w in (8, 12, 24)]:
    s = soma.System(**kw)
    with soma.Handle(s, graph_steps=4, move_warps=warps) as h:
        h.mc_steps(30)
        nx = s.grid[0]
        pA = np.repeat(0.5 + 0.4 * np.sin(2 * np.pi * (np.arange(nx) + 0.5) / nx), s.grid[1] * s.grid[2])
        tg = np.stack([pA, 1 - pA]).astype(np.float32)
        h.place(tg)
        h.set_umbrella(tg, 30.0)
        h.mc_steps(30)
        h.sync()
        pos, img, step = h.get_state()
        out.append([hashlib.sha256(pos.tobytes() + img.tobytes()).hexdigest(), int(h.accepted()), int(step)])
print(json.dumps(out))
'''


def _run(lib):
    code = RUN.replace("ROOT", repr(ROOT)).replace("LIB", repr(lib))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_runs_clean_and_matches_release():
    _build.build()
    _build.build(debug=True)
    release = _run(_build.LIB)
    checked = _run(_build.LIB_DEBUG)
    assert checked == release
    # every block shape steps the same trajectory
    for i in range(0, len(release), 3):
        assert release[i] == release[i + 1] == release[i + 2]
