"""The largest systems the ABI accepts (needs a GPU with about 200 GB free).

A system may hold up to 2^31 - 65 beads.  Two shapes at that limit: 67,108,861
chains of 32 beads on a 512^3 grid (2,147,483,552 beads, 16 per cell), and
2,147,483,583 single beads (N = 1, no bonds; 32 chains per warp, one bead per
lane) on a 256^3 grid.  After each step: the count sums equal the bead
numbers of each type, a sample of chains (the first and the last among them)
moves as the oracle moves them with the full system's fields, and the whole
grid equals a plain PyTorch binning of the GPU's positions by the same FP32
cell rule, done in chunks on the device.
"""
import numpy as np
import pytest

import gpu_util as G
from paper_2606_09356_b300 import soma

pytestmark = pytest.mark.gpu

LIMIT = 2**31 - 65

SHAPES = {
    "chains32": dict(n_poly=LIMIT // 32, N=32, n_A=16, box=(64.0, 64.0, 64.0), grid=(512, 512, 512), chiN=30.0,
                     kappaN=50.0, seed=7),
    "beads1": dict(n_poly=LIMIT, N=1, n_A=1, box=(32.0, 32.0, 32.0), grid=(256, 256, 256), chiN=0.0, kappaN=50.0,
                   A=0.1, seed=8),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


def _grid_counts(torch, s, pos_d):
    """[type][cell] counts of the positions by the cell rule: the FP32 product
    x (n/L), floored, clamped to n - 1; bead i < n_A is type A."""
    n = s.grid
    cps = [np.float32(n[a] / s.box[a]) for a in range(3)]
    out = torch.zeros(2 * s.n_cells, dtype=torch.int64, device=pos_d.device)
    chunk = (1 << 28) // s.N * s.N
    for b0 in range(0, s.n_beads, chunk):
        p = pos_d[b0:b0 + chunk]
        idx = [torch.clamp(torch.floor(p[:, a] * float(cps[a])), max=n[a] - 1).to(torch.int64) for a in range(3)]
        cell = (idx[0] * n[1] + idx[1]) * n[2] + idx[2]
        typ = (torch.arange(b0, b0 + p.shape[0], device=p.device, dtype=torch.int64) % s.N >= s.n_A).to(torch.int64)
        out += torch.bincount(typ * s.n_cells + cell, minlength=2 * s.n_cells)
        del p, idx, cell, typ
    return out.view(2, s.n_cells)


@pytest.mark.parametrize("shape", sorted(SHAPES))
def test_largest_system(shape):
    import torch
    s = soma.System(**SHAPES[shape])
    assert LIMIT - s.N < s.n_beads <= LIMIT
    need = 76 * s.n_beads + 72 * s.n_cells + (24 << 30)  # handle, sample buffers, chunked binning
    free, _ = torch.cuda.mem_get_info()
    if free < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")
    orc = G.oracle_for(s)
    k_b, _, _ = orc.params()
    band = G.band_for(s, k_b)
    N = s.N
    rng = np.random.default_rng(23)
    ids = np.unique(np.concatenate([[0, s.n_poly - 1], rng.choice(s.n_poly, 1022, replace=False)])).astype(np.uint32)
    sel = (ids[:, None].astype(np.int64) * N + np.arange(N)[None, :]).reshape(-1)
    box = np.array(s.box)
    pos_d = torch.empty((s.n_beads, 3), dtype=torch.float32, device="cuda")
    img_d = torch.empty((s.n_beads, 3), dtype=torch.int16, device="cuda")
    sel_d = torch.from_numpy(sel).cuda()

    def sample():
        _, _, step = h.get_state(pos=pos_d, img=img_d)
        torch.cuda.synchronize()
        p = pos_d[sel_d].double().cpu().numpy() + img_d[sel_d].double().cpu().numpy() * box
        return p, step

    with soma.Handle(s, graph_steps=0, sort_interval=0) as h:
        h.mc_steps(1)
        for _ in range(2):
            X0, step = sample()
            counts = h.get_density()
            assert counts[0].sum(dtype=np.int64) == s.n_poly * s.n_A
            assert counts[1].sum(dtype=np.int64) == s.n_poly * (N - s.n_A)
            w = orc.fields(counts)
            del counts
            Xs = X0.copy()  # the oracle moves the sample in place
            _, acc, margin, face = orc.mc_step_chains(Xs, ids, w, step, n_threads=G.NTHREADS)
            del w
            h.mc_steps(1)
            X1, _ = sample()
            moved = np.any(X1 != X0, axis=1)
            face_tol = 8.0 * float(np.spacing(np.float32(max(s.box))))
            sus = ((np.abs(margin) < band) | (face < face_tol)).reshape(-1, N)
            spread = sus.copy()
            spread[:, 1:] |= sus[:, :-1]
            spread[:, :-1] |= sus[:, 1:]
            ok = ~spread.reshape(-1)
            assert ok.mean() > 0.9  # most of the sample lies outside the decision band
            assert not (ok & (moved != acc.astype(bool))).any()
            assert (np.abs(X1 - Xs)[ok] / box).max() <= 1e-5
        # the whole grid from the final positions
        h.get_state(pos=pos_d, img=img_d)
        ref = _grid_counts(torch, s, pos_d)
        got = torch.from_numpy(h.get_density().astype(np.int64)).cuda()
        assert torch.equal(ref, got)
        assert h.accepted() > 0
