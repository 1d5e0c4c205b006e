"""Pins of the oracle against facts that do not come from the oracle itself.

Each ``pin_*`` function takes an oracle class (``oracle.Oracle`` or a build of
a mutated copy of its source) and returns a list of failure strings; an empty
list means the pin holds.  The facts used:

* Philox4x32-10: an independent implementation (Triton's, on its CPU
  interpreter) of the generator of Salmon et al. (SC'11); chi-square
  uniformity of the top and low bytes of 2^20 words.
* Gaussian-chain statistics of the initial configuration and of the
  chiN = kappaN = 0 dynamics: per-axis bond variance 1/(3(N-1)), <R_e^2> = 1,
  <R_g^2> = (N+1)/(6N); the harmonic chain's Boltzmann law is stationary.
* Acceptance at chiN = kappaN = 0: for a bead whose conditional position is
  Gaussian, dE given the displacement d is normal with variance twice its mean,
  so E[min(1, e^-dE)] = erfc(sqrt(mean)/2); averaged over the uniform cube.
* One bead in a frozen field: cell occupancy proportional to exp(-w(c)).
* An AB dimer on a 2^3 grid in a frozen field: the exact cell-pair law
  P(c1, c2) ~ exp(-w_A(c1) - w_B(c2)) prod_axes K(c1_a, c2_a), with K the
  Gaussian bond kernel integrated over a pair of periodic cells (erf sums).
* Density counts: brute-force numpy binning and the bead-count invariants.
* Fields: the exact central difference of the energy functional H_nb, and the
  exchange field chiN (phiB - phiA)/N of an incompressible cell.
* S(q) of ideal chains: (1/N) sum_ij s_i s_j exp(-q^2 |i-j| / (6(N-1))).
* Observables: rigid straight and right-angle chains (R_e^2, R_g^2 and the
  bond energy by hand), equipartition of the harmonic bond energy and the
  Gaussian-chain R_e^2, R_g^2 read through the observables themselves.
* Non-bonded energy: its absolute value on counts built by hand (uniform
  symmetric melt n_poly chiN/4, a one-cell excess, two hand-worked cells);
  the umbrella energy likewise.
* Model constants: k_b, the proposal half-width and rho_bar of the melt
  workloads as their definitions print them.
* A sample of chains stepped alone moves as inside the whole system.
* Umbrella fields: the exact central difference of H_nb + H_umb.
* Placement from target fields: the exact law of the bead-0 cell, the
  quantised target weights convolved with the uniform offset (piecewise-
  linear integrals, integrated exactly between their kinks), and Gaussian
  bond statistics of the placed chains.
* Boundary-zone conversion: the two-state Markov law of a molecule's type
  in a zone (binomial type counts after t steps), the binomial zone
  occupancy of the uniform bead 0 under certain flips, the Boltzmann law of
  a converted bead's type, and the ideal-chain S(q) of a two-type mixture.
"""
import os
import subprocess
import sys
import tempfile

import numpy as np
from numpy.polynomial.legendre import leggauss
from scipy.special import erf, erfc

NTHREADS = max(1, min(8, os.cpu_count() or 1))
HERE = os.path.dirname(os.path.abspath(__file__))


def _gl(a, b, n):
    x, w = leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (a + b), 0.5 * (b - a) * w


def _check(fails, name, value, expect, tol):
    if not (abs(value - expect) <= tol):
        fails.append(f"{name}: got {value:.6g}, expected {expect:.6g} +- {tol:.3g}")


# ---------------------------------------------------------------------------
def pin_philox_triton(O, n=512, seed=12345):
    rng = np.random.default_rng(seed)
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    with tempfile.TemporaryDirectory() as td:
        pc, pk, po = (os.path.join(td, f) for f in ("c.npy", "k.npy", "o.npy"))
        np.save(pc, ctr)
        np.save(pk, key)
        subprocess.check_call([sys.executable, os.path.join(HERE, "triton_philox_ref.py"), pc, pk, po])
        ref = np.load(po)
    got = O.philox(ctr, key)
    bad = np.nonzero((got != ref).any(axis=1))[0]
    return [f"philox differs from Triton's at {len(bad)} of {n} counters"] if len(bad) else []


def pin_philox_uniformity(O, n=1 << 18):
    """Chi-square of the top byte and of the low byte of 4n words from
    consecutive counters (256 bins each): within the 1e-4 tails of the
    chi-square law with 255 degrees of freedom."""
    from scipy.stats import chi2
    fails = []
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 2] = 7
    key = np.tile(np.array([[0x12345678, 0x9ABCDEF0]], np.uint32), (n, 1))
    w = O.philox(ctr, key).reshape(-1)
    lo, hi = chi2.ppf(1e-4, 255), chi2.ppf(1 - 1e-4, 255)
    for name, b in (("top byte", w >> 24), ("low byte", w & 0xFF)):
        cnt = np.bincount(b.astype(np.int64), minlength=256)
        e = w.size / 256
        x2 = float(((cnt - e) ** 2 / e).sum())
        if not (lo < x2 < hi):
            fails.append(f"philox {name} chi-square {x2:.1f} outside ({lo:.1f}, {hi:.1f})")
    return fails


# ---------------------------------------------------------------------------
def pin_init_statistics(O):
    fails = []
    n_poly, N = 8192, 16
    o = O(n_poly, N, 8, (4.0, 4.0, 4.0), (16, 16, 16), 0.0, 0.0, seed=7)
    pos = o.init().reshape(n_poly, N, 3)
    b = np.diff(pos, axis=1)
    nb = b.shape[0] * b.shape[1]
    for a in range(3):
        v = (b[:, :, a] ** 2).mean() * 3 * (N - 1)
        _check(fails, f"bond variance axis {a} x 3(N-1)", v, 1.0, 5 * np.sqrt(2.0 / nb))
    kurt = (b ** 4).mean() / ((b ** 2).mean() ** 2)
    _check(fails, "bond kurtosis", kurt, 3.0, 0.05)
    re2 = ((pos[:, -1] - pos[:, 0]) ** 2).sum(-1)
    _check(fails, "<R_e^2>", re2.mean(), 1.0, 5 * np.sqrt(2.0 / 3.0 / n_poly))
    cm = pos.mean(axis=1, keepdims=True)
    rg2 = ((pos - cm) ** 2).sum(-1).mean(-1)
    _check(fails, "<R_g^2>", rg2.mean(), (N + 1) / (6.0 * N), 5 * rg2.std() / np.sqrt(n_poly))
    x0 = pos[:, 0]
    if x0.min() < 0 or x0.max() >= 4.0:
        fails.append("first bead outside the box")
    for a in range(3):
        _check(fails, f"first bead mean axis {a}", x0[:, a].mean(), 2.0, 5 * np.sqrt(16 / 12 / n_poly))
    return fails


# ---------------------------------------------------------------------------
def _acceptance_ideal(N, A, kb, n=64):
    x, w = _gl(0.0, A, n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :] / A ** 3
    D = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    a_int = float((W * erfc(D * np.sqrt(kb / 2.0))).sum())
    a_end = float((W * erfc(D * np.sqrt(kb) / 2.0)).sum())
    return ((N - 2) * a_int + 2 * a_end) / N


def pin_ideal_dynamics(O, steps=120):
    """chiN = kappaN = 0: equilibrium bond statistics persist and the
    acceptance equals the Gaussian quadrature."""
    fails = []
    n_poly, N = 2048, 32
    o = O(n_poly, N, 16, (4.0, 4.0, 4.0), (16, 16, 16), 0.0, 0.0, seed=3)
    kb, A, _ = o.params()
    pos = o.init()
    res = o.run(pos, 0, steps, n_threads=NTHREADS, re2_trace=True, acc_trace=True)
    acc = res["accepted"] / (o.n_b * steps)
    expect = _acceptance_ideal(N, A, kb)
    _check(fails, "acceptance vs quadrature", acc, expect, 5 * np.sqrt(expect * (1 - expect) / (o.n_b * steps)) + 2e-4)
    p = pos.reshape(n_poly, N, 3)
    b2 = (np.diff(p, axis=1) ** 2).sum(-1).mean() * (N - 1)
    _check(fails, "<b^2>(N-1) after the run", b2, 1.0, 5 * np.sqrt(2.0 / 3.0 / (n_poly * (N - 1))))
    _check(fails, "time-averaged <R_e^2>", res["re2"].mean(), 1.0, 5 * np.sqrt(2.0 / 3.0 / n_poly))
    return fails


# ---------------------------------------------------------------------------
def _block_test(fails, name, samples, expect, zmax=5.5):
    """samples: [blocks, states] normalised frequencies; compare to expect."""
    mean = samples.mean(axis=0)
    se = samples.std(axis=0, ddof=1) / np.sqrt(samples.shape[0])
    se = np.maximum(se, 1e-12)
    z = (mean - expect) / se
    k = int(np.argmax(np.abs(z)))
    if abs(z[k]) > zmax:
        fails.append(f"{name}: state {k} freq {mean[k]:.5f} vs exact {expect[k]:.5f} (z={z[k]:.1f})")
    rel = np.abs(mean - expect).max()
    if rel > 0.01:
        fails.append(f"{name}: max abs deviation {rel:.4f}")


def pin_single_bead_field(O, blocks=16, per_block=15):
    fails = []
    rng = np.random.default_rng(11)
    for n_A, t in ((1, 0), (0, 1)):
        o = O(4096, 1, n_A, (1.0, 1.5, 2.0), (2, 3, 4), 0.0, 0.0, A=0.6, seed=5 + n_A)
        w = rng.normal(0.0, 0.8, size=(2, o.n_c))
        pos = o.init()
        o.run(pos, 0, 10, w_frozen=w, n_threads=NTHREADS)  # burn-in from the uniform start
        samples = []
        for b in range(blocks):
            r = o.run(pos, 10 + b * per_block, per_block, w_frozen=w, n_threads=NTHREADS, occ=True)
            occ = r["occ"].reshape(2, o.n_c)[t].astype(np.float64)
            samples.append(occ / occ.sum())
        p = np.exp(-w[t])
        _block_test(fails, f"single bead type {'AB'[t]} occupancy", np.array(samples), p / p.sum())
    return fails


# ---------------------------------------------------------------------------
def _bond_cell_kernel(L, n, kb, nx=96, images=6):
    """K[i, j] = int_{x in cell i} dx int db exp(-kb b^2) [x + b in cell j mod L]."""
    h = L / n
    K = np.zeros((n, n))
    s = np.sqrt(kb)
    for i in range(n):
        x, wx = _gl(i * h, (i + 1) * h, nx)
        for j in range(n):
            tot = np.zeros_like(x)
            for m in range(-images, images + 1):
                y0, y1 = j * h + m * L, (j + 1) * h + m * L
                tot += 0.5 * np.sqrt(np.pi / kb) * (erf(s * (y1 - x)) - erf(s * (y0 - x)))
            K[i, j] = (wx * tot).sum()
    return K


def pin_dimer_cell_pairs(O, blocks=16, per_block=15):
    fails = []
    rng = np.random.default_rng(21)
    box, grid = (1.0, 1.0, 1.0), (2, 2, 2)
    o = O(4096, 2, 1, box, grid, 0.0, 0.0, seed=9)
    kb, _, _ = o.params()
    w = rng.normal(0.0, 0.7, size=(2, o.n_c))
    Ks = [_bond_cell_kernel(box[a], grid[a], kb) for a in range(3)]
    cells = [(ix, iy, iz) for ix in range(2) for iy in range(2) for iz in range(2)]
    P = np.zeros((o.n_c, o.n_c))
    for c1, (a1, b1, z1) in enumerate(cells):
        for c2, (a2, b2, z2) in enumerate(cells):
            P[c1, c2] = np.exp(-w[0, c1] - w[1, c2]) * Ks[0][a1, a2] * Ks[1][b1, b2] * Ks[2][z1, z2]
    P /= P.sum()
    pos = o.init()
    o.run(pos, 0, 20, w_frozen=w, n_threads=NTHREADS)
    samples = []
    for b in range(blocks):
        r = o.run(pos, 20 + b * per_block, per_block, w_frozen=w, n_threads=NTHREADS, pair_hist=True)
        h = r["pair_hist"].astype(np.float64)
        samples.append(h / h.sum())
    _block_test(fails, "AB dimer cell-pair law", np.array(samples), P.reshape(-1))
    return fails


# ---------------------------------------------------------------------------
def pin_density_bruteforce(O):
    fails = []
    rng = np.random.default_rng(31)
    box, grid = (2.0, 3.0, 4.0), (8, 12, 16)
    n_poly, N, n_A = 300, 10, 4
    o = O(n_poly, N, n_A, box, grid, 0.0, 0.0, seed=1)
    pos = rng.uniform(-7.0, 9.0, size=(o.n_b, 3))
    pos[:5] = [[0.0, 0.0, 0.0], [2.0, 3.0, 4.0], [-2.0, -3.0, -4.0], [1.999999, 2.999999, 3.999999], [-1e-9, 0.25, 0.5]]
    got = o.density(pos)
    idx = []
    for a in range(3):
        xw = np.mod(pos[:, a], box[a])
        i = np.floor(xw * (grid[a] / box[a])).astype(np.int64)
        idx.append(np.clip(i, 0, grid[a] - 1))
    cell = (idx[0] * grid[1] + idx[1]) * grid[2] + idx[2]
    types = (np.arange(o.n_b) % N >= n_A).astype(np.int64)
    ref = np.zeros((2, o.n_c), np.int64)
    np.add.at(ref, (types, cell), 1)
    if not np.array_equal(got.astype(np.int64), ref):
        fails.append(f"density differs from brute force in {(got != ref).sum()} cells")
    if got[0].sum() != n_poly * n_A or got[1].sum() != n_poly * (N - n_A):
        fails.append("count sums differ from bead counts")
    return fails


def pin_fields_derivative(O):
    fails = []
    rng = np.random.default_rng(41)
    o = O(64, 16, 5, (2.0, 2.0, 2.0), (4, 4, 4), 23.0, 47.0, seed=1)
    counts = rng.integers(0, 40, size=(2, o.n_c)).astype(np.uint32)
    w = o.fields(counts)
    for t in range(2):
        for c in rng.choice(o.n_c, 12, replace=False):
            up, dn = counts.copy(), counts.copy()
            up[t, c] += 1
            dn[t, c] -= 1
            fd = (o.energy_nb(up) - o.energy_nb(dn)) / 2.0
            _check(fails, f"w[{t},{c}] vs dH/dn", w[t, c], fd, 1e-9 * max(1.0, abs(fd)) + 1e-9)
    _, _, rho = o.params()
    nA = rng.integers(0, 20, size=o.n_c)
    phiA = nA / rho
    inc = np.stack([phiA, 1.0 - phiA])
    wi = o.fields_from_phi(inc)
    _check(fails, "incompressible exchange field", float(np.abs((wi[0] - wi[1]) - 23.0 * (inc[1] - inc[0]) / 16).max()), 0.0, 1e-12)
    return fails


# ---------------------------------------------------------------------------
def pin_structure_factor_ideal(O, seeds=12):
    fails = []
    n_poly, N, n_A, L = 2048, 16, 8, 4.0
    ms = [(x, y, z) for x in range(-2, 3) for y in range(-2, 3) for z in range(-2, 3)
          if 0 < x * x + y * y + z * z <= 6]
    ms = np.array(ms, np.int32)
    shells = (ms ** 2).sum(1)
    s = np.where(np.arange(N) < n_A, 1.0, -1.0)
    ij = np.abs(np.arange(N)[:, None] - np.arange(N)[None, :])
    est = {k: [] for k in np.unique(shells)}
    for sd in range(seeds):
        o = O(n_poly, N, n_A, (L, L, L), (16, 16, 16), 0.0, 0.0, seed=100 + sd)
        S = o.structure_factor(o.init(), ms)
        for k in est:
            est[k].append(S[shells == k].mean())
    for k, v in est.items():
        q2 = (2 * np.pi / L) ** 2 * k
        exact = float((s[:, None] * s[None, :] * np.exp(-q2 * ij / (6.0 * (N - 1)))).sum() / N)
        v = np.array(v)
        se = v.std(ddof=1) / np.sqrt(len(v))
        _check(fails, f"S(q) shell |m|^2={k}", v.mean(), exact, 5 * se)
    return fails


# ---------------------------------------------------------------------------
# Bond-force-biased (smart) moves: detailed balance makes the same Boltzmann
# laws stationary, so the same closed forms pin them.
def pin_smart_ideal_dynamics(O, steps=300):
    fails = []
    n_poly, N = 4096, 32
    o = O(n_poly, N, 16, (4.0, 4.0, 4.0), (16, 16, 16), 0.0, 0.0, seed=13, move=1)
    pos = o.init()
    res = o.run(pos, 0, steps, n_threads=NTHREADS, re2_trace=True)
    p = pos.reshape(n_poly, N, 3)
    b2 = (np.diff(p, axis=1) ** 2).sum(-1).mean() * (N - 1)
    _check(fails, "smart: <b^2>(N-1) after the run", b2, 1.0, 5 * np.sqrt(2.0 / 3.0 / (n_poly * (N - 1))))
    _check(fails, "smart: time-averaged <R_e^2>", res["re2"].mean(), 1.0, 5 * np.sqrt(2.0 / 3.0 / n_poly))
    acc = res["accepted"] / (o.n_b * steps)
    if not (0.5 < acc < 1.0):
        fails.append(f"smart: acceptance {acc:.3f} outside (0.5, 1)")
    return fails


def pin_smart_single_bead_field(O, blocks=16, per_block=15):
    fails = []
    rng = np.random.default_rng(12)
    o = O(4096, 1, 1, (1.0, 1.5, 2.0), (2, 3, 4), 0.0, 0.0, A=0.6, seed=15, move=1)
    w = rng.normal(0.0, 0.8, size=(2, o.n_c))
    pos = o.init()
    o.run(pos, 0, 10, w_frozen=w, n_threads=NTHREADS)
    samples = []
    for b in range(blocks):
        r = o.run(pos, 10 + b * per_block, per_block, w_frozen=w, n_threads=NTHREADS, occ=True)
        occ = r["occ"].reshape(2, o.n_c)[0].astype(np.float64)
        samples.append(occ / occ.sum())
    p = np.exp(-w[0])
    _block_test(fails, "smart single bead occupancy", np.array(samples), p / p.sum())
    return fails


def pin_smart_dimer_cell_pairs(O, blocks=16, per_block=15):
    fails = []
    rng = np.random.default_rng(22)
    box, grid = (1.0, 1.0, 1.0), (2, 2, 2)
    o = O(4096, 2, 1, box, grid, 0.0, 0.0, seed=19, move=1)
    kb, _, _ = o.params()
    w = rng.normal(0.0, 0.7, size=(2, o.n_c))
    Ks = [_bond_cell_kernel(box[a], grid[a], kb) for a in range(3)]
    cells = [(ix, iy, iz) for ix in range(2) for iy in range(2) for iz in range(2)]
    P = np.zeros((o.n_c, o.n_c))
    for c1, (a1, b1, z1) in enumerate(cells):
        for c2, (a2, b2, z2) in enumerate(cells):
            P[c1, c2] = np.exp(-w[0, c1] - w[1, c2]) * Ks[0][a1, a2] * Ks[1][b1, b2] * Ks[2][z1, z2]
    P /= P.sum()
    pos = o.init()
    o.run(pos, 0, 20, w_frozen=w, n_threads=NTHREADS)
    samples = []
    for b in range(blocks):
        r = o.run(pos, 20 + b * per_block, per_block, w_frozen=w, n_threads=NTHREADS, pair_hist=True)
        h = r["pair_hist"].astype(np.float64)
        samples.append(h / h.sum())
    _block_test(fails, "smart AB dimer cell-pair law", np.array(samples), P.reshape(-1))
    return fails


def pin_normal_quantile(O):
    """The oracle's inverse normal CDF against scipy's (a library routine of
    the same definition) and the symmetry Phi^-1(1 - p) = -Phi^-1(p)."""
    from scipy.special import ndtri
    fails = []
    for p in (2.0 ** -25, 1e-6, 0.01, 0.2, 0.5, 0.7, 0.999, 1 - 2.0 ** -25):
        _check(fails, f"quantile({p})", O.normal_quantile(p), float(ndtri(p)), 1e-9)
        _check(fails, f"symmetry({p})", O.normal_quantile(1 - p) + O.normal_quantile(p), 0.0, 1e-8)
    return fails


# ---------------------------------------------------------------------------
def pin_umbrella_fields_derivative(O):
    fails = []
    rng = np.random.default_rng(43)
    o = O(64, 16, 5, (2.0, 2.0, 2.0), (4, 4, 4), 23.0, 47.0, seed=1)
    counts = rng.integers(1, 40, size=(2, o.n_c)).astype(np.uint32)
    target = rng.uniform(0.0, 2.0, size=(2, o.n_c))
    lam = 31.0
    w = o.fields_umbrella(counts, target, lam)

    def H(n):
        return o.energy_nb(n) + o.energy_umbrella(n, target, lam)

    for t in range(2):
        for c in rng.choice(o.n_c, 12, replace=False):
            up, dn = counts.copy(), counts.copy()
            up[t, c] += 1
            dn[t, c] -= 1
            fd = (H(up) - H(dn)) / 2.0
            _check(fails, f"umbrella w[{t},{c}] vs dH/dn", w[t, c], fd, 1e-9 * max(1.0, abs(fd)) + 1e-9)
    # at the target itself the restraint adds nothing
    _, _, rho = o.params()
    at = counts / rho
    _check(fails, "umbrella vanishes at the target", float(np.abs(o.fields_umbrella(counts, at, lam) -
                                                                  o.fields(counts)).max()), 0.0, 1e-12)
    return fails


def _offset_kernel(L, n, h, gl=4):
    """K[i, j] = P(cell of (i + U) L/n + h (2 U' - 1), periodic, is j)."""
    D = L / n
    x, wq = leggauss(gl)

    def overlap(xs, j):
        tot = np.zeros_like(xs)
        for m in range(-3, 4):
            a, b = j * D + m * L, (j + 1) * D + m * L
            tot += np.clip(np.minimum(xs + h, b) - np.maximum(xs - h, a), 0.0, None)
        return tot / (2 * h)

    K = np.zeros((n, n))
    for i in range(n):
        lo, hi = i * D, (i + 1) * D
        kinks = [lo, hi]
        for j in range(n + 1):
            for m in range(-3, 4):
                for sgn in (-1, 1):
                    k = j * D + m * L + sgn * h
                    if lo < k < hi:
                        kinks.append(k)
        kinks = np.unique(kinks)
        for a, b in zip(kinks[:-1], kinks[1:]):
            xs = 0.5 * (b - a) * x + 0.5 * (a + b)
            for j in range(n):
                K[i, j] += 0.5 * (b - a) * (wq * overlap(xs, j)).sum() / D
    return K


def pin_place_bead0_law(O):
    fails = []
    rng = np.random.default_rng(47)
    box, grid = (1.0, 0.75, 2.0), (4, 3, 5)
    n_poly = 300000
    o = O(n_poly, 1, 1, box, grid, 0.0, 0.0, A=0.2, seed=29)
    target = rng.uniform(0.0, 1.0, size=(2, o.n_c)).astype(np.float32)
    target[0, rng.choice(o.n_c, 7, replace=False)] = 0.0
    target[0, 3] = -0.5  # negative volume fractions carry no weight
    pos = o.place(target)
    q = np.where(target[0] > 0, np.floor(target[0].astype(np.float64) * 65536.0), 0.0)
    p0 = (q / q.sum()).reshape(grid)
    h = 0.5 / np.sqrt(3.0)
    Ks = [_offset_kernel(box[a], grid[a], h) for a in range(3)]
    P = np.einsum("abc,ai,bj,ck->ijk", p0, Ks[0], Ks[1], Ks[2]).reshape(-1)
    cells = np.array([o.cell_index(pos[k]) for k in range(0, n_poly)])
    cnt = np.bincount(cells, minlength=o.n_c)
    z = (cnt - n_poly * P) / np.sqrt(n_poly * P * (1 - P) + 1e-12)
    k = int(np.argmax(np.abs(z)))
    if abs(z[k]) > 5.0:
        fails.append(f"placed bead-0 cell {k}: {cnt[k]} vs exact {n_poly * P[k]:.1f} (z={z[k]:.1f})")
    _check(fails, "kernel rows sum to one", float(np.abs(Ks[2].sum(1) - 1).max()), 0.0, 1e-12)
    return fails


def pin_place_bond_statistics(O):
    fails = []
    rng = np.random.default_rng(53)
    n_poly, N = 8192, 16
    o = O(n_poly, N, 8, (4.0, 4.0, 4.0), (16, 16, 16), 0.0, 0.0, seed=31)
    target = rng.uniform(0.0, 1.0, size=(2, o.n_c)).astype(np.float32)
    pos = o.place(target).reshape(n_poly, N, 3)
    b = np.diff(pos, axis=1)
    nb = b.shape[0] * b.shape[1]
    for a in range(3):
        v = (b[:, :, a] ** 2).mean() * 3 * (N - 1)
        _check(fails, f"placed bond variance axis {a} x 3(N-1)", v, 1.0, 5 * np.sqrt(2.0 / nb))
    re2 = ((pos[:, -1] - pos[:, 0]) ** 2).sum(-1)
    _check(fails, "placed <R_e^2>", re2.mean(), 1.0, 5 * np.sqrt(2.0 / 3.0 / n_poly))
    return fails


# ---------------------------------------------------------------------------
def pin_wall_dimer_cell_pairs(O, blocks=16, per_block=15):
    """AB dimer on a 2^3 grid with hard walls in z: the z kernel has no
    periodic images (the restricted Boltzmann law is stationary)."""
    fails = []
    rng = np.random.default_rng(24)
    box, grid = (1.0, 1.0, 0.8), (2, 2, 2)
    for move in (0, 1):
        o = O(4096, 2, 1, box, grid, 0.0, 0.0, seed=37 + move, move=move, wall_z=1)
        kb, _, _ = o.params()
        w = rng.normal(0.0, 0.7, size=(2, o.n_c))
        Ks = [_bond_cell_kernel(box[0], grid[0], kb), _bond_cell_kernel(box[1], grid[1], kb),
              _bond_cell_kernel(box[2], grid[2], kb, images=0)]
        cells = [(ix, iy, iz) for ix in range(2) for iy in range(2) for iz in range(2)]
        P = np.zeros((o.n_c, o.n_c))
        for c1, (a1, b1, z1) in enumerate(cells):
            for c2, (a2, b2, z2) in enumerate(cells):
                P[c1, c2] = np.exp(-w[0, c1] - w[1, c2]) * Ks[0][a1, a2] * Ks[1][b1, b2] * Ks[2][z1, z2]
        P /= P.sum()
        pos = o.init()
        if not (pos[:, 2].min() >= 0 and pos[:, 2].max() < box[2]):
            fails.append("initial configuration outside the slab")
        o.run(pos, 0, 20, w_frozen=w, n_threads=NTHREADS)
        samples = []
        for b in range(blocks):
            r = o.run(pos, 20 + b * per_block, per_block, w_frozen=w, n_threads=NTHREADS, pair_hist=True)
            h = r["pair_hist"].astype(np.float64)
            samples.append(h / h.sum())
        if not (pos[:, 2].min() >= 0 and pos[:, 2].max() < box[2]):
            fails.append("a bead left the slab")
        _block_test(fails, f"wall dimer cell-pair law (move {move})", np.array(samples), P.reshape(-1))
    return fails


# ---------------------------------------------------------------------------
def pin_density_profile(O):
    """Counts built as (layer index + 1)(type + 1) give the profile
    (k + 1)(t + 1)/rho_bar exactly; random counts average, over the layers,
    to the global composition."""
    fails = []
    o = O(40, 8, 3, (2.0, 3.0, 4.0), (3, 4, 5), 10.0, 20.0, seed=1)
    _, _, rho = o.params()
    grid = (3, 4, 5)
    ix, iy, iz = np.meshgrid(*[np.arange(g) for g in grid], indexing="ij")
    idx = [ix.reshape(-1), iy.reshape(-1), iz.reshape(-1)]
    for axis in range(3):
        counts = np.stack([(idx[axis] + 1) * (t + 1) for t in range(2)]).astype(np.uint32)
        prof = o.density_profile(counts, axis)
        exact = np.stack([(np.arange(grid[axis]) + 1) * (t + 1) / rho for t in range(2)])
        _check(fails, f"profile axis {axis}", float(np.abs(prof - exact).max()), 0.0, 1e-12)
    rng = np.random.default_rng(5)
    counts = rng.integers(0, 9, size=(2, o.n_c)).astype(np.uint32)
    for axis in range(3):
        prof = o.density_profile(counts, axis)
        _check(fails, f"profile mean axis {axis}", float(np.abs(prof.mean(1) - counts.sum(1) / (o.n_c * rho)).max()),
               0.0, 1e-12)
    return fails


def pin_vertical_correlation(O):
    """Layers of counts proportional to 1 + cos(2 pi k z / nz) give
    C(dz) = cos(2 pi k dz / nz) when z is periodic; between walls a linear
    ramp n(z) = z pairs perfectly along z, so C(dz) is the ratio of the
    ramp's variance over the nz - dz layers that have a partner to its
    variance over all layers, ((nz - dz)^2 - 1) / (nz^2 - 1); C(0) = 1 for
    any field."""
    fails = []
    nz = 8
    o = O(10, 4, 2, (2.0, 2.0, 4.0), (2, 3, nz), 0.0, 0.0, seed=1)
    for k in (1, 2, 3):
        layer = np.rint(2 * (1 + np.cos(2 * np.pi * k * np.arange(nz) / nz)) * 1000).astype(np.int64)
        counts = np.zeros((2, o.n_c), np.uint32)
        counts[0] = np.tile(layer, o.n_c // nz)
        C = o.vertical_correlation(counts, 0)
        exact = np.cos(2 * np.pi * k * np.arange(nz) / nz)
        _check(fails, f"periodic cosine k={k}", float(np.abs(C - exact).max()), 0.0, 2e-3)
    nzw = 6
    ow = O(10, 4, 2, (2.0, 2.0, 4.0), (2, 3, nzw), 0.0, 0.0, seed=1, wall_z=1)
    counts = np.zeros((2, ow.n_c), np.uint32)
    counts[1] = np.tile(np.arange(nzw), ow.n_c // nzw).astype(np.uint32)
    C = ow.vertical_correlation(counts, 1)
    for dz in range(nzw):
        exact = ((nzw - dz) ** 2 - 1) / (nzw ** 2 - 1)
        _check(fails, f"walls ramp dz={dz}", C[dz], exact, 1e-12)
    rng = np.random.default_rng(9)
    counts = rng.integers(0, 7, size=(2, o.n_c)).astype(np.uint32)
    _check(fails, "C(0) of a random field", o.vertical_correlation(counts, 1)[0], 1.0, 1e-12)
    return fails


# ---------------------------------------------------------------------------
# Observables and the absolute scale of the non-bonded energy.
def _unit_vectors(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def pin_observables_rigid_chains(O):
    """Rigid chains whose observables are known by hand.  A straight chain of
    N beads with bond length l has R_e^2 = ((N-1) l)^2, R_g^2 =
    (N^2-1) l^2 / 12 (the variance of N equally spaced points) and bond
    energy k_b (N-1) l^2 with k_b = 3(N-1)/2.  A planar right-angle chain
    (n1 beads along one axis, then n2 along a perpendicular one, unit bonds)
    has R_e^2 = (n1-1)^2 + n2^2.  Chains of different lengths and directions
    make each mean over chains differ from a mean over beads or bonds."""
    fails = []
    rng = np.random.default_rng(51)
    N, n_poly = 12, 40
    o = O(n_poly, N, 5, (3.0, 3.0, 3.0), (6, 6, 6), 0.0, 0.0, seed=1)
    ell = rng.uniform(0.02, 0.3, size=n_poly)
    u = _unit_vectors(rng, n_poly)
    x0 = rng.uniform(-5.0, 8.0, size=(n_poly, 3))
    i = np.arange(N)
    pos = x0[:, None, :] + ell[:, None, None] * i[None, :, None] * u[:, None, :]
    got = o.observables(pos.reshape(-1, 3))
    kb = 1.5 * (N - 1)
    re2 = float(np.mean(((N - 1) * ell) ** 2))
    rg2 = float(np.mean((N * N - 1) * ell ** 2 / 12.0))
    eb = float(kb * (N - 1) * np.sum(ell ** 2))
    _check(fails, "straight chains R_e^2", got["Re2"], re2, 1e-12 * re2)
    _check(fails, "straight chains R_g^2", got["Rg2"], rg2, 1e-12 * rg2)
    _check(fails, "straight chains E_bond", got["Ebond"], eb, 1e-12 * eb)
    # right-angle chains: n1 = 5 beads along e1, then 7 beads along e2
    n1, n2 = 5, N - 5
    e1 = _unit_vectors(rng, 1)[0]
    e2 = np.cross(e1, _unit_vectors(rng, 1)[0])
    e2 /= np.linalg.norm(e2)
    shape = np.array([k * e1 for k in range(n1)] + [(n1 - 1) * e1 + k * e2 for k in range(1, n2 + 1)])
    pos = x0[:2, None, :] + 0.1 * shape[None]
    o2 = O(2, N, 5, (3.0, 3.0, 3.0), (6, 6, 6), 0.0, 0.0, seed=1)
    got = o2.observables(pos.reshape(-1, 3))
    re2 = 0.01 * ((n1 - 1) ** 2 + n2 ** 2)
    # R_g^2 of the corner chain from its two arms: coordinates along e1 are
    # 0..n1-1 then n2 times n1-1; along e2 n1 zeros then 1..n2.
    a = np.array(list(range(n1)) + [n1 - 1] * n2, float)
    b = np.array([0] * n1 + list(range(1, n2 + 1)), float)
    rg2 = 0.01 * (a.var() + b.var())
    _check(fails, "corner chain R_e^2", got["Re2"], re2, 1e-12)
    _check(fails, "corner chain R_g^2", got["Rg2"], rg2, 1e-12)
    _check(fails, "corner chain E_bond", got["Ebond"], 2 * kb * 0.01 * (N - 1), 1e-10)
    return fails


def pin_observables_equipartition(O, seeds=4):
    """Through the observables themselves, on Gaussian chains at chiN =
    kappaN = 0 (whose bond statistics pin_init_statistics pins in numpy):
    each of the 3(N-1) bond coordinates carries kT/2 in the harmonic bond
    energy, so <E_bond> per chain = 3(N-1)/2; <R_e^2> = 1; <R_g^2> =
    (N+1)/(6N)."""
    fails = []
    N, n_poly = 16, 4096
    re2, rg2, eb = [], [], []
    for sd in range(seeds):
        o = O(n_poly, N, 8, (4.0, 4.0, 4.0), (8, 8, 8), 0.0, 0.0, seed=61 + sd)
        g = o.observables(o.init())
        re2.append(g["Re2"])
        rg2.append(g["Rg2"])
        eb.append(g["Ebond"] / n_poly)
    # standard errors of the mean over seeds x chains, from the Gaussian law
    m = seeds * n_poly
    _check(fails, "<E_bond> per chain", np.mean(eb), 1.5 * (N - 1), 5 * np.sqrt(1.5 * (N - 1) / m))
    _check(fails, "<R_e^2>", np.mean(re2), 1.0, 5 * np.sqrt(2.0 / 3.0 / m))
    _check(fails, "<R_g^2>", np.mean(rg2), (N + 1) / (6.0 * N), 5 * 0.5 * (N + 1) / (6.0 * N) / np.sqrt(m))
    return fails


def pin_energy_nb_absolute(O):
    """H_nb = (rho_bar/N) sum_c [chiN phiA phiB + (kappaN/2)(phiA + phiB - 1)^2]
    on counts built by hand, so that its absolute scale (the rho_bar/N
    prefactor, the 1/2 of the compressibility term) is fixed and not only its
    derivatives:
    * phiA = phiB = 1/2 in every cell: H_nb = n_poly chiN / 4;
    * one cell of a pure-A melt with k beads too many: (rho_bar/N)(kappaN/2)(k/rho_bar)^2;
    * two cells worked out by hand, rho_bar = 4, N = 4 (prefactor 1):
      (2, 2) -> chiN/4; (5, 1) -> phi = (5/4, 1/4), chiN 5/16 + (kappaN/2)(1/4)."""
    fails = []
    chiN, kappaN = 23.0, 48.0
    # uniform symmetric melt: 64 chains of 16 beads, 4^3 cells, rho_bar = 16
    o = O(64, 16, 8, (2.0, 2.0, 2.0), (4, 4, 4), chiN, kappaN, seed=1)
    counts = np.full((2, o.n_c), 8, np.uint32)
    _check(fails, "uniform phi = 1/2 melt", o.energy_nb(counts), 64 * chiN / 4, 1e-9)
    # pure A, one cell with 4 extra beads: prefactor rho_bar/N = 1, excess 1/4
    counts = np.zeros((2, o.n_c), np.uint32)
    counts[0] = 16
    counts[0, 17] = 20
    _check(fails, "one-cell excess", o.energy_nb(counts), kappaN / 2 * (4 / 16) ** 2, 1e-12)
    # two cells, 2 chains of 4 beads
    o = O(2, 4, 2, (1.0, 1.0, 2.0), (1, 1, 2), chiN, kappaN, seed=1)
    counts = np.array([[2, 5], [2, 1]], np.uint32)
    _check(fails, "two hand-worked cells", o.energy_nb(counts), chiN / 4 + chiN * 5 / 16 + kappaN / 2 / 4, 1e-12)
    # and the same two cells with N = 8 beads per chain, one chain: prefactor 1/2
    o = O(1, 8, 4, (1.0, 1.0, 2.0), (1, 1, 2), chiN, kappaN, seed=1)
    _check(fails, "two cells, prefactor 1/2", o.energy_nb(counts), 0.5 * (chiN / 4 + chiN * 5 / 16 + kappaN / 2 / 4),
           1e-12)
    return fails



def pin_umbrella_energy_absolute(O):
    """H_umb = (rho_bar/N)(lambdaN/2) sum_c sum_t (phi_t - phi*_t)^2 on counts
    and targets built by hand: a pure-A melt at rho_bar = N = 16 (prefactor 1)
    held at phi = (1, 0) everywhere, the target off by 1/2 in one A cell and by
    1/4 in one B cell: (lambdaN/2)(1/4 + 1/16)."""
    fails = []
    lam = 31.0
    o = O(64, 16, 8, (2.0, 2.0, 2.0), (4, 4, 4), 23.0, 47.0, seed=1)
    counts = np.zeros((2, o.n_c), np.uint32)
    counts[0] = 16
    target = np.zeros((2, o.n_c))
    target[0] = 1.0
    target[0, 5] = 0.5
    target[1, 40] = 0.25
    _check(fails, "umbrella energy by hand", o.energy_umbrella(counts, target, lam), lam / 2 * (0.25 + 0.0625), 1e-12)
    return fails


def pin_params_workload_values(O):
    """The model constants of the melt workloads, as their definitions print
    them: k_b = 3(N-1)/2 is 46.5 for N = 32 and 94.5 for N = 64; the default
    proposal half-width 0.5/sqrt(N-1) is 0.0898 and 0.0630 to four digits and
    held as an FP32 number; rho_bar is 4, 2 and 4 beads per cell."""
    fails = []
    for (n_poly, N, L, g), kb_x, A_x, rho_x in (((512, 32, 4.0, 16), 46.5, 0.0898, 4.0),
                                                ((131072, 32, 16.0, 128), 46.5, 0.0898, 2.0),
                                                ((1048576, 64, 32.0, 256), 94.5, 0.0630, 4.0)):
        o = O(n_poly, N, N // 2, (L, L, L), (g, g, g), 20.0, 50.0, seed=1)
        kb, A, rho = o.params()
        _check(fails, f"k_b N={N}", kb, kb_x, 0.0)
        _check(fails, f"A N={N}", A, A_x, 5e-5)
        if A != float(np.float32(A)):
            fails.append(f"A N={N} is not an FP32 number")
        _check(fails, f"rho_bar {n_poly}x{N}", rho, rho_x, 0.0)
    return fails


def pin_step_chains_sample(O):
    """Chains interact only through the frozen fields within a step, so a
    sample of chains stepped alone (by logical id) moves exactly as inside
    the whole system, whose step the dynamics pins above fix."""
    fails = []
    rng = np.random.default_rng(71)
    o = O(300, 12, 5, (2.0, 2.0, 2.0), (8, 8, 8), 20.0, 50.0, seed=13, move=0)
    pos = o.init()
    w = o.fields(o.density(pos))
    for t in range(3):
        ids = np.sort(rng.choice(o.d.n_poly, 40, replace=False)).astype(np.uint32)
        sub = np.ascontiguousarray(pos.reshape(o.d.n_poly, -1)[ids].reshape(-1, 3))
        _, acc_s, _, _ = o.mc_step_chains(sub, ids, w, t)
        _, acc, _, _ = o.mc_step(pos, w, t)
        full = pos.reshape(o.d.n_poly, -1)[ids].reshape(-1, 3)
        if not np.array_equal(sub, full):
            fails.append(f"step {t}: sampled chains differ from the whole step")
        if not np.array_equal(acc_s, acc.reshape(o.d.n_poly, -1)[ids].reshape(-1)):
            fails.append(f"step {t}: sampled decisions differ from the whole step")
        w = o.fields(o.density(pos))
    return fails


# ---------------------------------------------------------------------------
# Molecule types and boundary-zone conversion (Sec. 3.2).
def _binomial_z(k, n, p):
    return (k - n * p) / np.sqrt(max(n * p * (1.0 - p), 1e-12))


def pin_conversion_markov(O, n=20000, steps=8):
    """With one zone covering the whole box, every chain's type is an
    independent two-state Markov chain with per-step probabilities a (0->1)
    and b (1->0): from type 0, P(type 1 after t steps) = pi (1 - (1-a-b)^t),
    pi = a/(a+b); the number of type-1 chains is binomial.  Each zone is
    tried on its own with unequal rates in the two directions."""
    fails = []
    L = 4.0
    for zone, rates in (("bottom", (0.30, 0.10)), ("top", (0.15, 0.45))):
        o = O(n, 2, 1, (L, L, L), (4, 4, 4), 0.0, 0.0, A=0.2, seed=31, wall_z=1)
        p = (rates[0], rates[1], 0.0, 0.0) if zone == "bottom" else (0.0, 0.0, rates[0], rates[1])
        o.set_conversion(0, L if zone == "bottom" else 0.0, L if zone == "top" else 0.0, p)
        k0 = 0 if zone == "bottom" else 2
        a, b = o.d.thr[k0] / 2.0**32, o.d.thr[k0 + 1] / 2.0**32
        pos = o.init()
        n1_prev = 0
        for t in range(steps):
            c4 = o.convert(pos, t)
            n1 = int(o.types.sum())
            if c4[k0] - c4[k0 + 1] != n1 - n1_prev or c4[2 - k0] or c4[3 - k0]:
                fails.append(f"{zone} zone: conversion counts {c4.tolist()} do not account for {n1 - n1_prev}")
            n1_prev = n1
            pt = a / (a + b) * (1.0 - (1.0 - a - b) ** (t + 1))
            z = _binomial_z(n1, n, pt)
            if abs(z) > 5.0:
                fails.append(f"{zone} zone step {t}: {n1} type-1 chains, expected {n * pt:.1f} (z={z:.1f})")
    return fails


def pin_conversion_zone_law(O, n=20000):
    """Bead 0 of the initial chains is uniform in the box, so with certain
    flips (p = 1) the first conversion turns exactly the chains whose bead 0
    lies in a zone: binomial with the zone's share of the box, per zone; the
    second flips them all back; the A-bead count follows the types."""
    fails = []
    L, lo, hi = 4.0, 0.5, 1.25
    for wall in (1, 0):
        o = O(n, 4, 3, (3.0, 3.0, L), (6, 6, 8), 0.0, 0.0, A=0.2, seed=32 + wall, wall_z=wall)
        o.set_conversion(1, lo, hi, (1.0, 1.0, 1.0, 1.0))
        pos = o.init()
        c4 = o.convert(pos, 0)
        for k, (cnt, share) in enumerate(((c4[0], lo / L), (c4[2], hi / L))):
            z = _binomial_z(int(cnt), n, share)
            if abs(z) > 5.0:
                fails.append(f"walls={wall}: zone {k} converted {cnt}, expected {n * share:.0f} (z={z:.1f})")
        n1 = int(o.types.sum())
        if n1 != c4[0] + c4[2]:
            fails.append(f"walls={wall}: {n1} type-1 chains after {c4.tolist()}")
        nA = int(o.density(pos)[0].sum())
        if nA != (n - n1) * 3 + n1 * 1:
            fails.append(f"walls={wall}: {nA} A beads for {n1} converted chains")
        o.convert(pos, 1)
        if int(o.types.sum()) != 0:
            fails.append(f"walls={wall}: certain flips left {int(o.types.sum())} chains converted")
    return fails


def pin_conversion_type_field(O, blocks=16, per_block=15):
    """Single beads of an A molecule converted to B at the first step (a
    zone covering the box, p(0->1) = 1, p(1->0) = 0) then move in a frozen
    field with the B field: occupancy proportional to exp(-w_B(c)), and no
    A bead left."""
    fails = []
    rng = np.random.default_rng(41)
    o = O(4096, 1, 1, (1.0, 1.5, 2.0), (2, 3, 4), 0.0, 0.0, A=0.6, seed=9)
    o.set_conversion(0, 2.0, 0.0, (1.0, 0.0, 0.0, 0.0))
    w = rng.normal(0.0, 0.8, size=(2, o.n_c))
    pos = o.init()
    o.run(pos, 0, 10, w_frozen=w, n_threads=NTHREADS)
    if int(o.types.sum()) != o.d.n_poly:
        fails.append(f"{int(o.types.sum())} of {o.d.n_poly} beads converted")
    samples = []
    for b in range(blocks):
        r = o.run(pos, 10 + b * per_block, per_block, w_frozen=w, n_threads=NTHREADS, occ=True)
        occ = r["occ"].reshape(2, o.n_c).astype(np.float64)
        if occ[0].sum() != 0 or occ[1].sum() == 0:
            fails.append("A beads counted after the conversion")
            return fails
        samples.append(occ[1] / occ[1].sum())
    p = np.exp(-w[1])
    _block_test(fails, "converted bead occupancy", np.array(samples), p / p.sum())
    return fails


def pin_conversion_structure_factor(O, seeds=12):
    """Ideal chains, every other one converted (its A block n_A_alt long):
    S(q) = (1/N) sum over the two molecule types, each with half the weight,
    of sum_ij s_i s_j exp(-q^2 |i-j| / (6(N-1)))."""
    fails = []
    n_poly, N, n_A, n_A_alt, L = 2048, 16, 8, 3, 4.0
    ms = np.array([(1, 0, 0), (0, 1, 1), (1, 1, 1), (2, 0, 0)], np.int32)
    ij = np.abs(np.arange(N)[:, None] - np.arange(N)[None, :])
    s0 = np.where(np.arange(N) < n_A, 1.0, -1.0)
    s1 = np.where(np.arange(N) < n_A_alt, 1.0, -1.0)
    types = (np.arange(n_poly) % 2).astype(np.uint8)
    est = []
    for sd in range(seeds):
        o = O(n_poly, N, n_A, (L, L, L), (16, 16, 16), 0.0, 0.0, seed=200 + sd)
        o.set_conversion(n_A_alt, 0.0, 0.0, (0.0, 0.0, 0.0, 0.0))
        o.set_types(types)
        est.append(o.structure_factor(o.init(), ms))
    est = np.array(est)
    for k, m in enumerate(ms):
        q2 = float(((2 * np.pi / L) ** 2) * (m ** 2).sum())
        K = np.exp(-q2 * ij / (6.0 * (N - 1)))
        exact = 0.5 * ((s0[:, None] * s0[None, :] * K).sum() + (s1[:, None] * s1[None, :] * K).sum()) / N
        se = est[:, k].std(ddof=1) / np.sqrt(seeds)
        _check(fails, f"S(q) with converted chains m={tuple(m)}", est[:, k].mean(), exact, 5 * se)
    return fails


ALL_PINS = {
    "philox_uniformity": pin_philox_uniformity,
    "philox_triton": pin_philox_triton,
    "init_statistics": pin_init_statistics,
    "ideal_dynamics": pin_ideal_dynamics,
    "single_bead_field": pin_single_bead_field,
    "dimer_cell_pairs": pin_dimer_cell_pairs,
    "density_bruteforce": pin_density_bruteforce,
    "fields_derivative": pin_fields_derivative,
    "structure_factor_ideal": pin_structure_factor_ideal,
    "observables_rigid_chains": pin_observables_rigid_chains,
    "observables_equipartition": pin_observables_equipartition,
    "energy_nb_absolute": pin_energy_nb_absolute,
    "umbrella_energy_absolute": pin_umbrella_energy_absolute,
    "params_workload_values": pin_params_workload_values,
    "step_chains_sample": pin_step_chains_sample,
    "smart_ideal_dynamics": pin_smart_ideal_dynamics,
    "smart_single_bead_field": pin_smart_single_bead_field,
    "smart_dimer_cell_pairs": pin_smart_dimer_cell_pairs,
    "normal_quantile": pin_normal_quantile,
    "umbrella_fields_derivative": pin_umbrella_fields_derivative,
    "place_bead0_law": pin_place_bead0_law,
    "place_bond_statistics": pin_place_bond_statistics,
    "wall_dimer_cell_pairs": pin_wall_dimer_cell_pairs,
    "density_profile": pin_density_profile,
    "vertical_correlation": pin_vertical_correlation,
    "conversion_markov": pin_conversion_markov,
    "conversion_zone_law": pin_conversion_zone_law,
    "conversion_type_field": pin_conversion_type_field,
    "conversion_structure_factor": pin_conversion_structure_factor,
}
