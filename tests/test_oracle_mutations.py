"""Plant plausible mistakes in a copy of the oracle source and check that the
pins catch each one (CPU only).  The mistakes live only in a temporary copy;
the oracle itself is never modified."""
import os
import subprocess
import tempfile

import pytest

import pins
from oracle import Oracle
from oracle.oracle import _SRC

# (name, text in soma_oracle.cpp, replacement, pin expected to catch it)
MUTATIONS = [
    ("bond constant doubled", "return 1.5 * (double)(d->N - 1);", "return 3.0 * (double)(d->N - 1);",
     "ideal_dynamics"),
    ("one-sided proposal", "A * (2.0 * unit_closed_open(r[a]) - 1.0)", "A * unit_closed_open(r[a])",
     "ideal_dynamics"),
    ("field term sign", "dE = k_b * dEb + wt[cell_of(d, rn)] - wt[cell_of(d, ri)];",
     "dE = k_b * dEb - wt[cell_of(d, rn)] + wt[cell_of(d, ri)];", "single_bead_field"),
    ("types swapped", "return i < nA ? 0 : 1;", "return i < nA ? 1 : 0;", "dimer_cell_pairs"),
    ("right neighbour dropped",
     "unit_closed_open(r[a]) - 1.0);\n        for (int j = i - 1; j <= i + 1; j += 2)",
     "unit_closed_open(r[a]) - 1.0);\n        for (int j = i - 1; j <= i - 1; j += 2)", "ideal_dynamics"),
    ("acceptance inverted", "bool ok = margin < 0.0;", "bool ok = margin > 0.0;", "ideal_dynamics"),
    ("cell axes transposed", "return (idx[0] * d->grid[1] + idx[1]) * d->grid[2] + idx[2];",
     "return (idx[2] * d->grid[1] + idx[1]) * d->grid[0] + idx[0];", "density_bruteforce"),
    ("uniform for ln u halved", "std::log(unit_open(r[3]))", "std::log(0.5 * unit_open(r[3]))",
     "ideal_dynamics"),
    ("chi term uses own type", "*wA = (d->chiN * phiB + d->kappaN * excess) / N;",
     "*wA = (d->chiN * phiA + d->kappaN * excess) / N;", "fields_derivative"),
    ("compressibility factor", "0.5 * d->kappaN * excess * excess", "d->kappaN * excess * excess",
     "fields_derivative"),
    ("philox key bump", "k1 += W1;", "k1 += W0;", "philox_triton"),
    ("init bond variance", "std::sqrt(1.0 / (3.0 * (double)(d->N - 1)))",
     "std::sqrt(1.0 / (2.0 * (double)(d->N - 1)))", "init_statistics"),
    ("composition sign lost", "double s = type_of(d, c, i) == 0 ? 1.0 : -1.0;", "double s = 1.0;",
     "structure_factor_ideal"),
    ("bond of second bead anchored to bead 0", "p[3 * i + 0] = p[3 * (i - 1) + 0] + sigma * z0;",
     "p[3 * i + 0] = p[0] + sigma * z0;", "init_statistics"),
    ("force-bias asymmetry term dropped", "bias = (rev - fwd) / (2.0 * s2);", "bias = 0.0;",
     "smart_ideal_dynamics"),
    ("force-bias drift sign flipped", "rn[a] = ri[a] + 0.5 * s2 * F[a] + std::sqrt(s2) * xi;",
     "rn[a] = ri[a] - 0.5 * s2 * F[a] + std::sqrt(s2) * xi;", "smart_ideal_dynamics"),
    ("force-bias reverse drift from the old force", "const double b = ri[a] - rn[a] - 0.5 * s2 * Fn[a];",
     "const double b = ri[a] - rn[a] - 0.5 * s2 * F[a];", "smart_ideal_dynamics"),
    ("normal quantile Newton step sign", "x -= f / dens;", "x += f / dens;", "normal_quantile"),
    ("force-bias normals from the wrong word", "normal_quantile(unit_open24(r[a]))",
     "normal_quantile(unit_open24(r[0]))", "smart_ideal_dynamics"),
    ("umbrella field doubled", "w[c] += lambdaN * (counts[c] / rho_bar - target[c]) / (double)d->N;",
     "w[c] += 2.0 * lambdaN * (counts[c] / rho_bar - target[c]) / (double)d->N;", "umbrella_fields_derivative"),
    ("umbrella field sign", "w[c] += lambdaN * (counts[c] / rho_bar - target[c]) / (double)d->N;",
     "w[c] += lambdaN * (target[c] - counts[c] / rho_bar) / (double)d->N;", "umbrella_fields_derivative"),
    ("placement offset dropped", "h * (2.0 * unit_closed_open(r2[a]) - 1.0);", "0.0;", "place_bead0_law"),
    ("placement offset width R_e/2 per axis", "const double h = 0.5 / std::sqrt(3.0);", "const double h = 0.5;",
     "place_bead0_law"),
    ("placement cell axes transposed",
     "const int64_t idx[3] = {cell / ((int64_t)d->grid[1] * d->grid[2]), (cell / d->grid[2]) % d->grid[1],\n"
     "                            cell % d->grid[2]};",
     "const int64_t idx[3] = {cell % d->grid[0], (cell / d->grid[0]) % d->grid[1],\n"
     "                            cell / ((int64_t)d->grid[0] * d->grid[1])};", "place_bead0_law"),
    ("wall ignored: z stays periodic", "if (d->wall_z && !(rn[2] >= 0.0 && rn[2] < d->box[2])) {",
     "if (false) {", "wall_dimer_cell_pairs"),
    ("profile averaged over the wrong cell count", "for (int i = 0; i < 2 * n; ++i) out[i] /= (double)m;",
     "for (int i = 0; i < 2 * n; ++i) out[i] /= (double)nc;", "density_profile"),
    ("correlation pairs wrap between walls", "        if (d->wall_z) continue;\n", "", "vertical_correlation"),
    ("placement weights of the other type", "const float* phi = target + (int64_t)(d->n_A > 0 ? 0 : 1) * nc;",
     "const float* phi = target + (int64_t)(d->n_A > 0 ? 1 : 0) * nc;", "place_bead0_law"),
    ("conversion directions swapped", "if ((uint64_t)r[0] < d->thr[2 * zone + m]) {",
     "if ((uint64_t)r[0] < d->thr[2 * zone + 1 - m]) {", "conversion_markov"),
    ("conversion zones swapped", "if ((uint64_t)r[0] < d->thr[2 * zone + m]) {",
     "if ((uint64_t)r[0] < d->thr[2 * (1 - zone) + m]) {", "conversion_markov"),
    ("top zone measured from the bottom", "const float zhi = (float)(L - d->zone_hi);",
     "const float zhi = (float)d->zone_hi;", "conversion_zone_law"),
    ("converted molecule keeps its A block", "? d->n_A_alt : d->n_A;", "? d->n_A : d->n_A;",
     "conversion_type_field"),
    ("conversion counts merged across directions", "if (counts4) counts4[2 * zone + m] += 1;",
     "if (counts4) counts4[2 * zone] += 1;", "conversion_markov"),
    ("bond energy without k_b", "out->Ebond = bond_k(d) * eb;", "out->Ebond = eb;", "observables_rigid_chains"),
    ("R_g^2 about bead 0", "g2 += (p[3 * i + a] - cm[a]) * (p[3 * i + a] - cm[a]);",
     "g2 += (p[3 * i + a] - p[a]) * (p[3 * i + a] - p[a]);", "observables_rigid_chains"),
    ("R_e^2 averaged per bead", "out->Re2 = re2 / d->n_poly;", "out->Re2 = re2 / (double)n_beads(d);",
     "observables_rigid_chains"),
    ("end-to-end vector to the second-last bead", "double v = p[3 * (N - 1) + a] - p[a];",
     "double v = p[3 * (N - 2) + a] - p[a];", "observables_rigid_chains"),
    ("bond energy over one axis", "      for (int a = 0; a < 3; ++a) {\n        double b = p[3 * i + a]",
     "      for (int a = 0; a < 1; ++a) {\n        double b = p[3 * i + a]", "observables_equipartition"),
    # consistent mistakes in the energy and its fields together: the fields
    # stay the energy's derivative, only its absolute value catches them
    ("energy prefactor rho_bar and fields without 1/N",
     [("return (double)d->n_poly / (double)nc * sum;", "return (double)n_beads(d) / (double)nc * sum;"),
      ("  const double N = (double)d->N;\n  double excess", "  const double N = 1.0;\n  double excess")],
     None, "energy_nb_absolute"),
    ("compressibility 1/2 dropped in the energy and doubled in the fields",
     [("0.5 * d->kappaN * excess * excess", "d->kappaN * excess * excess"),
      ("*wA = (d->chiN * phiB + d->kappaN * excess) / N;", "*wA = (d->chiN * phiB + 2.0 * d->kappaN * excess) / N;"),
      ("*wB = (d->chiN * phiA + d->kappaN * excess) / N;", "*wB = (d->chiN * phiA + 2.0 * d->kappaN * excess) / N;")],
     None, "energy_nb_absolute"),
    ("umbrella 1/2 dropped in the energy and doubled in the fields",
     [("return rho_bar / (double)d->N * 0.5 * lambdaN * sum;", "return rho_bar / (double)d->N * lambdaN * sum;"),
      ("w[c] += lambdaN * (counts[c] / rho_bar - target[c]) / (double)d->N;",
       "w[c] += 2.0 * lambdaN * (counts[c] / rho_bar - target[c]) / (double)d->N;")],
     None, "umbrella_energy_absolute"),
    ("proposal width 0.5/sqrt(N)", "0.5 / std::sqrt((double)(d->N - 1));", "0.5 / std::sqrt((double)d->N);",
     "params_workload_values"),
    ("proposal width kept in FP64", "  return (double)(float)a;\n", "  return a;\n", "params_workload_values"),
    ("sampled chains draw by their position in the sample",
     "const uint32_t chain = ids ? ids[c] : (uint32_t)c;", "const uint32_t chain = (uint32_t)c;",
     "step_chains_sample"),
]


@pytest.mark.parametrize("name,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_mutation(name, old, new, pin):
    # old is one anchor replaced by new, or a list of (anchor, replacement)
    # pairs planted together (new is then None)
    edits = old if new is None else [(old, new)]
    src = open(_SRC).read()
    for a, b in edits:
        assert src.count(a) == 1, f"mutation anchor not unique/found: {a}"
        src = src.replace(a, b)
    with tempfile.TemporaryDirectory() as td:
        cpp = os.path.join(td, "mut.cpp")
        so = os.path.join(td, "libmut.so")
        open(cpp, "w").write(src)
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", so, cpp])
        fails = pins.ALL_PINS[pin](Oracle.with_library(so))
    assert fails, f"pin {pin} did not catch the planted mistake '{name}'"
