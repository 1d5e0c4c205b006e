"""The oracle against facts that do not come from itself (CPU only).

See ``tests/pins.py`` for what each pin checks and why it is independent of
the oracle's own arithmetic.
"""
import pytest

import pins


@pytest.mark.parametrize("name", list(pins.ALL_PINS))
def test_oracle_pin(oracle_cls, name):
    fails = pins.ALL_PINS[name](oracle_cls)
    assert not fails, "\n".join(fails)


def test_dimer_kernel_normalisation():
    # The bond kernel summed over target cells is the Gaussian integral times
    # the cell width: sum_j K[i, j] = h sqrt(pi / k_b).
    import numpy as np
    K = pins._bond_cell_kernel(1.0, 2, 1.5)
    assert np.allclose(K.sum(axis=1), 0.5 * np.sqrt(np.pi / 1.5), rtol=1e-10)


def test_acceptance_quadrature_limits():
    # A -> 0 accepts every move; the quadrature is monotone in A.
    a_small = pins._acceptance_ideal(32, 1e-6, 46.5)
    a_mid = pins._acceptance_ideal(32, 0.0898, 46.5)
    a_big = pins._acceptance_ideal(32, 0.5, 46.5)
    assert abs(a_small - 1.0) < 1e-4
    assert a_small > a_mid > a_big > 0.0
