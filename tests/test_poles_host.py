"""The library's host pole rules (C++, own elliptic-function code) against the oracle's
(scipy elliptic functions): nodes and weights of eq. dFOP agree to rounding."""
import numpy as np
import pytest

import paper_1603_09724_gb300 as omm
from oracle import poles


@pytest.mark.parametrize("abc", [(-10.0, -2.0, -1.6), (-109.0, -103.3, -102.9), (-1630.0, -1615.0, -1614.83),
                                 (-1.0, 3.0, 3.05)])
@pytest.mark.parametrize("P", [2, 8, 16, 30])
def test_conformal_rule_matches_oracle(abc, P):
    z, w = omm.poles_fermi(*abc, P)
    zo, wo = poles.poles_conformal(*abc, P)
    scale = max(1.0, np.max(np.abs(zo)))
    np.testing.assert_allclose(z, zo, atol=1e-12 * scale)
    np.testing.assert_allclose(w, wo, atol=1e-12 * np.max(np.abs(wo)))


@pytest.mark.parametrize("P", [1, 4, 16])
def test_circle_rule_matches_oracle(P):
    z, w = omm.poles_circle(2.0, 0.75, P)
    zo, wo = poles.poles_circle(2.0, 0.75, P)
    np.testing.assert_allclose(z, zo, atol=1e-14)
    np.testing.assert_allclose(w, wo, atol=1e-14)


def test_default_shift_matches_oracle():
    from oracle import hamiltonian as ham
    from workloads import wells_2d
    V = wells_2d(32, 10.0, seed=2)
    assert omm.default_shift(2, 32, 10.0, V) == pytest.approx(ham.default_shift((32, 32), 10.0, V), rel=1e-14)
