"""Oracle pins: Philox4x32-10 known answers, the 53-bit uniform, and the protocol's weights
at their special points (Eq. (protocol))."""
import math
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert list(oracle.philox4x32_10(ctr, key)) == out


def test_u53_range_and_resolution():
    assert oracle.u53(0, 0) == 0.0
    assert oracle.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    # lowest bit of b that survives is bit 6; one step there is 2^-53
    assert oracle.u53(0, 1 << 6) == 2.0 ** -53
    assert oracle.u53(1 << 5, 0) == 2.0 ** -27


def test_protocol_weights_special_points():
    # alpha_sg(0) = alpha_sg(1) = 0, alpha_sg(1/2) = 1
    assert oracle.alpha_sg(0.0) == 0.0 and oracle.alpha_sg(1.0) == 0.0 and oracle.alpha_sg(0.5) == 1.0
    # alpha_g(1) = 1 to double precision, alpha_g(1/2) = 0, alpha_g(0) vanishingly small
    assert oracle.alpha_g(1.0) == 1.0
    assert oracle.alpha_g(0.5) == 0.0
    assert 0.0 <= oracle.alpha_g(0.0) < 1e-200
    # the soft grids switch on first: below 0.45 the full grid weight is negligible
    for a in np.linspace(0.0, 0.45, 10):
        assert oracle.alpha_g(a) < 1e-20
    # the unperturbed grid saturates by 0.51 to within its (2a-1)^2 envelope
    for a in np.linspace(0.51, 1.0, 10):
        assert math.isclose(oracle.alpha_g(a), (2 * a - 1) ** 2, rel_tol=1e-4)
    # no grid at all for the warming leg (alpha = NaN)
    assert oracle.alpha_sg(float("nan")) == 0.0 and oracle.alpha_g(float("nan")) == 0.0
    # beta = 1/(k_B T) with k_B in kcal/(mol K): kT at 300 K is about 0.596 kcal/mol
    assert abs(1.0 / oracle.beta(300.0) - 0.59616) < 1e-4
