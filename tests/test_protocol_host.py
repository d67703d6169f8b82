"""The scalar steps of protocol initialization that run on the host (the thermodynamic-length
parameter steps and the time-step rule, "Initialization") agree with the oracle's to rounding."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import protocol as P


@pytest.mark.parametrize("a", [0.0, 0.2, 0.45, 0.499, 0.5, 0.501, 0.6, 0.97])
def test_alpha_step(a):
    for sig in ([3.0, 0.0, 0.0], [0.0, 40.0, 0.0], [0.0, 0.0, 2.0], [1.5, 20.0, 0.7]):
        got = P.next_alpha(a, *sig, speed=0.2)
        want = oracle.next_alpha(a, *sig, 0.2)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-15)


def test_temperature_step_and_time_step_rule():
    for T, s_u in ((300.0, 4.0), (455.5, 9.1), (599.0, 0.5)):
        assert P.next_temperature(T, s_u, 0.3) == pytest.approx(oracle.next_temperature(T, s_u, 0.3), rel=1e-14)
    for dt in (0.1, 0.2, 2.0, 4.9, 5.0):
        for acc in (0.0, 0.05, 0.1, 0.3, 0.4, 0.6, 0.8, 0.81, 1.0):
            assert P.adapt_dt(dt, acc) == oracle.adapt_dt(dt, acc)
    assert math.isclose(P.d_alpha_g(0.5), 0.0, abs_tol=1e-15)
    assert np.sign(P.d_alpha_sg(0.2)) > 0 > np.sign(P.d_alpha_sg(0.8))
