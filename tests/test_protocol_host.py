"""The scalar steps of protocol initialization, which the library computes on the host (the
thermodynamic-length parameter steps, the time-step rule and the insertion rule: "Initialization",
"Equilibration and production"), agree with the oracle's to rounding.  No GPU is needed."""
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
    # invalid inputs are refused, not extrapolated
    from paper_1507_03703_gb300.algdock import AlgdockError
    for bad in ((-1.0, 1.0, 0.3), (300.0, -1.0, 0.3), (300.0, 1.0, 0.0)):
        with pytest.raises(AlgdockError):
            P.next_temperature(*bad)
    with pytest.raises(AlgdockError):
        P.next_alpha(1.5, 1.0, 1.0, 1.0, 0.2)
    with pytest.raises(AlgdockError):
        P.adapt_dt(2.0, 1.5)


def test_state_insertion_rule_matches_the_oracle():
    """protocol.insertions (the host's between-cycle rule) against oracle.split_ladder on random
    ladders and exchange counts of both legs: the same insertions, parameters equal to rounding."""
    from paper_1507_03703_gb300.protocol import insertions
    rng = np.random.default_rng(41)
    for trial in range(200):
        K = int(rng.integers(2, 12))
        if trial % 2:
            T = np.sort(rng.uniform(300, 600, K))
            A = np.full(K, np.nan)
        else:
            A = np.sort(rng.uniform(0, 1, K))
            T = 600.0 - 300.0 * A
        D = rng.uniform(0.5, 3.0, K)
        att = rng.integers(0, 50, K - 1)
        acc = np.minimum(att, rng.integers(0, 50, K - 1))
        hT, hA, hD, new = insertions(T, A, D, att, acc)
        oT, oA, oD, ins = oracle.split_ladder(T, A, D, att, acc)
        assert [n for n, _ in new] == ins
        assert all(lower == n - 1 for n, lower in new)
        # independent arithmetic (sqrt against a power of 1/2): equal to rounding
        assert np.allclose(hT, oT, rtol=1e-15, atol=0) and np.array_equal(hD, oD)
        assert np.array_equal(np.isnan(hA), np.isnan(oA))
        assert np.allclose(hA[~np.isnan(hA)], oA[~np.isnan(oA)], rtol=1e-15, atol=0)
