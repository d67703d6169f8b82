"""Oracle pins of the between-cycle state insertion ("Equilibration and production": a state is
inserted between neighbours whose exchange acceptance fell below 0.4 over the cycle, and its
configurations are drawn by sampling importance resampling from other states' samples).

- Nothing is inserted when every neighbour pair reaches the threshold, or when a pair was never
  attempted; a pair exactly at 0.4 keeps its gap.
- An inserted warming state sits at the geometric mean temperature (the ladder stays geometric
  when every gap is split), an inserted coupling state at the mean alpha with T on the protocol's
  line T(alpha); its time step is the neighbours' smaller one; the other states keep their order.
- Importance resampling from the lower neighbour's exact samples gives the new state's
  distribution: on harmonic wells the resampled variance is the new state's kT/k."""
import math

import numpy as np

import oracle


def test_no_insertion_above_threshold_or_without_attempts():
    T = [300.0, 400.0, 600.0]
    A = [np.nan] * 3
    D = [2.0] * 3
    T2, A2, D2, ins = oracle.split_ladder(T, A, D, [100, 0], [40, 0])
    assert ins == [] and np.array_equal(T2, T)
    _, _, _, ins = oracle.split_ladder(T, A, D, [100, 100], [39, 40])
    assert ins == [1]


def test_warming_midpoints_keep_a_geometric_ladder():
    T = 300.0 * 2.0 ** (np.arange(5) / 4.0)
    T2, A2, D2, ins = oracle.split_ladder(T, [np.nan] * 5, [2.0, 1.5, 2.0, 2.5, 2.0], [10] * 4, [0] * 4)
    assert ins == [1, 3, 5, 7] and len(T2) == 9
    assert np.allclose(T2, 300.0 * 2.0 ** (np.arange(9) / 8.0), rtol=1e-14)
    assert np.all(np.isnan(A2))
    assert list(D2) == [2.0, 1.5, 1.5, 1.5, 2.0, 2.0, 2.5, 2.0, 2.0]


def test_coupling_midpoints_follow_the_protocol_line():
    A = np.array([0.0, 0.2, 0.7, 1.0])
    T = 600.0 - 300.0 * A
    T2, A2, D2, ins = oracle.split_ladder(T, A, [2.0] * 4, [50, 50, 50], [10, 30, 5])
    assert ins == [1, 4]
    assert np.allclose(A2, [0.0, 0.1, 0.2, 0.7, 0.85, 1.0])
    assert np.allclose(T2, 600.0 - 300.0 * A2)


def test_resampling_from_the_lower_neighbour_gives_the_new_state():
    """Harmonic wells u_k = k_k x^2 / (2 kT): exact samples at stiffness 1, resampled into the
    state of stiffness 1.5 with weights exp(u_from - u_to), have variance kT / 1.5."""
    rng = np.random.default_rng(3)
    x = rng.normal(scale=1.0, size=20000)
    u_from, u_to = 0.5 * 1.0 * x * x, 0.5 * 1.5 * x * x
    idx = oracle.resample(u_from - u_to, 1000, seed=11, ctr=0)
    draws = x[idx]
    var = draws.var()
    se = var * math.sqrt(2.0 / len(draws)) * 1.5  # loose: draws repeat, add 50 %
    assert abs(var - 1.0 / 1.5) < 4 * se, (var, 1.0 / 1.5)
