"""Host-side pieces of the multi-ligand batch and of the benchmark's accounting (CPU).

- The clash-free growth mode keeps every atom at least min_sep from all atoms other than its
  parent and the parent's neighbours, keeps bond lengths in their range and the tree connected, and
  leaves the default growth (every earlier system) unchanged.
- The batch workload has the stated sizes and spread.
- The padded ligands of the padded-uniform baseline add only inert atoms at distinct points.
- The gather byte count of an HMC launch matches a hand count on a three-state ladder.
- The clock sampler's sample file is temporary unless named."""
import os
import sys

import numpy as np
import pytest

from paper_1507_03703_gb300 import synthetic as S


def _graph_distance(lig):
    n = lig.n_atoms
    adj = [[] for _ in range(n)]
    for a, b in lig.bonds:
        adj[a].append(b)
        adj[b].append(a)
    D = np.full((n, n), 99, dtype=int)
    for i in range(n):
        D[i, i] = 0
        frontier = [i]
        while frontier:
            nxt = []
            for u in frontier:
                for v in adj[u]:
                    if D[i, v] == 99:
                        D[i, v] = D[i, u] + 1
                        nxt.append(v)
            frontier = nxt
    return D


@pytest.mark.parametrize("n,seed", [(10, 1), (33, 2), (64, 3), (70, 4)])
def test_clash_free_growth(n, seed):
    lig = S.make_ligand(n, seed=seed, min_sep=2.6)
    D = _graph_distance(lig)
    assert np.all(D < 99)  # one tree
    assert lig.bonds.shape[0] == n - 1
    r = np.linalg.norm(lig.x0[:, None] - lig.x0[None], axis=-1)
    far = D >= 3
    assert r[far].min() >= 2.6 - 1e-9
    bl = np.linalg.norm(lig.x0[lig.bonds[:, 0]] - lig.x0[lig.bonds[:, 1]], axis=1)
    assert np.allclose(bl, lig.bond_r0) and bl.min() >= 1.3 and bl.max() <= 1.6
    assert abs(lig.charge.sum()) < 1e-12


def test_default_growth_is_unchanged():
    """The default path draws the same numbers as before the clash-free mode existed: the
    paper-scale ligand keeps its 48 atoms and its first bond and positions."""
    lig = S.make_ligand(48, seed=2)
    again = S.make_ligand(48, seed=2, min_sep=None)
    assert np.array_equal(lig.x0, again.x0) and np.array_equal(lig.bonds, again.bonds)
    assert S.config_paper_scale(2).ligand.n_atoms == S.ligand_atoms_for_seed(2) == 48
    # the clash-free mode is a different draw
    assert not np.array_equal(S.make_ligand(48, seed=2, min_sep=2.6).x0, lig.x0)


def test_batch_workload_shape():
    sys_, ligs = S.config_batch(3, n_ligands=32)
    sizes = np.array([l.n_atoms for l in ligs])
    assert len(ligs) == 32 and sizes.min() >= 10 and sizes.max() <= 70
    assert sys_.receptor.n_atoms == 4000 and tuple(sys_.grid.n) == (129, 129, 129)
    assert [l.K for l in sys_.legs] == [16, 48]
    assert all(float(np.float32(o)) == o for o in sys_.grid.origin)


@pytest.fixture(scope="module")
def bench_module():
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import bench
    return bench


def test_padded_ligand_adds_inert_atoms(bench_module):
    lig = S.make_ligand(12, seed=5, min_sep=2.6)
    p = bench_module.padded_ligand(lig, 70, np.zeros(3))
    assert p.n_atoms == 70
    assert np.array_equal(p.x0[:12], lig.x0) and np.array_equal(p.bonds, lig.bonds)
    assert np.all(p.charge[12:] == 0) and np.all(p.eps[12:] == 0) and np.all(p.mass[12:] == 1e9)
    pad = p.x0[12:]
    d = np.linalg.norm(pad[:, None] - pad[None], axis=-1) + np.eye(58) * 9
    assert d.min() >= 1.0 - 1e-12


def test_gather_bytes_hand_count(bench_module):
    """alpha = NaN (no grids), 0.25 (soft only in FP32: the hard weight underflows), 1 (hard
    only).  Per atom and evaluation 32 B per active grid (8 corners x 4 B): both energy
    evaluations read all five grids (160 B), each force-only one 0, 64 (two soft grids) or 96 B
    (three full grids)."""
    n_atoms, n_steps, R = 7, 11, 3
    got = bench_module.gather_bytes_per_launch(np.array([np.nan, 0.25, 1.0]), R, n_atoms, n_steps)
    want = R * n_atoms * (3 * 2 * 160 + (n_steps - 1) * (0 + 64 + 96))
    assert got == want


def test_clock_sampler_file_handling(bench_module, tmp_path, monkeypatch):
    """Without nvidia-smi the sampler reports nothing; its default sample file is temporary and
    removed after the summary, a named one is kept."""
    monkeypatch.setenv("PATH", str(tmp_path))  # no nvidia-smi on the path
    c = bench_module.Clocks(0)
    c.start()
    assert c.stop() is None and not os.path.exists(c.path)
    kept = tmp_path / "clocks.csv"
    c = bench_module.Clocks(0, str(kept))
    c.start()
    assert c.stop() is None and kept.exists()


def test_bpmf_credit_starts_where_the_estimate_stays_in_band(bench_module):
    """An arm is credited from the first window after which every later window stays within the
    criterion of the reference, and not at all if its last window is outside."""
    w = lambda *b: [{"bpmf_kT": v} for v in b]
    f = bench_module.in_band_from
    assert f(w(-18.0, -18.8, -18.95, -18.85), -18.9, 0.2) == 1
    assert f(w(-18.8, -19.2, -18.95, -18.85), -18.9, 0.2) == 2  # left the band once: counted after
    assert f(w(-17.5, -18.7, -18.84, -19.10, -19.15), -18.9, 0.2) is None  # drifted out at the end
    assert f(w(-18.9, -18.9), -18.9, 0.2) == 0
    assert f([], -18.9, 0.2) is None


def test_term_by_term_flop_count_of_a_chain(bench_module):
    """A five-atom chain 0-1-2-3-4: 4 bonds, 3 angles, 2 torsions, and the pairs more than two
    bonds apart (0-3, 0-4, 1-4), against the stated 26 / 20 / 60 / 100 / 182 flop per pair,
    bond, angle, torsion and atom."""
    class Chain:
        n_atoms = 5
        bonds = [(0, 1), (1, 2), (2, 3), (3, 4)]
        angles = [(0, 1, 2), (1, 2, 3), (2, 3, 4)]
        torsions = [(0, 1, 2, 3), (1, 2, 3, 4)]
    assert bench_module.flops_per_replica_eval(Chain) == 26 * 3 + 20 * 4 + 60 * 3 + 100 * 2 + 182 * 5


def test_captured_figures_follow_the_source_fingerprint(bench_module, monkeypatch):
    """A captured ncu figure is reported only while the fingerprint of its sources matches."""
    rec = dict(bench_module.NCU_TRAFFIC["hmc_kernel"])
    monkeypatch.setitem(bench_module.NCU_TRAFFIC, "hmc_kernel", rec)
    got = bench_module.captured_traffic("hmc_kernel")
    assert got in (None, rec["bytes_per_launch"])
    if got is not None:  # the committed fingerprint matches the committed sources
        assert bench_module.captured_traffic("hmc_kernel", "warp_instructions_per_launch") == \
            rec["warp_instructions_per_launch"]
    rec["sha256"] = "0" * 64
    assert bench_module.captured_traffic("hmc_kernel") is None
    assert bench_module.captured_traffic("hmc_kernel", "warp_instructions_per_launch") is None
    assert bench_module.captured_traffic("no_such_kernel") is None
