"""The bonded-force layout (algdock_gather_layout, host only): an arrangement of the same terms and
slots in which every slot still sits in the block of the atom its term acts on, the shared-memory
wavefront counts recomputed here from the model the header states (for the input order and for the
layout), fewer wavefronts than the input order, determinism, and the topologies it rejects."""
import numpy as np
import pytest

from paper_1507_03703_gb300 import algdock as AD
from paper_1507_03703_gb300 import synthetic as S


@pytest.fixture(scope="module", autouse=True)
def _library():
    try:
        AD.load_library()
    except (ImportError, OSError) as e:
        pytest.skip(str(e))


def _terms(lig):
    return [np.asarray(lig.bonds, np.int64).reshape(-1, 2), np.asarray(lig.angles, np.int64).reshape(-1, 3),
            np.asarray(lig.torsions, np.int64).reshape(-1, 4)]


def _wavefronts(ids):
    """One quarter-warp's 16-byte load: the most distinct addresses in one bank group (id mod 8)."""
    per_bank = {}
    for i in ids:
        per_bank.setdefault(i % 8, set()).add(i)
    return max(len(v) for v in per_bank.values())


def _cost(lig, order, slots, lane_run):
    """Total wavefronts per force evaluation of the three loads, from the layout alone."""
    na = len(lig.mass)
    T = _terms(lig)
    n = [len(t) for t in T]
    n_slots = 2 * n[0] + 3 * n[1] + 4 * n[2]
    if n_slots == 0:
        return 0
    counts = np.zeros(na, np.int64)
    for t in T:
        for row in t:
            for a in row:
                counts[a] += 1
    Lr = max(-(-n_slots // 32), -(-int(counts.max()) // 3))
    atom_of = np.repeat(np.arange(na), counts)
    total = 0
    # the bonded terms' position loads: kind by kind, round by round, role by role
    off = 0
    for k, t in enumerate(T):
        pos = order[off:off + n[k]]
        off += n[k]
        for rnd in range(-(-n[k] // 32)):
            for r in range(t.shape[1] if n[k] else 0):
                for q in range(4):
                    ps = [p for p in range(32 * rnd + 8 * q, 32 * rnd + 8 * q + 8) if p < n[k]]
                    if ps:
                        total += _wavefronts([int(t[pos[p], r]) for p in ps])
    # the gather's slot loads at each run position (a lane past the list reads the zero slot)
    for j in range(Lr):
        for q in range(4):
            ids = []
            for lane in range(8 * q, 8 * q + 8):
                e = lane_run[lane] * Lr + j
                ids.append(int(slots[e]) if e < n_slots else n_slots)
            total += _wavefronts(ids)
    # the owners' loads of each atom's k-th partial sum (an atom with fewer reads the zero slot)
    parts = [[] for _ in range(na)]
    for e in range(n_slots):
        if e % Lr == Lr - 1 or e + 1 == n_slots or atom_of[e + 1] != atom_of[e]:
            parts[atom_of[e]].append(int(slots[e]))
    for a0 in range(0, na, 32):
        for k in range(4):
            for q in range(4):
                atoms = [i for i in range(a0 + 8 * q, a0 + 8 * q + 8) if i < na]
                if atoms:
                    total += _wavefronts([parts[i][k] if k < len(parts[i]) else n_slots for i in atoms])
    return total


def _input_order_slots(lig):
    """The slot list of the input order: per atom, its slots in the order the terms list them."""
    na = len(lig.mass)
    b, a, t = _terms(lig)
    nb, nang, ntor = len(b), len(a), len(t)
    inc = [[] for _ in range(na)]
    for i, row in enumerate(b):
        for r in range(2):
            inc[row[r]].append(r * nb + i)
    for i, row in enumerate(a):
        for r in range(3):
            inc[row[r]].append(2 * nb + r * nang + i)
    for i, row in enumerate(t):
        for r in range(4):
            inc[row[r]].append(2 * nb + 3 * nang + r * ntor + i)
    return np.array([s for lst in inc for s in lst], np.int64)


def _check_arrangement(lig, lay):
    na = len(lig.mass)
    T = _terms(lig)
    n = [len(t) for t in T]
    order, slots, lane_run = lay["term_order"], lay["slots"].astype(np.int64), lay["lane_run"]
    off = 0
    for k in range(3):  # each kind's positions hold each of its terms once
        assert sorted(order[off:off + n[k]].tolist()) == list(range(n[k]))
        off += n[k]
    assert sorted(lane_run.tolist()) == list(range(32))
    n_slots = 2 * n[0] + 3 * n[1] + 4 * n[2]
    assert sorted(slots.tolist()) == list(range(n_slots))
    # every slot lies in the block of the atom its term's role acts on
    counts = np.zeros(na, np.int64)
    for t in T:
        np.add.at(counts, t.reshape(-1), 1)
    atom_of = np.repeat(np.arange(na), counts)
    base = [0, 2 * n[0], 2 * n[0] + 3 * n[1]]
    pos_order = [order[:n[0]], order[n[0]:n[0] + n[1]], order[n[0] + n[1]:]]
    for e, s in enumerate(slots):
        k = 2 if s >= base[2] and n[2] else (1 if s >= base[1] and n[1] else 0)
        r, p = divmod(int(s) - base[k], n[k])
        assert T[k][pos_order[k][p], r] == atom_of[e]


@pytest.mark.parametrize("which", ["paper", "small", "n96", "n33", "n5"])
def test_layout_is_a_valid_arrangement_with_the_stated_wavefronts(which):
    lig = {"paper": lambda: S.config_paper_scale(2).ligand, "small": lambda: S.config_small(1).ligand,
           "n96": lambda: S.make_ligand(96, seed=11), "n33": lambda: S.make_ligand(33, seed=12),
           "n5": lambda: S.make_ligand(5, seed=13)}[which]()
    lay = AD.gather_layout(lig)
    _check_arrangement(lig, lay)
    n_terms = sum(len(t) for t in _terms(lig))
    before, after = lay["wavefronts"]
    # the counts follow from the layout by the header's model
    assert _cost(lig, lay["term_order"], lay["slots"], lay["lane_run"]) == after
    ident = np.concatenate([np.arange(len(t)) for t in _terms(lig)]) if n_terms else np.zeros(0, np.int64)
    assert _cost(lig, ident, _input_order_slots(lig), np.arange(32)) == before
    assert after <= before
    if which == "paper":  # the 48-atom ligand: 358 wavefronts in the input order
        assert before == 358 and after <= 0.65 * before
    # deterministic, and the same from a second call (cached) as from the first
    again = AD.gather_layout(lig)
    for key in ("term_order", "slots", "lane_run"):
        assert np.array_equal(again[key], lay[key])


def test_layout_of_ligands_without_terms():
    lig = S.make_ligand(1, seed=3)
    lay = AD.gather_layout(lig)
    assert lay["wavefronts"] == (0, 0)
    assert lay["slots"].size == 0 and lay["term_order"].size == 0
    assert np.array_equal(lay["lane_run"], np.arange(32))


def test_layout_rejects_out_of_range_indices():
    lig = S.make_ligand(6, seed=4)
    bad = np.asarray(lig.bonds).copy()
    bad.reshape(-1, 2)[0, 1] = 6
    lig.bonds = bad
    with pytest.raises(AD.AlgdockError) as e:
        AD.gather_layout(lig)
    assert e.value.status == AD.E_INVALID
