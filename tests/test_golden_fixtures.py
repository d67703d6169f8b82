"""The stored oracle fixtures are what their generators write: the twenty-atom BPMF groups come
from tests/golden/make_bpmf_20atom.py under the protocol that script runs (no GPU needed)."""
import importlib.util
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _load_script():
    spec = importlib.util.spec_from_file_location("make_bpmf_20atom", os.path.join(HERE, "golden",
                                                                                     "make_bpmf_20atom.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_bpmf_20atom_fixture_matches_its_generator():
    gen = _load_script()
    d = json.load(open(os.path.join(HERE, "golden", "bpmf_20atom_oracle.json")))
    assert d["protocol"] == gen.PROTOCOL
    groups = [r["group"] for r in d["groups"]]
    assert groups == list(range(len(groups)))  # every group from 0 on, none twice
    v = np.array([r["bpmf_kT"] for r in d["groups"]])
    assert d["n_groups"] == len(v) and np.all(np.isfinite(v))
    assert abs(d["mean_kT"] - v.mean()) < 1e-12
    assert abs(d["standard_error_kT"] - v.std(ddof=1) / np.sqrt(len(v))) < 1e-12
