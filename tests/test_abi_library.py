"""The C-ABI library builds for sm_103a, loads, and exports every call include/algdock.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "algdock.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(algdock_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1507_03703_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ["algdock_grids_load", "algdock_hmc_cycle", "algdock_exchange", "algdock_reduced_energies",
              "algdock_mbar"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_declares_every_export():
    from paper_1507_03703_gb300 import algdock
    assert sorted(algdock.EXPORTS) == _declared()


def test_soft_elec_cap_matches_oracle_host_arithmetic(lib):
    """The one host-only call: the library's cap equals the oracle's for the same ligand."""
    import oracle
    from paper_1507_03703_gb300 import algdock
    from paper_1507_03703_gb300 import synthetic as S
    lig = S.make_ligand(30, seed=3)
    assert algdock.soft_elec_cap(lig) == pytest.approx(oracle.soft_elec_cap(lig), rel=1e-14)
    neutral = S.one_atom_ligand(charge=0.0)
    assert algdock.soft_elec_cap(neutral) == float("inf")


def test_create_without_a_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1507_03703_gb300 import algdock
    with pytest.raises(algdock.AlgdockError) as e:
        algdock.Context(0)
    assert e.value.status == algdock.E_CUDA
