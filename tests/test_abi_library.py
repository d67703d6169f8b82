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


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's sizes and offsets."""
    import shutil
    import subprocess
    from paper_1507_03703_gb300 import algdock
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"algdock_params": algdock.ParamsC, "algdock_run_desc": algdock.RunDescC,
               "algdock_array": algdock.ArrayC, "algdock_grid_desc": algdock.GridDesc,
               "algdock_restraint": algdock.RestraintC, "algdock_ligand": algdock.LigandC}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "algdock.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for cname, py in mirrors.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(py, f).offset, (cname, f)


def test_params_defaults(lib):
    """algdock_params_default (host only): the settings the library's run takes by default."""
    from paper_1507_03703_gb300 import algdock
    p = algdock.default_params()
    assert (p.n_steps, p.n_sweeps, p.max_sep, p.n_external) == (50, 25, 5, 0)
    assert (p.alpha_max, p.sigma_ext) == (algdock.ALPHA_MAX_EXTERNAL, algdock.SIGMA_TRANSLATION)
    assert (p.mbar_tol, p.mbar_max_iter, p.mbar_precision, p.checks) == (1e-10, 10000, 0, 0)
    q = algdock.default_params(n_steps=7, checks=1)
    assert (q.n_steps, q.checks, q.n_sweeps) == (7, 1, 25)
    with pytest.raises(TypeError):
        algdock.default_params(no_such_field=1)
