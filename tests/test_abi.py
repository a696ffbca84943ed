"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/mxe.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "mxe.h")).read()
    return sorted(set(re.findall(r"MXE_API\s+[\w\s\*]*?\b(mxe_\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("mxe_create", "mxe_destroy", "mxe_build_neighbors", "mxe_free_energy_grad", "mxe_relax",
              "mxe_diffuse_step"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_1910_01235_gb300 import mxe
    L = mxe.lib()
    for s in declared_symbols():
        assert hasattr(L, s), s
    assert set(declared_symbols()) == set(mxe.EXPORTS)


def test_status_strings():
    from paper_1910_01235_gb300 import mxe
    assert mxe.mxe_status_string(mxe.OK) == "ok"
    assert "max_iter" in mxe.mxe_status_string(mxe.ERR_NO_CONVERGE)


def test_workloads_do_not_load_cuda():
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r); import paper_1910_01235_gb300.workloads as w; "
            "w.config_vacancy_lattice(); import ctypes; "
            "print('mxe' in ' '.join(sys.modules))") % ROOT
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, check=True).stdout
    assert out.strip() == "False"
