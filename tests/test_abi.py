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


def test_create_batch_rejects_bad_arguments_before_touching_a_device():
    """Argument checks of mxe_create_batch run on the host: every rejected
    case returns MXE_ERR_ARG without a CUDA call (so this runs without a GPU)."""
    import ctypes as C
    from paper_1910_01235_gb300 import mxe, workloads as W
    L = mxe.lib()
    pot = mxe.make_potential(W.potential_single())
    boxes = (mxe.mxe_box * 2)(mxe.mxe_box((C.c_double * 3)(20.0, 20.0, 20.0)),
                              mxe.mxe_box((C.c_double * 3)(20.0, 20.0, 20.0)))
    ctx = C.c_void_p()

    def create(m, offsets, n, prec=mxe.FP64, bx=boxes):
        off = (C.c_int64 * len(offsets))(*offsets)
        return L.mxe_create_batch(C.byref(ctx), m, bx, off, C.byref(pot), n, prec, None)

    assert create(2, [1, 2, 4], 4) == mxe.ERR_ARG       # first offset not 0
    assert create(2, [0, 3, 2], 2) == mxe.ERR_ARG       # decreasing
    assert create(2, [0, 2, 4], 5) == mxe.ERR_ARG       # last offset != n
    assert create(-1, [0], 0) == mxe.ERR_ARG
    assert create((1 << 20) + 1, [0, 0], 0) == mxe.ERR_ARG
    assert create(2, [0, 2, 4], 4, prec=7) == mxe.ERR_ARG
    bad = (mxe.mxe_box * 2)(mxe.mxe_box((C.c_double * 3)(20.0, 20.0, 20.0)),
                            mxe.mxe_box((C.c_double * 3)(20.0, -1.0, 20.0)))
    assert create(2, [0, 2, 4], 4, bx=bad) == mxe.ERR_ARG
    assert ctx.value is None
