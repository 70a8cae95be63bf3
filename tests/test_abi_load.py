"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/dcsd.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "dcsd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dcsd_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    from paper_2401_11935_gb300 import build, _lib
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    lib = ctypes.CDLL(_lib.LIB_PATH)
    names = _declared()
    assert "dcsd_residual" in names and "dcsd_solve" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(_lib.EXPORTS) <= set(names)


def test_heff_host_arithmetic():
    # dcsd_heff is pure host arithmetic (no device needed)
    from paper_2401_11935_gb300 import _lib
    H, ev, si = _lib.dcsd_heff(-0.25, 0.01)
    assert H == [-0.25, 0.01, 0.01, -0.25]
    assert ev == [-0.26, -0.24] and si == 1
    H, ev, si = _lib.dcsd_heff(-0.25, -0.01)
    assert ev == [-0.26, -0.24] and si == 0
