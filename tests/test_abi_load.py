"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/dcsd.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

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


def _host_system():
    import numpy as np
    from synth import make_system
    s = make_system((2, 5, 12), seed=1)
    return [np.ascontiguousarray(x) for x in (s.fock_a, s.fock_b, s.B)], s


def test_init_checks_arguments_before_the_device():
    """dcsd_init refuses NULL pointers, bad dimensions and a bad memory kind
    with INVALID_ARG and its message, on any machine."""
    from paper_2401_11935_gb300 import _lib as L
    (fa, fb, B), s = _host_system()
    args = dict(n_c=s.n_c, n_v=s.n_v, naux=s.naux, eps=None, fock_a=fa.ctypes.data, fock_b=fb.ctypes.data,
                B=B.ctypes.data, mem_kind=L.MEM_HOST, stream=None)
    for change, words in (({"fock_a": None}, "NULL"), ({"B": None}, "NULL"), ({"n_c": -1}, "dimensions"),
                          ({"n_v": 0}, "dimensions"), ({"naux": 0}, "dimensions"), ({"mem_kind": 7}, "mem_kind")):
        with pytest.raises(L.DcsdError) as ei:
            L.dcsd_init(**{**args, **change})
        assert ei.value.status == 1 and words in str(ei.value), str(ei.value)


def test_no_device_fails_loudly():
    """Without a GPU the valid call returns NO_DEVICE, and the Engine raises:
    there is no CPU path to fall back to."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2401_11935_gb300 as P
    from paper_2401_11935_gb300 import _lib as L
    (fa, fb, B), s = _host_system()
    with pytest.raises(L.DcsdError) as ei:
        L.dcsd_init(s.n_c, s.n_v, s.naux, None, fa.ctypes.data, fb.ctypes.data, B.ctypes.data, L.MEM_HOST, None)
    assert ei.value.status == 7 and "no CUDA device" in str(ei.value)
    with pytest.raises(Exception):
        P.Engine.from_system(s)
