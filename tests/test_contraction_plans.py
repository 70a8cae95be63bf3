"""The library's contraction planner (every contraction of the residual,
its reverse mode and the solver goes through it: modes classified as batch,
row, column or summed, adjacent modes merged, strides per operand) executed
on the host through the C ABI (dcsd_einsum_host) against numpy.einsum, for
every contraction spec in the CUDA sources and the two adjoint specs the
reverse sweep derives from each, on contiguous and on strided, permuted
views.  No GPU needed."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _specs():
    found = set()
    src = os.path.join(ROOT, "paper_2401_11935_gb300", "csrc")
    for name in sorted(os.listdir(src)):
        if name.endswith(".cu"):
            found |= set(re.findall(r'"([a-zA-Z]+,[a-zA-Z]+->[a-zA-Z]*)"', open(os.path.join(src, name)).read()))
    out = set()
    for s in found:
        a, rest = s.split(",")
        b, c = rest.split("->")
        out |= {s, f"{c},{b}->{a}", f"{a},{c}->{b}"}  # forward and the two adjoints
    return sorted(out)


SPECS = _specs()


def _view(rng, shape, strided):
    """An array of the given shape: contiguous, or a permuted, sliced view
    of a larger buffer (strides neither contiguous nor ordered)."""
    if not strided or len(shape) == 0:
        return rng.normal(size=shape)
    perm = rng.permutation(len(shape))
    big = [shape[p] + int(rng.integers(0, 3)) for p in perm]
    base = rng.normal(size=big)
    sl = tuple(slice(0, shape[p]) for p in perm)
    v = base[sl].transpose(np.argsort(perm))
    assert v.shape == tuple(shape)
    return v


def test_specs_found():
    assert len(SPECS) > 100 and "sijcd,acbd->sijab" in SPECS


@pytest.mark.parametrize("strided", [False, True])
def test_plans_match_numpy_einsum(strided):
    from paper_2401_11935_gb300 import _lib
    rng = np.random.default_rng(11 if strided else 10)
    for spec in SPECS:
        a_s, rest = spec.split(",")
        b_s, c_s = rest.split("->")
        size = {ch: int(rng.integers(1, 5)) for ch in set(a_s + b_s + c_s)}
        A = _view(rng, [size[ch] for ch in a_s], strided)
        B = _view(rng, [size[ch] for ch in b_s], strided)
        cbuf = rng.normal(size=[size[ch] + 1 for ch in c_s]) if c_s else rng.normal(size=())
        Cv = cbuf[tuple(slice(0, size[ch]) for ch in c_s)] if c_s else cbuf
        if strided and Cv.ndim > 1:
            perm = rng.permutation(Cv.ndim)
            cbuf = np.ascontiguousarray(cbuf.transpose(perm))
            Cv = cbuf[tuple(slice(0, size[c_s[p]]) for p in perm)].transpose(np.argsort(perm))
        before = cbuf.copy()
        C0 = np.array(Cv)
        alpha, beta = 0.7, (0.0 if rng.random() < 0.3 else -1.3)
        _lib.dcsd_einsum_host(spec, alpha, A, B, beta, Cv)
        want = alpha * np.einsum(spec, A, B) + (beta * C0 if beta != 0.0 else 0.0)
        assert np.allclose(Cv, want, rtol=1e-12, atol=1e-12), spec
        # nothing outside the output view is written
        if Cv.ndim:
            inside = np.zeros(cbuf.size, dtype=bool)
            offs = (np.indices(Cv.shape).reshape(Cv.ndim, -1).T * (np.array(Cv.strides) // 8)).sum(1)
            start = (Cv.__array_interface__["data"][0] - cbuf.__array_interface__["data"][0]) // 8
            inside[start + offs] = True
            outside = ~inside.reshape(cbuf.shape)
            assert np.array_equal(cbuf[outside], before[outside]), spec


@pytest.mark.parametrize("spec,shapes", [
    ("ab,bc->ac", [(2, 3), (4, 2), (2, 2)]),   # size mismatch of b
    ("aab,bc->ac", [(2, 2, 3), (3, 2), (2, 2)]),  # repeated letter
    ("ab,cd->ac", [(2, 3), (2, 3), (2, 2)]),   # b and d summed in one operand only
    ("ab,bc->ad", [(2, 3), (3, 2), (2, 2)]),   # output letter absent from the inputs
])
def test_planner_rejects(spec, shapes):
    from paper_2401_11935_gb300 import _lib
    A, B, Cm = (np.zeros(s) for s in shapes)
    with pytest.raises(_lib.DcsdError):
        _lib.dcsd_einsum_host(spec, 1.0, A, B, 0.0, Cm)
