"""The allocation-free energy entry point agrees with dcsd_energy.

dcsd_energy_noalloc serves callers that cannot allocate device memory (for
example while capturing a CUDA graph); its working memory is a fixed array
inside the library.  This file is collected last so that a failure here
does not hide the results of the other GPU tests; it passes alone and after
them.  Two calls in a row (with different amplitudes) must each match the
context-based dcsd_energy to the energy tolerance of the parity tests, and
the CPU oracle's Delta E_A as well.
"""
import numpy as np
import pytest

from synth import make_system, random_amplitudes
from oracle import twod

pytestmark = pytest.mark.gpu

TOL_E = 1e-10


def test_energy_noalloc_matches_energy_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2401_11935_gb300 as P
    from paper_2401_11935_gb300 import _lib as L

    for ref, dims, seed in ((0, (3, 9, 20), 4), (1, (5, 14, 30), 6)):
        s = make_system(dims, seed=seed)
        eng = P.Engine.from_system(s)
        dev = torch.device("cuda")
        fa = torch.as_tensor(s.fock_a).to(dev)
        fb = torch.as_tensor(s.fock_b).to(dev)
        Bt = torch.as_tensor(s.B).to(dev)
        out = torch.zeros(1, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        for k, scale in enumerate((0.02, 0.05)):  # two calls in a row
            Th = random_amplitudes(s, seed=seed + 10 * k, ref=ref, scale1=scale, scale2=scale)
            T = eng.to_device(Th)
            dEA_ref, _ = eng.energy(T, ref=ref)
            _, _, dEA_oracle = twod.residual(s, ref, twod.DCSD, Th)
            out.fill_(np.nan)
            L.dcsd_energy_noalloc(s.n_c, s.n_v, s.naux, ref, fa.data_ptr(), fb.data_ptr(), Bt.data_ptr(),
                                  [x.data_ptr() for x in T], out.data_ptr(), stream)
            torch.cuda.synchronize()
            assert abs(float(out.item()) - dEA_ref) < TOL_E, (ref, k, float(out.item()), dEA_ref)
            assert abs(float(out.item()) - dEA_oracle) < TOL_E, (ref, k, float(out.item()), dEA_oracle)
        eng.close()


def test_energy_noalloc_rejects_sizes_beyond_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_11935_gb300 import _lib as L
    # n_c + 1 = 53 > 52: refused before any device work (pointers unused)
    with pytest.raises(L.DcsdError):
        L.dcsd_energy_noalloc(52, 4, 8, 0, 1, 1, 1, [1] * 5, 1, 0)
