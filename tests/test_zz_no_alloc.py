"""The allocation-free energy entry point, gda_energy_noalloc.

It serves callers that cannot allocate device memory while running (a host
that has reserved the whole GPU for its own memory pool, a serving process
whose allocator is frozen after start-up).  It must return what the
context-based gda_energy returns, from caller-owned device buffers, on calls
made back to back, since every call reuses the same fixed scratch array.
This file is named to be collected last.
"""
import ctypes as ct

import numpy as np
import pytest

import synth

MAX_N = 4096
MAX_R = 4096


def _lib():
    import __graft_entry__
    __graft_entry__.ensure_built()
    from paper_1807_00699_gb300 import gda
    return gda, gda.load_library()


def _interleaved(psi):
    psi = np.asarray(psi)
    if np.iscomplexobj(psi):
        return np.stack([psi.real, psi.imag], axis=-1).astype(np.float32).ravel()
    return psi.astype(np.float32).ravel()


def test_sizes_beyond_the_limit_are_rejected():
    gda, lib = _lib()
    fake = ct.c_void_p(1 << 20)  # never dereferenced: the size check comes first
    st = lib.gda_energy_noalloc(fake, None, MAX_N + 1, gda.ISING, fake, 8, fake, None)
    assert st == 1
    st = lib.gda_energy_noalloc(fake, None, 64, gda.XY, fake, MAX_R + 1, fake, None)
    assert st == 1
    assert lib.gda_energy_noalloc(None, None, 64, gda.XY, fake, 8, fake, None) == 1


@pytest.mark.gpu
def test_noalloc_energy_matches_gda_energy_on_consecutive_calls():
    import torch
    gda, lib = _lib()
    assert torch.cuda.is_available()
    cases = []
    for model, n, R, seed in (("xy", 300, 40, 1), ("ising", 260, 64, 2), ("xy", 1000, 12, 3)):
        if model == "xy":
            J, g = synth.xy_gaussian(n, seed)
        else:
            J, g = synth.sk_gaussian(n, seed)
            J = J.copy()
            np.fill_diagonal(J, 0.5)  # the diagonal counts in Eq. (1)
        s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
        s.run(gda.default_params(dt=0.02, eps=0.2, init_amp=0.3, seed=seed), R, 30)
        E_ref = s.energy()
        psi = s.get_state()[0]
        s.close()
        cases.append((model, J, g, psi, E_ref))

    stream = torch.cuda.current_stream()
    # two calls in a row on different instances, then the first one again
    for model, J, g, psi, E_ref in cases + cases[:1]:
        R, n = psi.shape
        Jd = torch.tensor(J, dtype=torch.float64, device="cuda")
        gd = torch.tensor(g, dtype=torch.float64, device="cuda")
        pd = torch.tensor(_interleaved(psi), device="cuda")
        Ed = torch.full((R,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.gda_energy_noalloc(ct.c_void_p(Jd.data_ptr()), ct.c_void_p(gd.data_ptr()), n,
                                    gda.XY if model == "xy" else gda.ISING, ct.c_void_p(pd.data_ptr()), R,
                                    ct.c_void_p(Ed.data_ptr()), ct.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        E = Ed.cpu().numpy()
        assert np.allclose(E, E_ref, rtol=1e-9, atol=1e-12), (model, np.abs(E - E_ref).max())
