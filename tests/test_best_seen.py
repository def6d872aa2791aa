"""The running best of the energy trace (gda_best_seen): the configuration a
restart held when a tracking evaluation found the lowest energy so far, kept by
the library and verified in FP64 / exact integers at the end."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gda():
    import torch

    import __graft_entry__
    assert torch.cuda.is_available()
    __graft_entry__.build()
    from paper_1807_00699_gb300 import gda as mod
    return mod


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_best_seen_matches_trace_minimum_xy(gda, prec):
    n, R = 300, 64
    J, g = synth.xy_gaussian(n, 21)
    s = gda.Solver(J, g, gda.XY)
    p = gda.BF16 if prec == "bf16" else gda.FP32
    s.run(gda.default_params(dt=0.05, eps=0.1, prec=p, energy_every=10, seed=4), R, 400)
    steps, Et, rs = s.trace()
    E, r, step, th = s.best_seen()
    k = int(np.argmin(Et))  # first occurrence of the lowest tracked energy
    assert step == steps[k] and r == rs[k]
    # the tracked value is the product with BF16 (or FP32) operands: BF16 rounds
    # J and the spins to 8 bits each, so it sits within ~1e-3 of the FP64 energy
    assert E == pytest.approx(Et[k], rel=1e-3 if prec == "bf16" else 1e-4)
    assert oracle.hamiltonian_theta(J, g, th) == pytest.approx(E, rel=1e-9, abs=1e-9)
    s.close()


def test_best_seen_exact_for_integer_ising(gda):
    n, R = 20, 64
    J, g = synth.ising_pm1(n, 3)
    s = gda.Solver(J, g, gda.ISING)
    s.run(gda.default_params(dt=0.01, eps=0.1, energy_every=25, seed=2), R, 1000)
    E, r, step, spins = s.best_seen()
    assert E == oracle.energies(J, g, spins.astype(np.float64)[None])[0]
    assert E == round(E)
    s.close()


def test_best_seen_spans_continuations_and_resets(gda):
    n, R = 200, 32
    J, g = synth.xy_gaussian(n, 5)
    s = gda.Solver(J, g, gda.XY)
    kw = dict(dt=0.05, eps=0.1, energy_every=20, seed=9)
    with pytest.raises(gda.GdaError) as e:  # nothing tracked yet
        s.run(gda.default_params(dt=0.05, eps=0.1, seed=9), R, 10)
        s.best_seen()
    assert e.value.status == 7
    s.run(gda.default_params(**kw), R, 100)
    E1, _, st1, _ = s.best_seen()
    tr1 = s.trace()[1].min()
    s.run(gda.default_params(init_mode=2, **kw), R, 200)
    E2, _, st2, _ = s.best_seen()
    tr2 = s.trace()[1].min()
    if tr2 < tr1:
        assert st2 > 100
    else:
        assert st2 == st1 and E2 == E1
    s.run(gda.default_params(**kw), R, 40)  # a fresh run starts a new record
    _, _, st3, _ = s.best_seen()
    assert st3 <= 40
    s.close()
