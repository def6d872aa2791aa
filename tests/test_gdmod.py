"""GD-mod (Eq. 6 with Delta_ij = gamma_i^inj + gamma_j^inj, per-restart K)
through the C ABI against the FP64 GD-mod oracle on the same seeded start."""
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
    __graft_entry__.ensure_built()
    from paper_1807_00699_gb300 import gda as mod
    return mod


def amp_err(psi, ref):
    num = np.abs(psi - ref).max(axis=1)
    den = np.maximum(np.abs(ref).max(axis=1), 1e-3)
    return (num / den).max()


KW = dict(dt=0.02, eps=0.2, eps_hat=0.5, gamma_c=3.0, beta0=0.3, gamma0=0.1, init_amp=0.3, seed=5)


@pytest.mark.parametrize("model,n,R", [("xy", 300, 20), ("ising", 257, 33), ("xy", 45, 3)])
def test_gdmod_200_steps_match_oracle(gda, model, n, R):
    J, g = synth.xy_gaussian(n, 7)
    if model == "ising":
        g = 0.05 * synth.normal(8, n)
    s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
    s.run(gda.default_params(coupling=gda.GDMOD, init_mode=1, **KW), R, 200)
    psi, gam = s.get_state()[:2]
    ref, rg, _ = oracle.gdmod_run(J, g, model, oracle.Params(init_mode=1, **KW), R, 200)
    assert amp_err(psi, ref) < 1e-4
    assert np.abs(gam - rg).max() < 1e-4 * max(1.0, np.abs(rg).max())
    s.close()


def test_gdmod_noise_parity_and_continuation(gda):
    n, R = 150, 12
    J, g = synth.xy_gaussian(n, 3)
    kw = dict(KW, noise_D=0.05)
    s = gda.Solver(J, g, gda.XY)
    s.run(gda.default_params(coupling=gda.GDMOD, init_mode=1, **kw), R, 40)
    s.run(gda.default_params(coupling=gda.GDMOD, init_mode=2, **kw), R, 60)
    psi = s.get_state()[0]
    t = gda.Solver(J, g, gda.XY)
    t.run(gda.default_params(coupling=gda.GDMOD, init_mode=1, **kw), R, 100)
    assert np.array_equal(psi, t.get_state()[0])  # resuming within the context is exact
    ref = oracle.gdmod_run(J, g, "xy", oracle.Params(init_mode=1, **kw), R, 100)[0]
    assert amp_err(psi, ref) < 1e-4
    s.close()
    t.close()


def test_gdmod_energies_and_trace(gda):
    n, R = 200, 16
    J, g = synth.xy_gaussian(n, 12)
    s = gda.Solver(J, g, gda.XY)
    s.run(gda.default_params(coupling=gda.GDMOD, init_mode=1, energy_every=25, **KW), R, 100)
    tr = []
    oracle.gdmod_run(J, g, "xy", oracle.Params(init_mode=1, energy_every=25, **KW), R, 100, trace=tr)
    steps, E, r = s.trace()
    assert list(steps) == [t[0] for t in tr]
    assert np.allclose(E, [t[1] for t in tr], rtol=1e-4)
    psi = s.get_state()[0].astype(np.complex128)
    assert np.allclose(s.energy(), oracle.energies(J, g, oracle.project(psi)), rtol=1e-9, atol=1e-9)
    s.close()


def test_gdmod_rejections(gda):
    J, g = synth.xy_gaussian(40, 1)
    s = gda.Solver(J, g, gda.XY)
    for kw in (dict(prec=gda.BF16), dict(integ=gda.RK4), dict(noise_D=0.1, noise_decay=1),
               dict(schedule=gda.RESIDENT)):
        with pytest.raises(gda.GdaError) as e:
            s.run(gda.default_params(coupling=gda.GDMOD, **kw), 4, 1)
        assert e.value.status == 6  # GDA_ERR_UNSUPPORTED
    # continuing needs a GD-mod coupling state for the same R
    s.run(gda.default_params(), 4, 2)
    with pytest.raises(gda.GdaError) as e:
        s.run(gda.default_params(coupling=gda.GDMOD, init_mode=2), 4, 1)
    assert e.value.status == 7  # GDA_ERR_STATE
    with pytest.raises(gda.GdaError):
        s.run(gda.default_params(coupling=5), 4, 1)
    s.close()
