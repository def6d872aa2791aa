"""Sparse coupling product (GDA_SPARSE: ELL gather over the nonzeros of J)
through the C ABI against the FP64 oracle, which applies the same J densely:
the sum over the nonzeros is the coupling sum of Eq. (2) with the zero terms
left out."""
import numpy as np
import pytest

import oracle
import synth
from oracle.gda_oracle import coupling_operand

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


def regular3(n, seed):
    J, _ = synth.sparse_3regular(n, seed)
    return J / 10.0  # weights in [-1, 1]: |lambda| <= 3


def start(model, n, R, seed):
    psi = synth.initial_amplitudes(n, R, seed, 0.3, model == "xy")
    gam = (0.1 * synth.normal(seed + 2, R * n)).astype(np.float32).astype(np.float64).reshape(R, n)
    return psi, gam, np.ones(R)


@pytest.mark.parametrize("model,n,R", [("xy", 300, 70), ("ising", 258, 150), ("ising", 46, 1)])
def test_sparse_coupling_matches_oracle(gda, model, n, R):
    J = regular3(n, 3)
    X = synth.initial_amplitudes(n, R, 5, 1.0, model == "xy")
    s = gda.Solver(J, None, gda.XY if model == "xy" else gda.ISING)
    Y = s.coupling(X, gda.SPARSE)
    ref = X @ coupling_operand(J).T
    assert np.abs(Y - ref).max() <= 1e-6 * np.abs(ref).max()
    s.close()


@pytest.mark.parametrize("integ", ["euler", "rk4"])
@pytest.mark.parametrize("model,n,R", [("xy", 300, 40), ("ising", 258, 90), ("ising", 130, 33)])
def test_sparse_200_steps_match_oracle(gda, integ, model, n, R):
    J = regular3(n, 7)
    g = 0.05 * synth.normal(8, n) if model == "ising" else synth.xy_gaussian(n, 8)[1]
    psi0, gam0, beta0 = start(model, n, R, 2)
    s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
    s.set_state(psi0, gam0, beta0, 0)
    kw = dict(dt=0.02, eps=0.2, eps_hat=0.3, beta0=0.4)
    s.run(gda.default_params(prec=gda.SPARSE, integ=gda.RK4 if integ == "rk4" else gda.EULER, init_mode=2,
                             **kw), R, 200)
    psi, gam, beta = s.get_state()[:3]
    ref, rg, rb = oracle.run(J, g, model, oracle.Params(integ=integ, **kw), R, 200,
                             state=(psi0, gam0, beta0))
    assert amp_err(psi, ref) < 1e-4
    assert np.abs(gam - rg).max() < 1e-4 * max(1.0, np.abs(rg).max())
    s.close()


@pytest.mark.parametrize("model,R", [("xy", 24), ("ising", 23)])
def test_sparse_noise_decay_and_resume(gda, model, R):
    # noise with decay uses the same density partial sums as the FP32 path;
    # resuming from a saved state is bit-identical to one run
    n = 200
    J = regular3(n, 11)
    g = synth.xy_gaussian(n, 2)[1]
    kw = dict(dt=0.02, eps=0.2, noise_D=0.05, noise_decay=1, seed=77, prec=gda.SPARSE, init_amp=0.1)
    m = gda.XY if model == "xy" else gda.ISING
    a = gda.Solver(J, g, m)
    a.run(gda.default_params(init_mode=1, **kw), R, 60)
    full = a.get_state()
    b = gda.Solver(J, g, m)
    b.run(gda.default_params(init_mode=1, **kw), R, 25)
    mid = b.get_state()
    c = gda.Solver(J, g, m)
    c.set_state(mid[0], mid[1], mid[2], mid[3])
    c.run(gda.default_params(init_mode=2, **kw), R, 35)
    for x, y in zip(full[:3], c.get_state()[:3]):
        assert np.array_equal(x, y)
    pk = {k: v for k, v in kw.items() if k != "prec"}
    ref = oracle.run(J, g, model, oracle.Params(init_mode=1, **pk), R, 60)[0]
    assert amp_err(full[0], ref) < 1e-4
    for s in (a, b, c):
        s.close()


def test_sparse_trace_and_final_energies(gda):
    n, R = 800, 32  # the size of the paper's sparse benchmark graphs
    J, _ = synth.sparse_3regular(n, 5)
    s = gda.Solver(J, None, gda.ISING)
    s.run(gda.default_params(dt=0.005, eps=0.1, prec=gda.SPARSE, energy_every=50, seed=3), R, 200)
    tr = []
    oracle.run(J, None, "ising", oracle.Params(dt=0.005, eps=0.1, energy_every=50, seed=3), R, 200, trace=tr)
    steps, E, r = s.trace()
    assert list(steps) == [t[0] for t in tr]
    assert np.allclose(E, [t[1] for t in tr], rtol=1e-4)
    psi = s.get_state()[0].astype(np.float64)
    assert np.allclose(s.energy(), oracle.energies(J, np.zeros(n), oracle.project(psi)), rtol=1e-9, atol=1e-9)
    s.close()


def test_sparse_rejects_dense_rows(gda):
    n = 100
    J, g = synth.xy_gaussian(n, 1)  # 99 nonzeros per row
    s = gda.Solver(J, g, gda.XY)
    with pytest.raises(gda.GdaError) as e:
        s.run(gda.default_params(prec=gda.SPARSE), 4, 1)
    assert e.value.status == 6  # GDA_ERR_UNSUPPORTED
    s.run(gda.default_params(prec=gda.FP32), 4, 1)  # the context stays usable
    # a row of exactly 64 nonzeros is accepted
    J2 = np.zeros((n, n))
    J2[0, 1:65] = 0.1
    J2[1:65, 0] = 0.1
    s2 = gda.Solver(J2, None, gda.ISING)
    X = synth.initial_amplitudes(n, 3, 4, 1.0, False)
    assert np.abs(s2.coupling(X, gda.SPARSE) - X @ J2.T).max() < 1e-6
    s.close()
    s2.close()


@pytest.mark.parametrize("model,R", [("ising", 5), ("xy", 2)])
def test_sparse_large_staged_form_matches_oracle(gda, model, R):
    """N = 14 336: the staged Euler kernel's 1024-thread form (one CTA per SM;
    a ragged pair for odd R), with noise and the ramp, against the oracle."""
    n = 14336
    J = regular3(n, 21)
    g = 0.05 * synth.normal(22, n) if model == "ising" else 0.05 * synth.normal(23, n)
    kw = dict(dt=0.02, eps=0.2, eps_hat=0.3, beta0=0.4, noise_D=0.02, seed=6, init_amp=0.3)
    s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
    s.run(gda.default_params(prec=gda.SPARSE, init_mode=1, **kw), R, 3)
    psi, gam = s.get_state()[:2]
    ref, rg, _ = oracle.run(J, g, model, oracle.Params(init_mode=1, **kw), R, 3)
    assert amp_err(psi, ref) < 1e-4
    assert np.abs(gam - rg).max() < 1e-4 * max(1.0, np.abs(rg).max())
    s.close()
