"""FP8 coupling operands (E4M3 J0 with per-row scales, E4M3 amplitudes at a
fixed scale) through the C ABI against the FP8-operand oracle."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle.gda_oracle import coupling_operand, fp8_coupling

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gda():
    import torch

    import __graft_entry__
    assert torch.cuda.is_available()
    __graft_entry__.ensure_built()
    from paper_1807_00699_gb300 import gda as mod
    return mod


def instance(model, n, seed):
    if model == "xy":
        return synth.xy_gaussian(n, seed)
    J, g = synth.sk_gaussian(n, seed)
    return J / math.sqrt(n), 0.05 * synth.normal(seed + 1, n)


def amp_err(psi, ref):
    num = np.abs(psi - ref).max(axis=1)
    den = np.maximum(np.abs(ref).max(axis=1), 1e-3)
    return (num / den).max()


# FP32 accumulation of exact E4M3 products against the oracle's FP64 sum:
# relative to sum_j |J0_ij X8_j| the difference is a few K 2^-24.
def coupling_tol(J0, X):
    return 1e-5 * (np.abs(X) @ np.abs(J0).T) + 1e-30


MODELS = [("xy", 300, 70), ("ising", 300, 150), ("xy", 129, 3), ("ising", 45, 1), ("ising", 1000, 300)]


@pytest.mark.parametrize("model,n,R", MODELS)
def test_fp8_coupling_matches_oracle(gda, model, n, R):
    J, g = instance(model, n, 11)
    X = synth.initial_amplitudes(n, R, 5, 1.0, model == "xy")
    s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
    Y = s.coupling(X, gda.FP8)
    J0 = coupling_operand(J)
    ref = fp8_coupling(J0, X)
    if model == "xy":
        tol = coupling_tol(J0, X.real) + coupling_tol(J0, X.imag)
    else:
        tol = coupling_tol(J0, X)
    assert np.all(np.abs(Y - ref) <= tol), np.abs(Y - ref).max()
    s.close()


def test_fp8_coupling_saturation_zero_row_and_subnormals(gda):
    n, R = 200, 9
    J, g = instance("ising", n, 4)
    J[17, :] = 0.0
    J[:, 17] = 0.0
    X = synth.initial_amplitudes(n, R, 8, 1.0, False)
    X[0, :50] = 12.0            # beyond 448 / 64 = 7: saturates
    X[1, :] *= 2.0 ** -10       # E4M3 subnormal range of X * 64
    X[2, 60:80] = -7.5
    s = gda.Solver(J, g, gda.ISING)
    Y = s.coupling(X, gda.FP8)
    J0 = coupling_operand(J)
    ref = fp8_coupling(J0, X)
    assert np.all(np.abs(Y - ref) <= coupling_tol(J0, X))
    assert np.all(Y[:, 17] == 0.0)
    s.close()


@pytest.mark.parametrize("model,n,R", MODELS[:2])
def test_fp8_euler_step_matches_fp8_operand_oracle(gda, model, n, R):
    J, g = instance(model, n, 9)
    psi0 = synth.initial_amplitudes(n, R, 2, 0.3, model == "xy")
    gam0 = (0.1 * synth.normal(4, R * n)).astype(np.float32).astype(np.float64).reshape(R, n)
    beta0 = np.ones(R)
    s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
    s.set_state(psi0, gam0, beta0, 0)
    s.run(gda.default_params(dt=0.02, eps=0.2, prec=gda.FP8, init_mode=2), R, 1)
    psi, gam = s.get_state()[:2]
    op = oracle.Params(dt=0.02, eps=0.2, operand="fp8")
    ref, rg, _ = oracle.run(J, g, model, op, R, 1, state=(psi0, gam0, beta0))
    assert amp_err(psi, ref) < 1e-5
    assert np.abs(gam - rg).max() < 1e-5
    s.close()


def test_fp8_rk4_step_matches_fp8_operand_oracle(gda):
    # RK4 stage states are rounded to E4M3 from FP32 (device) and FP64
    # (oracle); a stage value on an E4M3 rounding boundary may round apart,
    # moving Y by one E4M3 step of one operand.  The bound allows that.
    model, n, R = "xy", 300, 40
    J, g = instance(model, n, 9)
    psi0 = synth.initial_amplitudes(n, R, 2, 0.3, True)
    gam0 = np.zeros((R, n))
    s = gda.Solver(J, g, gda.XY)
    s.set_state(psi0, gam0, np.ones(R), 0)
    s.run(gda.default_params(dt=0.02, eps=0.2, prec=gda.FP8, integ=gda.RK4, init_mode=2), R, 1)
    psi = s.get_state()[0]
    ref = oracle.run(J, g, model, oracle.Params(integ="rk4", dt=0.02, eps=0.2, operand="fp8"), R, 1,
                     state=(psi0, gam0, np.ones(R)))[0]
    assert amp_err(psi, ref) < 2e-4
    s.close()


def test_fp8_resume_is_bit_identical(gda):
    n, R = 200, 24
    J, g = instance("xy", n, 3)
    kw = dict(dt=0.02, eps=0.2, noise_D=0.05, noise_decay=1, eps_hat=0.3, beta0=0.3, seed=77, prec=gda.FP8)
    a = gda.Solver(J, g, gda.XY)
    a.run(gda.default_params(init_mode=0, **kw), R, 60)
    full = a.get_state()
    b = gda.Solver(J, g, gda.XY)
    b.run(gda.default_params(init_mode=0, **kw), R, 25)
    mid = b.get_state()
    c = gda.Solver(J, g, gda.XY)
    c.set_state(mid[0], mid[1], mid[2], mid[3])
    c.run(gda.default_params(init_mode=2, **kw), R, 35)
    res = c.get_state()
    for x, y in zip(full[:3], res[:3]):
        assert np.array_equal(x, y)
    for s in (a, b, c):
        s.close()


def test_fp8_tracking_and_final_energies(gda):
    # The energy trace of an FP8 run is the BF16 product of the projected
    # spins; the final energies are FP64.  Both against the oracle on the
    # device's final state.
    n, R = 257, 33
    J, g = instance("xy", n, 21)
    s = gda.Solver(J, g, gda.XY)
    s.run(gda.default_params(dt=0.05, eps=0.1, prec=gda.FP8, energy_every=50, seed=3), R, 200)
    psi = s.get_state()[0]
    E = s.energy()
    ref = oracle.energies(J, g, oracle.project(psi.astype(np.complex128)))
    assert np.allclose(E, ref, rtol=1e-9, atol=1e-9)
    steps, Et, rt = s.trace()
    assert list(steps) == [50, 100, 150, 200]
    assert Et[-1] == pytest.approx(ref.min(), rel=2e-3)
    s.close()


def test_fp8_quality_close_to_bf16(gda):
    # Not amplitude-pinned: E4M3 operands perturb the coupling sum by ~2^-4
    # per term.  The best FP64 energy of an FP8 run stays within 1 % of the
    # BF16 run's on the same start.
    n, R = 400, 64
    J, g = instance("ising", n, 31)
    best = {}
    for prec in (gda.BF16, gda.FP8):
        s = gda.Solver(J, g, gda.ISING)
        s.run(gda.default_params(dt=0.05, eps=0.1, prec=prec, seed=5, schedule=gda.PER_STEP), R, 1500)
        best[prec] = s.energy().min()
        s.close()
    assert best[gda.FP8] <= best[gda.BF16] + 0.01 * abs(best[gda.BF16])
