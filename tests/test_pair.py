"""Two-SM tensor-core tiles (GDA_SCHEDULE_PAIR: clusters of two CTAs sharing
256 x BN tcgen05 cta_group::2 tiles) against the one-SM per-step kernel and
the operand-rounding oracle, for each tile width the chooser can pick."""
import math

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


def instance(model, n, seed):
    if model == "xy":
        return synth.xy_gaussian(n, seed)
    J, g = synth.sk_gaussian(n, seed)
    return J / math.sqrt(n), 0.05 * synth.normal(seed + 1, n)


def run_both(gda, model, n, R, prec, steps, **kw):
    J, g = instance(model, n, 3)
    out = []
    for sched in (gda.PER_STEP, gda.PAIR):
        s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
        s.run(gda.default_params(dt=0.02, eps=0.2, prec=prec, schedule=sched, init_amp=0.3, seed=4, **kw), R, steps)
        out.append(s.get_state())
        s.close()
    return J, g, out


# sizes chosen so that the pair tile width is 128 (first: the smallest tensor
# memory allocation), then 224 / 256
@pytest.mark.parametrize("model,n,R", [("ising", 256, 200), ("xy", 500, 100)])
def test_pair_bn128_matches_single_sm(gda, model, n, R):
    _, _, (a, b) = run_both(gda, model, n, R, gda.BF16, 50)
    assert amp_err(b[0], a[0]) < 1e-5
    assert np.abs(b[1] - a[1]).max() < 1e-5


def test_pair_one_step_matches_bf16_operand_oracle(gda):
    model, n, R = "xy", 512, 150
    J, g = instance(model, n, 9)
    psi0 = synth.initial_amplitudes(n, R, 2, 0.3, True)
    gam0 = (0.1 * synth.normal(4, R * n)).astype(np.float32).astype(np.float64).reshape(R, n)
    s = gda.Solver(J, g, gda.XY)
    s.set_state(psi0, gam0, np.ones(R), 0)
    s.run(gda.default_params(dt=0.02, eps=0.2, prec=gda.BF16, schedule=gda.PAIR, init_mode=2), R, 1)
    ref = oracle.run(J, g, model, oracle.Params(dt=0.02, eps=0.2, operand="bf16"), R, 1,
                     state=(psi0, gam0, np.ones(R)))[0]
    assert amp_err(s.get_state()[0], ref) < 1e-5
    s.close()


@pytest.mark.parametrize("model,n,R,prec", [("ising", 2048, 2048, "bf16"), ("ising", 2048, 1700, "bf16"),
                                            ("xy", 1024, 1024, "bf16"), ("ising", 2048, 2048, "fp8")])
def test_pair_wide_tiles_match_single_sm(gda, model, n, R, prec):
    p = gda.FP8 if prec == "fp8" else gda.BF16
    _, _, (a, b) = run_both(gda, model, n, R, p, 20, noise_D=0.02, noise_decay=1)
    assert amp_err(b[0], a[0]) < 1e-5
    assert np.abs(b[1] - a[1]).max() < 1e-5


def test_pair_energy_tracking_and_rk4(gda):
    n, R = 512, 96
    J, g = instance("xy", n, 5)
    res = []
    for sched in (gda.PER_STEP, gda.PAIR):
        s = gda.Solver(J, g, gda.XY)
        s.run(gda.default_params(dt=0.02, eps=0.2, prec=gda.BF16, integ=gda.RK4, schedule=sched, energy_every=10,
                                 seed=2, init_amp=0.2), R, 40)
        res.append((s.get_state()[0], s.trace()[1]))
        s.close()
    assert amp_err(res[1][0], res[0][0]) < 1e-5
    assert np.allclose(res[1][1], res[0][1], rtol=1e-6)


def test_pair_rejects_odd_row_blocks(gda):
    J, g = instance("xy", 300, 1)  # 3 row blocks of 128
    s = gda.Solver(J, g, gda.XY)
    with pytest.raises(gda.GdaError) as e:
        s.run(gda.default_params(prec=gda.BF16, schedule=gda.PAIR), 8, 1)
    assert e.value.status == 6
    with pytest.raises(gda.GdaError):
        s.run(gda.default_params(prec=gda.FP32, schedule=gda.PAIR), 8, 1)
    s.close()


# ---- the resident kernel's two-SM form (GDA_SCHEDULE_RESIDENT_PAIR)

@pytest.mark.parametrize("model,n,R", [("ising", 256, 200), ("xy", 500, 100), ("xy", 1000, 1024)])
def test_resident_pair_matches_resident(gda, model, n, R):
    """60 steps in 100-step segments of 20 (tracking), with noise decay (the
    density sums of every row block) and the coupling ramp: the pair form
    against the one-SM resident kernel, state and trace."""
    J, g = instance(model, n, 3)
    out = []
    for sched in (gda.RESIDENT, gda.RESIDENT_PAIR):
        s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
        s.run(gda.default_params(dt=0.02, eps=0.2, prec=gda.BF16, schedule=sched, init_amp=0.3, seed=4,
                                 energy_every=20, noise_D=0.01, noise_decay=1, beta0=0.5, eps_hat=0.1), R, 60)
        out.append((s.get_state(), s.trace()))
        s.close()
    (a, ta), (b, tb) = out
    assert amp_err(b[0], a[0]) < 1e-5
    assert np.abs(b[1] - a[1]).max() < 1e-5
    assert np.allclose(b[2], a[2], rtol=1e-6)
    assert list(ta[0]) == list(tb[0]) and np.allclose(tb[1], ta[1], rtol=1e-5)


def test_resident_pair_one_step_matches_bf16_operand_oracle(gda):
    model, n, R = "xy", 512, 150
    J, g = instance(model, n, 9)
    psi0 = synth.initial_amplitudes(n, R, 2, 0.3, True)
    gam0 = (0.1 * synth.normal(4, R * n)).astype(np.float32).astype(np.float64).reshape(R, n)
    s = gda.Solver(J, g, gda.XY)
    s.set_state(psi0, gam0, np.ones(R), 0)
    s.run(gda.default_params(dt=0.02, eps=0.2, prec=gda.BF16, schedule=gda.RESIDENT_PAIR, init_mode=2), R, 1)
    ref = oracle.run(J, g, model, oracle.Params(dt=0.02, eps=0.2, operand="bf16"), R, 1,
                     state=(psi0, gam0, np.ones(R)))[0]
    assert amp_err(s.get_state()[0], ref) < 1e-5
    s.close()


def test_resident_pair_rejects_odd_row_blocks(gda):
    J, g = instance("xy", 300, 1)  # 3 row blocks of 128
    s = gda.Solver(J, g, gda.XY)
    with pytest.raises(gda.GdaError) as e:
        s.run(gda.default_params(prec=gda.BF16, schedule=gda.RESIDENT_PAIR), 8, 1)
    assert e.value.status == 6
    s.close()
