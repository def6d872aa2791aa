"""Batched runs (many instances in one launch per step) against the oracle
and against single-instance runs of the same instances and seeds."""
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


def mix(gda):
    out = []
    for k, (n, R, xy) in enumerate([(50, 16, True), (130, 40, False), (300, 100, True), (300, 16, False),
                                    (129, 256, True), (1, 3, False)]):
        J, g = synth.xy_gaussian(n, 100 + k)  # N(0, 1/N) couplings keep dt = 0.05 stable
        if not xy:
            g = np.zeros(n)
        out.append((J, g, gda.XY if xy else gda.ISING, R))
    return out


def test_batch_equals_single_instance_runs(gda):
    insts = mix(gda)
    b = gda.Batch(insts, seed=2024)
    kw = dict(dt=0.05, eps=0.2, eps_hat=0.3, beta0=0.4, noise_D=0.02, init_mode=1, init_amp=0.2, prec=gda.BF16)
    b.run(gda.default_params(**kw), 150)  # one captured chunk of 100 steps, then 50 single launches
    Eb, rb = b.best()
    for k, (J, g, model, R) in enumerate(insts):
        s = gda.Solver(J, g, model)
        s.run(gda.default_params(seed=b.instance_seed(k), schedule=gda.PER_STEP, **kw), R, 150)
        psi, gam, beta, _ = s.get_state()
        bpsi, bgam, bbeta = b.get_state(k)
        assert np.array_equal(psi, bpsi), k
        assert np.array_equal(gam, bgam) and np.array_equal(beta, bbeta), k
        E = s.energy()
        assert Eb[k] == pytest.approx(E.min(), rel=1e-9, abs=1e-9) and E[rb[k]] == pytest.approx(E.min(), rel=1e-9)
        s.close()
    b.close()


def ragged_mix(gda):
    """N = 1, 50, 129, 300, Ising and XY, fields on the XY instances."""
    out = []
    for k, (n, R, xy) in enumerate([(1, 3, False), (50, 16, True), (129, 40, False), (129, 24, True),
                                    (300, 100, False), (300, 70, True), (50, 33, False)]):
        J, g = synth.xy_gaussian(n, 300 + k)
        if not xy:
            g = np.zeros(n)
        out.append((J, g, gda.XY if xy else gda.ISING, R))
    return out


KW_MIX = dict(dt=0.05, eps=0.2, eps_hat=0.3, beta0=0.4, noise_D=0.02, init_mode=1, init_amp=0.2)


def test_batch_one_step_matches_bf16_operand_oracle(gda):
    """Every instance of a ragged batch after one BF16 step (noise, coupling
    ramp) against the oracle with BF16-rounded coupling operands."""
    insts = ragged_mix(gda)
    b = gda.Batch(insts, seed=99)
    b.run(gda.default_params(prec=gda.BF16, **KW_MIX), 1)
    for k, (J, g, model, R) in enumerate(insts):
        name = "xy" if model == gda.XY else "ising"
        op = oracle.Params(seed=b.instance_seed(k), operand="bf16", **KW_MIX)
        ref, rg, rb = oracle.run(J, g, name, op, R, 1)
        psi, gam, beta = b.get_state(k)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(psi - ref).max() < 1e-5 * scale, k
        assert np.abs(gam - rg).max() < 1e-5 * max(1.0, np.abs(rg).max()), k
        assert np.allclose(beta, rb, rtol=1e-6), k
    b.close()


def test_batch_fp64_best_energies_match_oracle(gda):
    """After 50 batched steps, each instance's reported best energy is the
    oracle's Eq. (1) minimum over its restarts' projected spins."""
    insts = ragged_mix(gda)
    b = gda.Batch(insts, seed=5)
    b.run(gda.default_params(prec=gda.BF16, **KW_MIX), 50)
    Eb, rb = b.best()
    for k, (J, g, model, R) in enumerate(insts):
        psi = b.get_state(k)[0]
        S = oracle.project(psi.astype(np.complex128) if model == gda.XY else psi.astype(np.float64))
        E = oracle.energies(J, g, S)
        assert Eb[k] == pytest.approx(E.min(), rel=1e-9, abs=1e-9), k
        assert E[rb[k]] == pytest.approx(E.min(), rel=1e-9, abs=1e-9), k
    b.close()


def test_batch_tile_widths_agree(gda):
    insts = mix(gda)[:4]
    out = []
    for bn in (128, 256):
        b = gda.Batch(insts, seed=7)
        b.set_tile(bn)
        b.run(gda.default_params(dt=0.05, eps=0.2, init_amp=0.2, prec=gda.BF16), 30)
        out.append([b.get_state(k)[0] for k in range(len(insts))])
        b.close()
    for x, y in zip(*out):
        assert np.abs(x - y).max() <= 1e-5 * max(1.0, np.abs(x).max())


def test_batch_rejects_unsupported(gda):
    b = gda.Batch(mix(gda)[:2], seed=1)
    with pytest.raises(gda.GdaError):
        b.run(gda.default_params(prec=gda.FP32), 5)
    with pytest.raises(gda.GdaError):
        b.run(gda.default_params(prec=gda.BF16, integ=gda.RK4), 5)
    b.close()
