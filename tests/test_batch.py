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
    __graft_entry__.ensure_built()
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


def test_batch_own_settings_and_start_equal_single_instance_runs(gda):
    """Instances with their own dt, eps, rho_th, ramp (gda_batch_set_params) and
    base amplitudes (gda_batch_set_init_base, init_mode 3) follow exactly the
    single-instance runs with those settings and that start."""
    insts = mix(gda)[:5]
    b = gda.Batch(insts, seed=77)
    own = {0: dict(dt=0.05, eps=0.3, rho_th=1.2, beta0=0.6, eps_hat=0.2),
           3: dict(dt=0.03, eps=0.05, rho_th=0.8, beta0=1.0, eps_hat=0.0)}
    rng = np.random.default_rng(3)
    bases = {}
    for k in (0, 1, 4):
        n = insts[k][0].shape[0]
        xy = insts[k][2] == gda.XY
        bases[k] = 0.1 * (rng.normal(size=n) + (1j * rng.normal(size=n) if xy else 0.0))
        b.set_init_base(k, bases[k])
    for k, st in own.items():
        b.set_params(k, gda.default_params(**st))
    run = dict(dt=0.05, eps=0.2, rho_th=1.0, beta0=0.4, eps_hat=0.3, noise_D=0.02, init_amp=0.05, prec=gda.BF16)
    b.run(gda.default_params(init_mode=3, **run), 130)
    for k, (J, g, model, R) in enumerate(insts):
        kw = dict(run, **own.get(k, {}))
        s = gda.Solver(J, g, model)
        if k in bases:
            s.set_init_base(bases[k])
        s.run(gda.default_params(seed=b.instance_seed(k), schedule=gda.PER_STEP, init_mode=3 if k in bases else 1,
                                 **kw), R, 130)
        psi, gam, beta, _ = s.get_state()
        bpsi, bgam, bbeta = b.get_state(k)
        assert np.array_equal(psi, bpsi), k
        assert np.array_equal(gam, bgam) and np.array_equal(beta, bbeta), k
        s.close()
    # back to the run's settings for instance 0
    b.set_params(0, None)
    b.run(gda.default_params(init_mode=1, **run), 10)
    J, g, model, R = insts[0]
    s = gda.Solver(J, g, model)
    s.run(gda.default_params(seed=b.instance_seed(0), schedule=gda.PER_STEP, init_mode=1, **run), R, 10)
    assert np.array_equal(s.get_state()[0], b.get_state(0)[0])
    s.close()
    b.close()


def test_batch_continuation_across_chunks(gda):
    """A batched run split into calls of 70, 100 and 33 steps (partial chunks,
    a replayed chunk) equals one call of 203 steps."""
    insts = mix(gda)[:4]
    kw = dict(dt=0.05, eps=0.2, noise_D=0.01, init_amp=0.2, prec=gda.BF16)
    a = gda.Batch(insts, seed=4)
    a.run(gda.default_params(init_mode=1, **kw), 203)
    b = gda.Batch(insts, seed=4)
    b.run(gda.default_params(init_mode=1, **kw), 70)
    b.run(gda.default_params(init_mode=2, **kw), 100)
    b.run(gda.default_params(init_mode=2, **kw), 33)
    for k in range(len(insts)):
        assert np.array_equal(a.get_state(k)[0], b.get_state(k)[0]), k
    assert a.launch_mode() in (0, 1)
    a.close()
    b.close()


def test_batch_schedules_agree(gda):
    """One persistent launch per chunk (steps ordered by tile flags) and one
    launch per step give the same bits, at both tile widths."""
    insts = mix(gda)
    kw = dict(dt=0.05, eps=0.2, eps_hat=0.1, beta0=0.5, noise_D=0.01, init_amp=0.2, prec=gda.BF16)
    out = {}
    for sched in (gda.RESIDENT, gda.PER_STEP):
        for bn in (128, 256):
            b = gda.Batch(insts, seed=21)
            b.set_schedule(sched)
            b.set_tile(bn)
            b.run(gda.default_params(init_mode=1, **kw), 130)
            out[(sched, bn)] = [b.get_state(k)[0] for k in range(len(insts))]
            b.close()
    ref = out[(gda.RESIDENT, 128)]
    for key, states in out.items():
        for k, (x, y) in enumerate(zip(ref, states)):
            if key[1] == 128:
                assert np.array_equal(x, y), (key, k)
            else:  # another tile width sums the same products in another order
                assert np.abs(x - y).max() <= 1e-5 * max(1.0, np.abs(x).max()), (key, k)
    with pytest.raises(gda.GdaError):
        gda.Batch(insts[:1], seed=1).set_schedule(gda.PAIR)
