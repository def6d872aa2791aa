"""GPU path (through the C ABI) against the CPU FP64 oracle on the same
seeded inputs.  Sizes span several 128-row / 64-row tiles with ragged tails
in spins, columns and the K dimension."""
import math
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL_AMP = 1e-4  # FP32 path vs FP64 oracle, relative per restart


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


def start_state(model, n, R, seed, amp=0.3):
    psi = synth.initial_amplitudes(n, R, seed, amp, model == "xy")
    gam = (0.1 * synth.normal(seed + 2, R * n)).astype(np.float32).astype(np.float64).reshape(R, n)
    beta = np.ones(R)
    return psi, gam, beta


MODELS = [("xy", 300, 70), ("ising", 300, 150), ("xy", 129, 3), ("ising", 45, 1)]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("model,n,R", MODELS)
def test_coupling_product(gda, prec, model, n, R):
    J, g = instance(model, n, 11)
    X = synth.initial_amplitudes(n, R, 5, 1.0, model == "xy")
    s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
    Y = s.coupling(X, gda.BF16 if prec == "bf16" else gda.FP32)
    J0 = oracle.gda_oracle.coupling_operand(J)
    if prec == "bf16":
        ref = oracle.round_bf16(X) @ oracle.round_bf16(J0).T
    else:
        ref = X @ J0.T
    err = np.abs(Y - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err
    s.close()


@pytest.mark.parametrize("integ", ["euler", "rk4"])
@pytest.mark.parametrize("model,n,R", MODELS)
def test_fp32_amplitudes_200_steps(gda, integ, model, n, R):
    J, g = instance(model, n, 3)
    psi0, gam0, beta0 = start_state(model, n, R, 8)
    s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
    s.set_state(psi0, gam0, beta0, 0)
    p = gda.default_params(dt=0.02, eps=0.2, integ=gda.RK4 if integ == "rk4" else gda.EULER, init_mode=2)
    s.run(p, R, 200)
    psi, gam, beta, step = s.get_state()
    op = oracle.Params(integ=integ, dt=0.02, eps=0.2)
    ref, rg, rb = oracle.run(J, g, model, op, R, 200, state=(psi0, gam0, beta0))
    assert step == 200
    assert amp_err(psi, ref) < TOL_AMP
    assert np.abs(gam - rg).max() < TOL_AMP * max(1.0, np.abs(rg).max())
    s.close()


@pytest.mark.parametrize("integ", ["euler", "rk4"])
@pytest.mark.parametrize("decay", [0, 1])
def test_noise_and_ramp_parity(gda, integ, decay):
    model, n, R = "xy", 200, 12
    J, g = instance(model, n, 4)
    s = gda.Solver(J, g, gda.XY)
    kw = dict(dt=0.02, eps=0.2, eps_hat=0.5, beta0=0.2, noise_D=0.05, noise_decay=decay, seed=1234567,
              init_mode=0)
    p = gda.default_params(integ=gda.RK4 if integ == "rk4" else gda.EULER, **kw)
    s.run(p, R, 200)
    psi, gam, beta, _ = s.get_state()
    op = oracle.Params(integ=integ, **kw)
    ref, rg, rb = oracle.run(J, g, model, op, R, 200)
    assert amp_err(psi, ref) < TOL_AMP
    assert np.allclose(beta, rb, rtol=1e-5)
    s.close()


def test_real_noise_parity(gda):
    n, R = 150, 9
    J, g = instance("ising", n, 6)
    s = gda.Solver(J, g, gda.ISING)
    kw = dict(dt=0.02, eps=0.2, noise_D=0.1, noise_decay=1, seed=99, init_mode=0)
    s.run(gda.default_params(**kw), R, 150)
    psi = s.get_state()[0]
    ref = oracle.run(J, g, "ising", oracle.Params(**kw), R, 150)[0]
    assert amp_err(psi, ref) < TOL_AMP
    s.close()


@pytest.mark.parametrize("model", ["xy", "ising"])
def test_init_mode_1_bit_exact(gda, model):
    n, R = 77, 5
    J, g = instance(model, n, 1)
    s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
    s.run(gda.default_params(init_mode=1, init_amp=0.25, seed=2 ** 40 + 17), R, 0)
    psi = s.get_state()[0]
    ref = oracle.init_amplitudes(2 ** 40 + 17, R, n, 0.25, model == "xy")
    assert np.array_equal(psi.astype(ref.dtype), ref)
    s.close()


@pytest.mark.parametrize("integ", ["euler", "rk4"])
@pytest.mark.parametrize("model,n,R", MODELS[:2])
def test_bf16_steps_match_bf16_operand_oracle(gda, integ, model, n, R):
    J, g = instance(model, n, 9)
    psi0, gam0, beta0 = start_state(model, n, R, 2)
    s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
    s.set_state(psi0, gam0, beta0, 0)
    p = gda.default_params(dt=0.02, eps=0.2, prec=gda.BF16, integ=gda.RK4 if integ == "rk4" else gda.EULER,
                           init_mode=2)
    s.run(p, R, 1)
    psi = s.get_state()[0]
    op = oracle.Params(integ=integ, dt=0.02, eps=0.2, operand="bf16")
    ref = oracle.run(J, g, model, op, R, 1, state=(psi0, gam0, beta0))[0]
    assert amp_err(psi, ref) < 1e-5
    s.close()


def test_bf16_trajectory_close_to_fp32(gda):
    # Not amplitude-pinned: BF16 operands perturb the coupling sum by ~2^-9.
    model, n, R = "xy", 300, 32
    J, g = instance(model, n, 5)
    psi0, gam0, beta0 = start_state(model, n, R, 4)
    out = {}
    for prec in (gda.FP32, gda.BF16):
        s = gda.Solver(J, g, gda.XY)
        s.set_state(psi0, gam0, beta0, 0)
        s.run(gda.default_params(dt=0.02, eps=0.2, prec=prec, init_mode=2), R, 100)
        out[prec] = s.get_state()[0]
        s.close()
    assert amp_err(out[gda.BF16], out[gda.FP32]) < 2e-2


def test_ising_integer_energies_bit_exact_n20(gda):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "ising_pm1_n20_ground.txt")) if l[0] != "#"]
    for seed, e_min in rows[:3]:
        J, g = synth.ising_pm1(20, int(seed))
        s = gda.Solver(J, g, gda.ISING)
        s.run(gda.default_params(dt=0.01, eps=0.1, rho_th=1.0, init_mode=1, init_amp=1e-3, seed=int(seed)), 64,
              2000)
        E = s.energy()
        psi = s.get_state()[0]
        S = oracle.project(psi.astype(np.float64))
        exact = np.array([oracle.hamiltonian_int(J, x) for x in S], dtype=np.float64)
        assert np.array_equal(E, exact)
        Eb, rb, cfg = s.best()
        assert Eb == E.min() and rb == int(np.argmin(E))
        assert oracle.hamiltonian_int(J, cfg.astype(np.float64)) == Eb
        assert Eb == int(e_min)  # the GD run finds the enumerated ground state
        s.close()


@pytest.mark.parametrize("n,R", [(300, 40), (1000, 8), (1, 1)])
def test_xy_energies_fp64(gda, n, R):
    J, g = synth.xy_gaussian(n, 2) if n > 1 else (np.zeros((1, 1)), np.array([0.07]))
    J = J.copy()
    np.fill_diagonal(J, 0.3 * synth.normal(9, n))  # a diagonal counts in Eq. (1)
    s = gda.Solver(J, g, gda.XY)
    s.run(gda.default_params(dt=0.05, eps=0.2, init_mode=1, init_amp=0.5, seed=4), R, 50)
    E = s.energy()
    psi = s.get_state()[0].astype(np.complex128)
    ref = oracle.energies(J, g, oracle.project(psi))
    assert np.allclose(E, ref, rtol=1e-9, atol=1e-12)
    Eb, rb, th = s.best()
    assert rb == int(np.argmin(E)) and Eb == E[rb]
    assert oracle.hamiltonian_theta(J, g, th) == pytest.approx(Eb, rel=1e-9, abs=1e-12)
    s.close()


def test_non_integer_ising_energy_fp64(gda):
    J, g = instance("ising", 260, 7)
    s = gda.Solver(J, g, gda.ISING)
    s.run(gda.default_params(dt=0.05, eps=0.2, init_amp=0.1, seed=3), 20, 100)
    E = s.energy()
    S = oracle.project(s.get_state()[0].astype(np.float64))
    assert np.allclose(E, oracle.energies(J, g, S), rtol=1e-9, atol=1e-12)
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("integ", ["euler", "rk4"])
def test_resume_is_bit_identical(gda, prec, integ):
    n, R = 200, 24
    J, g = instance("xy", n, 3)
    kw = dict(dt=0.02, eps=0.2, noise_D=0.05, noise_decay=1, eps_hat=0.3, beta0=0.3, seed=77,
              prec=gda.BF16 if prec == "bf16" else gda.FP32, integ=gda.RK4 if integ == "rk4" else gda.EULER)
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
    assert res[3] == 60
    for x, y in zip(full[:3], res[:3]):
        assert np.array_equal(x, y)
    for s in (a, b, c):
        s.close()


def test_trace_matches_oracle_energies(gda):
    n, R = 150, 16
    J, g = instance("xy", n, 12)
    s = gda.Solver(J, g, gda.XY)
    s.run(gda.default_params(dt=0.05, eps=0.2, init_amp=0.2, seed=5, energy_every=25), R, 100)
    steps, E, r = s.trace()
    tr = []
    oracle.run(J, g, "xy", oracle.Params(dt=0.05, eps=0.2, init_amp=0.2, seed=5, energy_every=25), R, 100, trace=tr)
    assert list(steps) == [t[0] for t in tr]
    assert np.allclose(E, [t[1] for t in tr], rtol=1e-4)
    s.close()


def test_divergence_is_reported(gda):
    J, g = synth.uniform_dense(64, 1)
    s = gda.Solver(J, g, gda.ISING)
    s.run(gda.default_params(dt=5.0, init_amp=1.0), 8, 50)
    with pytest.raises(gda.GdaError) as ei:
        s.sync()
    assert ei.value.status == 4
    s.close()


def test_invalid_params(gda):
    J, g = synth.ising_pm1(10, 0)
    s = gda.Solver(J, g, gda.ISING)
    with pytest.raises(gda.GdaError):
        s.run(gda.default_params(dt=-1.0), 4, 1)
    with pytest.raises(gda.GdaError):
        s.run(gda.default_params(init_mode=2), 4, 1)  # nothing to resume
    with pytest.raises(gda.GdaError):
        s.energy()
    s.close()


def test_deterministic(gda):
    J, g = instance("ising", 300, 2)
    outs = []
    for _ in range(2):
        s = gda.Solver(J, g, gda.ISING)
        s.run(gda.default_params(prec=gda.BF16, noise_D=0.02, noise_decay=1, init_mode=0, seed=3), 130, 40)
        outs.append(s.get_state())
        s.close()
    for x, y in zip(outs[0][:3], outs[1][:3]):
        assert np.array_equal(x, y)


def test_kernel_launches_counted(gda):
    J, g = synth.ising_pm1(20, 1)
    s = gda.Solver(J, g, gda.ISING)
    before = s.kernel_launches()
    s.run(gda.default_params(), 8, 10)
    s.sync()
    assert s.kernel_launches() - before >= 10
    s.close()


@pytest.mark.parametrize("model,n,R", [("xy", 300, 70), ("ising", 260, 150), ("xy", 1000, 1024)])
def test_resident_schedule_equals_per_step(gda, model, n, R):
    # The resident kernel keeps psi and gamma in tensor memory across steps;
    # its arithmetic and MMA order are those of the per-step kernel, so the
    # two schedules must agree bit for bit (noise with decay, beta ramp,
    # tracking segments of 16 steps included).
    J, g = instance(model, n, 21)
    kw = dict(dt=0.02, eps=0.2, eps_hat=0.3, beta0=0.4, noise_D=0.03, noise_decay=1, seed=5, init_mode=1,
              init_amp=0.2, prec=gda.BF16, energy_every=16)
    out = {}
    for sched in (gda.PER_STEP, gda.RESIDENT):
        s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
        s.run(gda.default_params(schedule=sched, **kw), R, 40)
        out[sched] = (s.get_state(), s.trace(), s.energy())
        s.close()
    (sa, ta, ea), (sb, tb, eb) = out[gda.PER_STEP], out[gda.RESIDENT]
    for x, y in zip(sa[:3], sb[:3]):
        assert np.array_equal(x, y)
    assert sa[3] == sb[3] == 40
    for x, y in zip(ta, tb):
        assert np.array_equal(x, y)
    assert np.array_equal(ea, eb)


def test_resident_schedule_rejects_rk4(gda):
    J, g = instance("xy", 64, 1)
    s = gda.Solver(J, g, gda.XY)
    with pytest.raises(gda.GdaError) as ei:
        s.run(gda.default_params(prec=gda.BF16, integ=gda.RK4, schedule=gda.RESIDENT), 8, 2)
    assert ei.value.status == 6
    s.close()


@pytest.mark.parametrize("model,n,R,seed", [("xy", 1000, 1024, 1), ("ising", 4096, 4096, 3)])
def test_full_size_sampled_restarts(gda, model, n, R, seed):
    # The benchmark's XY instance (resident kernel) and the SK N = R = 4096
    # shape (per-step kernel, wide tiles), BF16 with the coupling ramp, a few
    # steps; sampled restarts are recomputed by the oracle on their own
    # (restarts are independent) with BF16-rounded operands.
    if model == "xy":
        J, g = synth.xy_gaussian(n, seed)
        dt = 0.05
    else:
        J, g = synth.sk_gaussian(n, seed)
        dt = 0.1 / math.sqrt(n)
    kw = dict(dt=dt, eps=0.1, eps_hat=0.05, beta0=0.2, init_amp=0.1, seed=seed)
    s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
    s.run(gda.default_params(init_mode=1, prec=gda.BF16, **kw), R, 3)
    psi, gam, beta, step = s.get_state()
    E = s.energy()
    idx = [0, 1, R // 2 - 1, R // 2, R - 2, R - 1]
    psi0 = oracle.init_amplitudes(seed, R, n, 0.1, model == "xy")[idx]
    st = (psi0, np.zeros((len(idx), n)), np.full(len(idx), 0.2))
    ref, rg, rb = oracle.run(J, g, model, oracle.Params(operand="bf16", **kw), len(idx), 3, state=st)
    assert amp_err(psi[idx], ref) < 1e-4
    assert np.allclose(beta[idx], rb, rtol=1e-6)
    Eref = oracle.energies(J, g, oracle.project(psi[idx].astype(ref.dtype)))
    assert np.allclose(E[idx], Eref, rtol=1e-9, atol=1e-9)
    Eb, rb_, _ = s.best(with_cfg=False)
    assert Eb == E.min() and rb_ == int(np.argmin(E))
    s.close()


@pytest.mark.parametrize("model", ["xy", "ising"])
def test_init_mode_3_base_plus_perturbation_bit_exact(gda, model):
    n, R = 77, 5
    J, g = instance(model, n, 1)
    s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
    base = synth.initial_amplitudes(n, 1, 9, 0.7, model == "xy")[0]
    s.set_init_base(base)
    s.run(gda.default_params(init_mode=3, init_amp=0.25, seed=77), R, 0)
    psi = s.get_state()[0]
    pert = oracle.init_amplitudes(77, R, n, 0.25, model == "xy")
    # FP32 sum of the FP32 base and the FP32 perturbation
    if model == "xy":
        ref = ((base.real.astype(np.float32) + pert.real.astype(np.float32)).astype(np.float64)
               + 1j * (base.imag.astype(np.float32) + pert.imag.astype(np.float32)).astype(np.float64))
    else:
        ref = (base.astype(np.float32) + pert.astype(np.float32)).astype(np.float64)
    assert np.array_equal(psi.astype(ref.dtype), ref)
    s.close()


def test_headline_xy_schedule_300_steps(gda):
    """The XY N = 1000, R = 1024 workload's exact parameters (dt = 0.05,
    eps = 0.1, tracking every 100 steps, seeded 1e-3 start) for 300 steps:
    the resident kernel equals per-step launches bit for bit (state and trace),
    and the FP64 energies of the returned spins equal the oracle's Eq. (1)."""
    n, R = 1000, 1024
    J, g = synth.xy_gaussian(n, 1)
    kw = dict(dt=0.05, eps=0.1, rho_th=1.0, init_mode=1, init_amp=1e-3, seed=1, energy_every=100, prec=gda.BF16)
    out = {}
    for sched in (gda.RESIDENT, gda.PER_STEP):
        s = gda.Solver(J, g, gda.XY)
        s.run(gda.default_params(schedule=sched, **kw), R, 300)
        psi = s.get_state()[0]
        out[sched] = (psi, s.trace(), s.energy(), s.trace_energy())
        s.close()
    a, b = out[gda.RESIDENT], out[gda.PER_STEP]
    assert np.array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    ref = oracle.energies(J, g, oracle.project(a[0].astype(np.complex128)))
    assert np.allclose(a[2], ref, rtol=1e-9, atol=0)
