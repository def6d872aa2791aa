"""Pins of the oracle's time stepping (Eqs. 2, 5, 6; Sec. 2 integrators)
against closed forms, the paper's density/phase form (Eqs. 3-4), its fixed
point (Eqs. 7-8) and its Ising penalty (Sec. 1, Sec. 3)."""
import math
import os

import numpy as np
import pytest

import synth
import oracle
from oracle import (Params, add_noise, energies, euler_step, field_drive,
                    hamiltonian_int, project, rhs, rk4_step, round_bf16, run)
from oracle.gda_oracle import coupling_operand

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _logistic_rho(t, gamma, rho0):
    e = math.exp(2 * gamma * t)
    return gamma * rho0 * e / (gamma + rho0 * (e - 1))


@pytest.mark.parametrize("integ,order", [("euler", 1), ("rk4", 4)])
def test_single_spin_logistic_convergence_order(integ, order):
    # One uncoupled spin with a fixed gain (eps = 0): d rho/dt = 2 rho (gamma - rho).
    gamma, psi0, T = 0.8, 0.1, 3.0
    errs = []
    for dt in (0.02, 0.01):
        p = Params(integ=integ, dt=dt, eps=0.0, gamma0=gamma, init_mode=0)
        psi, _, _ = run(np.zeros((1, 1)), None, "ising", p, 1, int(round(T / dt)),
                        state=(np.array([[psi0]]), np.array([[gamma]]), np.array([1.0])))
        errs.append(abs(psi[0, 0] ** 2 - _logistic_rho(T, gamma, psi0 ** 2)))
    ratio = errs[0] / errs[1]
    assert ratio == pytest.approx(2.0 ** order, rel=0.15)
    assert errs[1] < (5e-3 if order == 1 else 1e-9)


def test_coupling_index_and_orientation():
    # Only J_01 = 1 (asymmetric on purpose): d psi_0/dt picks up +psi_1, psi_1 does not see psi_0.
    J = np.zeros((2, 2))
    J[0, 1] = 1.0
    a, dt = 0.3, 0.1
    p = Params(dt=dt, eps=0.0)
    st = (np.array([[0.0, a]]), np.zeros((1, 2)), np.ones(1))
    psi, _, _ = euler_step(st, coupling_operand(J), np.zeros(2), p, "ising")
    assert psi[0, 0] == pytest.approx(dt * a, rel=1e-15)
    assert psi[0, 1] == pytest.approx(a - dt * a ** 3, rel=1e-15)


def test_diagonal_excluded_from_dynamics():
    p = Params(dt=0.05, eps=0.0, gamma0=0.5)
    st = (np.array([[0.2]]), np.array([[0.5]]), np.ones(1))
    a = run(np.array([[7.0]]), None, "ising", p, 1, 20, state=st)[0]
    b = run(np.array([[0.0]]), None, "ising", p, 1, 20, state=st)[0]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("integ", ["euler", "rk4"])
def test_gain_ramp_is_linear_at_zero_amplitude(integ):
    # psi = 0 stays 0 without noise or field; Eq. (5) then gives gamma = gamma0 + eps rho_th t.
    J, _ = synth.xy_gaussian(10, 1)
    p = Params(integ=integ, dt=0.01, eps=0.3, rho_th=1.7, gamma0=-0.4, init_mode=0)
    psi, gam, _ = run(J, np.zeros(10), "xy", p, 3, 250)
    assert np.all(psi == 0)
    assert np.allclose(gam, -0.4 + 0.3 * 1.7 * 2.5, rtol=1e-12)
    assert np.all(gam == gam[0, 0])  # all gains equal while the densities are equal (Fig. 1, first stage)


@pytest.mark.parametrize("integ", ["euler", "rk4"])
def test_coupling_strength_ramp_closed_form(integ):
    # Eq. (6) with Delta = 1, K = beta J: d beta/dt = eps_hat (1 - beta).
    # Euler: 1 - beta_n = (1 - beta0)(1 - eps_hat dt)^n; RK4: amplification 1 + z + z^2/2 + z^3/6 + z^4/24.
    eh, dt, b0, n = 0.4, 0.05, 0.1, 60
    p = Params(integ=integ, dt=dt, eps=0.0, beta0=b0, eps_hat=eh, init_mode=0)
    _, _, beta = run(np.zeros((3, 3)), None, "ising", p, 2, n)
    z = -eh * dt
    amp = 1 + z if integ == "euler" else 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    assert np.allclose(1 - beta, (1 - b0) * amp ** n, rtol=1e-12)
    assert abs(beta[0] - (1 - (1 - b0) * math.exp(-eh * dt * n))) < (1e-2 if integ == "euler" else 1e-8)


def test_coupling_scaled_by_beta():
    J, _ = synth.xy_gaussian(6, 2)
    psi = synth.initial_amplitudes(6, 2, 4, 0.5, True)
    gam = np.zeros((2, 6))
    p = Params()
    f1, _, _ = rhs(psi, gam, np.array([1.0, 1.0]), coupling_operand(J), np.zeros(6), p, "xy")
    f2, _, _ = rhs(psi, gam, np.array([0.25, 0.25]), coupling_operand(J), np.zeros(6), p, "xy")
    local = psi * (gam - np.abs(psi) ** 2)
    assert np.allclose(f2 - local, 0.25 * (f1 - local), rtol=1e-13, atol=1e-15)


def test_cartesian_matches_density_phase_form():
    # Eqs. (3)-(4): (1/2) rho_i' = (gamma_i - rho_i) rho_i + sum_{j!=i} J_ij sqrt(rho_i rho_j) cos th_ij
    #                              + sum_q h_qi rho_i^{q/2} cos(q th_i)
    #               th_i' = -sum_{j!=i} J_ij sqrt(rho_j / rho_i) sin th_ij - sum_q h_qi rho_i^{q/2-1} sin(q th_i)
    n = 7
    J, g = synth.xy_gaussian(n, 3, field=0.6)
    psi = synth.initial_amplitudes(n, 1, 8, 1.2, True)[0]
    gam = synth.normal(4, n)
    for model, h2 in (("xy", 0.0), ("ising_h2", 0.9)):
        p = Params(rho_th=1.3, h2=h2)
        h1 = field_drive(g, p.rho_th)
        f, _, _ = rhs(psi[None], gam[None], np.ones(1), coupling_operand(J), h1, p, model)
        f = f[0]
        rho, th = np.abs(psi) ** 2, np.angle(psi)
        half_rho_dot = np.real(np.conj(psi) * f)
        th_dot = np.imag(np.conj(psi) * f) / rho
        for i in range(n):
            cs = sum(J[i, j] * math.sqrt(rho[i] * rho[j]) * math.cos(th[i] - th[j]) for j in range(n) if j != i)
            sn = sum(J[i, j] * math.sqrt(rho[j] / rho[i]) * math.sin(th[i] - th[j]) for j in range(n) if j != i)
            exp_r = (gam[i] - rho[i]) * rho[i] + cs + h1[i] * math.sqrt(rho[i]) * math.cos(th[i]) \
                + h2 * rho[i] * math.cos(2 * th[i])
            exp_t = -sn - h1[i] / math.sqrt(rho[i]) * math.sin(th[i]) - h2 * math.sin(2 * th[i])
            assert half_rho_dot[i] == pytest.approx(exp_r, rel=1e-12, abs=1e-12)
            assert th_dot[i] == pytest.approx(exp_t, rel=1e-12, abs=1e-12)


def test_fixed_point_gains_eq7_and_total_eq8():
    # At the fixed point rho_i = rho_th and (Eq. 7, q = 1 drive)
    # gamma_i = rho_th - sum_{j!=i} J_ij cos th_ij - h_1i rho_th^{-1/2} cos th_i,
    # so sum_i gamma_i = N rho_th + H_s with H_s of Eq. (8).
    n = 12
    J, g = synth.xy_gaussian(n, 4, field=0.05)
    J = 3.0 * J
    p = Params(integ="rk4", dt=0.05, eps=0.1, rho_th=1.0, init_mode=1, init_amp=0.1, seed=1)
    psi, gam, _ = run(J, g, "xy", p, 1, 16000)
    psi, gam = psi[0], gam[0]
    rho, th = np.abs(psi) ** 2, np.angle(psi)
    h1 = field_drive(g, p.rho_th)
    assert np.abs(rho - p.rho_th).max() < 1e-3
    coup = np.array([sum(J[i, j] * math.cos(th[i] - th[j]) for j in range(n) if j != i) for i in range(n)])
    pred = p.rho_th - coup - h1 * np.cos(th)
    assert np.abs(gam - pred).max() < 1e-3
    H_s = -coup.sum() - np.sum(h1 * np.cos(th))
    assert gam.sum() == pytest.approx(n * p.rho_th + H_s, abs=5e-3)
    # with zero diagonal and rho_th = 1, H_s is Eq. (1)'s H of the projected spins
    assert H_s == pytest.approx(energies(J, g, project(psi[None]))[0], rel=1e-12)


def test_field_drive_sign_single_spin():
    # J = 0, g > 0: Eq. (1) is minimal at theta = pi, and by Eq. (7)
    # gamma -> rho_th - h_1 cos(pi) / sqrt(rho_th) = 1 - g.
    p = Params(integ="rk4", dt=0.05, eps=0.2, rho_th=1.0, init_mode=1, init_amp=0.05, seed=2)
    psi, gam, _ = run(np.zeros((1, 1)), np.array([0.5]), "ising", p, 4, 6000)
    assert np.allclose(psi, -1.0, atol=1e-4)
    assert np.allclose(gam, 0.5, atol=1e-3)


def test_complex_h2_mode_real_start_equals_real_mode():
    # Real psi(0), real J, no noise: h_2 conj(psi) = h_2 psi, so the complex
    # h_2 mode stays real and equals the real model with gamma0 shifted by h_2.
    n = 9
    J, _ = synth.uniform_dense(n, 5, a=1.0)
    base = Params(integ="rk4", dt=0.02, eps=0.1, init_mode=1, init_amp=0.05, seed=7)
    psi_r, gam_r, _ = run(J, None, "ising", base.with_(gamma0=0.3), 3, 400)
    from oracle import init_amplitudes
    psi0 = init_amplitudes(7, 3, n, 0.05, complex_=False) + 0j
    psi_c, gam_c, _ = run(J, None, "ising_h2", base.with_(h2=0.3), 3, 400,
                          state=(psi0, np.zeros((3, n)), np.ones(3)))
    assert np.all(psi_c.imag == 0)
    assert np.allclose(psi_c.real, psi_r, rtol=1e-12, atol=1e-14)
    assert np.allclose(gam_c + 0.3, gam_r, rtol=1e-12, atol=1e-12)


def test_h2_penalty_forces_binary_phases():
    # Sec. 1: h_2 > max_i sum_j |J_ij| makes the phases 0 or pi (Ising).
    n = 10
    J, _ = synth.ising_pm1(n, 2)
    h2 = 1.2 * np.abs(J).sum(1).max()
    p = Params(integ="rk4", dt=0.01, eps=0.1, rho_th=1.0, h2=h2, init_mode=1, init_amp=0.1, seed=3)
    psi, _, _ = run(J, None, "ising_h2", p, 4, 3000)
    th = np.angle(psi)
    dist = np.minimum(np.abs(np.sin(th)), 1.0)
    assert dist.max() < 1e-3


def test_noise_vanishes_at_threshold():
    p = Params(noise_D=0.5, noise_decay=1, rho_th=1.0, dt=0.01)
    old = np.full((2, 5), 1.1 + 0j)
    new = np.full((2, 5), 0.3 + 0.1j)
    assert np.array_equal(add_noise(new, old, 4, p, True), new)
    below = add_noise(new, old * 0.5, 4, p, True)  # mean rho = 0.3025
    d = (below - new) / (math.sqrt(p.dt) * 0.5 * (1 - 0.3025))
    from oracle import noise_xi
    assert np.allclose(d, noise_xi(p.seed, 4, 2, 5, True), rtol=1e-12)


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.concatenate([synth.normal(1, 5000) * 10.0 ** synth.normal(2, 5000),
                        [1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, 65504.0, 1e-40]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(round_bf16(x), ref)


def test_gda_finds_brute_force_ground_state_n20():
    # N = 20 dense +-1 couplings, R = 64, 2000 Euler steps, dt = 0.01, eps = 0.1, rho_th = 1.
    rows = [l.split() for l in open(os.path.join(GOLDEN, "ising_pm1_n20_ground.txt")) if l[0] != "#"]
    for seed, e_min in rows[:4]:
        J, g = synth.ising_pm1(20, int(seed))
        p = Params(integ="euler", dt=0.01, eps=0.1, rho_th=1.0, init_mode=1, init_amp=1e-3, seed=int(seed))
        psi, _, _ = run(J, g, "ising", p, 64, 2000)
        S = project(psi)
        E = [hamiltonian_int(J, s) for s in S]
        assert min(E) == int(e_min)


def test_round_e4m3_matches_torch():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8 in this torch")
    x = np.concatenate([synth.normal(3, 20000) * 10.0 ** (2 * synth.normal(4, 20000)),
                        [0.0, 448.0, 449.0, 1e6, -1e6, 2.0 ** -9, 1.5 * 2.0 ** -9, 0.5 * 2.0 ** -9, 240.0, 232.0]])
    x = x.astype(np.float32)
    ref = torch.tensor(np.clip(x, -448, 448)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_e4m3(x), ref)


def test_e4m3_table_closed_form():
    from oracle.gda_oracle import _E4M3
    assert _E4M3[0] == 0 and _E4M3[1] == 2.0 ** -9 and _E4M3[8] == 2.0 ** -6
    assert _E4M3[-1] == 448.0 and len(_E4M3) == 127 and np.all(np.diff(_E4M3) > 0)


def test_fp8_coupling_exact_on_representable_operands():
    # Row maxima 1 and 0.5 give scales 1/448 and 1/896; J0 / s and psi * 64
    # then round to the E4M3 values 448 J0 / max and 64 psi, so the FP8
    # product equals J0 psi up to the FP32 rounding of s.  A dropped row
    # scale or amplitude scale fails here.
    rng = np.random.default_rng(5)
    n = 12
    U = rng.choice([-1.0, -0.5, 0.5, 1.0, 0.0], size=(n, n))
    J = np.triu(U, 1)
    J = J + J.T
    J[3] *= 0.5
    J[:, 3] *= 0.5
    J[3, 3] = 0.0
    J[7, :] = 0.0  # an isolated spin: scale 1, zero row
    J[:, 7] = 0.0
    X = rng.choice([-0.75, -0.25, 0.0, 0.125, 0.5, 3.0], size=(4, n))
    s = oracle.fp8_coupling_scales(J)
    assert s[7] == 1.0 and s[3] == pytest.approx(np.abs(J[3]).max() / 448.0, rel=1e-7)
    assert np.array_equal(oracle.round_e4m3(X * 64), X * 64)
    mx = np.abs(J).max(1)
    mx[7] = 448.0
    assert np.array_equal(oracle.round_e4m3(J / s[:, None].astype(np.float32)), 448.0 * J / mx[:, None])
    from oracle.gda_oracle import fp8_coupling
    err = np.abs(fp8_coupling(J, X) - X @ J.T)
    assert np.all(err <= 2.0 ** -23 * (np.abs(X) @ np.abs(J).T))


def test_fp8_coupling_within_e4m3_rounding_bound():
    # Each operand is rounded to 3 mantissa bits (relative error <= 2^-4 in
    # the normal range), so |Y8 - Y| <= sum_j |J0_ij||X_j| (2^-3 + 2^-8),
    # plus the subnormal floor of the amplitude operand.
    from oracle.gda_oracle import fp8_coupling
    n = 200
    J, _ = synth.xy_gaussian(n, 3)
    J0 = coupling_operand(J)
    X = synth.initial_amplitudes(n, 6, 4, 1.0, False)
    Y8, Y = fp8_coupling(J0, X), X @ J0.T
    bound = (np.abs(X) @ np.abs(J0).T) * (2.0 ** -3 + 2.0 ** -8) + np.abs(J0).sum(1)[None, :] * 2.0 ** -16
    assert np.all(np.abs(Y8 - Y) <= bound)
    assert np.abs(Y8 - Y).max() > 1e-4 * np.abs(Y).max()  # the rounding is really applied
    # saturation: amplitudes beyond 448 / 64 = 7 are clipped
    X2 = np.full((1, n), 10.0)
    assert np.allclose(fp8_coupling(J0, X2), fp8_coupling(J0, np.full((1, n), 7.0)))


@pytest.mark.parametrize("q", [2, 3, 4, 5])
def test_resonant_drive_matches_density_phase_form(q):
    # Eqs. (3)-(4) with one resonant term: the q:1 drive h_q conj(psi)^(q-1)
    # adds h_q rho^(q/2) cos(q th) to rho'/2 and -h_q rho^(q/2-1) sin(q th) to th'
    n = 6
    J, g = synth.xy_gaussian(n, 5, field=0.3)
    psi = synth.initial_amplitudes(n, 1, 9, 1.1, True)[0]
    gam = synth.normal(2, n)
    p = Params(rho_th=1.2, q=q, hq=0.7)
    h1 = field_drive(g, p.rho_th)
    f0 = rhs(psi[None], gam[None], np.ones(1), coupling_operand(J), h1, Params(rho_th=1.2), "xy")[0][0]
    f = rhs(psi[None], gam[None], np.ones(1), coupling_operand(J), h1, p, "xy")[0][0]
    d = f - f0
    rho, th = np.abs(psi) ** 2, np.angle(psi)
    assert np.allclose(np.real(np.conj(psi) * d), 0.7 * rho ** (q / 2) * np.cos(q * th), rtol=1e-12, atol=1e-13)
    assert np.allclose(np.imag(np.conj(psi) * d) / rho, -0.7 * rho ** (q / 2 - 1) * np.sin(q * th),
                       rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("q", [2, 3, 5, 6])
def test_potts_projection_nearest_root(q):
    w = oracle.potts_roots(q)
    assert np.allclose(np.abs(w), 1.0) and np.allclose(w ** q, 1.0)
    rng = np.random.default_rng(q)
    th = rng.uniform(-np.pi, np.pi, 500)
    z = rng.uniform(0.1, 3.0, 500) * np.exp(1j * th)
    s = oracle.project(z, q)
    k = np.mod(np.round(th * q / (2 * np.pi)), q).astype(int)  # nearest root by angle
    assert np.allclose(s, w[k])
    assert oracle.project(np.array([0j]), q)[0] == w[0]
    assert np.array_equal(oracle.project(np.array([2.0 + 0j, -3.0 + 0j]), 2), np.array([1.0, -1.0]))


def test_resonant_drive_locks_single_spin_phase():
    # one uncoupled spin, gain fixed: the phase settles on the nearest multiple
    # of 2 pi / q (th' = -h_q rho^(q/2-1) sin(q th) drives sin(q th) to 0 stably
    # at the roots)
    q = 3
    th0 = np.array([0.3, 1.8, -2.5, 2.2])
    psi0 = 0.8 * np.exp(1j * th0)
    J = np.zeros((4, 4))
    p = Params(dt=0.01, eps=0.0, q=q, hq=0.5, gamma0=1.0, init_mode=0)
    psi, _, _ = run(J, None, "xy", p, 1, 4000, state=(psi0[None], np.ones((1, 4)), np.ones(1)))
    want = np.exp(2j * np.pi * np.mod(np.round(th0 * q / (2 * np.pi)), q) / q)
    assert np.allclose(psi[0] / np.abs(psi[0]), want, atol=1e-6)


def test_potts_gd_finds_brute_force_ground_state():
    # q = 3 Potts (XY energy of Eq. 1 with phases 2 pi k / 3), N = 7: all 3^7
    # configurations enumerated; GD with the q:1 drive reaches the minimum
    q, n = 3, 7
    J, _ = synth.xy_gaussian(n, 11)
    w = oracle.potts_roots(q)
    ks = np.array(np.meshgrid(*[np.arange(q)] * n, indexing="ij")).reshape(n, -1).T
    E_all = energies(J, np.zeros(n), w[ks])
    p = Params(dt=0.02, eps=0.1, q=q, hq=2.0, init_amp=0.1, seed=3)
    psi, _, _ = run(J, None, "xy", p, 32, 3000)
    E = energies(J, np.zeros(n), oracle.project(psi, q))
    assert E.min() == pytest.approx(E_all.min(), abs=1e-9)
