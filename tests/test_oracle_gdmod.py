"""Pins of the GD-mod oracle (Eq. 6 with Delta_ij = gamma_i^inj + gamma_j^inj
and a per-restart coupling matrix K): reduction to the GD step, a brute-force
coupling sum, the exact discrete solution of the K equation, and the
ferromagnetic ground state with Delta K -> J at the fixed point."""
import numpy as np
import pytest

import synth
from oracle import Params, energies, euler_step, gdmod_euler_step, gdmod_rhs, gdmod_run, project
from oracle.gda_oracle import coupling_operand, field_drive


def _state(n, R, seed, cplx):
    psi = synth.initial_amplitudes(n, R, seed, 0.5, cplx)
    gamma = 0.3 * synth.normal(seed + 1, R * n).reshape(R, n)
    return psi, gamma


def test_uniform_gain_reduces_to_gd_step():
    # eps_hat = 0 and uniform gamma = c: Delta = 2 (c + gamma_c) everywhere and
    # K = beta0 J0, so one GD-mod step is a GD step with beta = 2 (c + gamma_c) beta0.
    n, R = 17, 3
    J, g = synth.xy_gaussian(n, 2)
    J0 = coupling_operand(J)
    h1 = field_drive(g, 1.3)
    psi, _ = _state(n, R, 4, True)
    c = 0.35
    gamma = np.full((R, n), c)
    p = Params(dt=0.02, eps=0.2, rho_th=1.3, eps_hat=0.0, gamma_c=0.8)
    K = np.broadcast_to(0.6 * J0, (R, n, n)).copy()
    a = gdmod_euler_step((psi, gamma, K), J0, h1, p)
    b = euler_step((psi, gamma, np.full(R, 2 * (c + 0.8) * 0.6)), J0, h1, p, "xy")
    assert np.allclose(a[0], b[0], rtol=0, atol=1e-14)
    assert np.allclose(a[1], b[1], rtol=0, atol=1e-14)
    assert np.array_equal(a[2], K)


def test_coupling_sum_brute_force():
    # Y_i = sum_{j != i} (gamma_i + gamma_j + 2 gamma_c) K_ij psi_j by loops, with a
    # non-uniform gain and a K that is not symmetric (it need not stay so).
    n, R = 7, 2
    rng = np.random.default_rng(3)
    psi = rng.normal(size=(R, n)) + 1j * rng.normal(size=(R, n))
    gamma = rng.normal(size=(R, n))
    K = rng.normal(size=(R, n, n))
    for r in range(R):
        np.fill_diagonal(K[r], 0.0)
    J0 = np.zeros((n, n))
    p = Params(gamma_c=0.4, eps=0.0, eps_hat=0.0)
    f, _, _ = gdmod_rhs(psi, gamma, K, J0, np.zeros(n), p)
    rho = np.abs(psi) ** 2
    Y = f - psi * (gamma - rho)
    for r in range(R):
        for i in range(n):
            want = sum((gamma[r, i] + gamma[r, j] + 0.8) * K[r, i, j] * psi[r, j] for j in range(n) if j != i)
            assert Y[r, i] == pytest.approx(want, rel=1e-13, abs=1e-13)


def test_K_equation_exact_discrete_solution():
    # psi = 0 and eps = 0 keep gamma fixed; then Euler on Eq. (6) is linear per
    # element: K_n - J/Delta = (1 - dt eps_hat Delta)^n (K_0 - J/Delta).
    n, R, steps = 9, 2, 40
    J, _ = synth.xy_gaussian(n, 5)
    J0 = coupling_operand(J)
    gamma = 0.2 * synth.normal(6, R * n).reshape(R, n)
    p = Params(dt=0.05, eps=0.0, eps_hat=0.7, gamma_c=1.0)
    psi = np.zeros((R, n), dtype=np.complex128)
    K0 = np.broadcast_to(0.3 * J0, (R, n, n)).copy()
    st = (psi, gamma, K0)
    for _ in range(steps):
        st = gdmod_euler_step(st, J0, np.zeros(n), p)
    ginj = gamma + 1.0
    D = ginj[:, :, None] + ginj[:, None, :]
    Kstar = J0[None] / D
    want = Kstar + (1 - p.dt * p.eps_hat * D) ** steps * (K0 - Kstar)
    assert np.allclose(st[2], want, rtol=1e-12, atol=1e-14)
    assert np.array_equal(st[1], gamma) and np.all(st[0] == 0)


def test_ferromagnet_reaches_aligned_ground_state_and_target_coupling():
    # J_ij = 1: the ground state is all spins aligned (E = -N(N-1)); at the fixed
    # point every amplitude has rho = rho_th and Delta_ij K_ij = J_ij (Eq. 6).
    # There gamma_i = rho_th - (N - 1) = -6, so gamma_c = 10 keeps the injection
    # gamma^inj = gamma + gamma_c (and Delta) positive.
    n, R = 8, 4
    J = np.ones((n, n)) - np.eye(n)
    p = Params(dt=0.01, eps=0.5, eps_hat=1.0, gamma_c=10.0, beta0=0.2, init_amp=0.1, seed=2)
    psi, gamma, K = gdmod_run(J, None, "ising", p, R, 6000)
    E = energies(J, np.zeros(n), project(psi))
    assert np.all(E == -n * (n - 1))
    assert np.allclose(np.abs(psi) ** 2, 1.0, atol=1e-6)
    assert np.allclose(gamma, 1.0 - (n - 1), atol=1e-6)
    ginj = gamma + 10.0
    DK = (ginj[:, :, None] + ginj[:, None, :]) * K
    assert np.allclose(DK, J[None] * np.ones((R, 1, 1)), atol=1e-6)


def test_run_rejects_rk4_and_counts_noise_steps():
    with pytest.raises(ValueError):
        gdmod_run(np.zeros((3, 3)), None, "ising", Params(integ="rk4"), 1, 1)
    # resuming at step0 draws the same noise as the uninterrupted run
    J, g = synth.xy_gaussian(12, 1)
    p = Params(dt=0.02, noise_D=0.1, seed=9, init_amp=0.2)
    full = gdmod_run(J, g, "xy", p, 3, 10)
    half = gdmod_run(J, g, "xy", p, 3, 4)
    rest = gdmod_run(J, g, "xy", p, 3, 6, state=half, step0=4)
    for x, y in zip(full, rest):
        assert np.array_equal(x, y)
