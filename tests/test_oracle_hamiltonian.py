"""Pins of the oracle's Eq. (1) evaluators and brute-force search against
closed forms (ferromagnet, Mattis), symmetries and special cases."""
import math

import numpy as np
import pytest

import synth
from oracle import (brute_force_ising, energies, hamiltonian, hamiltonian_int,
                    hamiltonian_theta, project)

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def test_ferromagnet_aligned_closed_form():
    # J_ij = c for i != j: every aligned configuration has H = -c N (N - 1).
    n, c = 9, 0.7
    J = np.full((n, n), c)
    np.fill_diagonal(J, 0.0)
    g = np.zeros(n)
    for phi in (0.0, 1.3, -2.9):
        assert hamiltonian_theta(J, g, np.full(n, phi)) == pytest.approx(-c * n * (n - 1), rel=1e-14)
    e, s = brute_force_ising(J, g)
    assert e == pytest.approx(-c * n * (n - 1), rel=1e-14)
    assert abs(s.sum()) == n


def test_mattis_ground_state_closed_form():
    # J = v v^T with zero diagonal: H(s) = -(sum v_i s_i)^2 + sum v_i^2, minimal
    # at s = sign(v) with H = -(sum |v_i|)^2 + sum v_i^2 (Ising and XY alike).
    v = synth.normal(11, 14)
    J = synth.mattis(v)
    g = np.zeros(14)
    exact = -np.sum(np.abs(v)) ** 2 + np.sum(v ** 2)
    e, s = brute_force_ising(J, g)
    assert e == pytest.approx(exact, rel=1e-12)
    assert np.array_equal(s, np.sign(v)) or np.array_equal(s, -np.sign(v))
    # the XY energy of any phase configuration is bounded below by the same value
    theta = 2 * math.pi * synth.uniform01(5, 200 * 14).reshape(200, 14)
    H = energies(J, g, np.exp(1j * theta))
    assert np.all(H >= exact - 1e-9)
    assert hamiltonian(J, g, np.exp(1j * np.where(v > 0, 0.0, math.pi))) == pytest.approx(exact, rel=1e-12)


def test_integer_mattis_exact():
    v = np.array([3, -1, 4, -1, 5, -9, 2, 6, -5, 3], dtype=np.float64)
    J = synth.mattis(v)
    exact = -int(np.sum(np.abs(v))) ** 2 + int(np.sum(v ** 2))
    assert hamiltonian_int(J, np.sign(v)) == exact
    e, _ = brute_force_ising(J, np.zeros(len(v)))
    assert e == exact


def test_global_rotation_invariance_xy():
    J, _ = synth.xy_gaussian(30, 2)
    g = np.zeros(30)
    theta = 2 * math.pi * synth.uniform01(9, 30)
    h0 = hamiltonian_theta(J, g, theta)
    for phi in (0.4, 2.0, 5.5):
        assert hamiltonian_theta(J, g, theta + phi) == pytest.approx(h0, rel=1e-12, abs=1e-12)


def test_field_sign_single_spin():
    # Eq. (1) with J = 0: H = g cos(theta); for g > 0 the minimum is theta = pi.
    J = np.zeros((1, 1))
    g = np.array([2.5])
    assert hamiltonian(J, g, np.array([1.0])) == pytest.approx(2.5)
    assert hamiltonian(J, g, np.array([-1.0])) == pytest.approx(-2.5)
    e, s = brute_force_ising(J, g)
    assert e == pytest.approx(-2.5) and s[0] == -1.0


def test_diagonal_counts_in_energy():
    # Eq. (1) sums all ordered pairs: a pure diagonal contributes -sum_i J_ii.
    d = np.array([1.5, -2.0, 0.25])
    J = np.diag(d)
    for s in ([1, 1, 1], [1, -1, 1], [-1, -1, 1]):
        assert hamiltonian(J, np.zeros(3), np.array(s, float)) == pytest.approx(-d.sum())


def test_vectorised_energies_match_eq1():
    J, g = synth.xy_gaussian(25, 6)
    theta = 2 * math.pi * synth.uniform01(1, 4 * 25).reshape(4, 25)
    H = energies(J, g, np.exp(1j * theta))
    for r in range(4):
        assert H[r] == pytest.approx(hamiltonian_theta(J, g, theta[r]), rel=1e-12)
    J2, g2 = synth.ising_pm1(16, 3)
    S = np.where(synth.uniform01(2, 3 * 16).reshape(3, 16) < 0.5, 1.0, -1.0)
    H2 = energies(J2, g2, S)
    for r in range(3):
        assert H2[r] == hamiltonian_int(J2, S[r])


def test_projection_rules():
    assert np.array_equal(project(np.array([0.0, -0.0, 2.0, -1e-30])), [1.0, 1.0, 1.0, -1.0])
    z = project(np.array([0j, 3 + 4j]))
    assert z[0] == 1.0 and z[1] == pytest.approx(0.6 + 0.8j)


def test_brute_force_golden_n20():
    rows = [l.split() for l in open(f"{GOLDEN}/ising_pm1_n20_ground.txt") if l[0] != "#"]
    for seed, e in rows[:2]:
        J, g = synth.ising_pm1(20, int(seed))
        got, s = brute_force_ising(J, g)
        assert got == int(e)
        assert hamiltonian_int(J, s) == int(e)


def test_brute_force_is_minimum_small():
    # N = 8: compare with an explicit loop over all 256 configurations.
    J, g = synth.uniform_dense(8, 4)
    g = 0.5 * synth.normal(3, 8)
    best = min(hamiltonian(J, g, np.array([1.0 - 2.0 * ((k >> b) & 1) for b in range(8)]))
               for k in range(256))
    assert brute_force_ising(J, g)[0] == pytest.approx(best, rel=1e-13)
