"""Pins of the proposal-network oracle: finite differences, closed forms,
symmetries."""
import math

import numpy as np
import pytest

import synth
from oracle import mlp_oracle as mo


def _rand(seed, *shape):
    return np.random.default_rng(seed).normal(size=shape)


def test_backward_matches_finite_differences():
    p = mo.init_params(3) + 0.05 * _rand(4, mo.NPARAM)  # nonzero biases too
    X = _rand(5, 9, mo.DIN)
    dO = _rand(6, 9, mo.DOUT)

    def f(q):
        return float(np.sum(dO * mo.forward(q, X)[0]))

    g = mo.backward(p, mo.forward(p, X)[1], dO)
    idx = np.random.default_rng(7).choice(mo.NPARAM, 80, replace=False)
    idx = np.concatenate([idx, [0, mo.NPARAM - 1, 1024, 1024 + 128, 1024 + 128 + 16384]])
    h = 1e-6
    for k in idx:
        e = np.zeros(mo.NPARAM)
        e[k] = h
        fd = (f(p + e) - f(p - e)) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-5, abs=1e-7), k


def test_forward_closed_form_and_relu():
    d = {name: np.zeros(shape) for name, shape in mo.SHAPES}
    d["W1"][0, 0] = 1.0
    d["W2"][0, 0] = 2.0
    d["W3"][0, 0] = 3.0
    d["b3"][:] = [0.5, -1.0, 0.25, 2.0, -3.0]
    X = np.zeros((4, mo.DIN))
    X[:, 0] = [1.5, -2.0, 0.0, 4.0]
    O, _ = mo.forward(mo.pack(d), X)
    assert np.allclose(O[:, 0], 6.0 * np.maximum(X[:, 0], 0) + 0.5)
    assert np.allclose(O[:, 1:], np.broadcast_to([-1.0, 0.25, 2.0, -3.0], (4, 4)))


def test_loss_symmetry_minimum_and_gradient():
    offs = [0, 6, 11]
    cplx = [0, 1]
    S = np.zeros((11, 2))
    S[:6, 0] = np.sign(_rand(1, 6))
    th = _rand(2, 5)
    S[6:, 0], S[6:, 1] = np.cos(th), np.sin(th)
    T = _rand(3, 2, 3)
    O = _rand(4, 11, mo.DOUT)
    dO, L = mo.proposal_loss(O, S, T, offs, cplx, 0.5)
    # global sign / phase of the target spins does not change the loss
    S2 = S.copy()
    S2[:6] *= -1
    z = np.exp(1j * 0.7) * (S[6:, 0] + 1j * S[6:, 1])
    S2[6:, 0], S2[6:, 1] = z.real, z.imag
    assert np.allclose(mo.proposal_loss(O, S2, T, offs, cplx, 0.5)[1], L)
    # zero at a rotated copy of the targets with matching settings
    O0 = np.zeros_like(O)
    O0[:6, 0] = -S[:6, 0]
    w = np.exp(-1j * 1.1) * (S[6:, 0] + 1j * S[6:, 1])
    O0[6:, 0], O0[6:, 1] = w.real, w.imag
    O0[:6, 2:] = T[0]
    O0[6:, 2:] = T[1]
    assert np.allclose(mo.proposal_loss(O0, S, T, offs, cplx, 0.5)[1], 0.0, atol=1e-24)
    # dO is the gradient of the summed loss
    h = 1e-7
    for (i, k) in [(0, 0), (3, 0), (7, 0), (8, 1), (2, 3), (9, 4), (5, 1)]:
        e = np.zeros_like(O)
        e[i, k] = h
        fd = (mo.proposal_loss(O + e, S, T, offs, cplx, 0.5)[1].sum()
              - mo.proposal_loss(O - e, S, T, offs, cplx, 0.5)[1].sum()) / (2 * h)
        assert fd == pytest.approx(dO[i, k], rel=1e-5, abs=1e-9)


def test_features_mattis_closed_form():
    v = synth.normal(4, 12)
    J = synth.mattis(v)  # J0 = v v^T - diag(v^2)
    F = mo.features(J, None, xy=False)
    sv, sv2 = v.sum(), (v * v).sum()
    nrm = np.abs(v) * np.sqrt(sv2 - v * v)
    assert np.allclose(F[:, 0], v * (sv - v) / nrm)
    assert np.allclose(F[:, 1], np.abs(v) * (np.abs(v).sum() - np.abs(v)) / (math.sqrt(12) * nrm))
    assert np.allclose(F[:, 2], nrm)
    mx = np.array([np.abs(v[i]) * np.max(np.abs(np.delete(v, i))) for i in range(12)])
    assert np.allclose(F[:, 3], mx / nrm)

    def apply(x):  # J0 x without forming J0
        return v * (v @ x) - v * v * x

    def normed(y):
        return y / np.sqrt(np.mean(y * y))

    v1 = normed(apply(np.ones(12)))
    f5 = normed(apply(v1))
    assert np.allclose(F[:, 5], f5)
    assert np.allclose(F[:, 6], normed(apply(f5)))
    assert np.all(F[:, 7] == 0) and np.all(mo.features(J, np.ones(12), True)[:, [4, 7]] == 1)


def test_adam_first_step_closed_form():
    p = _rand(1, 50)
    g = _rand(2, 50)
    q, m1, m2 = mo.adam_step(p, g, np.zeros(50), np.zeros(50), 0.01, 0.9, 0.999, 1e-8, 1)
    assert np.allclose(q, p - 0.01 * g / (np.abs(g) + 1e-8))
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)


def test_proposal_head_centre_limits_and_invariances():
    """The head's settings sit at the middle of their ranges for zero outputs,
    at the ends for large outputs, and depend only on the spin-mean of the
    outputs; the base is the scaled amplitude outputs."""
    rng = np.random.default_rng(3)
    O = np.zeros((7, 5))
    _, st = mo.proposal_head(O, False, 0.1)
    assert np.allclose(st, [0.26, 1.25, 0.55], rtol=0, atol=1e-15)
    O[:, 2:5] = 50.0
    assert np.allclose(mo.proposal_head(O, False, 0.1)[1], [0.5, 2.0, 1.0], atol=1e-15)
    O[:, 2:5] = -50.0
    assert np.allclose(mo.proposal_head(O, False, 0.1)[1], [0.02, 0.5, 0.1], atol=1e-15)
    O = rng.normal(size=(40, 5))
    b, st = mo.proposal_head(O, True, 0.25)
    # one setting moved by one output alone: s(m) recovered from the setting
    m = O[:, 2:5].mean(0)
    assert np.isclose((st[0] - 0.02) / 0.48, 1 / (1 + np.exp(-m[0])), rtol=1e-14)
    assert np.isclose((st[2] - 0.1) / 0.9, 1 / (1 + np.exp(-m[2])), rtol=1e-14)
    perm = rng.permutation(40)
    assert np.allclose(mo.proposal_head(O[perm], True, 0.25)[1], st, rtol=1e-14)
    assert np.allclose(mo.proposal_head(np.concatenate([O, O]), True, 0.25)[1], st, rtol=1e-14)
    assert np.array_equal(b, 0.25 * O[:, 0] + 0.25j * O[:, 1])
    br, _ = mo.proposal_head(O, False, 0.25)
    assert br.dtype == np.float64 and np.array_equal(br, 0.25 * O[:, 0])
