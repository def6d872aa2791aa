"""Plain CPU FP64 oracle of the learned proposal network (test infrastructure only).

The proposal is not in the paper: a network that maps an instance's couplings
J (and field g) to initial amplitudes and run settings of the GD algorithm.
This module restates its definitions in FP64 numpy so that the CUDA kernels
can be checked:

* per-spin features (8 per spin), J0 = J without its diagonal, row i:
  f0 = sum_j J0_ij / |J0_i|, f1 = sum_j |J0_ij| / (sqrt(N) |J0_i|), f2 = |J0_i|,
  f3 = max_j |J0_ij| / |J0_i|, f4 = g_i, f5 = normalised J0 v1 with
  v1 = normalised J0 1, f6 = normalised J0 f5, f7 = 1 for XY else 0
  (normalised: divided by the root mean square over the spins; 0/0 = 0);
* a 3-layer perceptron 8 -> 128 -> 128 -> 5 with ReLU hidden layers;
* the training loss: the squared distance of the predicted amplitudes to the
  target spins after the best global sign (Ising) or phase (XY), plus a
  weighted squared error of the instance-mean of outputs 2..4 against target
  settings;
* one Adam step (Kingma & Ba, ICLR 2015) with bias correction;
* the head that turns an instance's outputs into a start and settings: base
  amplitudes amp * O[:, 0] (+ i amp * O[:, 1] for XY) and, with s the
  logistic function and m the mean over the spins of O[:, 2:5],
  eps = 0.02 + 0.48 s(m0), rho_th = 0.5 + 1.5 s(m1), beta0 = 0.1 + 0.9 s(m2).

Pins (tests/test_oracle_mlp.py): finite differences of the loss through the
forward pass check the hand-written backward pass; closed forms on tiny
networks check the forward pass; the loss is checked for its symmetry and its
minimum; the features are checked on a Mattis instance in closed form; the
head's settings are checked at the logistic function's centre and limits, and
for their invariance under a permutation or a repetition of the spins.
"""
from __future__ import annotations

import math

import numpy as np

DIN, DH, DOUT = 8, 128, 5
SHAPES = [("W1", (DH, DIN)), ("b1", (DH,)), ("W2", (DH, DH)), ("b2", (DH,)), ("W3", (DOUT, DH)), ("b3", (DOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p: np.ndarray) -> dict:
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed: int) -> np.ndarray:
    """He-style initial weights from a seeded generator, zero biases."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, math.sqrt(2.0 / DIN), (DH, DIN)), "b1": np.zeros(DH),
         "W2": rng.normal(0, math.sqrt(2.0 / DH), (DH, DH)), "b2": np.zeros(DH),
         "W3": rng.normal(0, math.sqrt(1.0 / DH), (DOUT, DH)), "b3": np.zeros(DOUT)}
    return pack(d)


def _rms_normalise(y: np.ndarray) -> np.ndarray:
    rms = math.sqrt(float(np.mean(y * y)))
    return y / rms if rms > 0 else np.zeros_like(y)


def features(J: np.ndarray, g: np.ndarray | None, xy: bool) -> np.ndarray:
    """Per-spin features [N][8] (definitions in the module docstring)."""
    J0 = np.array(J, dtype=np.float64, copy=True)
    np.fill_diagonal(J0, 0.0)
    N = J0.shape[0]
    nrm = np.sqrt(np.sum(J0 * J0, axis=1))
    inv = np.where(nrm > 0, 1.0 / np.where(nrm > 0, nrm, 1.0), 0.0)
    F = np.zeros((N, DIN))
    F[:, 0] = J0.sum(1) * inv
    F[:, 1] = np.abs(J0).sum(1) * inv / math.sqrt(N)
    F[:, 2] = nrm
    F[:, 3] = np.abs(J0).max(1) * inv if N > 1 else 0.0
    F[:, 4] = 0.0 if g is None else np.asarray(g, dtype=np.float64)
    v1 = _rms_normalise(J0 @ np.ones(N))
    F[:, 5] = _rms_normalise(J0 @ v1)
    F[:, 6] = _rms_normalise(J0 @ F[:, 5])
    F[:, 7] = 1.0 if xy else 0.0
    return F


def forward(p: np.ndarray, X: np.ndarray):
    """O [M][5] and the cache (pre- and post-activations) of the MLP."""
    w = unpack(p)
    z1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(z2, 0.0)
    O = h2 @ w["W3"].T + w["b3"]
    return O, (X, z1, h1, z2, h2)


def backward(p: np.ndarray, cache, dO: np.ndarray) -> np.ndarray:
    """Gradient of sum_m dO[m] . O[m] with respect to the parameter vector."""
    w = unpack(p)
    X, z1, h1, z2, h2 = cache
    g = {"W3": dO.T @ h2, "b3": dO.sum(0)}
    d2 = (dO @ w["W3"]) * (z2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(0)
    d1 = (d2 @ w["W2"]) * (z1 > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(0)
    return pack(g)


def proposal_loss(O: np.ndarray, S: np.ndarray, Tset: np.ndarray, offsets, cplx, wset: float):
    """Per-instance loss and dLoss/dO (definitions in the module docstring).
    S: [M][2] target spins (re, im); Tset: [n_inst][3]."""
    dO = np.zeros_like(O)
    losses = []
    for b in range(len(offsets) - 1):
        i0, i1 = offsets[b], offsets[b + 1]
        n = i1 - i0
        a = O[i0:i1, 0] + (1j * O[i0:i1, 1] if cplx[b] else 0.0)
        s = S[i0:i1, 0] + (1j * S[i0:i1, 1] if cplx[b] else 0.0)
        ip = np.sum(np.conj(s) * a)  # <s, a>
        if cplx[b]:
            u = ip / abs(ip) if abs(ip) > 0 else 1.0
        else:
            u = 1.0 if ip.real >= 0 else -1.0
        e = a - u * s
        lamp = float(np.sum(np.abs(e) ** 2)) / n
        dO[i0:i1, 0] = 2 * e.real / n
        if cplx[b]:
            dO[i0:i1, 1] = 2 * e.imag / n
        p = O[i0:i1, 2:5].mean(0)
        d = p - Tset[b]
        dO[i0:i1, 2:5] = 2 * wset * d / n
        losses.append(lamp + wset * float(np.sum(d * d)))
    return dO, np.array(losses)


def adam_step(p, g, m1, m2, lr, b1, b2, eps, t):
    """One Adam step with bias correction; returns new (p, m1, m2)."""
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** t)
    vh = m2 / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2


def proposal_head(O: np.ndarray, cplx: bool, amp: float):
    """(base, settings) of one instance from its outputs O [N][5]: base [N]
    (complex for XY) and settings (eps, rho_th, beta0)."""
    O = np.asarray(O, dtype=np.float64)
    base = amp * O[:, 0] + (1j * amp * O[:, 1] if cplx else 0.0)
    m = O[:, 2:5].mean(0)
    sig = [1.0 / (1.0 + math.exp(-x)) for x in m]
    settings = np.array([0.02 + 0.48 * sig[0], 0.5 + 1.5 * sig[1], 0.1 + 0.9 * sig[2]])
    return base, settings
