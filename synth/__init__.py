"""Seeded synthetic coupling instances for the gain-dissipative solver.

This module holds the input generators shared by the tests, the CPU oracle and
the benchmark. It contains none of the method's arithmetic: it only draws
couplings J and fields g with the shapes and value distributions of the
paper's workloads (dense random couplings, Sec. 2; Max-Cut-like +-1 graphs,
Sec. 3) and of the benchmark configurations.

All randomness comes from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here so the streams
are identical on every platform and numpy version.  A symmetric matrix is made
by drawing its strict upper triangle in row-major order and mirroring it; the
diagonal is zero.
"""
from __future__ import annotations

import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of the SplitMix64 stream started at `seed`."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normal doubles (Box-Muller on pairs of uniforms)."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:n]


def symmetric_from_upper(vals: np.ndarray, n: int) -> np.ndarray:
    """Symmetric n x n matrix whose strict upper triangle (row-major) is `vals`."""
    J = np.zeros((n, n), dtype=np.float64)
    iu = np.triu_indices(n, 1)
    J[iu] = vals
    J[(iu[1], iu[0])] = vals
    return J


def _n_upper(n: int) -> int:
    return n * (n - 1) // 2


def ising_pm1(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Dense J with off-diagonal entries uniform in {-1, +1}, g = 0."""
    bits = splitmix64(seed, _n_upper(n)) >> np.uint64(63)
    vals = 1.0 - 2.0 * bits.astype(np.float64)
    return symmetric_from_upper(vals, n), np.zeros(n)


def xy_gaussian(n: int, seed: int, field: float = 0.1) -> tuple[np.ndarray, np.ndarray]:
    """Dense J_ij ~ N(0, 1/n) and g_i ~ U[-field, field]."""
    J = symmetric_from_upper(normal(seed, _n_upper(n)) / math.sqrt(n), n)
    g = field * (2.0 * uniform01(seed ^ 0x5DEECE66D, n) - 1.0)
    return J, g


def sk_gaussian(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Sherrington-Kirkpatrick couplings J_ij ~ N(0, 1), g = 0."""
    return symmetric_from_upper(normal(seed, _n_upper(n)), n), np.zeros(n)


def ternary(n: int, seed: int, density: float = 0.5) -> tuple[np.ndarray, np.ndarray]:
    """J_ij = 0 with probability 1-density, else +-1 with equal odds; g = 0."""
    u = uniform01(seed, 2 * _n_upper(n))
    keep = u[0::2] < density
    sign = np.where(u[1::2] < 0.5, -1.0, 1.0)
    return symmetric_from_upper(np.where(keep, sign, 0.0), n), np.zeros(n)


def uniform_dense(n: int, seed: int, a: float = 10.0) -> tuple[np.ndarray, np.ndarray]:
    """Dense J_ij ~ U[-a, a], g = 0 (the paper's 'dense' matrices, Sec. 2)."""
    u = uniform01(seed, _n_upper(n))
    return symmetric_from_upper(a * (2.0 * u - 1.0), n), np.zeros(n)


def sparse_3regular(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """The paper's 'sparse' matrices (Sec. 2): every node has exactly three
    neighbours; each edge weight is uniform on an interval whose two bounds are
    drawn from {-10, -3, 3, 10}.  Built by the configuration model with
    rejection of self-loops and multi-edges; n*3 must be even."""
    if (3 * n) % 2:
        raise ValueError("3-regular graph needs an even node count")
    bounds = np.array([-10.0, -3.0, 3.0, 10.0])
    attempt = 0
    while True:
        u = uniform01(seed + 7919 * attempt, 3 * n)
        stubs = np.repeat(np.arange(n), 3)[np.argsort(u, kind="stable")]
        a, b = stubs[0::2], stubs[1::2]
        ok = not np.any(a == b)
        if ok:
            key = np.minimum(a, b) * n + np.maximum(a, b)
            ok = len(np.unique(key)) == len(key)
        if ok:
            break
        attempt += 1
    m = len(a)
    w = uniform01(seed ^ 0xA5A5A5A5, 3 * m)
    lo = bounds[(w[0::3] * 4).astype(int)]
    hi = bounds[(w[1::3] * 4).astype(int)]
    val = lo + (hi - lo) * w[2::3]
    J = np.zeros((n, n))
    J[a, b] = val
    J[b, a] = val
    return J, np.zeros(n)


def mattis(v: np.ndarray) -> np.ndarray:
    """Mattis couplings J = v v^T with zero diagonal."""
    v = np.asarray(v, dtype=np.float64)
    J = np.outer(v, v)
    np.fill_diagonal(J, 0.0)
    return J


def batched_mix(count: int, seed: int, n_lo: int = 50, n_hi: int = 2000,
                r_lo: int = 16, r_hi: int = 256) -> list[dict]:
    """Serving mix: N log-uniform in [n_lo, n_hi], half Ising ternary couplings
    (density 0.5), half XY Gaussian N(0, 1/N) couplings, R uniform in
    [r_lo, r_hi].  Returns descriptors; matrices are drawn lazily with
    `make_instance`."""
    u = uniform01(seed, 3 * count)
    out = []
    for k in range(count):
        n = int(math.floor(math.exp(math.log(n_lo) + u[3 * k] * (math.log(n_hi) - math.log(n_lo)))))
        r = r_lo + int(u[3 * k + 1] * (r_hi - r_lo + 1))
        model = "ising" if k % 2 == 0 else "xy"
        out.append({"n": n, "r": r, "model": model, "seed": seed * 1000003 + k})
    return out


def make_instance(desc: dict) -> tuple[np.ndarray, np.ndarray]:
    if desc["model"] == "ising":
        return ternary(desc["n"], desc["seed"], 0.5)
    J, _ = xy_gaussian(desc["n"], desc["seed"])
    return J, np.zeros(desc["n"])


def initial_amplitudes(n: int, r: int, seed: int, a: float, complex_: bool) -> np.ndarray:
    """Seeded initial amplitudes, each real component ~ U(-a, a), shape (r, n).
    Values are float32-representable so both sides start from the same state."""
    k = r * n * (2 if complex_ else 1)
    x = (a * (2.0 * uniform01(seed, k) - 1.0)).astype(np.float32).astype(np.float64)
    if complex_:
        return (x[0::2] + 1j * x[1::2]).reshape(r, n)
    return x.reshape(r, n)
