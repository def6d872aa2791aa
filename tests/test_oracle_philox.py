"""Pins of the oracle's counter-based generator and noise/initial-state maps."""
import math
import os

import numpy as np
import pytest

from oracle import (box_muller, init_amplitudes, noise_xi, philox4x32_10,
                    philox_generic, philox_uniform)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M32 = (0xD2511F53, 0xCD9E8D57)
W32 = (0x9E3779B9, 0xBB67AE85)


def test_philox4x32_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        got = [int(x) for x in philox4x32_10(*w[:6])]
        assert got == w[6:], line
        assert list(philox_generic(w[:4], w[4:6], 32, M32, W32)) == w[6:]


def test_philox_round_structure_matches_numpy_4x64():
    # numpy's Philox bit generator is Philox4x64-10; it increments the counter
    # before each block.  The same round function with 64-bit words and the
    # 4x64 constants must reproduce its raw output.
    M = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
    W = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)
    key = [0x0123456789ABCDEF, 0x0FEDCBA987654321]
    for start in (0, 41, 2 ** 40):
        bg = np.random.Philox(key=key, counter=[start, 0, 0, 0])
        raw = [int(x) for x in bg.random_raw(8)]
        assert raw[:4] == list(philox_generic((start + 1, 0, 0, 0), key, 64, M, W))
        assert raw[4:] == list(philox_generic((start + 2, 0, 0, 0), key, 64, M, W))


def test_vectorised_matches_scalar():
    rng = np.random.default_rng(0)
    c = rng.integers(0, 2 ** 32, size=(6, 50), dtype=np.uint64)
    out = philox4x32_10(*c)
    for k in range(50):
        assert [int(o[k]) for o in out] == list(philox_generic(c[:4, k], c[4:, k], 32, M32, W32))


def test_uniform_map_is_open_and_fp32_exact():
    x = np.array([0, 1, 511, 512, 2 ** 32 - 1], dtype=np.uint64)
    u = philox_uniform(x)
    assert u.min() > 0 and u.max() < 1
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert u[0] == 0.5 * 2 ** -23 and u[3] == 1.5 * 2 ** -23


def test_box_muller_moments():
    _, _, x2, x3 = philox4x32_10(np.arange(200000), 7, 0, 0, 1, 2)
    z0, z1 = box_muller(philox_uniform(x2), philox_uniform(x3))
    z = np.concatenate([z0, z1])
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert abs(np.mean(z0 * z1)) < 0.01


def test_noise_layout_and_variance():
    R, N = 8, 300
    xr = noise_xi(5, 3, R, N, complex_=False)
    # restarts 0..3 share one Philox call: their four values are z0..z3 of it
    x0, x1, x2, x3 = philox4x32_10(np.arange(N), 0, 3, 0, 5, 0)
    z0, z1 = box_muller(philox_uniform(x0), philox_uniform(x1))
    z2, z3 = box_muller(philox_uniform(x2), philox_uniform(x3))
    assert np.allclose(xr[:4], np.stack([z0, z1, z2, z3]), rtol=0, atol=0)
    xc = noise_xi(5, 3, R, N, complex_=True)
    assert np.allclose(xc[1], (z2 + 1j * z3) / math.sqrt(2), rtol=0, atol=0)
    big = noise_xi(1, 0, 64, 4096, complex_=True)
    assert abs(big.real.var() - 0.5) < 0.01 and abs(big.imag.var() - 0.5) < 0.01
    # steps and seeds change the stream
    assert not np.array_equal(noise_xi(5, 4, R, N, False), xr)
    assert not np.array_equal(noise_xi(6, 3, R, N, False), xr)


def test_init_amplitudes_range():
    p = init_amplitudes(3, 16, 500, 0.25, complex_=True)
    assert p.shape == (16, 500)
    assert np.abs(p.real).max() < 0.25 and np.abs(p.imag).max() < 0.25
    assert abs(p.real.mean()) < 0.01
    r = init_amplitudes(3, 16, 500, 0.25, complex_=False)
    assert np.array_equal(r, p.real)
