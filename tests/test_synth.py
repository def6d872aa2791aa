"""The seeded input generators (synth/): the SplitMix64 stream against its
published reference outputs, and the structure each instance family promises
(symmetry, zero diagonal, degrees, ranges, moments)."""
import math

import numpy as np

import synth


def test_splitmix64_reference_outputs():
    # published reference outputs of SplitMix64 (Steele, Lea, Flood 2014) for
    # the states 0 and 1234567
    assert [int(x) for x in synth.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(x) for x in synth.splitmix64(1234567, 2)] == [6457827717110365317, 3203168211198807973]
    # offsets continue the same stream
    assert np.array_equal(synth.splitmix64(7, 5)[2:], synth.splitmix64(7, 3, offset=2))


def test_uniform_and_normal_moments():
    u = synth.uniform01(3, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    z = synth.normal(4, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.05  # Gaussian kurtosis


def _symmetric_zero_diag(J):
    return np.array_equal(J, J.T) and np.all(np.diag(J) == 0)


def test_dense_families():
    n = 300
    J, g = synth.ising_pm1(n, 1)
    assert _symmetric_zero_diag(J) and set(np.unique(J[np.triu_indices(n, 1)])) == {-1.0, 1.0} and np.all(g == 0)
    J, g = synth.xy_gaussian(n, 2)
    off = J[np.triu_indices(n, 1)]
    assert _symmetric_zero_diag(J) and abs(off.var() * n - 1.0) < 0.05 and np.all(np.abs(g) <= 0.1)
    J, _ = synth.sk_gaussian(n, 3)
    assert _symmetric_zero_diag(J) and abs(J[np.triu_indices(n, 1)].var() - 1.0) < 0.05
    J, _ = synth.ternary(n, 4, 0.5)
    off = J[np.triu_indices(n, 1)]
    assert _symmetric_zero_diag(J) and set(np.unique(off)) <= {-1.0, 0.0, 1.0}
    assert abs(np.mean(off == 0) - 0.5) < 0.02
    J, _ = synth.uniform_dense(n, 5)
    assert _symmetric_zero_diag(J) and np.abs(J).max() <= 10.0


def test_sparse_3regular_graph():
    n = 800
    J, g = synth.sparse_3regular(n, 6)
    assert _symmetric_zero_diag(J) and np.all(g == 0)
    assert np.all(np.count_nonzero(J, axis=1) == 3)  # every node has exactly three neighbours
    w = J[J != 0]
    assert np.abs(w).max() <= 10.0
    assert np.array_equal(J, synth.sparse_3regular(n, 6)[0])  # seeded
    assert not np.array_equal(J, synth.sparse_3regular(n, 7)[0])


def test_mattis_and_batched_mix():
    v = synth.normal(1, 9)
    J = synth.mattis(v)
    assert np.allclose(J, np.outer(v, v) - np.diag(v * v))
    mix = synth.batched_mix(400, 2)
    ns = np.array([d["n"] for d in mix])
    rs = np.array([d["r"] for d in mix])
    assert ns.min() >= 50 and ns.max() <= 2000 and rs.min() >= 16 and rs.max() <= 256
    assert [d["model"] for d in mix[:4]] == ["ising", "xy", "ising", "xy"]
    # log-uniform N: about half the instances below the geometric mean of the range
    assert abs(np.mean(ns < math.sqrt(50 * 2000)) - 0.5) < 0.08


def test_initial_amplitudes_are_float32_and_bounded():
    x = synth.initial_amplitudes(50, 7, 3, 0.25, True)
    assert x.shape == (7, 50) and np.iscomplexobj(x)
    assert np.all(np.abs(x.real) <= 0.25) and np.all(np.abs(x.imag) <= 0.25)
    assert np.array_equal(x.real.astype(np.float32).astype(np.float64), x.real)
    y = synth.initial_amplitudes(50, 7, 3, 0.25, False)
    assert y.dtype == np.float64 and np.array_equal(y.astype(np.float32).astype(np.float64), y)
