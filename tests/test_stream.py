"""The persistent streaming schedule (one launch per tracking segment, steps
ordered by per-tile flags) against per-step launches of the same tiles: the
same bits, with and without two-SM tiles, BF16 and FP8, noise with decay, the
coupling ramp and tracking; and one step against the BF16-operand oracle."""
import math

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


def _run(gda, J, g, model, R, steps, **kw):
    s = gda.Solver(J, g, model)
    s.run(gda.default_params(**kw), R, steps)
    out = s.get_state(), s.trace()
    s.close()
    return out


# (two-SM tiles need an even number of 128-row blocks)
CASES = [("xy", 300, 70, "stream"), ("ising", 512, 300, "stream"), ("xy", 200, 40, "stream_pair"),
         ("ising", 700, 200, "stream_pair")]


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("model,n,R,sched", CASES)
def test_stream_equals_per_step(gda, model, n, R, sched, prec):
    J, g = synth.xy_gaussian(n, 40 + n)
    if model == "ising":
        g = np.zeros(n)
    m = gda.XY if model == "xy" else gda.ISING
    p = gda.BF16 if prec == "bf16" else gda.FP8
    kw = dict(dt=0.05, eps=0.2, eps_hat=0.3, beta0=0.4, noise_D=0.02, noise_decay=1, seed=77, init_amp=0.2,
              energy_every=16, prec=p)
    ref_sched = gda.PAIR if sched == "stream_pair" else gda.PER_STEP
    (a_state, a_tr) = _run(gda, J, g, m, R, 40, schedule=ref_sched, **kw)
    (b_state, b_tr) = _run(gda, J, g, m, R, 40, schedule=gda.STREAM_PAIR if sched == "stream_pair" else gda.STREAM,
                           **kw)
    for x, y in zip(a_state[:3], b_state[:3]):
        assert np.array_equal(x, y)
    assert a_state[3] == b_state[3] == 40
    for x, y in zip(a_tr, b_tr):
        assert np.array_equal(x, y)


def test_stream_one_step_matches_bf16_operand_oracle(gda):
    n, R = 300, 70
    J, g = synth.xy_gaussian(n, 9)
    s = gda.Solver(J, g, gda.XY)
    s.run(gda.default_params(dt=0.05, eps=0.2, prec=gda.BF16, schedule=gda.STREAM, seed=3, init_amp=0.3), R, 1)
    psi = s.get_state()[0]
    ref = oracle.run(J, g, "xy", oracle.Params(dt=0.05, eps=0.2, seed=3, init_amp=0.3, operand="bf16"), R, 1)[0]
    assert np.abs(psi - ref).max() < 1e-5 * max(1.0, np.abs(ref).max())
    s.close()


def test_stream_full_size_sk(gda):
    """SK N = R = 4096 (the headline size, two-SM tiles): 30 streamed steps in
    two segments equal per-step two-SM launches bit for bit."""
    n, R = 4096, 4096
    J, _ = synth.sk_gaussian(n, 0)
    kw = dict(dt=0.1 / math.sqrt(n), eps=0.03, beta0=0.5, eps_hat=0.05, seed=100, prec=gda.BF16, energy_every=15)
    a = _run(gda, J, None, gda.ISING, R, 30, schedule=gda.PAIR, **kw)
    b = _run(gda, J, None, gda.ISING, R, 30, schedule=gda.STREAM, **kw)
    assert np.array_equal(a[0][0], b[0][0]) and np.array_equal(a[0][1], b[0][1])
    assert np.array_equal(a[1][1], b[1][1])


def test_stream_rejects_rk4_and_fp32(gda):
    J, g = synth.xy_gaussian(40, 1)
    s = gda.Solver(J, g, gda.XY)
    for kw in (dict(prec=gda.BF16, integ=gda.RK4), dict(prec=gda.FP32)):
        with pytest.raises(gda.GdaError) as e:
            s.run(gda.default_params(schedule=gda.STREAM, **kw), 4, 2)
        assert e.value.status == 6
    s.close()
