"""Failure detection on the device: every wait of the resident tensor-core
kernel has a time limit after which the launch aborts, drains its copies and
MMAs, frees its tensor memory and reports GDA_ERR_TIMEOUT.  The test makes one
tile withhold its step flag (a flag nothing else sets), so the waits of its
column run out after a short limit; the same context then runs a clean solve
that matches the oracle."""
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


def test_withheld_flag_times_out_and_context_recovers(gda):
    n, R = 300, 70  # 3 row blocks x 2 column blocks (XY: 140 columns)
    J, g = synth.xy_gaussian(n, 12)
    s = gda.Solver(J, g, gda.XY)
    bad = gda.default_params(dt=0.05, eps=0.1, prec=gda.BF16, schedule=gda.RESIDENT, seed=5,
                             withhold_flag=2, wait_s=0.02)
    s.run(bad, R, 10)
    with pytest.raises(gda.GdaError) as e:
        s.sync()
    assert e.value.status == 5  # GDA_ERR_TIMEOUT
    # the error flag is cleared and the context keeps working
    s.sync()
    kw = dict(dt=0.05, eps=0.1, prec=gda.BF16, seed=5, init_amp=0.2)
    s.run(gda.default_params(schedule=gda.RESIDENT, **kw), R, 1)
    psi = s.get_state()[0]
    op = oracle.Params(dt=0.05, eps=0.1, seed=5, init_amp=0.2, operand="bf16")
    ref = oracle.run(J, g, "xy", op, R, 1)[0]
    assert np.abs(psi - ref).max() < 1e-5 * max(1.0, np.abs(ref).max())
    # and a longer clean run equals the per-step schedule bit for bit
    s.run(gda.default_params(schedule=gda.RESIDENT, **kw), R, 40)
    a = s.get_state()[0]
    s.run(gda.default_params(schedule=gda.PER_STEP, **kw), R, 40)
    b = s.get_state()[0]
    assert np.array_equal(a, b)
    s.close()


def test_short_limit_alone_does_not_abort(gda):
    n, R = 300, 70
    J, g = synth.xy_gaussian(n, 13)
    s = gda.Solver(J, g, gda.XY)
    s.run(gda.default_params(dt=0.05, eps=0.1, prec=gda.BF16, schedule=gda.RESIDENT, seed=1, wait_s=0.05), R, 50)
    s.sync()
    s.close()


def test_wait_limit_is_validated(gda):
    J, g = synth.xy_gaussian(40, 1)
    s = gda.Solver(J, g, gda.XY)
    for bad in (dict(wait_s=-1.0), dict(wait_s=float("nan")), dict(withhold_flag=-3)):
        with pytest.raises(gda.GdaError) as e:
            s.run(gda.default_params(**bad), 4, 1)
        assert e.value.status == 1
    s.close()


def test_withheld_flag_times_out_in_the_two_sm_form(gda):
    """The same failure in the resident kernel's two-SM form: the pair's waits
    on each other (stages counted on the even CTA's barriers, accumulators
    freed by both epilogues) end on the limit too, and the context recovers."""
    n, R = 500, 70  # 4 row blocks (2 pairs) x 2 column blocks
    J, g = synth.xy_gaussian(n, 14)
    s = gda.Solver(J, g, gda.XY)
    bad = gda.default_params(dt=0.05, eps=0.1, prec=gda.BF16, schedule=gda.RESIDENT_PAIR, seed=5,
                             withhold_flag=2, wait_s=0.02)
    s.run(bad, R, 10)
    with pytest.raises(gda.GdaError) as e:
        s.sync()
    assert e.value.status == 5  # GDA_ERR_TIMEOUT
    s.sync()
    kw = dict(dt=0.05, eps=0.1, prec=gda.BF16, seed=5, init_amp=0.2)
    s.run(gda.default_params(schedule=gda.RESIDENT_PAIR, **kw), R, 1)
    psi = s.get_state()[0]
    op = oracle.Params(dt=0.05, eps=0.1, seed=5, init_amp=0.2, operand="bf16")
    ref = oracle.run(J, g, "xy", op, R, 1)[0]
    assert np.abs(psi - ref).max() < 1e-5 * max(1.0, np.abs(ref).max())
    s.close()
