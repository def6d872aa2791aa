"""Host side of the learned proposal (no GPU): the settings mapping agrees with
the oracle's head, its inverse gives the training targets, the run parameters
switch the coupling ramp on below beta0 = 1, and the hit rule of the
evaluation takes the first FP64-verified trace point."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo
from paper_1807_00699_gb300 import proposal


@pytest.mark.parametrize("m", [(0.0, 0.0, 0.0), (1.3, -0.7, 2.2), (-4.0, 3.5, -0.1)])
def test_settings_mapping_matches_the_oracle_head(m):
    O = np.zeros((3, 5))
    O[:, 2:5] = m
    _, want = mo.proposal_head(O, False, proposal.AMP)
    got = proposal.settings_from_outputs(np.array(m))
    assert np.allclose([got["eps"], got["rho_th"], got["beta0"]], want, rtol=1e-14)


@pytest.mark.parametrize("st", [(0.05, 1.0, 0.3), (0.2, 1.0, 1.0), (0.49, 1.9, 0.95), (0.03, 0.6, 0.15)])
def test_training_targets_invert_the_mapping(st):
    o = proposal.outputs_from_settings(*st)
    back = proposal.settings_from_outputs(np.array(o))
    # settings inside the clipped range come back; beta0 = 1 sits at the clip
    want = [min(st[0], 0.02 + 0.48 * (1 - 1e-3)), st[1], min(st[2], 0.1 + 0.9 * (1 - 1e-3))]
    assert np.allclose([back["eps"], back["rho_th"], back["beta0"]], want, rtol=1e-12)


def test_run_params_ramp_and_grid():
    p = proposal.run_params({"eps": 0.1, "rho_th": 1.0, "beta0": 0.5}, dt=0.05)
    assert p.eps_hat == proposal.RAMP and p.beta0 == 0.5 and p.dt == 0.05
    q = proposal.run_params({"eps": 0.1, "rho_th": 1.0, "beta0": 1.0}, dt=0.05)
    assert q.eps_hat == 0.0
    assert len(proposal.GRID) == 6 and all(r == 1.0 for _, r, _ in proposal.GRID)


def test_first_hit_is_the_first_fp64_point_at_or_below_the_target():
    st = np.array([25, 50, 75, 100])
    E = np.array([-1.0, -3.0, -2.0, -3.5])
    assert proposal._first_hit(st, E, -3.0) == 50
    assert proposal._first_hit(st, E, -3.2) == 100
    assert proposal._first_hit(st, E, -4.0) is None
