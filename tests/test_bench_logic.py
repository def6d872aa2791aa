"""Host logic of the benchmark's time-to-target scoring (no GPU): the target is
set by the best FP64 energy of any arm, an arm's hit is its first trace point
whose FP64-evaluated configuration reaches the target (the tracking energy
alone decides nothing), and its time is prorated by steps."""
import numpy as np
import pytest

import bench


def arm(E64, Et, E_all, steps, total, t_run, t_pre=0.0, extra=None):
    return {"E64": np.array(E64, float), "Et": np.array(Et, float), "E_all": np.array(E_all, float),
            "steps": np.array(steps), "total_steps": total, "t_run": t_run, "t_pre": t_pre, "extra": extra}


def test_target_hit_and_prorated_time():
    arms = {
        # tracking claims the target at step 100, FP64 only at step 300
        "a": arm([-1.0, -5.0, -9.995], [-9.999, -5.0, -9.995], [-9.99, -9.5], [100, 200, 300], 300, 3.0),
        "b": arm([-2.0, -10.0, -10.0], [-2.0, -10.0, -10.0], [-10.0], [100, 200, 300], 300, 3.0, t_pre=0.5,
                 extra={"eps": 0.2}),
    }
    out = bench.score_arms(arms, "a")
    assert out["E_star_fp64"] == -10.0 and out["target_E"] == pytest.approx(-9.99)
    a, b = out["a"], out["b"]
    assert a["steps_to_target"] == 300 and a["ttt_s"] == pytest.approx(3.0)
    assert a["steps_tracking_only"] == 100  # reported, but not what the hit is judged on
    assert a["E_fp64_at_hit"] == -9.995
    assert b["steps_to_target"] == 200 and b["ttt_s"] == pytest.approx(0.5 + 2.0)
    assert b["proposal_s"] == 0.5 and b["settings"] == {"eps": 0.2}
    assert out["speedup_b_vs_a"] == pytest.approx(3.0 / 2.5)
    assert a["gap_rel"] == pytest.approx(1e-3) and b["gap_rel"] == 0.0
    assert a["success_prob"] == 0.5 and b["success_prob"] == 1.0


def test_base_that_never_hits_gives_a_lower_bound():
    arms = {
        "slow": arm([-1.0, -2.0], [-1.0, -2.0], [-2.0], [50, 100], 100, 10.0),
        "fast": arm([-3.0, -3.0], [-3.0, -3.0], [-3.0], [50, 100], 100, 1.0),
    }
    out = bench.score_arms(arms, "slow")
    assert out["slow"]["ttt_s"] is None and out["slow"]["E_fp64_at_hit"] is None
    assert out["fast"]["ttt_s"] == pytest.approx(0.5)
    assert "speedup_fast_vs_slow" not in out
    assert out["speedup_fast_vs_slow_lower_bound"] == pytest.approx(10.0 / 0.5)


def test_energy_trace_without_entries():
    # an arm whose run traced nothing still sets E* through its final energies
    arms = {"x": arm([], [], [-4.0, -3.0], [], 10, 1.0), "y": arm([-4.0], [-4.0], [-1.0], [10], 10, 1.0)}
    out = bench.score_arms(arms, "y")
    assert out["E_star_fp64"] == -4.0
    assert out["x"]["ttt_s"] is None and out["y"]["steps_to_target"] == 10


def test_clock_summary_reads_the_throttle_reasons():
    c = bench.ClockSampler(0)
    assert c.summary()["reasons"] == ["unavailable"]
    na, act = "Not Active", "Active"
    c.samples = [["1695", "2070", "1390.2", na, na, na, act],
                 ["1650", "2070", "1398.0", na, na, na, act],
                 ["2070", "2070", "900.5", na, na, na, na],
                 ["[N/A]", "2070", "[N/A]", na, na, na, na]]
    s = c.summary()
    assert s["sm_mhz"] == 1695.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["sw_power_cap"]
    c.samples.append(["1200", "2070", "1000", na, act, na, na])
    assert bench.ClockSampler.summary(c)["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
