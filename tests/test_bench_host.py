"""Host-side logic of bench.py: the time-to-target rule (with and without the
hybrid's polish) and the algorithmic SFU counts behind the roofline."""
import numpy as np

import bench


def _log(f_inc, t_ns):
    return {"f_inc": np.array(f_inc, float), "t_ns": np.array(t_ns, np.int64)}


def test_time_to_target_first_level_within_tolerance():
    fs = -418.9828872724337
    logs = [_log([-300.0, fs + 1e-3, fs + 1e-5, fs], [1_000_000, 2_000_000, 3_000_000, 4_000_000])]
    out = bench.time_to_target(logs, 0, [fs])
    # |f - f*| <= 1e-6 |f*| = 4.19e-4: level 2 (1e-5 away) is the first
    assert out["reached"] and out["level"] == 2 and abs(out["seconds"] - 3e-3) < 1e-12


def test_time_to_target_not_reached_reports_the_gap():
    logs = [_log([5.0, 1.0], [10, 20]), _log([0.0, 0.0], [10, 20])]
    out = bench.time_to_target(logs, 0, [0.0, 0.0])
    assert not out["reached"] and out["problems_reached"] == 1 and out["seconds"] is None
    assert out["worst_final_rel_gap"] == 1.0


def test_time_to_target_counts_the_polished_incumbent_at_the_run_end():
    fs = -418.9828872724337
    logs = [_log([-300.0, -400.0], [1_000, 2_000])]
    out = bench.time_to_target(logs, 0, [fs], final_f=[fs + 1e-9], run_s=0.39)
    assert out["reached"] and out["reached_by_polish"] == 1 and out["seconds"] == 0.39 and "level" not in out
    out = bench.time_to_target(logs, 0, [fs], final_f=[-400.0], run_s=0.39)
    assert not out["reached"]


def test_time_to_target_without_closed_form():
    out = bench.time_to_target([_log([1.0], [1])], 0, [None])
    assert out["reached"] is None


def test_sfu_counts():
    # Gaussian step: lg2, sqrt, cos; the acceptance test: lg2; Schwefel's new term: sqrt, sin
    assert bench.sfu_per_step("schwefel", 256) == 6
    assert bench.sfu_per_step("schwefel", 256, "uniform") == 3
    assert bench.sfu_per_step("rot_rastrigin", 1024) == 1028
    assert bench.sfu_per_step("rot_schwefel", 128, "uniform") == 2 * 128 + 1


def test_convergence_curve_means_the_replicas_at_each_checkpoint():
    fs = -400.0
    a = np.array([-200.0, -300.0, -380.0, -396.0])  # relative errors 0.5, 0.25, 0.05, 0.01
    b = np.array([-100.0, -200.0, -400.0, -400.0])  # 0.75, 0.5, 0, 0
    out = bench.convergence_curve([a, b], fs, (1, 2, 3, 4))
    assert np.allclose(out, [0.625, 0.375, 0.025, 0.005], rtol=0, atol=1e-15)
    # a checkpoint past the end of a run takes its last level
    assert np.allclose(bench.convergence_curve([a], fs, (4, 9)), [0.01, 0.01], rtol=0, atol=1e-15)


def test_convergence_versions_explore_equal_points_per_level():
    # V0 runs one chain of C * L steps per level, V1 and V2 C chains of L steps
    assert bench.CONV_C * bench.CONV_L == 1 * (bench.CONV_C * bench.CONV_L)
    assert bench.CONV_CHECKPOINTS[-1] == 1146 and list(bench.CONV_CHECKPOINTS) == sorted(set(bench.CONV_CHECKPOINTS))


def test_surrogate_mode_is_for_rotated_workloads_only():
    import pytest
    w = bench.Workload("rot_schwefel_n128", 0, False, "gaussian", 0, True)
    assert w.surrogate and w.config()["workload"].endswith("_surrogate")
    with pytest.raises(SystemExit):
        bench.Workload("schwefel_n256", 0, False, "gaussian", 0, True)


def test_launch_counts_per_run():
    class H:
        def describe(self):
            return [{"kind": "fp32_thread"}]
    # the plain sweep: start stamp, then per level the sweep, the argmin/restart and the advance
    assert bench.Workload("schwefel_n256").launches_per_run(H()) == 1 + 200 * 3
    # delayed acceptance adds, per level, the training steps and 4 launches per Metropolis step
    w = bench.Workload("rot_schwefel_n128", 2, False, "gaussian", 0, True)
    per_level = 1 + bench.DA_TRAIN_STEPS * bench.DA_LAUNCHES_PER_TRAIN_STEP + 6 + 4 * w.L + bench.DA_INSERTS + 1
    assert w.launches_per_run(H()) == 1 + 2 + 2 + 2 * (per_level + 3)
