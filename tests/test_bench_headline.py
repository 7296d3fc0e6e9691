"""Host logic of the benchmark line, on the CPU. The headline choice
(bench.choose_headline): `value` is the rate of the fastest precision whose
final iteration met the tolerance in the run, with its step time, its
host-buffer run and its launch count; with none, the FP32 rate stays and no
at-tolerance rate is claimed. The batched workload's CPU baseline
(bench.batched_cpu_baseline): whole trajectories, one per thread."""
import copy

import bench


def line(fp32_ok, refined_ok, mixed_ok):
    return {
        "value": 3.0e9, "ms_per_step": 6.7, "steps": 20, "dtype": "f32",
        "config": {"precision": "fp32"},
        "per_method": {"ieks": "fp32 figures"},
        "fp32": {"value": 3.0e9, "ms_per_step": 6.7, "per_method": {"ieks": "fp32 figures"}},
        "refined": {"value": 2.4e9, "ms_per_step": 8.8, "per_method": {"ieks": "refined figures"}},
        "mixed": {"value": 0.96e9, "ms_per_step": 21.8},
        "e2e": {"value": 2.7e9, "precision": "fp32"},
        "e2e_by_precision": {"fp32": {"value": 2.7e9, "precision": "fp32"},
                             "refined": {"value": 2.1e9, "precision": "refined"}},
        "parity": {"within_tol": {"fp32_final_iteration": fp32_ok, "refined_final_iteration": refined_ok,
                                  "mixed_final_iteration": mixed_ok}},
    }


def test_fp32_is_the_headline_when_it_meets_the_tolerance():
    r = line(True, True, True)
    bench.choose_headline(r)
    assert r["at_oracle_tol"]["precision"] == "fp32" and r["value"] == 3.0e9
    assert r["config"]["precision"] == "fp32" and r["e2e"]["precision"] == "fp32"
    assert r["gpu_launches"] == 7 * 2 * 20


def test_refined_is_the_headline_when_fp32_misses():
    r = line(False, True, True)
    bench.choose_headline(r)
    assert r["at_oracle_tol"] == {"precision": "refined", "value": 2.4e9, "unit": bench.UNIT}
    assert r["value"] == 2.4e9 and r["ms_per_step"] == 8.8
    assert r["config"]["precision"] == "refined" and r["e2e"]["precision"] == "refined"
    assert r["per_method"] == {"ieks": "refined figures"}
    assert r["gpu_launches"] == 12 * 2 * 20


def test_mixed_only_and_none():
    r = line(False, False, True)
    bench.choose_headline(r)
    assert r["at_oracle_tol"]["precision"] == "mixed" and r["dtype"] == "f32 (final iteration f64)"
    r = line(False, False, False)
    before = copy.deepcopy(r)
    bench.choose_headline(r)
    assert r["at_oracle_tol"] is None and r["value"] == before["value"]
    assert r["config"]["precision"].startswith("fp32 (no precision met")


def test_batched_cpu_baseline_times_whole_trajectories_on_all_cores():
    from paper_2102_00514_gb300 import synth
    wl = synth.ct_bearings([30, 50, 20, 40, 10], seed=3, omega0_halfwidth=1.0)
    rec = bench.batched_cpu_baseline(wl, iters=2, budget_states=100, cores=3)
    assert rec["kind"] == "oracle" and rec["cores"] == 3 and rec["unit"] == bench.UNIT
    n = int(rec["sample"].split(" of ")[0])
    assert 1 <= n <= 5 and rec["value"] > 0
    # whole trajectories, at most the budget of states unless one alone exceeds it
    steps = int(rec["sample"].split("(")[1].split(" steps")[0])
    assert steps <= 100 or n == 1


def test_per_state_errors_are_relative_to_each_state():
    import numpy as np
    b = np.array([[1.0, 0.0, 3.0], [0.0, 2.0, 4.0]])
    a = b + np.array([[0.1, 0.0, 0.0], [0.0, 0.0, 0.5]])
    e = bench.per_state_errors(a, b)
    assert np.allclose(e, [0.1, 0.0, 0.1])
    assert bench.per_state_max(a, b) == e.max()
