"""bench.py's output contract, on the CPU: the headline line carries every
key the contract names, stays a few KB however large the legs' detail is,
and is valid JSON with non-finite numbers replaced by null."""
import json
import math

import pytest

import bench


def _base():
    return {
        "metric": bench.METRIC, "value": 1.37e12, "unit": "spin-updates/s", "n_gpus": 1, "steps": 20,
        "warmup": 5, "ms_per_step": 149.9, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": bench.WORKLOAD_NAME, **bench.WORKLOAD, "updates_per_step": 2.048e11,
                   "l2": "flushed", "launch": {"group_trials": 32, "strips": 0, "threads": 640, "grid_ctas": 152}},
        "e2e": {"value": 1.2e12, "unit": "spin-updates/s", "h2d_bytes_per_step": 120000,
                "d2h_bytes_per_step": 20484096, "ms_per_step": 170.0},
        "gpu_launches": 20,
        "roofline": {"bound": "alu", "achieved": 13.6, "peak": 20.1, "unit": "Tops/s (32-bit IMAD)",
                     "frac": 0.68, "traffic": 787712, "kernel": "anneal_flow_kernel", "peak_source": "x"},
        "cpu_baseline": {"value": 6.3e8, "unit": "spin-updates/s", "cores": 16, "kind": "oracle", "sample": "s",
                         "single_core": {"value": 4e7, "sample": "s"},
                         "ttt_99_9": {"50x50": {"TTT_s": 0.5, "r": 2.0}, "200x100": {"TTT_s": 1e3, "r": math.inf}}},
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 20},
        "ttt_99_9": {"best_cut": 13810, "target": 13797, "P_s": 0.01, "r": 456.2, "STT_sweeps": 4.5e6,
                     "TTT_s_throughput_form": 0.0668, "TTT_s_latency_form": 0.3, "cut_mean": 13780.1,
                     "cut_min": 13700},
    }


def _legs():
    big = [{"seed": s, **{f"form{j}@{b}": {"P_s": 0.1, "mean_cut": 13000.123456, "wall_s": 0.2, "TTT_s": None}
                          for j in range(5) for b in range(4)}} for s in range(32)]
    return {
        "draw16": {"value": 1.9e12, "roofline": {"frac": 0.47}, "ms_per_step": 107.0},
        "batched": {"value": 1.46e12, "updates": 2.5e12},
        "graph": {"random_2000v_19990e_w1": {"value": 5.2e10}, "torus_200x100_as_graph": {"value": 5.5e11}},
        "pt": {"value": 1.2e12, "coldest": {"best_cut": 13772, "mean_cut": 13700.5}},
        "campaign": {"budgets": [{"sweeps": s, "highest": 13800 + i, "mean": 13700.0,
                                  "histogram": {"first_cut": 13600, "counts": list(range(300))}}
                                 for i, s in enumerate((1000, 3000, 10000, 30000, 100000, 300000))]},
        "learned": {"summary": {"median_TTT_s": {"plain_batched": 0.029, "learned_end_batched": 0.0286}},
                    "per_seed": big},
        "trace": {"error": "RuntimeError: " + "x" * 1000},
    }


def test_headline_has_the_contract_keys_and_is_compact():
    text = bench.headline_line(_base(), _legs())
    assert "\n" not in text
    assert len(text) <= bench.HEADLINE_MAX_BYTES
    line = json.loads(text)
    for k in bench.HEADLINE_KEYS:
        assert k in line, k
    assert line["value"] > 0 and line["unit"] == "spin-updates/s"
    assert line["roofline"]["frac"] == pytest.approx(0.68)
    assert line["cpu_baseline"]["cores"] == 16
    assert line["cpu_baseline"]["ttt_99_9"]["200x100"]["r"] is None      # inf -> null, still valid JSON
    assert set(line["legs"]) == set(_legs())
    assert line["legs"]["campaign"]["highest"][0] == 13800
    assert line["legs"]["learned"]["median_TTT_s"]["plain_batched"] == pytest.approx(0.029)
    assert len(line["legs"]["trace"]["error"]) <= 200


def test_oversized_leg_summaries_are_moved_off_the_headline():
    legs = _legs()
    legs["learned"]["summary"]["padding"] = ["x" * 50] * 200
    line = json.loads(bench.headline_line(_base(), legs))
    assert line["legs"]["learned"] == "on its own line"
    assert line["legs"]["campaign"]["highest"][0] == 13800      # the others stay


def test_headline_rejects_missing_keys_and_oversize():
    base = _base()
    del base["roofline"]
    with pytest.raises(KeyError):
        bench.headline_line(base, {})
    base = _base()
    base["config"]["padding"] = "x" * 7000
    with pytest.raises(ValueError):
        bench.headline_line(base, {})


def test_reference_sample_is_stratified_over_the_schedule():
    inst = {"n": 20000}
    jobs = bench.oracle_sample_jobs(bench.WORKLOAD, inst, 16, 1000)
    starts = [j[5] for j in jobs]                                        # (inst, betas, seed, t0, count, k0)
    assert starts == [p * 10000 // 16 for p in range(15)] + [9000]        # the last slice ends at sweep 10,000
    assert [j[3] for j in jobs] == list(range(16)) and all(j[4] == 1 for j in jobs)   # trial p in process p
    full = bench.synth.linear_betas(0.1, 3.0, 10000)
    for j in jobs:                                                       # each a slice of the full schedule
        assert len(j[1]) == 1000 and (j[1] == full[j[5]:j[5] + 1000]).all()


def test_form_stats_targets_success_and_time_to_target():
    """bench's per-instance statistics on hand-made cuts: target = ceil(0.999
    x the best cut of any listed form at any budget); P_s per form and budget;
    TTT per instance = min over budgets of (wall per trial) x r(P_s), Eq. 3-5."""
    np = pytest.importorskip("numpy")
    T = 2
    res = {
        # instance 1: best cut 1000 -> target 999
        (10, 1): {"a": (np.array([999, 990]), 2.0, None), "b": (np.array([900, 900]), 1.0, None)},
        (20, 1): {"a": (np.array([1000, 1000]), 4.0, None), "b": (np.array([998, 997]), 2.0, None)},
        # instance 2: best cut 2001 (form b) -> target ceil(1998.999) = 1999
        (10, 2): {"a": (np.array([1998, 1990]), 2.0, None), "b": (np.array([2001, 1000]), 1.0, None)},
        (20, 2): {"a": (np.array([1999, 1000]), 4.0, None), "b": (np.array([1999, 1999]), 2.0, None)},
    }
    out = bench._form_stats(res, ["a", "b"], T)
    ps = out["P_s"]
    assert ps["a@10"][0] == pytest.approx(0.25) and ps["a@20"][0] == pytest.approx(0.75)
    assert ps["b@10"][0] == pytest.approx(0.25) and ps["b@20"][0] == pytest.approx(0.5)
    # standard error over the two instances: std(ddof=1) / sqrt(2)
    assert ps["a@20"][1] == pytest.approx(np.std([1.0, 0.5], ddof=1) / math.sqrt(2))
    r_half = math.log(0.01) / math.log(0.5)
    # a: instance 1 best at S=20 (P=1, 2 ms/trial); instance 2 at S=20 (P=0.5, 2 ms/trial)
    # b: instance 1 never reaches 999; instance 2: S=20 (P=1, 1 ms/trial) beats S=10 (P=0.5, 0.5 ms x r)
    ta, tb = out["TTT_s"]["a"], out["TTT_s"]["b"]
    assert ta["reached"] == 2 and tb["reached"] == 1
    assert ta["median"] == pytest.approx(np.median([2e-3, 2e-3 * r_half]))
    assert tb["median"] is None                       # half or fewer reached: no median
    assert tb["mean_reached"] == pytest.approx(min(0.5e-3 * r_half, 1e-3))
    # restricting the forms lowers instance 2's best cut to 1999 -> target 1998
    only_a = bench._form_stats(res, ["a"], T)
    assert only_a["P_s"]["a@10"][0] == pytest.approx((0.5 + 0.5) / 2)
