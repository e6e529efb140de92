"""Host logic of the benchmark (no GPU): workload descriptions of both arms,
the roofline and bandwidth arithmetic on given timings, the source-matched
traffic lookup, the serving stream and the FIFO latency model."""
import argparse
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _args(**kw):
    d = dict(power_fine=4, gradient="matched", workload="paper", storage="f32")
    d.update(kw)
    return argparse.Namespace(**d)


def test_workload_descriptions(bench):
    w, m = bench.workload_description(_args())
    assert "256x256x128" in w and "4 per finer level" in w and m == bench.PAPER_METRIC
    w, m = bench.workload_description(_args(workload="cube40"))
    assert "256x256x256" in w and "40 views" in w and m == bench.METRIC
    w, m = bench.workload_description(_args(workload="lowdose", storage="bf16", gradient="eq6"))
    assert "256x256x256" in w and "360 views" in w and "bf16" in w and "Eq. 6" in w and "low-dose" in m
    w, _ = bench.workload_description(_args(power_fine=0))
    assert "20 power iterations per level" in w


def test_roofline_and_bandwidth_arithmetic(bench):
    from paper_1001_0599_gb300 import synthetic
    wl = synthetic.workload("paper")
    nnz0 = 19262253600
    # 30 finest-level transpose steps of 5 ms, fewer elsewhere
    prof = {"back_project_step": (100, 400.0), "forward_residual": (100, 200.0), "rof_persistent": (100, 20.0)}
    levels = {0: {"back_project_step": (30, 150.0), "forward_residual": (30, 80.0)},
              1: {"back_project_step": (30, 70.0)}, 2: {"back_project_step": (40, 50.0)}}
    r = bench.roofline(prof, levels, wl)
    assert r["kernel"] == "back_project_step" and r["level"] == 0 and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(2 * nnz0 / 5e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert set(r["levels"]) == {0, 1, 2}
    b = bench.projector_bandwidth(levels, wl)
    nvox, nray = 256 * 256 * 128, 40 * 384 * 512
    assert b["back_project_step"]["algorithmic_bytes"] == 4 * (nray + 2 * nvox)
    assert b["forward_residual"]["algorithmic_gbs"] == pytest.approx(4 * (nvox + 2 * nray) / (80.0 / 30 / 1e3) / 1e9)
    assert b["forward_residual"]["samples_per_s"] == pytest.approx(nnz0 / 8 / (80.0 / 30 / 1e3))


def test_traffic_follows_the_sources(bench, tmp_path, monkeypatch):
    # a capture counts only while the kernel's sources hash as they did
    import json
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"back_project_step/paper/L0": {"dram_bytes_per_launch": 123, "sources_sha1": "abc"}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sources_sha1", lambda names: "abc")
    assert bench.measured_traffic("back_project_step", "paper", 0) == 123
    assert bench.measured_traffic("back_project_step", "lowdose", 0) is None
    monkeypatch.setattr(bench, "sources_sha1", lambda names: "def")
    assert bench.measured_traffic("back_project_step", "paper", 0) is None


def test_serve_stream_and_fifo_model(bench):
    a, b = bench.serve_stream(64), bench.serve_stream(64)
    assert a == b and len(a) == 64
    assert {x[0] for x in a} <= set(range(len(bench.SERVE_GRIDS)))
    # one-at-a-time queue: the second job waits for the first
    assert bench.fifo_latencies([0.0, 0.5, 5.0], [1.0, 1.0, 1.0]) == [1.0, 1.5, 1.0]


def test_oracle_model_counts_every_operation_once(bench):
    # two levels with made-up unit costs: P^T's per-call part is paid once per
    # call, its per-view part per view; ROF per call, per accepted step, per reduction
    units = [{"views": 40, "p_view": 0.1, "pt_call": 1.0, "pt_view": 0.2, "rof_call": 0.5, "rof_step": 0.3,
              "rof_trial": 0.05},
             {"views": 40, "p_view": 0.2, "pt_call": 2.0, "pt_view": 0.4, "rof_call": 1.0, "rof_step": 0.6,
              "rof_trial": 0.1}]
    sched = {"levels": [{"power": 20, "fbs": [{"n_inner": 3, "backtracks": 2}]},
                        {"power": 4, "fbs": [{"n_inner": 1, "backtracks": 0}, {"n_inner": 2, "backtracks": 5}]}]}
    pp0 = 0.1 * 40 + 1.0 + 0.2 * 40
    pp1 = 0.2 * 40 + 2.0 + 0.4 * 40
    want = 20 * pp0 + (pp0 + 0.5 + 3 * 0.3 + 2 * 0.05) + 4 * pp1 + (pp1 + 1.0 + 0.6) + (pp1 + 1.0 + 2 * 0.6 + 5 * 0.1)
    assert bench.oracle_model_seconds(units, sched) == pytest.approx(want)


def test_schedule_from_reconstruction_statistics(bench):
    from types import SimpleNamespace
    from paper_1001_0599_gb300 import synthetic
    wl = synthetic.workload("paper")
    its = [SimpleNamespace(level=0, n_inner=4, backtracks=1)] * 40 + \
          [SimpleNamespace(level=1, n_inner=3, backtracks=0)] * 30 + [SimpleNamespace(level=2, n_inner=2, backtracks=2)] * 30
    st = SimpleNamespace(n_iters=100, iters=its)
    sched = bench.schedule_from_stats(st, wl, 4)
    assert [lv["power"] for lv in sched["levels"]] == [20, 4, 4]
    assert [len(lv["fbs"]) for lv in sched["levels"]] == [40, 30, 30]
    assert sched["levels"][2]["fbs"][0] == {"n_inner": 2, "backtracks": 2}


def test_serve_summary_reports_step_reuse(bench):
    # the default line's serve block carries both back-to-back rates when the
    # server reused step sizes, and a null second rate when it did not
    load = {"load": 0.8, "p50_s": 0.2, "p99_s": 1.0, "scans_per_min": 200.0, "sequential_p50_s": 0.5,
            "sequential_p99_s": 2.5, "gpu_s_per_scan": 0.3, "graph_replays": 32}
    res = {"scans": 32, "loads": [load], "sequential": {"scans_per_min": 218.0},
           "server_burst": {"scans_per_min": 412.0},
           "server_burst_without_step_reuse": {"scans_per_min": 286.0}, "reuse_steps": True,
           "bit_identical_to_sequential": True, "concurrency": 4, "config": {"workload": "mix"}, "clocks": {}}
    out = bench.serve_summary(res)
    assert out["server_burst_scans_per_min"] == 412.0
    assert out["server_burst_without_step_reuse_scans_per_min"] == 286.0
    assert out["reuse_steps"] is True and out["loads"][0]["p99_s"] == 1.0
    assert "gpu_s_per_scan" not in out["loads"][0]
    res.update(server_burst_without_step_reuse=None, reuse_steps=False)
    out = bench.serve_summary(res)
    assert out["server_burst_without_step_reuse_scans_per_min"] is None and out["reuse_steps"] is False
