"""The bench line's roofline arithmetic (host logic, no GPU): the algorithmic
bytes per coordinate update, achieved bandwidth and fraction of the peak from a
handle's counters, and when a committed DRAM-traffic figure may be reported
beside them (only for the kernel sources, workload and kernel choice it was
taken on)."""
import argparse
import json

import pytest

import bench


def _args(dtype="f64", omega=16, tau=65536):
    return argparse.Namespace(dtype=dtype, omega=omega, tau=tau, n=4_000_000, unfused=False)


def _counters(val_bytes, xg_bytes, updates, per_col, moving_frac, launches, kernel_ms):
    return {"val_bytes": val_bytes, "xg_bytes": xg_bytes, "updates": updates,
            "gathered_nnz": updates * per_col, "scattered_nnz": int(round(updates * moving_frac)) * per_col,
            "iter_launches": launches, "iter_kernel_ms": kernel_ms}


@pytest.mark.parametrize("dtype,val_bytes,xg_bytes,per_update", [("f64", 8, 8, 357), ("f32", 4, 4, 223),
                                                                ("bf16", 2, 4, 190)])
def test_algorithmic_bytes_per_update_at_the_bench_workload(monkeypatch, dtype, val_bytes, xg_bytes, per_update):
    # omega = 16: 16 gathered entries per update; about 1.1% of the steps move and are scattered.
    # Per gathered entry: value + row index + g_r; per update: x read and written (FP64), 1/L_i
    # (residual dtype) and the column's start and length (8 B); per scattered entry: value + row
    # index + g_r read and written.  With 1 launch of 1 ms the achieved GB/s is the bytes / 1e6.
    monkeypatch.setattr(bench, "measured_peaks", lambda: (1000.0, "measured"))
    monkeypatch.setattr(bench, "traffic_per_update", lambda a, t: (None, None))
    updates = 1_000_000
    st = _counters(val_bytes, xg_bytes, updates, 16, 0.011, 1, 1.0)
    roof, avg_s, launches = bench.kernel_roofline(_args(dtype), st, None, dtype)
    assert launches == 1 and avg_s == pytest.approx(1e-3)
    assert roof["alg_bytes_per_launch"] / updates == pytest.approx(per_update, abs=0.5)
    assert roof["achieved"] == pytest.approx(roof["alg_bytes_per_launch"] / 1e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 1000.0)
    assert roof["traffic"] is None and roof["bound"] == "hbm" and roof["unit"] == "GB/s"


def test_roofline_is_per_launch(monkeypatch):
    # four launches of 0.5 ms processing 400 updates in all: per launch 100 updates; a committed
    # traffic of 500 B per update becomes 50000 B per launch
    monkeypatch.setattr(bench, "measured_peaks", lambda: (2000.0, "measured"))
    tuning = {"kernel": 0, "lanes_per_col": 1, "threads_per_block": 448, "heads": 1, "zero_cert": 0}
    monkeypatch.setattr(bench, "traffic_per_update", lambda a, t: (500.0, t))
    st = {"val_bytes": 8, "xg_bytes": 8, "updates": 400, "gathered_nnz": 400 * 10, "scattered_nnz": 20,
          "iter_launches": 4, "iter_kernel_ms": 2.0}
    roof, avg_s, launches = bench.kernel_roofline(_args(), st, tuning, "f64")
    alg = 4000 * 20 + 400 * 32 + 20 * 28
    assert roof["alg_bytes_per_launch"] == pytest.approx(alg / 4)
    assert roof["avg_launch_ms"] == pytest.approx(0.5)
    assert roof["achieved"] == pytest.approx(alg / 4 / 0.5e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 2000.0)
    assert roof["traffic"] == pytest.approx(500.0 * 100)
    assert roof["traffic_taken_at"] == tuning
    assert roof["kernel"].startswith("k_fused_pipe_wide")


def _write_traffic(tmp_path, src_hash):
    prof = tmp_path / "profiles"
    prof.mkdir()
    pipe = {"kernel": 0, "lanes_per_col": 1, "threads_per_block": 448, "heads": 1, "zero_cert": 0}
    warp = {"kernel": 5, "lanes_per_col": 1, "threads_per_block": 512, "heads": 1, "zero_cert": -1}
    d = {"src_hash": src_hash, "workloads": {
        "f64/omega16/tau65536": {"dram_bytes_per_update": 587.1, "tuning": pipe},
        "f64/omega128/tau65536": {"dram_bytes_per_update": 2426.6, "tuning": warp}}}
    (prof / "fused_kernel_traffic.json").write_text(json.dumps(d))


@pytest.mark.parametrize("tuning,expect", [
    ({"kernel": 0, "lanes_per_col": 1, "threads_per_block": 448, "heads": 1, "zero_cert": 0}, 587.1),
    ({"kernel": 0, "lanes_per_col": 1, "threads_per_block": 256, "heads": 1, "zero_cert": 0}, 587.1),
    ({"kernel": 0, "lanes_per_col": 1, "threads_per_block": 448, "heads": 1, "zero_cert": -1}, 587.1),
    ({"kernel": 0, "lanes_per_col": 1, "threads_per_block": 448, "heads": 1, "zero_cert": 1}, None),
    ({"kernel": 0, "lanes_per_col": 1, "threads_per_block": 448, "heads": 0, "zero_cert": 0}, None),
    ({"kernel": 1, "lanes_per_col": 2, "threads_per_block": 0, "heads": 1, "zero_cert": 0}, None),
    ({"kernel": 3, "lanes_per_col": 1, "threads_per_block": 448, "heads": 1, "zero_cert": 0}, None),
    (None, None),
])
def test_traffic_is_reported_only_for_the_kernel_it_was_taken_on(monkeypatch, tmp_path, tuning, expect):
    # the block size may differ; the kernel, lanes per column, column heads and (outside the
    # warp-cooperative kernel, whose -1 is its own adaptive rule) the certificate may not
    _write_traffic(tmp_path, "cafe")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "cafe")
    got, taken_at = bench.traffic_per_update(_args(), tuning)
    assert got == expect
    assert (taken_at is None) == (expect is None)


def test_traffic_of_the_warp_kernel_keeps_its_adaptive_certificate(monkeypatch, tmp_path):
    _write_traffic(tmp_path, "cafe")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "cafe")
    warp = {"kernel": 5, "lanes_per_col": 1, "threads_per_block": 512, "heads": 1}
    assert bench.traffic_per_update(_args(omega=128), dict(warp, zero_cert=-1))[0] == 2426.6
    assert bench.traffic_per_update(_args(omega=128), dict(warp, zero_cert=1))[0] is None
    assert bench.traffic_per_update(_args(omega=128), dict(warp, zero_cert=0))[0] is None


def test_stale_or_missing_traffic_is_not_reported(monkeypatch, tmp_path):
    _write_traffic(tmp_path, "cafe")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    pipe = {"kernel": 0, "lanes_per_col": 1, "threads_per_block": 448, "heads": 1, "zero_cert": 0}
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "beef")        # sources changed since
    assert bench.traffic_per_update(_args(), pipe) == (None, None)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "cafe")
    assert bench.traffic_per_update(_args(dtype="bf16"), pipe) == (None, None)   # no entry for the workload
    assert bench.traffic_per_update(_args(omega=2), pipe) == (None, None)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "nowhere"))
    assert bench.traffic_per_update(_args(), pipe) == (None, None)


def test_committed_traffic_summary_is_consistent():
    # each committed figure is its mean DRAM bytes per launch over the updates of one launch
    # (62 iterations of tau = 65536), taken on a named kernel choice
    with open(bench.os.path.join(bench.ROOT, "profiles", "fused_kernel_traffic.json")) as f:
        d = json.load(f)
    assert len(d["src_hash"]) == 16
    assert set(d["workloads"]) >= {"f64/omega16/tau65536", "f32/omega16/tau65536", "bf16/omega16/tau65536",
                                   "f64/omega128/tau65536"}
    for key, e in d["workloads"].items():
        assert e["updates_per_launch"] == 62 * 65536, key
        per = (e["dram_read_bytes_per_launch"] + e["dram_write_bytes_per_launch"]) / e["updates_per_launch"]
        assert e["dram_bytes_per_update"] == pytest.approx(per, abs=0.06), key
        assert set(e["tuning"]) == {"kernel", "lanes_per_col", "threads_per_block", "heads", "zero_cert"}, key


def test_peak_falls_back_when_the_measured_file_is_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6784.5}))
    assert bench.measured_peaks() == (6784.5, "measured")
