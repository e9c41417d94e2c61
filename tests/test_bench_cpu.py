"""The benchmark's roofline bookkeeping on the CPU: per-kernel achieved bandwidth and
fraction of the peak from two model-info snapshots, the slowest kernel's fraction, the
time-weighted fraction, and the DRAM-traffic record, which is reported only while the
kernel sources hash to the value it was captured on."""
import json

import bench


def _info(fn, fms, sn, sms, an, ams):
    return {"fwd_step_launches": fn, "fwd_step_ms": fms, "store_step_launches": sn,
            "store_step_ms": sms, "adj_step_launches": an, "adj_step_ms": ams}


def test_kernel_stats_arithmetic():
    npts, peak = 1_000_000, 1000.0   # 1 M points, a 1000 GB/s peak
    i0 = _info(0, 0.0, 0, 0.0, 0, 0.0)
    # 10 forward steps of 0.02 ms, 5 stores of 0.03 ms, 20 reverse steps of 0.05 ms
    i1 = _info(10, 0.2, 5, 0.15, 20, 1.0)
    kern, summ = bench.kernel_stats(i0, i1, npts, peak, traffic=False)
    f, s, a = kern["fwd_step_3d"], kern["store_step_3d"], kern["adj_step_3d"]
    assert (f["launches"], s["launches"], a["launches"]) == (10, 5, 20)
    # GB/s = bytes per point x points / average seconds
    assert abs(f["GB/s"] - bench.BYTES_FWD * npts / 0.02e-3 / 1e9) < 1e-9
    assert abs(s["GB/s"] - bench.BYTES_STORE * npts / 0.03e-3 / 1e9) < 1e-9
    assert abs(a["GB/s"] - bench.BYTES_ADJ * npts / 0.05e-3 / 1e9) < 1e-9
    assert f["frac"] == round(f["GB/s"] / peak, 4)
    assert summ["min_frac"] == min(f["frac"], s["frac"], a["frac"])
    tw = (bench.BYTES_FWD * 10 + bench.BYTES_STORE * 5 + bench.BYTES_ADJ * 20) * npts \
        / ((0.2 + 0.15 + 1.0) * 1e-3) / 1e9 / peak
    assert summ["time_weighted_frac"] == round(tw, 4)
    assert all(k["traffic"] is None for k in kern.values())


def test_kernel_stats_without_launches_of_a_kind():
    i0 = _info(0, 0.0, 0, 0.0, 0, 0.0)
    kern, summ = bench.kernel_stats(i0, _info(4, 0.4, 0, 0.0, 4, 0.8), 1000, 100.0,
                                    traffic=False)
    assert kern["store_step_3d"]["frac"] is None and kern["store_step_3d"]["GB/s"] is None
    assert summ["min_frac"] == min(kern["fwd_step_3d"]["frac"], kern["adj_step_3d"]["frac"])


def test_traffic_record_is_gated_by_the_source_hash(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    rec = {"fwd_step_3d": {"bytes_per_launch": 123456, "source_hash": bench.kernel_source_hash()},
           "adj_step_3d": {"bytes_per_launch": 654321, "source_hash": "0" * 16}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["fwd_step_3d"]["source_hash"])
    assert bench.recorded_traffic("fwd_step_3d") == 123456.0
    assert bench.recorded_traffic("adj_step_3d") is None      # captured on other sources
    assert bench.recorded_traffic("store_step_3d") is None    # no record
