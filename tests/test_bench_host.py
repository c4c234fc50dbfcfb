"""Host-side pieces of the benchmark: the per-workload roofline arithmetic."""
import json
import os

import bench


def test_workload_rooflines_use_the_oracle_work_counts():
    work = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "work_per_frame.json")))
    wl = {
        "c1_cascl_128_64_L4": dict(value=1.0, frames=10000, ms=0.1),
        "c3_1024_512_L8": {"f32_unpruned": dict(frames=100000, ms=10.0), "i16_pruned": dict(frames=100000, ms=20.0)},
        "c2_fa_2048_1723": {"f32_4.5dB": dict(frames=200000, ms=10.0)},
        "c4_uneven_500k": dict(frames=500000),
    }
    bench.add_workload_rooflines(wl, 2000.0, sms=152)
    peak = 152 * 128 * 2000.0 * 1e6 / 1e9
    r = wl["c1_cascl_128_64_L4"]["roofline"]
    assert r["peak"] == peak and r["bound"] == "alu"
    assert abs(r["achieved"] - work["c1_cascl_128_64_L4_L4_unpruned"]["fg_elems"] * 10000 / 1e-4 / 1e9) < 1e-6
    assert wl["c3_1024_512_L8"]["i16_pruned"]["roofline"]["work"] == "c3_1024_512_L8_L8_pruned"
    assert wl["c3_1024_512_L8"]["f32_unpruned"]["roofline"]["work"] == "c3_1024_512_L8_L8_unpruned"
    assert wl["c2_fa_2048_1723"]["f32_4.5dB"]["latency_ms_batch"] == 10.0
    assert "roofline" not in wl["c4_uneven_500k"]
    wl2 = {"c1_cascl_128_64_L4": dict(frames=1, ms=1.0)}
    bench.add_workload_rooflines(wl2, None, sms=152)
    assert "roofline" not in wl2["c1_cascl_128_64_L4"]
