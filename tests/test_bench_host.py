"""Host-side pieces of the benchmark: the roofline arithmetic and the
interpolation of the SNR at a target frame error rate."""
import json
import os

import pytest

import bench


def test_workload_rooflines_use_the_oracle_work_counts():
    work = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "work_per_frame.json")))
    wl = {
        "c1_cascl_128_64_L4": dict(value=1.0, frames=10000, ms=0.1, work="c1_cascl_128_64_L4_L4_unpruned",
                                   quant="f32"),
        "c3_1024_512_L8": {"i16_pruned_2.0dB": dict(frames=100000, ms=20.0, quant="i16",
                                                    work="c3_1024_512_L8_L8_pruned")},
        "c4_uneven_500k": dict(frames=500000),
    }
    bench.add_workload_rooflines(wl, 2000.0, sms=152)
    r = wl["c1_cascl_128_64_L4"]["roofline"]
    upd = work["c1_cascl_128_64_L4_L4_unpruned"]["fg_elems"] * 10000 / 1e-4
    # shared-memory model: 12 bytes per float update against 128 B/clk/SM
    assert r["bound"] == "smem" and r["peak"] == 128 * 152 * 2000.0 * 1e6 / 1e9
    assert r["achieved"] == pytest.approx(upd * 12 / 1e9)
    assert r["models"]["alu"]["peak"] == 152 * 128 * 2000.0 * 1e6 / 1e9
    assert r["models"]["alu"]["achieved"] == pytest.approx(upd / 1e9)
    r16 = wl["c3_1024_512_L8"]["i16_pruned_2.0dB"]["roofline"]
    upd16 = work["c3_1024_512_L8_L8_pruned"]["fg_elems"] * 100000 / 0.02
    assert r16["achieved"] == pytest.approx(upd16 * 6 / 1e9)
    assert "roofline" not in wl["c4_uneven_500k"]
    wl2 = {"c1_cascl_128_64_L4": dict(frames=1, ms=1.0, work="c1_cascl_128_64_L4_L4_unpruned")}
    bench.add_workload_rooflines(wl2, None, sms=152)
    assert "roofline" not in wl2["c1_cascl_128_64_L4"]


def test_issue_and_dram_models_need_a_profile():
    m = bench.roofline_models(1000, 100, 1e-3, "i8", 2000.0, 152, hbm_gbs=6780.0)
    assert set(m) == {"smem", "alu"}
    assert m["smem"]["achieved"] == pytest.approx(1000 * 100 / 1e-3 * 3 / 1e9)
    m = bench.roofline_models(1000, 100, 1e-3, "f32", 2000.0, 152, hbm_gbs=6780.0,
                              prof={"dram_bytes_per_frame": 10 ** 6, "warp_instructions_per_frame": 4 * 10 ** 5})
    assert m["dram"]["achieved"] == pytest.approx(100 * 1e6 / 1e-3 / 1e9)
    assert m["dram"]["frac"] == pytest.approx(m["dram"]["achieved"] / 6780.0)
    assert m["issue"]["peak"] == pytest.approx(152 * 4 * 2000.0 * 1e6 / 1e9)


def test_snr_at_fer_interpolates_in_log_domain():
    pts = [(1.0, 1e-2), (1.5, 1e-3), (2.0, 1e-5)]
    assert bench.snr_at_fer(pts, 1e-3) == pytest.approx(1.5)
    assert bench.snr_at_fer(pts, 1e-4) == pytest.approx(1.75)
    assert bench.snr_at_fer(pts, 1e-7) is None


def test_both_arms_report_the_same_config():
    assert bench.headline_config("f32", bench.BATCH, 1) == bench.headline_config()


def test_bench_source_refers_only_to_names_it_defines():
    """The benchmark's GPU-only code paths cannot run here, so check by
    reading: every global a function reads exists at module level (or is a
    builtin), and every name a function deletes is assigned in it."""
    import ast
    import builtins
    import os
    import symtable
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py")
    src = open(path).read()
    top = symtable.symtable(src, path, "exec")
    module_names = set(top.get_identifiers())
    bad = []

    def walk(t):
        for ch in t.get_children():
            if ch.get_type() == "function":
                for s in ch.get_symbols():
                    n = s.get_name()
                    if s.is_global() and s.is_referenced() and n not in module_names and not hasattr(builtins, n):
                        bad.append((ch.get_name(), n))
            walk(ch)

    walk(top)
    for f in ast.walk(ast.parse(src)):
        if isinstance(f, (ast.FunctionDef, ast.AsyncFunctionDef)):
            assigned = {n.id for n in ast.walk(f) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Store)}
            assigned |= {a.arg for a in f.args.args + f.args.kwonlyargs}
            for d in (n for n in ast.walk(f) if isinstance(n, ast.Delete)):
                for tg in d.targets:
                    for nm in ast.walk(tg):
                        if isinstance(nm, ast.Name) and nm.id not in assigned:
                            bad.append((f.name, nm.id))
    assert not bad, bad


@pytest.mark.parametrize("key", ["c2_2048_1723_L32_unpruned", "c3_1024_512_L8_L8_pruned_n64",
                                 "c2_2048_1723_L1_pruned_n32", "c1_cascl_128_64_L4_L4_unpruned"])
def test_stored_work_counts_are_the_oracles(key):
    """The stored per-frame work counts the rooflines use are what the oracle
    counts now (the generator, tests/golden/make_work_counts.py, is the
    only writer)."""
    import importlib.util
    import json
    import os
    import numpy as np
    import oracle
    import synth
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("make_work_counts", os.path.join(here, "golden", "make_work_counts.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    stored = json.load(open(os.path.join(here, "golden", "work_per_frame.json")))[key]
    name, L, pk = next((n, l, p) for n, l, p in gen.CASES if f"{n}_L{l}_{p or 'unpruned'}" == key)
    d = synth.load_code(name)
    code = oracle.Code(d["frozen"], d["crc_len"], d["crc_poly"], d["punct"], d["systematic"])
    st = oracle.Stats()
    oracle.decode(code, np.full(code.N - code.P, 3.0), L, oracle.CASCL,
                  oracle.pruning(**gen.PRUNINGS[pk]) if pk else None, oracle.F32, stats=st)
    assert (st.fg_elems, st.node_steps, st.sorts, st.cand_total) == (
        stored["fg_elems"], stored["node_steps"], stored["sorts"], stored["cand_total"])
