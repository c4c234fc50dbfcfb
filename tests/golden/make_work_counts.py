"""Algorithmic work per frame of the benchmark workloads, counted by the oracle:
f/g LLR updates summed over active paths, node steps, steps that discard
candidates, and candidates offered.  The counts depend only on the code, the
list size and the pruning (never on the data), so one frame suffices.
Writes tests/golden/work_per_frame.json.  Run: python tests/golden/make_work_counts.py"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import synth  # noqa: E402

CASES = [
    ("c2_2048_1723", 32, None), ("c2_2048_1723", 32, "pruned"), ("c2_2048_1723", 1, None),
    ("c2_2048_1723", 1, "pruned"), ("c1_cascl_128_64_L4", 4, None), ("c3_1024_512_L8", 8, None),
    ("c3_1024_512_L8", 8, "pruned"),
] + [("ls_2048_1024", L, pk) for L in (1, 2, 4, 8, 16, 32) for pk in (None, "pruned")] + [
    ("c2_2048_1723", L, "pruned") for L in (2, 4, 8, 16)] + [
    (f"ln_{n}_{n // 2}", 8, None) for n in (4096, 8192)] + [
    ("c2_2048_1723", 1, "pruned_n32"), ("c2_2048_1723", 32, "pruned_n32"), ("c3_1024_512_L8", 8, "pruned_n64")]

# pruning settings by name: the paper's node set (R0/R1/REP/SPC4, Chase-2,
# SPC flips of 4), and the same restricted to nodes of 32 (SPC of any size)
# or 64 leaves and more
PRUNINGS = {"pruned": dict(mask=15, rep_max=0, spc_max=4, r1_t=2, spc_t=4),
            "pruned_n32": dict(mask=15, rep_max=0, spc_max=0, r1_t=2, spc_t=4, node_min=17),
            "pruned_n64": dict(mask=15, rep_max=0, spc_max=4, r1_t=2, spc_t=4, node_min=33)}


def main():
    out = {}
    for name, L, pk in CASES:
        d = synth.load_code(name)
        code = oracle.Code(d["frozen"], d["crc_len"], d["crc_poly"], d["punct"], d["systematic"])
        pr = oracle.pruning(**PRUNINGS[pk]) if pk else None
        st = oracle.Stats()
        llr = np.full(code.N - code.P, 3.0)
        oracle.decode(code, llr, L, oracle.CASCL, pr, oracle.F32, stats=st)
        out[f"{name}_L{L}_{pk or 'unpruned'}"] = dict(
            fg_elems=st.fg_elems, node_steps=st.node_steps, sorts=st.sorts, cand_total=st.cand_total,
            N=code.N, K=code.K, K_info=code.K_info, L=L)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "work_per_frame.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
