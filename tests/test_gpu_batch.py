"""Uneven batches: one persistent launch over many codes, list sizes and
number formats must decode every frame exactly like the oracle, exactly like
one launch per work item, and exactly like a CUDA-graph replay of itself."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import QMAP, gpu_code, make_inputs, unpack_info

pytestmark = pytest.mark.gpu

CTX = ["u00", "u01", "u02", "u04", "u05", "u09", "u16", "u22", "u27", "u30", "u36", "u41", "u43", "u47"]


def build_parts(seed=0, frames=(20, 70)):
    import torch
    from paper_1710_08314_gb300 import polarscl as ps
    rng = np.random.default_rng(seed)
    parts, refs = [], []
    for k, name in enumerate(CTX):
        d = synth.load_code(name)
        n = int(rng.integers(*frames))
        quant = "i8" if k % 3 == 2 else ("i16" if k % 5 == 4 else "f32")
        prune = (k % 2 == 1)
        code, info, llr = make_inputs(d, n, d["ebn0_db"] + 0.5, 100 + k)
        g = gpu_code(d)
        pdict = dict(mask=15, rep_max=8 if quant == "i8" else 0, spc_max=4, r1_t=2, spc_t=4)
        parts.append(dict(code=g, llr=torch.from_numpy(llr).cuda(), L=d["L"], algo=ps.PSCL_CASCL,
                          quant=QMAP[quant][0], prune=ps.pruning(**pdict) if prune else None))
        refs.append((code, llr, d["L"], quant, oracle.pruning(**pdict) if prune else None))
    return parts, refs


def test_batch_matches_oracle_plain_and_graph():
    import torch
    from paper_1710_08314_gb300.polarscl import Batch
    parts, refs = build_parts()
    b = Batch(parts)
    b.run()
    torch.cuda.synchronize()
    got = [tuple(t.cpu().numpy().copy() for t in b.outputs(i)) for i in range(len(parts))]
    for i, (code, llr, L, quant, pr) in enumerate(refs):
        r = oracle.decode_batch(code, llr.astype(np.float64), L, oracle.CASCL, pr, QMAP[quant][1], want_pm=False)
        bits = unpack_info(got[i][0], code.K_info)
        assert np.array_equal(bits, r["info"]), f"item {i} ({CTX[i]}): info bits differ from the oracle"
        assert np.array_equal(got[i][1], r["status"]), f"item {i} ({CTX[i]}): status differs"
    # one launch per item: identical
    b.info_pool.zero_()
    b.status_pool.zero_()
    b.run_plain()
    torch.cuda.synchronize()
    for i in range(len(parts)):
        info, st = b.outputs(i)
        assert np.array_equal(info.cpu().numpy(), got[i][0]) and np.array_equal(st.cpu().numpy(), got[i][1])
    # captured in a CUDA graph and replayed: identical
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run()
    b.info_pool.zero_()
    b.status_pool.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for i in range(len(parts)):
        info, st = b.outputs(i)
        assert np.array_equal(info.cpu().numpy(), got[i][0]) and np.array_equal(st.cpu().numpy(), got[i][1])
    b.close()


def test_batch_rejects_adaptive_items():
    from paper_1710_08314_gb300 import polarscl as ps
    from paper_1710_08314_gb300.polarscl import Batch
    import torch
    d = synth.load_code("u09")
    g = gpu_code(d)
    with pytest.raises(ps.PsclError):
        Batch([dict(code=g, llr=torch.zeros((4, d["N"] - d["P"]), device="cuda"), L=4, algo=ps.PSCL_FASCL)])
