"""The autotuner measures schedule knobs; whatever it picks, results stay
bit-exact, and its cache round-trips."""
import os

import numpy as np
import pytest

import synth
from gpu_helpers import gpu_code, make_inputs

pytestmark = pytest.mark.gpu


def test_autotune_picks_applies_and_caches(tmp_path):
    import torch
    from paper_1710_08314_gb300 import autotune, polarscl as ps
    d = synth.load_code("c3_1024_512_L8")
    g = gpu_code(d)
    _, _, llr = make_inputs(d, 512, 2.0, 3)
    t = torch.from_numpy(llr).cuda()
    ref_info, ref_st, _ = g.decode(t, 8, ps.PSCL_CASCL, None, ps.PSCL_I16)
    path = str(tmp_path / "tune.json")
    (w, f, b, r), measured = autotune.tuned(g, 8, ps.PSCL_I16, t, path=path)
    assert measured and w in autotune.WARPS_GRID and f in autotune.FUSE_GRID and b in autotune.BLOCK_GRID
    assert r in (autotune.RESIDENT_LO, autotune.RESIDENT_HI)
    info, st, _ = g.decode(t, 8, ps.PSCL_CASCL, None, ps.PSCL_I16)
    assert torch.equal(info, ref_info) and torch.equal(st, ref_st)
    g2 = gpu_code(d)
    (w2, f2, b2, r2), measured2 = autotune.tuned(g2, 8, ps.PSCL_I16, None, path=path)
    assert not measured2 and (w2, f2, b2, r2) == (w, f, b, r)
    assert os.path.exists(path)


@pytest.mark.parametrize("wpb", [1, 2, 8])
def test_warps_per_block_gives_identical_results(wpb):
    """Frames per block (warps per block x 32/L) changes only the launch."""
    from paper_1710_08314_gb300 import polarscl as ps
    from gpu_helpers import gpu_decode
    for name, L, n in [("c2_2048_1723", 32, 300), ("c3_1024_512_L8", 8, 500)]:
        d = synth.load_code(name)
        _, _, llr = make_inputs(d, n, 3.0 if d["N"] == 2048 else 1.5, 40 + wpb)
        g = gpu_code(d)
        ref = gpu_decode(g, llr, L, "cascl", "f32")
        ps.pscl_code_tune(g.handle, L, ps.PSCL_F32, 20, 4, None, wpb)
        got = gpu_decode(g, llr, L, "cascl", "f32")
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("quant", ["f32", "i16", "i8"])
@pytest.mark.parametrize("wps,res", [(16, 16), (40, 16), (24, 28), (48, 28)])
def test_register_variant_and_slice_sizing_give_identical_results(quant, wps, res):
    """The register cap (resident warps) and the slice sizing (which may
    leave shared memory to the L1 cache) change only the launch, with and
    without pruned nodes."""
    from paper_1710_08314_gb300 import polarscl as ps, pruning
    from gpu_helpers import gpu_decode, QMAP
    d = synth.load_code("c3_1024_512_L8")
    _, _, llr = make_inputs(d, 400, 1.5, 60 + wps + res)
    for pr in [None, pruning(15, rep_max=8 if quant == "i8" else 0), pruning(15, rep_max=0, spc_max=0, node_min=9)]:
        g = gpu_code(d)
        ref = gpu_decode(g, llr, 8, "cascl", quant, pr)
        ps.pscl_code_tune(g.handle, 8, QMAP[quant][0], wps, 4, pr, 4, res)
        got = gpu_decode(g, llr, 8, "cascl", quant, pr)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)
