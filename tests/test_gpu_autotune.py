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
    (w, f, b), measured = autotune.tuned(g, 8, ps.PSCL_I16, t, path=path)
    assert measured and w in autotune.WARPS_GRID and f in autotune.FUSE_GRID and b in autotune.BLOCK_GRID
    info, st, _ = g.decode(t, 8, ps.PSCL_CASCL, None, ps.PSCL_I16)
    assert torch.equal(info, ref_info) and torch.equal(st, ref_st)
    g2 = gpu_code(d)
    (w2, f2, b2), measured2 = autotune.tuned(g2, 8, ps.PSCL_I16, None, path=path)
    assert not measured2 and (w2, f2, b2) == (w, f, b)
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
