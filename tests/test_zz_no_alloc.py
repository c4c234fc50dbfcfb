"""pscl_decode_static: decoding that allocates nothing, for callers that cannot
allocate device memory while they decode.  Its results must equal
pscl_decode's, call after call, even though every call reuses the same
static scratch inside the library."""
import numpy as np
import pytest

import synth
from gpu_helpers import gpu_code, make_inputs

pytestmark = pytest.mark.gpu


def _decode_both(g, llr, L, algo, prune, quant):
    import torch
    from paper_1710_08314_gb300 import polarscl as ps
    t = torch.from_numpy(llr).cuda()
    n = t.shape[0]
    out = []
    for fn in (ps.pscl_decode, ps.pscl_decode_static):
        info = torch.full((n, g.nbytes), 0xAA, dtype=torch.uint8, device="cuda")
        status = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        pm = torch.full((n, L), -1.0, dtype=torch.float32, device="cuda")
        fn(g.handle, t, n, L, algo, prune, quant, info, status, pm)
        torch.cuda.synchronize()
        out.append((info.cpu().numpy(), status.cpu().numpy(), pm.cpu().numpy()))
    return out


@pytest.mark.parametrize("name,L,algo,quant,prune", [
    ("c2_2048_1723", 32, 1, 0, None),          # CA-SCL, float, N = 2048: scratch in use
    ("c1_cascl_128_64_L4", 4, 3, 2, "i8"),     # adaptive (frame lists in the scratch), int8
])
def test_static_scratch_matches_pscl_decode_twice(name, L, algo, quant, prune):
    from paper_1710_08314_gb300 import polarscl as ps
    d = synth.load_code(name)
    g = gpu_code(d)
    pr = ps.pruning(15, rep_max=8) if prune else None
    ps.pscl_prepare(g.handle, pr)           # set-up: the schedule upload allocates here
    for call, seed in enumerate([31, 32]):  # two calls in a row share the scratch
        _, _, llr = make_inputs(d, 700, 3.0 if d["N"] == 2048 else 1.0, seed)
        (ia, sa, pa), (ib, sb, pb) = _decode_both(g, llr, L, algo, pr, quant)
        assert np.array_equal(ia, ib), f"call {call}: info bits differ"
        assert np.array_equal(sa, sb), f"call {call}: status differs"
        assert np.array_equal(pa, pb), f"call {call}: path metrics differ"


def test_static_scratch_rejects_oversized_and_unprepared_calls():
    import torch
    from paper_1710_08314_gb300 import polarscl as ps
    d = synth.load_code("c1_cascl_128_64_L4")
    g = gpu_code(d)
    t = torch.zeros((8, 128), device="cuda")
    info = torch.empty((8, g.nbytes), dtype=torch.uint8, device="cuda")
    status = torch.empty((8,), dtype=torch.int32, device="cuda")
    # adaptive decoding keeps two frame lists of 4 bytes per frame in the scratch:
    # 5 million frames need 40 MB > 32 MiB and must be refused before any launch
    ps.pscl_prepare(g.handle, None)
    with pytest.raises(ps.PsclError) as e:
        ps.pscl_decode_static(g.handle, t, 5_000_000, 4, 3, None, 0, info, status)
    assert e.value.code == ps.PSCL_EINVAL and "static scratch" in str(e.value)
    # a pruning setting whose schedule was never prepared is refused, not built
    with pytest.raises(ps.PsclError) as e:
        ps.pscl_decode_static(g.handle, t, 8, 4, 1, ps.pruning(15, rep_max=2), 0, info, status)
    assert "pscl_prepare" in str(e.value)


def test_static_calls_leave_device_memory_unchanged():
    """After set-up, further static calls take no device memory: the free
    memory that cudaMemGetInfo reports is the same before and after them (the GPU
    is this process's alone while the tests run)."""
    import torch
    from paper_1710_08314_gb300 import polarscl as ps
    d = synth.load_code("c2_2048_1723")
    g = gpu_code(d)
    ps.pscl_prepare(g.handle, None)
    _, _, llr = make_inputs(d, 256, 3.0, 41)
    t = torch.from_numpy(llr).cuda()
    info = torch.empty((256, g.nbytes), dtype=torch.uint8, device="cuda")
    status = torch.empty((256,), dtype=torch.int32, device="cuda")
    ps.pscl_decode_static(g.handle, t, 256, 32, ps.PSCL_CASCL, None, ps.PSCL_F32, info, status)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        ps.pscl_decode_static(g.handle, t, 256, 32, ps.PSCL_CASCL, None, ps.PSCL_F32, info, status)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
