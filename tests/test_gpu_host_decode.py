"""pscl_decode_host (host buffers, transfers overlapped with chunked decodes)
gives the same bits, status words as pscl_decode on the same LLRs, for batches
below and above the chunking threshold, page-locked and pageable buffers,
adaptive schedules and fixed point; argument errors are reported before
anything runs."""
import numpy as np
import pytest

import synth
from gpu_helpers import AMAP, QMAP, gpu_code, make_inputs

pytestmark = pytest.mark.gpu


def _device_decode(g, llr, L, algo, quant, pr):
    import torch
    t = torch.from_numpy(llr).cuda()
    info, status, _ = g.decode(t, L, AMAP[algo][0], pr, QMAP[quant][0])
    torch.cuda.synchronize()
    return info.cpu().numpy(), status.cpu().numpy()


def _host_decode(g, llr, L, algo, quant, pr, pinned):
    import torch
    from paper_1710_08314_gb300 import polarscl as ps
    n = llr.shape[0]
    if pinned:
        llr_h = torch.from_numpy(llr).pin_memory()
        info_h = torch.zeros((n, g.nbytes), dtype=torch.uint8).pin_memory()
        status_h = torch.zeros((n,), dtype=torch.int32).pin_memory()
    else:
        llr_h = np.ascontiguousarray(llr)
        info_h = np.zeros((n, g.nbytes), dtype=np.uint8)
        status_h = np.zeros((n,), dtype=np.int32)
    stream = torch.cuda.current_stream()
    ps.pscl_decode_host(g.handle, llr_h, n, L, AMAP[algo][0], pr, QMAP[quant][0], info_h, status_h, stream)
    stream.synchronize()
    if pinned:
        return info_h.numpy(), status_h.numpy()
    return info_h, status_h


@pytest.mark.parametrize("n", [1, 777, 9000, 20000])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_decode_equals_device_decode(n, pinned):
    d = synth.load_code("c2_2048_1723")
    _, _, llr = make_inputs(d, n, 3.5, 1200 + n)
    g = gpu_code(d)
    ref = _device_decode(g, llr, 32, "cascl", "f32", None)
    got = _host_decode(g, llr, 32, "cascl", "f32", None, pinned)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


@pytest.mark.parametrize("algo,quant", [("fascl", "f32"), ("fascl", "i8"), ("cascl", "i16")])
def test_host_decode_adaptive_and_fixed_point(algo, quant):
    from paper_1710_08314_gb300 import pruning
    d = synth.load_code("c3_1024_512_L8")
    n = 17000
    _, _, llr = make_inputs(d, n, 1.5, 1300)
    g = gpu_code(d)
    pr = pruning(15, rep_max=8 if quant == "i8" else 0)
    ref = _device_decode(g, llr, 8, algo, quant, pr)
    got = _host_decode(g, llr, 8, algo, quant, pr, True)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_host_decode_repeated_calls_and_growth():
    """Later calls on the same stream reuse (and grow) the staging buffer
    only after the earlier ones are done with it."""
    d = synth.load_code("c2_2048_1723")
    g = gpu_code(d)
    for n, seed in [(9000, 1), (9000, 2), (30000, 3), (5000, 4)]:
        _, _, llr = make_inputs(d, n, 3.5, 1400 + seed)
        ref = _device_decode(g, llr, 32, "cascl", "f32", None)
        got = _host_decode(g, llr, 32, "cascl", "f32", None, True)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_host_decode_argument_errors():
    from paper_1710_08314_gb300 import polarscl as ps
    d = synth.load_code("c1_cascl_128_64_L4")
    g = gpu_code(d)
    llr = np.zeros((4, 128), dtype=np.float32)
    info = np.zeros((4, g.nbytes), dtype=np.uint8)
    st = np.zeros((4,), dtype=np.int32)
    with pytest.raises(ps.PsclError):
        ps.pscl_decode_host(g.handle, llr, -1, 4, ps.PSCL_CASCL, None, ps.PSCL_F32, info, st)
    with pytest.raises(ps.PsclError):
        ps.pscl_decode_host(g.handle, llr, 4, 3, ps.PSCL_CASCL, None, ps.PSCL_F32, info, st)
    with pytest.raises(ps.PsclError):
        ps.pscl_decode_host(g.handle, None, 4, 4, ps.PSCL_CASCL, None, ps.PSCL_F32, info, st)
    ps.pscl_decode_host(g.handle, llr, 0, 4, ps.PSCL_CASCL, None, ps.PSCL_F32, info, st)
