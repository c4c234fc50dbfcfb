"""Serving loop: requests of mixed codes and list sizes decoded by the
device-resident loop must equal pscl_decode frame by frame, whether a
request runs alone or inside a busy mix; malformed requests, a full ring and
an idle producer are reported on the host without touching the GPU."""
import time

import numpy as np
import pytest

import synth
from gpu_helpers import gpu_code, make_inputs

pytestmark = pytest.mark.gpu

MCS = ["mcs_128_40", "mcs_256_128", "mcs_512_256", "mcs_1024_512", "mcs_2048_1723"]


def _contexts():
    codes, ctx = [], []
    for name in MCS:
        d = synth.load_code(name)
        g = gpu_code(d)
        codes.append((d, g))
        ctx.append((g, d["L"], None))
    return codes, ctx


def _wait(server, tickets, timeout_s=60.0):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets):
        for c in server.poll():
            done[c.ticket] = c
        if time.time() - t0 > timeout_s:
            raise AssertionError(f"only {len(done)} of {len(tickets)} requests completed")
        time.sleep(0.0005)
    return done


def _reference(g, llr, L):
    from paper_1710_08314_gb300 import polarscl as ps
    info, st, _ = g.decode(llr, L, ps.PSCL_CASCL, None, ps.PSCL_F32)
    return info, st


def test_requests_alone_and_in_the_mix_equal_pscl_decode():
    import torch
    from paper_1710_08314_gb300.polarscl import Server
    codes, ctx = _contexts()
    rng = np.random.default_rng(5)
    reqs = []
    for r in range(40):
        k = int(rng.integers(0, len(MCS)))
        d, g = codes[k]
        n = int(rng.integers(1, 40))
        _, _, llr = make_inputs(d, n, d["ebn0_db"] - 0.5, 1000 + r)
        t = torch.from_numpy(llr).cuda()
        reqs.append((k, t, torch.zeros((n, g.nbytes), dtype=torch.uint8, device="cuda"),
                     torch.zeros((n,), dtype=torch.int32, device="cuda")))
    torch.cuda.synchronize()
    # while the server runs, only stream-level waits: a device-wide
    # synchronize would wait for the persistent serving kernel itself
    srv = Server(ctx, ring_slots=64, max_frames=64, idle_timeout_ms=20000)
    try:
        # request 0 alone
        k0, t0, i0, s0 = reqs[0]
        tk = srv.submit(k0, t0, i0, s0)
        _wait(srv, [tk])
        alone = (i0.clone(), s0.clone())
        i0.zero_()
        s0.zero_()
        torch.cuda.current_stream().synchronize()
        # all of them at once, request 0 in the middle of the mix
        order = list(range(1, 20)) + [0] + list(range(20, 40))
        tickets = []
        for r in order:
            k, t, i, s = reqs[r]
            while True:
                tk = srv.submit(k, t, i, s)
                if tk is not None:
                    break
                srv.poll()
            tickets.append(tk)
        done = _wait(srv, tickets)
        assert all(c.status == 0 for c in done.values())
    finally:
        srv.stop()
    assert torch.equal(alone[0], reqs[0][2]) and torch.equal(alone[1], reqs[0][3])
    for r, (k, t, i, s) in enumerate(reqs):
        ri, rs = _reference(codes[k][1], t, codes[k][0]["L"])
        assert torch.equal(ri, i), f"request {r}: info differs from pscl_decode"
        assert torch.equal(rs, s), f"request {r}: status differs from pscl_decode"


def test_malformed_full_and_idle_are_reported_on_the_host():
    import torch
    from paper_1710_08314_gb300 import polarscl as ps
    from paper_1710_08314_gb300.polarscl import Server
    codes, ctx = _contexts()
    d, g = codes[0]
    llr = torch.zeros((8, 128), device="cuda")
    info = torch.zeros((8, g.nbytes), dtype=torch.uint8, device="cuda")
    st = torch.zeros((8,), dtype=torch.int32, device="cuda")
    nine = torch.zeros((9, 128), device="cuda")
    torch.cuda.synchronize()
    srv = Server(ctx[:1], ring_slots=4, max_frames=8, max_inflight=8, idle_timeout_ms=400)
    try:
        with pytest.raises(ps.PsclError):          # unknown context
            srv.submit(3, llr, info, st)
        with pytest.raises(ps.PsclError):          # more frames than a request may hold
            srv.submit(0, nine, info, st)
        # admission: 8 frames fill the budget; the next request is deferred, not dropped
        t1 = srv.submit(0, llr, info, st)
        assert t1 is not None
        t2 = srv.submit(0, llr[:1], info[:1], st[:1])
        assert t2 is None
        _wait(srv, [t1])
        t2 = srv.submit(0, llr[:1], info[:1], st[:1])
        assert t2 is not None
        _wait(srv, [t2])
        # the producer goes quiet: the device loop leaves on its idle budget
        t0 = time.time()
        while srv.status()["running"] and time.time() - t0 < 10:
            time.sleep(0.05)
        stt = srv.status()
        assert not stt["running"] and stt["device_status"] == ps.PSCL_ETIMEDOUT
    finally:
        srv.stop()


def test_burst_of_large_requests_all_complete():
    """Every idle warp races for the frames of the oldest request; no request
    may be skipped while frames of it are still unclaimed."""
    import torch
    from paper_1710_08314_gb300.polarscl import Server
    codes, ctx = _contexts()
    reqs = []
    for r in range(24):
        k = 4 if r % 3 else 0          # mostly (2048, 1723) L = 32: one frame per task
        d, g = codes[k]
        n = 200 if k == 4 else 37
        _, _, llr = make_inputs(d, n, d["ebn0_db"], 2000 + r)
        reqs.append((k, torch.from_numpy(llr).cuda(), torch.zeros((n, g.nbytes), dtype=torch.uint8, device="cuda"),
                     torch.zeros((n,), dtype=torch.int32, device="cuda")))
    torch.cuda.synchronize()
    srv = Server(ctx, ring_slots=32, max_frames=256, idle_timeout_ms=20000)
    try:
        tickets = [srv.submit(k, t, i, s) for k, t, i, s in reqs]
        assert all(t is not None for t in tickets)
        _wait(srv, tickets, timeout_s=120.0)
    finally:
        srv.stop()
    for r, (k, t, i, s) in enumerate(reqs):
        ri, rs = _reference(codes[k][1], t, codes[k][0]["L"])
        assert torch.equal(ri, i) and torch.equal(rs, s), f"request {r} differs from pscl_decode"


def test_reused_request_buffers_are_read_afresh():
    """A client that refills the same LLR buffer for its next request must
    get the new frames decoded (the device loop outlives any cache)."""
    import torch
    from paper_1710_08314_gb300.polarscl import Server
    codes, ctx = _contexts()
    d, g = codes[1]
    n = 64
    contents = []
    for r in range(6):
        _, _, llr = make_inputs(d, n, d["ebn0_db"], 3000 + r)
        contents.append(torch.from_numpy(llr).cuda())
    llr_buf = torch.zeros_like(contents[0])
    info = torch.zeros((n, g.nbytes), dtype=torch.uint8, device="cuda")
    st = torch.zeros((n,), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    srv = Server(ctx, ring_slots=8, max_frames=64, idle_timeout_ms=20000)
    got = []
    try:
        for r in range(6):
            llr_buf.copy_(contents[r])
            torch.cuda.current_stream().synchronize()
            tk = srv.submit(1, llr_buf, info, st)
            assert tk is not None
            _wait(srv, [tk])
            got.append((info.clone(), st.clone()))
            torch.cuda.current_stream().synchronize()
    finally:
        srv.stop()
    for r in range(6):
        ri, rs = _reference(g, contents[r], d["L"])
        assert torch.equal(ri, got[r][0]) and torch.equal(rs, got[r][1]), f"request {r}: stale input"
