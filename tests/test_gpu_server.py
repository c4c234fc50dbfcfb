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


def test_mixed_formats_and_pruning_in_one_server_equal_the_oracle():
    """One server holding float, int16 and int8 contexts, pruned and
    unpruned: every served frame equals the oracle's decode of it (bits and
    status), whether it was decoded beside requests of other formats."""
    import torch
    from paper_1710_08314_gb300 import pruning
    from paper_1710_08314_gb300.polarscl import Server
    from oracle_pool import OraclePool
    from gpu_helpers import QMAP, unpack_info
    import oracle
    P_ALL = dict(mask=15, rep_max=0, spc_max=4, r1_t=2, spc_t=4)
    P_I8 = dict(mask=15, rep_max=8, spc_max=4, r1_t=2, spc_t=4)
    spec = [("mcs_256_128", 8, None, "f32"), ("mcs_512_256", 16, P_ALL, "f32"),
            ("mcs_1024_512", 16, P_I8, "i8"), ("mcs_2048_1723", 32, None, "i16"),
            ("mcs_128_40", 8, P_ALL, "i16"), ("mcs_2048_1723", 32, P_I8, "i8")]
    ctx, codes = [], []
    for name, L, p, q in spec:
        d = synth.load_code(name)
        g = gpu_code(d)
        codes.append((d, g))
        ctx.append((g, L, pruning(**p) if p else None, QMAP[q][0]))
    rng = np.random.default_rng(9)
    reqs = []
    for r in range(36):
        k = r % len(spec)
        d, g = codes[k]
        n = int(rng.integers(1, 9 if d["N"] == 2048 else 33))
        code, _, llr = make_inputs(d, n, d["ebn0_db"] - 0.5, 4000 + r)
        reqs.append((k, code, llr, torch.from_numpy(llr).cuda(),
                     torch.zeros((n, g.nbytes), dtype=torch.uint8, device="cuda"),
                     torch.zeros((n,), dtype=torch.int32, device="cuda")))
    torch.cuda.synchronize()
    with OraclePool() as pool:
        srv = Server(ctx, ring_slots=64, max_frames=64, idle_timeout_ms=20000)
        try:
            tickets = []
            for k, _, _, t, i, s in reqs:
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
        for r, (k, code, llr, _, i, s) in enumerate(reqs):
            name, L, p, q = spec[k]
            oi, os_, _ = pool.decode(code, llr, L, oracle.CASCL, QMAP[q][1], p)
            gi = unpack_info(i.cpu().numpy(), code.K_info)
            assert np.array_equal(gi, oi), f"request {r} ({name}, {q}): info differs from the oracle"
            assert np.array_equal(s.cpu().numpy(), os_), f"request {r} ({name}, {q}): status differs"


def test_admission_by_device_byte_budget():
    """With a byte budget, a request is admitted only while the device bytes
    of the frames in flight (LLR rows, outputs, scratch share) fit; the next
    one is deferred until a completion frees its share, and a request larger
    than the whole budget is refused."""
    import torch
    from paper_1710_08314_gb300 import polarscl as ps
    from paper_1710_08314_gb300.polarscl import Server
    codes, ctx = _contexts()
    d, g = codes[4]                      # (2048, 1723), L = 32
    probe = Server(ctx[4:5], ring_slots=8, max_frames=64, idle_timeout_ms=2000)
    try:
        info4 = probe.context_info(0)
    finally:
        probe.stop()
    per = info4["bytes_per_frame"]
    assert per >= (d["N"]) * 4 + g.nbytes + 4
    assert info4["smem_per_warp"] > 0 and info4["scratch_per_warp"] > 0
    budget = 10 * per                    # ten frames in flight at most
    _, _, llr = make_inputs(d, 16, d["ebn0_db"], 5000)
    t = torch.from_numpy(llr).cuda()
    info = torch.zeros((16, g.nbytes), dtype=torch.uint8, device="cuda")
    st = torch.zeros((16,), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    srv = Server(ctx[4:5], ring_slots=8, max_frames=64, idle_timeout_ms=20000, hbm_budget=budget)
    try:
        with pytest.raises(ps.PsclError) as e:   # 11 frames can never fit
            srv.submit(0, t[:11], info[:11], st[:11])
        assert e.value.code == ps.PSCL_EINVAL
        t1 = srv.submit(0, t[:6], info[:6], st[:6])
        assert t1 is not None
        t2 = srv.submit(0, t[6:11], info[6:11], st[6:11])   # 6 + 5 > 10: deferred
        assert t2 is None
        t3 = srv.submit(0, t[6:10], info[6:10], st[6:10])   # 6 + 4 fits
        assert t3 is not None
        _wait(srv, [t1, t3])
        t2 = srv.submit(0, t[10:16], info[10:16], st[10:16])
        assert t2 is not None
        _wait(srv, [t2])
    finally:
        srv.stop()
    ri, rs = _reference(g, t, d["L"])
    assert torch.equal(ri, info) and torch.equal(rs, st)


def test_every_warp_leaves_together_on_the_idle_budget():
    """A few warps, idle at different times: when the idle budget runs out all
    of them leave, the host sees PSCL_ETIMEDOUT, and a submit afterwards is
    refused instead of waiting for a loop that is gone."""
    import torch
    from paper_1710_08314_gb300 import polarscl as ps
    from paper_1710_08314_gb300.polarscl import Server
    codes, ctx = _contexts()
    d, g = codes[1]
    _, _, llr = make_inputs(d, 40, d["ebn0_db"], 6000)
    t = torch.from_numpy(llr).cuda()
    info = torch.zeros((40, g.nbytes), dtype=torch.uint8, device="cuda")
    st = torch.zeros((40,), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    srv = Server(ctx, ring_slots=8, max_frames=64, idle_timeout_ms=300, max_warps=16)
    try:
        tk = srv.submit(1, t[:3], info[:3], st[:3])
        _wait(srv, [tk])
        time.sleep(0.15)                 # some warps idle for a while ...
        tk = srv.submit(1, t[3:40], info[3:40], st[3:40])
        _wait(srv, [tk])                 # ... others just worked
        t0 = time.time()
        while srv.status()["running"] and time.time() - t0 < 10:
            time.sleep(0.02)
        stt = srv.status()
        assert not stt["running"] and stt["device_status"] == ps.PSCL_ETIMEDOUT
        assert srv.poll() == []
        with pytest.raises(ps.PsclError):
            srv.submit(1, t[:1], info[:1], st[:1])
    finally:
        srv.stop()
    ri, rs = _reference(g, t, d["L"])
    assert torch.equal(ri, info) and torch.equal(rs, st)


@pytest.mark.parametrize("seed", [13, 14, 15])
def test_thousands_of_small_requests_from_a_busy_producer(seed):
    """Many tiny requests published as fast as the host can: idle warps keep
    opening new tickets concurrently; every request must complete once and
    decode exactly as pscl_decode does."""
    import torch
    from paper_1710_08314_gb300.polarscl import Server
    codes, ctx = _contexts()
    d, g = codes[0]
    n_req = 3000
    _, _, llr = make_inputs(d, 4 * n_req, d["ebn0_db"], 7000)
    t = torch.from_numpy(llr).cuda()
    info = torch.zeros((4 * n_req, g.nbytes), dtype=torch.uint8, device="cuda")
    st = torch.zeros((4 * n_req,), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    sizes = rng.integers(1, 5, n_req)
    srv = Server(ctx, ring_slots=64, max_frames=8, idle_timeout_ms=3000)
    done = {}
    try:
        tickets = []
        for r in range(n_req):
            lo = 4 * r
            n = int(sizes[r])
            while True:
                try:
                    tk = srv.submit(0, t[lo:lo + n], info[lo:lo + n], st[lo:lo + n])
                except Exception as e:
                    raise AssertionError(f"request {r}: {e}; {srv.status()}; exit {srv.debug_exit()}; "
                                         f"outstanding {srv.debug_slots()}")
                if tk is not None:
                    break
                for c in srv.poll():
                    done[c.ticket] = c
            tickets.append(tk)
        t0 = time.time()
        while len(done) < n_req and time.time() - t0 < 60:
            for c in srv.poll():
                done[c.ticket] = c
        assert len(done) == n_req and set(done) == set(tickets)
        assert all(c.status == 0 for c in done.values())
    finally:
        srv.stop()
    ri, rs = _reference(g, t, d["L"])
    for r in range(n_req):
        lo, n = 4 * r, int(sizes[r])
        assert torch.equal(ri[lo:lo + n], info[lo:lo + n]) and torch.equal(rs[lo:lo + n], st[lo:lo + n]), r
