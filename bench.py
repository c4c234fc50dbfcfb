"""Benchmark: batched CA-SCL decoding of the (2048, 1723 incl. CRC-32) polar
code with L = 32 on one GB300 (info Mb/s), plus the end-to-end rate through
the C ABI with host buffers, the roofline of the decode kernel and the CPU
oracle's rate on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step decodes one batch of B frames (LLR ingest and quantisation, f/g
updates, partial sums, path metrics, top-L selection, lazy path copy, CRC
check and info-bit extraction: the whole hot path).  Inputs are synthetic:
uniform info bits, systematic encoding, BPSK over AWGN at 4.5 dB (the
headline; the same decode is also timed at 3.5 dB).

    python bench.py --study spc4plus|lsweep   # the slower studies, one JSON line each
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c2_2048_1723"
EBN0_DB = 4.5
L_LIST = 32
BATCH = 16384            # frames per step: 134 MB of LLRs, larger than L2
ALGO_CASCL = 1
QUANT = {"f32": 0, "i16": 1, "i8": 2}


ALGO_NAMES = {"cascl": "CA-SCL", "sc": "SC", "fascl": "FA-SSCL"}


def headline_config(quant: str = "f32", batch: int = BATCH, ws: int = 1, algo: str = "cascl",
                    pruned: bool = False, node_min: int = 0) -> dict:
    """The workload both arms report (so that their lines compare);
    --algo / --pruned select another decode of the same frames (profiling)."""
    pn = ("pruned" + (f" (nodes of {node_min}+ leaves)" if node_min > 2 else "")) if pruned else "unpruned"
    return {"workload": f"{ALGO_NAMES[algo]} (2048,1723 incl. CRC-32) L=32 {quant} "
                        f"{pn}, BPSK-AWGN {EBN0_DB} dB, GA frozen set at 4.5 dB",
            "frames_per_step": batch, "l2": "inputs larger than L2 (134 MB LLRs per step)",
            "parallelism": f"replicas x{ws}"}


def max_over_ranks(value: float, device: str = "cuda") -> float:
    """Largest value over all ranks (the slowest rank's time), or the value
    itself without a process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def log(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on the host cores (spawned workers)
def _oracle_worker(args):
    name, llr_rows, L = args
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    import synth
    d = synth.load_code(name)
    code = oracle.Code(d["frozen"], d["crc_len"], d["crc_poly"], d["punct"], d["systematic"])
    t0 = time.perf_counter()
    if llr_rows:
        oracle.decode_batch(code, np.asarray(llr_rows, dtype=np.float64), L, oracle.CASCL, None, oracle.F32,
                            want_pm=False)
    return time.perf_counter() - t0, len(llr_rows)


class OraclePool:
    """The oracle on every host core: a pool of spawned workers, warmed up
    (imports, library load) before anything is timed."""

    def __init__(self):
        import multiprocessing as mp
        import numpy as np
        import oracle
        import synth
        self.cores = len(os.sched_getaffinity(0))
        self.pool = mp.get_context("spawn").Pool(self.cores)
        d = synth.load_code(WORKLOAD)
        self.code = oracle.Code(d["frozen"], d["crc_len"], d["crc_poly"], d["punct"], d["systematic"])
        self.pool.map(_oracle_worker, [(WORKLOAD, [], L_LIST)] * self.cores)
        # seconds per frame on one core, from one frame
        llr = self.frames(1, 5)
        t0 = time.perf_counter()
        oracle.decode_batch(self.code, llr.astype(np.float64), L_LIST, oracle.CASCL, None, oracle.F32,
                            want_pm=False)
        self.per_frame = time.perf_counter() - t0

    def frames(self, n, seed):
        import oracle
        import synth
        info = synth.info_bits(n, self.code.K_info, seed)
        x = oracle.encode(self.code, info)
        return synth.bpsk_awgn_llr(x, synth.sigma_for(EBN0_DB, self.code.K_info / self.code.N), seed + 1)

    def rate(self, seconds, seed):
        """Info Mb/s over about `seconds` of decoding on all cores."""
        n = max(self.cores, int(self.cores * seconds / max(self.per_frame, 1e-4)))
        llr = self.frames(n, seed)
        chunks = [llr[i::self.cores].tolist() for i in range(self.cores)]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(WORKLOAD, ch, L_LIST) for ch in chunks])
        wall = time.perf_counter() - t0
        frames = sum(r[1] for r in res)
        sample = (f"{frames} frames of the same workload ((2048,1723) CA-SCL L=32 f32, {EBN0_DB} dB) on "
                  f"{self.cores} worker processes; {wall:.1f} s of decoding (workers started and warmed up first)")
        return frames * self.code.K_info / wall / 1e6, sample

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_oracle_rate(seconds=20.0, seed=99):
    p = OraclePool()
    try:
        v, sample = p.rate(seconds, seed)
        one = oracle_single_thread(p, seconds=6.0, seed=seed + 1)
        return v, p.cores, sample, one
    finally:
        p.close()


def oracle_single_thread(pool, seconds, seed):
    """The oracle on one thread of this process (the paper's figures are
    single-core): info Mb/s over about `seconds` of decoding."""
    import numpy as np
    import oracle
    n = max(1, int(seconds / max(pool.per_frame, 1e-4)))
    llr = pool.frames(n, seed).astype(np.float64)
    t0 = time.perf_counter()
    oracle.decode_batch(pool.code, llr, L_LIST, oracle.CASCL, None, oracle.F32, want_pm=False)
    wall = time.perf_counter() - t0
    return {"value": n * pool.code.K_info / wall / 1e6, "unit": "Mb/s", "cores": 1,
            "sample": f"{n} frames of the same workload on one thread, {wall:.1f} s"}


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    pool = OraclePool()
    per_step = []
    sample = ""
    try:
        for s in range(args.warmup + args.steps):
            v, sample = pool.rate(5.0, 1000 + s)
            if s >= args.warmup:
                per_step.append(v)
    finally:
        pool.close()
    value = sum(per_step) / len(per_step)
    line = {
        "impl": "reference", "metric": "info Mb/s per GB300 (CA-SCL N=2048 K=1723 L=32) bit-exact",
        "value": value, "unit": "Mb/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": headline_config("f32", BATCH, ws),
        "cpu_baseline": {"value": value, "unit": "Mb/s", "cores": pool.cores, "kind": "oracle",
                         "sample": "the CPU oracle (plain C, list copies) on the host cores, each step about 5 s "
                                   "of decoding: " + sample},
        "e2e": {"value": value, "unit": "Mb/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"pscl_clocks_{os.getpid()}_{index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# Further workloads, reported beside the headline (same JSON line).
def _gen_frames(code, n, ebn0_db, gen, sigma_per_frame=None):
    """Synthetic frames on the device: random info bits -> library encoder ->
    BPSK-AWGN channel.  Returns (info_packed, llr)."""
    import torch
    import synth
    info = torch.randint(0, 256, (n, code.nbytes), generator=gen, device="cuda", dtype=torch.uint8)
    if code.K_info % 8:
        info[:, -1] &= (0xFF << (8 - code.K_info % 8)) & 0xFF
    x = code.encode(info)
    keep = None
    if code.puncture is not None:
        keep = torch.from_numpy(np.flatnonzero(code.puncture == 0)).cuda()
    sig = sigma_per_frame if sigma_per_frame is not None else synth.sigma_for(ebn0_db, code.K_info / (code.N - code.P))
    llr = synth.torch_bpsk_awgn_llr(x, sig, gen, keep)
    return info, llr


def _timed(fn, reps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _each(fn, reps):
    """Device time of each of `reps` calls (ms), after one warm-up call."""
    import torch
    fn()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record()
    for r in range(reps):
        fn()
        ev[r + 1].record()
    torch.cuda.synchronize()
    return [ev[r].elapsed_time(ev[r + 1]) for r in range(reps)]


def pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * len(xs)))] if xs else None


def batch_latency(fn, reps=20):
    """p50 / p99 / max of the device time of one batch decode over `reps`
    back-to-back calls (ms)."""
    t = _each(fn, reps)
    return {"batch_p50_ms": pct(t, 0.5), "batch_p99_ms": pct(t, 0.99), "batch_max_ms": max(t), "reps": reps}


def frame_latency(code, llr1, L, algo, prune, quant, reps=30):
    """Latency of one frame decoded alone (one launch per stage): the GPU
    counterpart of the paper's per-frame latency, median over `reps` (ms)."""
    import torch
    from paper_1710_08314_gb300 import polarscl as ps
    o = torch.empty((1, code.nbytes), dtype=torch.uint8, device="cuda")
    st = torch.empty((1,), dtype=torch.int32, device="cuda")
    t = _each(lambda: ps.pscl_decode(code.handle, llr1, 1, L, algo, prune, quant, o, st, None, None), reps)
    return pct(t, 0.5)


def _code(name):
    import synth
    from paper_1710_08314_gb300 import Code
    d = synth.load_code(name)
    return d, Code(d["frozen"], d["crc_len"], d["crc_poly"], d["punct"], d["systematic"])


def _decode_fn(code, llr, n, L, algo, prune, quant, o, st):
    from paper_1710_08314_gb300 import polarscl as ps
    return lambda: ps.pscl_decode(code.handle, llr, n, L, algo, prune, quant, o, st, None, None)


def run_c1(gen):
    """Plain CA-SCL (128, 64 incl. CRC-8), L = 4, f32, no pruning, 2.0 dB, 10,000 frames."""
    import torch
    from paper_1710_08314_gb300 import autotune
    d, code = _code("c1_cascl_128_64_L4")
    info, llr = _gen_frames(code, 10000, 2.0, gen)
    autotune.tuned(code, 4, 0, llr)
    out = torch.empty_like(info)
    st = torch.empty((10000,), dtype=torch.int32, device="cuda")
    fn = _decode_fn(code, llr, 10000, 4, 1, None, 0, out, st)
    ms = _timed(fn)
    fer = float((out != info).any(dim=1).float().mean())
    lat = batch_latency(fn)
    lat["frame_ms"] = frame_latency(code, llr[:1], 4, 1, None, 0)
    return dict(value=10000 * code.K_info / ms / 1e3, unit="Mb/s", ms=ms, frames=10000, fer=fer, latency=lat,
                work="c1_cascl_128_64_L4_L4_unpruned", quant="f32")


C2_SNRS = (3.5, 3.75, 4.0, 4.25, 4.5)


def run_c2(gen, snrs=C2_SNRS, frames=1000000):
    """Adaptive FA-SSCL (2048, 1723 incl. CRC-32), Lmax = 32, pruned
    (R0/R1/REP/SPC4; REP8- for int8), f32 and int8, 10^6 frames per point;
    "_n32": the same node types restricted to nodes of 32 or more leaves,
    SPC of any size (the smaller nodes decoded in register subtrees).
    Per-frame latency as in the paper's Table 3: a frame that stops at list
    size L costs the single-frame decodes of stages 1, 2, ..., L (measured
    one launch per stage); L_avg weighs them by the measured stop histogram,
    L_worst is a frame that fails every stage (pure-noise LLRs)."""
    import torch
    from paper_1710_08314_gb300 import pruning, polarscl as ps
    from paper_1710_08314_gb300 import autotune
    d, code = _code("c2_2048_1723")
    out = {}
    Ls = [1, 2, 4, 8, 16, 32]
    variants = [(0, "f32", "", pruning(15, rep_max=0)), (2, "i8", "", pruning(15, rep_max=8)),
                (0, "f32", "_n32", pruning(15, rep_max=0, spc_max=0, node_min=17)),
                (2, "i8", "_n32", pruning(15, rep_max=8, spc_max=0, node_min=17))]
    for quant, qn, tag, pr in variants:
        stage_ms = None
        for snr in sorted(snrs, reverse=True):
            info, llr = _gen_frames(code, frames, snr, gen)
            if stage_ms is None:
                # a sample of two waves of the one-path first stage (32 frames per warp)
                autotune.tuned(code, 32, quant, llr[:1 << 18].contiguous(), prune=pr, algo=ps.PSCL_FASCL)
                # per-stage single-frame latency (each stage a CA-SCL(L) decode)
                stage_ms = {L: frame_latency(code, llr[:1], L, ps.PSCL_CASCL if L > 1 else ps.PSCL_SC, pr, quant)
                            for L in Ls}
                noise = torch.randn((1, code.N), generator=gen, device="cuda")
                worst = frame_latency(code, noise, 32, ps.PSCL_FASCL, pr, quant)
            o = torch.empty_like(info)
            st = torch.empty((frames,), dtype=torch.int32, device="cuda")
            fn = _decode_fn(code, llr, frames, 32, ps.PSCL_FASCL, pr, quant, o, st)
            ms = _timed(fn, reps=2)
            Lu = ((st >> 8) & 0xFF).cpu().numpy()
            hist = {str(int(L)): int((Lu == L).sum()) for L in Ls}
            cum = {L: sum(stage_ms[l] for l in Ls if l <= L) for L in Ls}
            l_avg = sum(hist[str(L)] * cum[L] for L in Ls) / frames
            bl = batch_latency(_decode_fn(code, llr[:16384], 16384, 32, ps.PSCL_FASCL, pr, quant, o, st))
            out[f"{qn}{tag}_{snr}dB"] = dict(value=frames * code.K_info / ms / 1e3, unit="Mb/s", frames=frames,
                                             fer=float((o != info).any(dim=1).float().mean()), final_L_hist=hist,
                                             ms=ms, quant=qn, work="c2_2048_1723_L1_pruned" + tag,
                                        latency=dict(frame_avg_ms=l_avg, frame_worst_ms=worst,
                                                     stage_frame_ms={str(L): v for L, v in stage_ms.items()},
                                                     batch16k_p50_ms=bl["batch_p50_ms"],
                                                     batch16k_p99_ms=bl["batch_p99_ms"]))
            del info, llr, o, st
            torch.cuda.empty_cache()
    return out


C3_SNRS = (1.0, 1.5, 2.0, 2.5, 3.0)


def run_c3(gen, snrs=C3_SNRS, frames=2000000):
    """CA-SCL (1024, 512 incl. CRC-16), L = 8: pruned vs unpruned, int16 and
    f32, 2x10^6 frames per point; "pruned_n64": nodes of 64 or more leaves
    only."""
    import torch
    from paper_1710_08314_gb300 import pruning
    from paper_1710_08314_gb300 import autotune
    d, code = _code("c3_1024_512_L8")
    out = {}
    variants = [("f32", 0, "unpruned", None), ("f32", 0, "pruned", pruning(15, rep_max=0)),
                ("f32", 0, "pruned_n64", pruning(15, rep_max=0, node_min=33)),
                ("i16", 1, "unpruned", None), ("i16", 1, "pruned", pruning(15, rep_max=0)),
                ("i16", 1, "pruned_n64", pruning(15, rep_max=0, node_min=33))]
    tuned = set()
    for snr in snrs:
        info, llr = _gen_frames(code, frames, snr, gen)
        o = torch.empty_like(info)
        st = torch.empty((frames,), dtype=torch.int32, device="cuda")
        for qn, quant, pn, pr in variants:
            if (qn, pn) not in tuned:
                autotune.tuned(code, 8, quant, llr[:16384].contiguous(), prune=pr)
                tuned.add((qn, pn))
            fn = _decode_fn(code, llr, frames, 8, 1, pr, quant, o, st)
            ms = _timed(fn, reps=2)
            e = dict(value=frames * code.K_info / ms / 1e3, unit="Mb/s", frames=frames, snr_db=snr,
                     fer=float((o != info).any(dim=1).float().mean()), ms=ms, quant=qn,
                     work="c3_1024_512_L8_L8_" + pn)
            if snr == 2.0:
                lat = batch_latency(_decode_fn(code, llr[:16384], 16384, 8, 1, pr, quant, o, st))
                lat["frame_ms"] = frame_latency(code, llr[:1], 8, 1, pr, quant)
                e["latency"] = lat
            out[f"{qn}_{pn}_{snr}dB"] = e
        del info, llr, o, st
        torch.cuda.empty_cache()
    return out


def run_lsweep(gen, snrs=(1.5, 2.0, 2.5), frames=32768):
    """List-size sweep on the (2048, 1024 incl. CRC-32) code (Sec. III-B-1,
    Fig. 3): throughput, FER and single-frame latency for L = 1 ... 32, tree
    pruned (CA-SSCL, R0/R1/REP/SPC4 as the figure) and unpruned; L = 1 is SC."""
    import torch
    from paper_1710_08314_gb300 import pruning, polarscl as ps
    d, code = _code("ls_2048_1024")
    out = {}
    for snr in snrs:
        info, llr = _gen_frames(code, frames, snr, gen)
        o = torch.empty_like(info)
        st = torch.empty((frames,), dtype=torch.int32, device="cuda")
        for pn, pr in [("pruned", pruning(15, rep_max=0)), ("unpruned", None)]:
            for L in (1, 2, 4, 8, 16, 32):
                algo = ps.PSCL_SC if L == 1 else ps.PSCL_CASCL
                fn = _decode_fn(code, llr, frames, L, algo, pr, 0, o, st)
                ms = _timed(fn, reps=3)
                e = dict(value=frames * code.K_info / ms / 1e3, unit="Mb/s", frames=frames, ms=ms, quant="f32",
                         fer=float((o != info).any(dim=1).float().mean()), work=f"ls_2048_1024_L{L}_{pn}")
                if snr == 2.0:
                    e["latency"] = dict(frame_ms=frame_latency(code, llr[:1], L, algo, pr, 0))
                out[f"{pn}_L{L}_{snr}dB"] = e
        del info, llr, o, st
    return out


def run_c4(gen, total=500000, seed=7):
    """Uneven batch: 500,000 frames over 48 code contexts (N 128..2048, rate
    1/4..8/9, L 1..32, CRC-8/16/32, 0-20 % quasi-uniform puncturing, Eb/N0 per
    frame uniform in 0-5 dB), f32 and int8 contexts; persistent launch vs one
    launch per work item vs CUDA-graph replay."""
    import torch
    import synth
    from paper_1710_08314_gb300 import polarscl as ps
    from paper_1710_08314_gb300.polarscl import Batch
    names = json.load(open(os.path.join(ROOT, "tests", "golden", "codes", "uneven_index.json")))
    rng = np.random.default_rng(seed)
    counts = np.bincount(rng.integers(0, len(names), total), minlength=len(names))
    parts, refs = [], []
    for k, name in enumerate(names):
        d, code = _code(name)
        n = int(counts[k])
        ebn0 = torch.from_numpy(rng.uniform(0.0, 5.0, n)).cuda()
        rate = code.K_info / (code.N - code.P)
        sig = torch.sqrt(1.0 / (2.0 * rate * torch.pow(10.0, ebn0 / 10.0))).float()
        info, llr = _gen_frames(code, n, None, gen, sigma_per_frame=sig)
        quant = ps.PSCL_I8 if k % 2 else ps.PSCL_F32
        parts.append(dict(code=code, llr=llr, L=d["L"], algo=ps.PSCL_CASCL, quant=quant))
        refs.append(info)
    b = Batch(parts)
    n_launch, n_tasks, scratch = ps.pscl_batch_info(b.handle)
    ms_p = _timed(b.run)
    res_p = b.info_pool.clone()
    ms_plain = _timed(b.run_plain)
    same = bool(torch.equal(res_p, b.info_pool))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run()
    ms_g = _timed(graph.replay)
    same_g = bool(torch.equal(res_p, b.info_pool))
    lat = batch_latency(graph.replay, reps=10)
    bits = sum(int(r.shape[0]) * p["code"].K_info for r, p in zip(refs, parts))
    errs = 0
    for i, r in enumerate(refs):
        info, _ = b.outputs(i)
        errs += int((info != r).any(dim=1).sum())
    b.close()
    return dict(frames=total, contexts=len(names), launches=n_launch, tasks=n_tasks,
                persistent=dict(value=bits / ms_p / 1e3, unit="Mb/s", ms=ms_p, frames_per_s=total / ms_p * 1e3),
                plain_per_item=dict(value=bits / ms_plain / 1e3, unit="Mb/s", ms=ms_plain,
                                    launches=len(parts)),
                graph_replay=dict(value=bits / ms_g / 1e3, unit="Mb/s", ms=ms_g),
                speedup_vs_plain=ms_plain / ms_p, identical_outputs=same and same_g, fer=errs / total,
                latency=lat)


def run_c5(rates=(10e3, 50e3, 200e3, 1e6, 2e6, 4e6, 8e6), seconds=2.0, seed=11):
    """Serving: Poisson arrivals of requests (1..256 frames) over five MCS
    contexts; latency from arrival to observed completion, p50/p99.  The
    offered rate grows until the loop no longer keeps up (achieved below 90 %
    of offered), which shows where p99 breaks."""
    import time as _t
    import torch
    import synth
    from paper_1710_08314_gb300.polarscl import Server
    names = ["mcs_128_40", "mcs_256_128", "mcs_512_256", "mcs_1024_512", "mcs_2048_1723"]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    ctxs, pools = [], []
    R = 1024
    for name in names:
        d, code = _code(name)
        _, llr = _gen_frames(code, 256 * 8, d["ebn0_db"], gen)
        ctxs.append((code, d["L"], None))
        pools.append((code, llr))
    outs = [(torch.empty((R, 256, c.nbytes), dtype=torch.uint8, device="cuda"),
             torch.empty((R, 256), dtype=torch.int32, device="cuda")) for c, _ in pools]
    torch.cuda.synchronize()
    res = {}
    rng = np.random.default_rng(seed)
    srv = Server(ctxs, ring_slots=R, max_frames=256, idle_timeout_ms=5000)
    try:
        for rate in rates:
            mean_req = 128.5
            req_rate = rate / mean_req
            n_req = max(20, int(req_rate * seconds))
            gaps = rng.exponential(1.0 / req_rate, n_req)
            ctx = rng.integers(0, len(names), n_req)
            sizes = rng.integers(1, 257, n_req)
            arrive = {}
            lat = []
            frames_done = 0
            t0 = _t.monotonic_ns()
            sched = t0 + np.cumsum(gaps * 1e9).astype(np.int64)
            i = 0
            pending = 0
            deadline = t0 + int((seconds + 30) * 1e9)
            while (i < n_req or pending) and _t.monotonic_ns() < deadline:
                now = _t.monotonic_ns()
                while i < n_req and sched[i] <= now:
                    k, n = int(ctx[i]), int(sizes[i])
                    code, llr = pools[k]
                    off = (i * 256) % (llr.shape[0] - 256)
                    slot = i % R
                    tk = srv.submit(k, llr[off:off + n], outs[k][0][slot, :n], outs[k][1][slot, :n])
                    if tk is None:
                        break  # full: deferred (arrival time kept)
                    arrive[tk] = (int(sched[i]), n)
                    i += 1
                    pending += 1
                for c in srv.poll():
                    a, n = arrive.pop(c.ticket)
                    lat.append((c.t_done_ns - a) / 1e6)
                    frames_done += n
                    pending -= 1
            wall = (_t.monotonic_ns() - t0) / 1e9
            log(f"serving rate {rate:.0f}: {len(lat)}/{n_req} requests, {pending} pending, {wall:.1f} s, "
                f"status {srv.status()}")
            if pending or i < n_req:
                res["stalled"] = dict(rate=rate, pending=pending, unsubmitted=n_req - i)
            lat.sort()
            res[f"{int(rate)}"] = dict(offered_frames_per_s=rate, achieved_frames_per_s=frames_done / wall,
                                       requests=len(lat), p50_ms=lat[len(lat) // 2] if lat else None,
                                       p99_ms=lat[int(len(lat) * 0.99)] if lat else None,
                                       max_ms=lat[-1] if lat else None)
            if "stalled" in res:
                break
            if frames_done / wall < 0.9 * rate:
                res["saturation"] = dict(offered_frames_per_s=rate, achieved_frames_per_s=frames_done / wall)
                break
    finally:
        try:
            srv.stop()
        except Exception as e:  # the device loop did not leave: report, do not wait on it
            res["stop_error"] = repr(e)
    return res


def _c5_child(q):
    try:
        import torch
        torch.cuda.set_device(0)
        q.put(run_c5())
    except Exception as e:  # report to the parent
        q.put({"error": repr(e)})


def run_c5_isolated(timeout_s=300.0):
    """The serving workload in a child process of its own: a serving loop
    that did not stop would otherwise hold up the whole benchmark (a device
    context cannot be torn down under a running kernel); the child is
    stopped after timeout_s and the headline line is still printed."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_c5_child, args=(q,))
    p.start()
    try:
        res = q.get(timeout=timeout_s)
    except Exception:
        res = {"error": f"serving workload did not finish within {timeout_s:.0f} s"}
    p.join(timeout=30)
    if p.is_alive():
        p.kill()
        p.join(timeout=30)
    return res


PROFILE = os.path.join(ROOT, "profiles", "scl_kernel_f32_cascl_2048_1723_L32_unpruned.md")
# bytes an on-chip f/g update moves: two operands read, one result written
BYTES_PER_UPDATE = {"f32": 12, "i16": 6, "i8": 3}


def profile_figures() -> dict:
    """Per-frame DRAM bytes and warp instructions of the headline decode,
    from the ncu capture summarised in profiles/, or {} when the kernel
    sources changed since that capture."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1710_08314_gb300", "csrc")
    try:
        txt = open(PROFILE).read()
        sha = txt.split("kernel_sources_sha1:")[1].split()[0]
        h = hashlib.sha1()
        for f in ("scl_kernel.cuh", "internal.h", "api.cu"):
            h.update(open(os.path.join(csrc, f), "rb").read())
        if h.hexdigest()[:16] != sha:
            return {}
        out = {"dram_bytes_per_frame": int(txt.split("dram_bytes_per_frame:")[1].split()[0])}
        if "warp_instructions_per_frame:" in txt:
            out["warp_instructions_per_frame"] = int(txt.split("warp_instructions_per_frame:")[1].split()[0])
        return out
    except (OSError, IndexError, ValueError):
        return {}


def profiled_traffic(frames: int):
    """DRAM bytes of one decode launch of `frames` frames (scratch traffic
    grows with the frame count), or None when the profile is stale."""
    per = profile_figures().get("dram_bytes_per_frame")
    return per * frames if per else None


def roofline_models(fg_per_frame, frames, seconds, quant, mhz, sms, hbm_gbs=None, prof=None):
    """Every roofline the decoder could meet, for `frames` frames decoded in
    `seconds` at `mhz` sampled SM clock:
      smem  -- on-chip operand traffic of the algorithmic f/g updates (two
               reads and a write per update) vs 128 B/clk per SM;
      alu   -- f/g updates vs one per FP32 lane per clock;
      issue -- warp instructions (ncu, per frame) vs 4 per SM per clock;
      dram  -- measured DRAM traffic (ncu, per frame) vs the measured HBM copy
               bandwidth.  The last two only with a current profile."""
    upd = fg_per_frame * frames / seconds
    smem_peak = 128 * sms * mhz * 1e6 / 1e9
    smem = upd * BYTES_PER_UPDATE[quant] / 1e9
    alu_peak = sms * 128 * mhz * 1e6 / 1e9
    out = {"smem": {"achieved": smem, "peak": smem_peak, "unit": "GB/s", "frac": smem / smem_peak},
           "alu": {"achieved": upd / 1e9, "peak": alu_peak, "unit": "Gop/s", "frac": upd / 1e9 / alu_peak}}
    prof = prof or {}
    if prof.get("warp_instructions_per_frame"):
        ips = prof["warp_instructions_per_frame"] * frames / seconds / 1e9
        peak = sms * 4 * mhz * 1e6 / 1e9
        out["issue"] = {"achieved": ips, "peak": peak, "unit": "G warp-instr/s", "frac": ips / peak}
    if prof.get("dram_bytes_per_frame") and hbm_gbs:
        gbs = prof["dram_bytes_per_frame"] * frames / seconds / 1e9
        out["dram"] = {"achieved": gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": gbs / hbm_gbs,
                       "note": "scratch traffic measured by ncu, not algorithmic bytes"}
    return out


def add_workload_rooflines(wl, mhz, sms=None):
    """On-chip (shared-memory model) and ALU roofline fractions for every
    throughput workload entry that names its oracle work count ("work": f/g
    updates per frame of that code, list size and pruning; the adaptive one
    counts its L = 1 stage only, a lower bound) and its number format."""
    path = os.path.join(ROOT, "tests", "golden", "work_per_frame.json")
    if not mhz or not os.path.exists(path):
        return
    work = json.load(open(path))
    if sms is None:
        import torch
        sms = torch.cuda.get_device_properties(0).multi_processor_count

    def visit(entry):
        if not isinstance(entry, dict):
            return
        if "ms" in entry and entry.get("work") in work and "frames" in entry:
            m = roofline_models(work[entry["work"]]["fg_elems"], entry["frames"], entry["ms"] / 1e3,
                                entry.get("quant", "f32"), mhz, sms)
            entry["roofline"] = dict(bound="smem", **m["smem"], models=m)
            return
        for v in entry.values():
            visit(v)

    visit(wl)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fer_at(code, L, pr, snr, frames, gen, chunk=1 << 20):
    """Frame error rate and decode time (CA-SCL, f32) over `frames` frames."""
    import torch
    from paper_1710_08314_gb300 import polarscl as ps
    errs = done = 0
    ms = 0.0
    while done < frames:
        n = min(chunk, frames - done)
        info, llr = _gen_frames(code, n, snr, gen)
        o = torch.empty_like(info)
        st = torch.empty((n,), dtype=torch.int32, device="cuda")
        ms += _timed(_decode_fn(code, llr, n, L, ps.PSCL_CASCL, pr, 0, o, st), reps=1)
        errs += int((o != info).any(dim=1).sum())
        done += n
        del info, llr, o, st
    return errs / frames, ms, errs


def snr_at_fer(points, target):
    """Eb/N0 where log10(FER) crosses log10(target), interpolated linearly
    between the two measured points around it (None if not bracketed)."""
    import math
    pts = sorted(points)
    for (s0, f0), (s1, f1) in zip(pts, pts[1:]):
        if f0 >= target > f1 and f0 > 0:
            if f1 <= 0:
                return s1
            a, b = math.log10(f0), math.log10(f1)
            return s0 + (math.log10(target) - a) / (b - a) * (s1 - s0)
    return None


def run_study(name):
    """--study spc4plus: SPC4 vs SPC4+ nodes (Sec. III-B-2, Table 2): for each
    code of the study, list size 8 and 32, the Eb/N0 at which CA-SSCL reaches
    FER 1e-4 and the throughput, with SPC nodes limited to size 4 and
    unlimited.  --study lsweep: the list-size sweep at more SNR points."""
    import torch
    from paper_1710_08314_gb300 import pruning
    torch.cuda.set_device(0)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2024)
    out = {"study": name}
    if name == "lsweep":
        out["results"] = run_lsweep(gen, snrs=(1.0, 1.5, 2.0, 2.5, 3.0), frames=1 << 18)
        print(json.dumps(out), flush=True)
        return
    target, fine = 1e-4, 1_000_000
    res = {}
    for n in (256, 1024, 4096):
        for rn in ("13", "12", "23"):
            cname = f"spc_{n}_r{rn}"
            try:
                d, code = _code(cname)
            except Exception as e:  # the code length is beyond the kernels
                res[cname] = {"error": repr(e)}
                continue
            for L in (8, 32):
                row = {}
                for tag, spc_max in (("spc4", 4), ("spc4plus", 0)):
                    pr = pruning(15, rep_max=0, spc_max=spc_max)
                    # coarse search for the waterfall, then fine points
                    s, pts = 0.0, []
                    while s <= 6.0:
                        f, _, _ = fer_at(code, L, pr, s, 20000, gen)
                        if f < 3e-2:
                            break
                        s += 0.5
                    s0 = max(0.0, s - 0.5)
                    while s0 <= 7.0:
                        f, ms, e = fer_at(code, L, pr, s0, fine, gen)
                        pts.append((s0, f))
                        if f < target / 2 or e == 0:
                            break
                        s0 += 0.25
                    _, ms_last, _ = fer_at(code, L, pr, pts[-1][0], 1 << 20, gen)
                    row[tag] = {"snr_at_fer_1e-4": snr_at_fer(pts, target), "points": pts,
                                "throughput_mbps": (1 << 20) * code.K_info / ms_last / 1e3,
                                "throughput_snr_db": pts[-1][0]}
                a, b = row["spc4"], row["spc4plus"]
                if a["snr_at_fer_1e-4"] is not None and b["snr_at_fer_1e-4"] is not None:
                    row["snr_loss_db"] = b["snr_at_fer_1e-4"] - a["snr_at_fer_1e-4"]
                row["throughput_gain_pct"] = 100.0 * (b["throughput_mbps"] / a["throughput_mbps"] - 1.0)
                res[f"{cname}_L{L}"] = row
                log(f"{cname} L={L}: {row.get('snr_loss_db')} dB, {row['throughput_gain_pct']:.1f} %")
    out["results"] = res
    print(json.dumps(out), flush=True)


def headline_inputs(code, B, ebn0_db, gen):
    """B frames at ebn0_db: random bits -> library encoder -> channel, on the device."""
    import torch
    import synth
    info_in = torch.randint(0, 256, (B, code.nbytes), generator=gen, device="cuda", dtype=torch.uint8)
    if code.K_info % 8:
        info_in[:, -1] &= (0xFF << (8 - code.K_info % 8)) & 0xFF
    x = code.encode(info_in)
    llr = synth.torch_bpsk_awgn_llr(x, synth.sigma_for(ebn0_db, code.K_info / (code.N - code.P)), gen)
    return info_in, llr


def timed_steps(step, steps, stream, dist=None):
    """Device time of each of `steps` steps (CUDA events on the launching
    stream, synchronised and barriered on both sides)."""
    import torch
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for s in range(steps):
        step()
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return [ev[s].elapsed_time(ev[s + 1]) for s in range(steps)], ev[0].elapsed_time(ev[-1])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--quant", default="f32", choices=list(QUANT))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true", help="skip the further workloads")
    ap.add_argument("--study", choices=["spc4plus", "lsweep"], help="run one study instead (one JSON line)")
    ap.add_argument("--algo", default="cascl", choices=list(ALGO_NAMES),
                    help="decode of the timed step (default: the metric's CA-SCL)")
    ap.add_argument("--pruned", action="store_true", help="R0/R1/REP/SPC4 tree pruning in the timed step")
    ap.add_argument("--node-min", type=int, default=0, help="with --pruned: smallest pruned node (leaves)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    if args.study:
        return run_study(args.study)

    ws, rank, local = dist_env()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        log("oracle CPU baseline")
        cpu = cpu_oracle_rate(seconds=20.0, seed=99)  # before any CUDA use
        log("oracle CPU baseline done")

    import torch

    import synth
    from paper_1710_08314_gb300 import Code, polarscl as ps

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    d = synth.load_code(WORKLOAD)
    code = Code(d["frozen"], d["crc_len"], d["crc_poly"], d["punct"], d["systematic"])
    B, K_info = args.batch, code.K_info
    quant = QUANT[args.quant]
    from paper_1710_08314_gb300 import pruning as _pruning
    ALGO = {"cascl": ALGO_CASCL, "sc": 0, "fascl": 3}[args.algo]
    PRUNE = _pruning(15, rep_max=8 if args.quant == "i8" else 0, node_min=args.node_min) if args.pruned else None
    # synthetic inputs (resident in HBM): bits -> library encoder -> channel
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234 + rank)
    info_in, llr = headline_inputs(code, B, EBN0_DB, gen)
    info_out = torch.empty((B, code.nbytes), dtype=torch.uint8, device="cuda")
    status = torch.empty((B,), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    # schedule knobs from the autotuner (cached per GPU model and code)
    from paper_1710_08314_gb300 import autotune
    log("headline: tuning")
    # one-path and adaptive decodes start with 32 frames per warp: their
    # sample covers two waves of those
    sample = llr[:8192] if args.algo == "cascl" else llr[:1 << 18]
    tuning, measured = autotune.tuned(code, L_LIST, quant, sample.contiguous(), prune=PRUNE, algo=ALGO)
    log(f"headline: tuned {tuning}, timing")
    cur = {"llr": llr}

    def step():
        ps.pscl_decode(code.handle, cur["llr"], B, L_LIST, ALGO, PRUNE, quant, info_out, status, None, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches_per_step = ps.pscl_debug_last_launches()

    # device-timed region
    with ClockSampler(local) as clk:
        per_launch_ms, total_ms = timed_steps(step, args.steps, stream, dist)
    total_ms = max_over_ranks(total_ms)
    ms_per_step = total_ms / args.steps
    frames_all = B * args.steps * ws
    value = frames_all * K_info / (total_ms / 1e3) / 1e6

    # correctness of what was timed: frame errors vs the transmitted bits
    fer = float((info_out != info_in).any(dim=1).float().mean().item())
    crc_fail = float(((status & 1) == 0).float().mean().item())

    # the same decode at 3.5 dB (the low end of the workload's SNR range)
    log("headline at 3.5 dB")
    info35, llr35 = headline_inputs(code, B, 3.5, gen)
    cur["llr"] = llr35
    for _ in range(args.warmup):
        step()
    per35, tot35 = timed_steps(step, args.steps, stream, dist)
    tot35 = max_over_ranks(tot35)
    at35 = {"value": frames_all * K_info / (tot35 / 1e3) / 1e6, "unit": "Mb/s", "ms_per_step": tot35 / args.steps,
            "fer": float((info_out != info35).any(dim=1).float().mean().item()),
            "batch_p50_ms": pct(per35, 0.5), "batch_p99_ms": pct(per35, 0.99)}
    cur["llr"] = llr
    del info35, llr35

    # end to end through the C ABI's host-buffer decode: page-locked host LLRs
    # in, host bits and status out (copies overlapped with the decodes)
    llr_h = llr.cpu().pin_memory()
    info_h = torch.empty((B, code.nbytes), dtype=torch.uint8).pin_memory()
    status_h = torch.empty((B,), dtype=torch.int32).pin_memory()

    log("headline: end to end through host buffers")

    def e2e_step():
        ps.pscl_decode_host(code.handle, llr_h, B, L_LIST, ALGO, PRUNE, quant, info_h, status_h, stream)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    _, e2e_ms = timed_steps(e2e_step, args.steps, stream, dist)
    e2e_value = frames_all * K_info / (max_over_ranks(e2e_ms) / 1e3) / 1e6
    frame_ms = frame_latency(code, llr[:1], L_LIST, ALGO, PRUNE, quant)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # rooflines of the decode kernel: algorithmic f/g updates per frame (the
    # oracle's count for this code and L) over the measured launch time
    wpath = os.path.join(ROOT, "tests", "golden", "work_per_frame.json")
    wkey = f"{WORKLOAD}_L{1 if args.algo == 'sc' else L_LIST}_{'pruned' if args.pruned else 'unpruned'}"
    work = json.load(open(wpath)).get(wkey) if os.path.exists(wpath) and args.algo != "fascl" else None
    clocks = clk.summary()
    peaks = measured_peaks()
    avg_launch_s = (sum(per_launch_ms) / len(per_launch_ms)) / 1e3 / max(1, launches_per_step)
    roof = None
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = clocks.get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1440.0
    if work:
        prof = profile_figures() if args.quant == "f32" and B >= 4096 and args.algo == "cascl" \
            and not args.pruned else {}
        models = roofline_models(work["fg_elems"], B, avg_launch_s, args.quant, mhz, sms, peaks.get("hbm_gbs"), prof)
        sm = models["smem"]
        roof = {"bound": "smem", "achieved": sm["achieved"], "peak": sm["peak"], "unit": "GB/s", "frac": sm["frac"],
                "traffic": prof["dram_bytes_per_frame"] * B if prof.get("dram_bytes_per_frame") else None,
                "note": (f"on-chip operand bytes of the algorithmic f/g updates ({work['fg_elems']} per frame, "
                         f"{BYTES_PER_UPDATE[args.quant]} B each) vs 128 B/clk/SM ({sms} SMs x {mhz:.0f} MHz "
                         f"sampled); traffic = DRAM bytes per launch from the ncu profile"),
                "models": models}
    line = {
        "metric": "info Mb/s per GB300 (CA-SCL N=2048 K=1723 L=32) bit-exact",
        "value": value, "unit": "Mb/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.quant, "data": "synthetic",
        "config": headline_config(args.quant, B, ws, args.algo, args.pruned, args.node_min),
        "e2e": {"value": e2e_value, "unit": "Mb/s", "h2d_bytes_per_step": int(llr.numel() * 4),
                "d2h_bytes_per_step": int(info_out.numel() + status.numel() * 4)},
        "gpu_launches": launches_per_step * args.steps,
        "tuning": {"warps_per_sm": tuning[0], "fuse_leaves": tuning[1], "warps_per_block": tuning[2],
                   "resident_warps": tuning[3] or tuning[0], "measured_now": measured},
        "roofline": roof,
        "clocks": clocks,
        "fer": fer, "crc_fail_rate": crc_fail,
        "A_bits_per_s_Mb": value * (K_info + code.crc_len) / K_info,
        "at_3_5dB": at35,
        "latency": {"frame_ms": frame_ms, "batch_p50_ms": pct(per_launch_ms, 0.5),
                    "batch_p99_ms": pct(per_launch_ms, 0.99), "batch_frames": B},
    }
    if cpu:
        line["cpu_baseline"] = {"value": cpu[0], "unit": "Mb/s", "cores": cpu[1], "kind": "oracle",
                                "sample": cpu[2], "single_thread": cpu[3]}
    if not args.headline_only:
        del llr, llr_h
        torch.cuda.empty_cache()
        g2 = torch.Generator(device="cuda")
        g2.manual_seed(77)
        wl = {}
        for key, fn in [("c1_cascl_128_64_L4", run_c1), ("c3_1024_512_L8", run_c3), ("c2_fa_2048_1723", run_c2),
                        ("l_sweep_2048_1024", run_lsweep), ("c4_uneven_500k", run_c4)]:
            log(f"workload {key}")
            try:
                wl[key] = fn(g2)
            except Exception as e:  # report, do not hide the headline
                wl[key] = {"error": repr(e)}
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        log("workload c5_serving")
        wl["c5_serving"] = run_c5_isolated()
        try:
            add_workload_rooflines(wl, mhz, sms)
        except Exception as e:
            log(f"workload rooflines: {e!r}")
        line["workloads"] = wl
        srv = wl.get("c5_serving", {})
        p99 = [v.get("p99_ms") for k, v in srv.items() if isinstance(v, dict) and k.isdigit()
               and v.get("p99_ms") is not None and v.get("achieved_frames_per_s", 0) >= 0.9 * v["offered_frames_per_s"]]
        line["p99_latency_ms_mixed_load"] = max(p99) if p99 else None
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
