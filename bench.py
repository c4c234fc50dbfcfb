"""Benchmark: batched CA-SCL decoding of the (2048, 1723 incl. CRC-32) polar
code with L = 32 on one GB300 (info Mb/s), plus the end-to-end rate through
the C ABI with host buffers, the roofline of the decode kernel and the CPU
oracle's rate on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step decodes one batch of B frames (LLR ingest and quantisation, f/g
updates, partial sums, path metrics, top-L selection, lazy path copy, CRC
check and info-bit extraction: the whole hot path).  Inputs are synthetic:
uniform info bits, systematic encoding, BPSK over AWGN at 4.5 dB.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c2_2048_1723"
EBN0_DB = 4.5
L_LIST = 32
BATCH = 16384            # frames per step: 134 MB of LLRs, larger than L2
ALGO_CASCL = 1
QUANT = {"f32": 0, "i16": 1, "i8": 2}


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
    oracle.decode_batch(code, np.asarray(llr_rows, dtype=np.float64), L, oracle.CASCL, None, oracle.F32,
                        want_pm=False)
    return time.perf_counter() - t0, len(llr_rows)


def cpu_oracle_rate(n_frames_target, seed=99, max_seconds=25.0):
    """Info Mb/s of the oracle over a bounded sample of the workload, frames
    split across all host cores.  Returns (value, cores, sample description)."""
    import multiprocessing as mp

    import numpy as np
    import oracle
    import synth
    d = synth.load_code(WORKLOAD)
    cores = len(os.sched_getaffinity(0))
    code = oracle.Code(d["frozen"], d["crc_len"], d["crc_poly"], d["punct"], d["systematic"])
    # calibrate on one frame, then size the sample to ~max_seconds of work
    info = synth.info_bits(1, code.K_info, seed)
    x = oracle.encode(code, info)
    llr = synth.bpsk_awgn_llr(x, synth.sigma_for(EBN0_DB, code.K_info / code.N), seed + 1)
    t0 = time.perf_counter()
    oracle.decode_batch(code, llr.astype(np.float64), L_LIST, oracle.CASCL, None, oracle.F32, want_pm=False)
    per = time.perf_counter() - t0
    n = int(max(cores, min(n_frames_target, cores * max(1, int(max_seconds / max(per, 1e-3))))))
    info = synth.info_bits(n, code.K_info, seed + 2)
    x = oracle.encode(code, info)
    llr = synth.bpsk_awgn_llr(x, synth.sigma_for(EBN0_DB, code.K_info / code.N), seed + 3)
    chunks = [llr[i::cores].tolist() for i in range(cores)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(WORKLOAD, ch, L_LIST) for ch in chunks if ch])
    wall = time.perf_counter() - t0
    frames = sum(r[1] for r in res)
    value = frames * code.K_info / wall / 1e6
    sample = (f"{frames} frames of the same workload ((2048,1723) CA-SCL L=32 f32, {EBN0_DB} dB), "
              f"split over {cores} spawned processes; wall {wall:.1f} s incl. process start")
    return value, cores, sample


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    per_step = []
    cpu = None
    for s in range(args.warmup + args.steps):
        v, cores, sample = cpu_oracle_rate(n_frames_target=16, seed=1000 + s, max_seconds=6.0)
        if s >= args.warmup:
            per_step.append(v)
            cpu = (v, cores, sample)
    value = sum(per_step) / len(per_step)
    line = {
        "impl": "reference", "metric": "info Mb/s per GB300 (CA-SCL N=2048 K=1723 L=32) bit-exact",
        "value": value, "unit": "Mb/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "CA-SCL (2048,1723 incl. CRC-32) L=32 f32 unpruned, BPSK-AWGN 4.5 dB",
                   "note": "the CPU oracle (plain C, list copies) on the host cores; each step a bounded sample"},
        "cpu_baseline": {"value": value, "unit": "Mb/s", "cores": cpu[1], "kind": "oracle", "sample": cpu[2]},
        "e2e": {"value": value, "unit": "Mb/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

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


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--quant", default="f32", choices=list(QUANT))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)

    ws, rank, local = dist_env()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(n_frames_target=64, seed=99, max_seconds=20.0)  # before any CUDA use

    import numpy as np
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
    B, N, K_info = args.batch, code.N, code.K_info
    quant = QUANT[args.quant]
    # synthetic inputs (resident in HBM): bits -> library encoder -> channel
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234 + rank)
    info_in = torch.randint(0, 256, (B, code.nbytes), generator=gen, device="cuda", dtype=torch.uint8)
    if K_info % 8:
        info_in[:, -1] &= (0xFF << (8 - K_info % 8)) & 0xFF
    x = code.encode(info_in)
    sigma = synth.sigma_for(EBN0_DB, K_info / (N - code.P))
    llr = synth.torch_bpsk_awgn_llr(x, sigma, gen)
    del x
    info_out = torch.empty((B, code.nbytes), dtype=torch.uint8, device="cuda")
    status = torch.empty((B,), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        ps.pscl_decode(code.handle, llr, B, L_LIST, ALGO_CASCL, None, quant, info_out, status, None, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches_per_step = ps.pscl_debug_last_launches()

    # device-timed region
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for s in range(args.steps):
            step()
            ev[s + 1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    per_launch_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    t = torch.tensor([total_ms], device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    frames_all = B * args.steps * ws
    value = frames_all * K_info / (total_ms / 1e3) / 1e6

    # correctness of what was timed: frame errors vs the transmitted bits
    fer = float((info_out != info_in).any(dim=1).float().mean().item())
    crc_fail = float(((status & 1) == 0).float().mean().item())

    # end to end through the C ABI: pinned host LLRs -> device -> decode -> host bits
    llr_h = llr.cpu().pin_memory()
    info_h = torch.empty((B, code.nbytes), dtype=torch.uint8).pin_memory()
    status_h = torch.empty((B,), dtype=torch.int32).pin_memory()
    llr_d = torch.empty_like(llr)

    def e2e_step():
        llr_d.copy_(llr_h, non_blocking=True)
        ps.pscl_decode(code.handle, llr_d, B, L_LIST, ALGO_CASCL, None, quant, info_out, status, None, stream)
        info_h.copy_(info_out, non_blocking=True)
        status_h.copy_(status, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    te = torch.tensor([e0.elapsed_time(e1)], device="cuda")
    if dist:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = frames_all * K_info / (float(te.item()) / 1e3) / 1e6

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the decode kernel: algorithmic element updates per frame
    # (f/g LLR updates, counted by the oracle for this code and L) / kernel time
    work = json.load(open(os.path.join(ROOT, "tests", "golden", "work_per_frame.json"))).get(
        f"{WORKLOAD}_L{L_LIST}_unpruned", None) if os.path.exists(
        os.path.join(ROOT, "tests", "golden", "work_per_frame.json")) else None
    clocks = clk.summary()
    peaks = measured_peaks()
    avg_launch_s = (sum(per_launch_ms) / len(per_launch_ms)) / 1e3 / max(1, launches_per_step)
    roof = None
    if work:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        mhz = clocks.get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1440.0
        peak_gops = sms * 128 * mhz * 1e6 / 1e9
        achieved = work["fg_elems"] * B / avg_launch_s / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_gops, "unit": "Gop/s",
                "frac": achieved / peak_gops, "traffic": None,
                "note": (f"f/g LLR updates ({work['fg_elems']} per frame) per second vs one update per "
                         f"FP32 lane per clock ({sms} SMs x 128 lanes x {mhz:.0f} MHz sampled)")}
    line = {
        "metric": "info Mb/s per GB300 (CA-SCL N=2048 K=1723 L=32) bit-exact",
        "value": value, "unit": "Mb/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.quant, "data": "synthetic",
        "config": {"workload": f"CA-SCL (2048,1723 incl. CRC-32) L=32 {args.quant} unpruned, BPSK-AWGN "
                               f"{EBN0_DB} dB, GA frozen set at 4.5 dB",
                   "frames_per_step": B, "l2": "inputs larger than L2 (134 MB LLRs per step)",
                   "parallelism": f"replicas x{ws}"},
        "e2e": {"value": e2e_value, "unit": "Mb/s", "h2d_bytes_per_step": int(llr.numel() * 4),
                "d2h_bytes_per_step": int(info_out.numel() + status.numel() * 4)},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
        "clocks": clocks,
        "fer": fer, "crc_fail_rate": crc_fail,
        "A_bits_per_s_Mb": value * (K_info + code.crc_len) / K_info,
    }
    if cpu:
        line["cpu_baseline"] = {"value": cpu[0], "unit": "Mb/s", "cores": cpu[1], "kind": "oracle",
                                "sample": cpu[2]}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
