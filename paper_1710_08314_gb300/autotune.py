"""Autotuner for the decoder's launch and schedule knobs, measured on the GPU.

For a code, list size, number format and pruning setting it times decodes of
a sample batch over a grid of
  - the warps per SM each warp's shared-memory slice is sized for (more
    warps hide more latency, fewer keep more LLR layers on chip; sizing for
    more warps than are resident leaves shared memory to the L1 cache), and
  - the largest unpruned subtree decoded in registers (node fusion),
with the register cap following the slice sizing; then, at the best fusion,
over the slice sizing with the other register cap (the resident warps), and
at the best of those over the warps per block (frames per block =
warps x 32/L: the granularity of shared-memory allocation and of block
scheduling).  It keeps the fastest, applies it to the code (pscl_code_tune)
and stores it in a JSON cache keyed by the GPU model and a digest of the
code, so later runs reuse it without measuring (PSCL_RETUNE=1 measures
again).  Results never depend on the tuning; only time.
"""
from __future__ import annotations

import hashlib
import json
import os
import threading

from . import polarscl as ps

DEFAULT_CACHE = os.environ.get(
    "PSCL_TUNE_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json"))
WARPS_GRID = (8, 12, 16, 20, 24, 28, 32, 40)
RESIDENT_LO, RESIDENT_HI = 16, 28
FUSE_GRID = (2, 4, 8)
BLOCK_GRID = (2, 4, 8)
_lock = threading.Lock()


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def code_digest(code) -> str:
    h = hashlib.sha1()
    h.update(bytes(code.frozen.tobytes()))
    if code.puncture is not None:
        h.update(bytes(code.puncture.tobytes()))
    h.update(f"{code.crc_len}".encode())
    return h.hexdigest()[:16]


def cache_key(code, L, quant, prune, algo=ps.PSCL_CASCL) -> str:
    pk = "none" if prune is None or prune.mask == 0 else (
        f"{prune.mask}-{prune.rep_max}-{prune.spc_max}-{prune.r1_t}-{prune.spc_t}-{prune.r1_max}"
        + (f"-m{prune.node_min}" if prune.node_min > 2 else ""))
    return f"{gpu_name()}|N{code.N}|K{code.K}|P{code.P}|{code_digest(code)}|L{L}|q{quant}|a{algo}|{pk}"


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
        fh.write("\n")
    os.replace(tmp, path)


def measure(code, llr, L, quant, prune=None, algo=ps.PSCL_CASCL, warps_grid=WARPS_GRID, fuse_grid=FUSE_GRID,
            block_grid=BLOCK_GRID, reps=3):
    """Time every (slice warps, fusion) pair on the sample LLRs with the
    register cap the slice sizing implies, then the slice sizings with the
    other register cap at the best fusion, then the warps per block at the
    best setting; returns the list of results (ms per decode) and the best."""
    import torch
    n = int(llr.shape[0])
    info = torch.empty((n, code.nbytes), dtype=torch.uint8, device=llr.device)
    status = torch.empty((n,), dtype=torch.int32, device=llr.device)
    results = []

    def run(w, f, b, r):
        ps.pscl_code_tune(code.handle, L, quant, w, f, prune, b, r)
        ps.pscl_prepare(code.handle, prune)
        ps.pscl_decode(code.handle, llr, n, L, algo, prune, quant, info, status, None, None)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ps.pscl_decode(code.handle, llr, n, L, algo, prune, quant, info, status, None, None)
        e1.record()
        torch.cuda.synchronize()
        results.append(dict(warps_per_sm=w, fuse=f, warps_per_block=b, resident_warps=r,
                            ms=e0.elapsed_time(e1) / reps))

    def auto(w):
        return RESIDENT_HI if w >= 24 else RESIDENT_LO

    for w in warps_grid:
        for f in fuse_grid:
            run(w, f, 4, auto(w))
    best = min(results, key=lambda r: r["ms"])
    other = RESIDENT_LO if best["resident_warps"] == RESIDENT_HI else RESIDENT_HI
    for w in warps_grid:
        run(w, best["fuse"], 4, other)
    best = min(results, key=lambda r: r["ms"])
    for b in block_grid:
        if b != 4:
            run(best["warps_per_sm"], best["fuse"], b, best["resident_warps"])
    best = min(results, key=lambda r: r["ms"])
    return results, best


def tuned(code, L, quant, llr_sample=None, prune=None, algo=ps.PSCL_CASCL, path: str = DEFAULT_CACHE,
          remeasure: bool = False):
    """Apply cached tuning for this (code, L, format, pruning) or measure it on
    llr_sample and cache it.  Returns the applied (warps_per_sm, fuse,
    warps_per_block, resident_warps) and whether it was measured now.  An
    adaptive or one-path decode runs all its stages with the entry of the
    list size it is called with, so it is tuned by timing whole decodes of
    that algorithm (the sample should fill the GPU at the first stage's 32
    frames per warp)."""
    key = cache_key(code, L, quant, prune, algo)
    with _lock:
        cache = load_cache(path)
    hit = cache.get(key)
    remeasure = remeasure or os.environ.get("PSCL_RETUNE", "0") == "1"
    if hit and not remeasure:
        wpb = hit.get("warps_per_block", 4)
        res = hit.get("resident_warps", 0)
        ps.pscl_code_tune(code.handle, L, quant, hit["warps_per_sm"], hit["fuse"], prune, wpb, res)
        ps.pscl_prepare(code.handle, prune)  # schedules for the tuned fusion size
        return (hit["warps_per_sm"], hit["fuse"], wpb, res), False
    if llr_sample is None:
        return None, False
    results, best = measure(code, llr_sample, L, quant, prune, algo)
    ps.pscl_code_tune(code.handle, L, quant, best["warps_per_sm"], best["fuse"], prune, best["warps_per_block"],
                      best["resident_warps"])
    ps.pscl_prepare(code.handle, prune)
    with _lock:
        cache = load_cache(path)
        cache[key] = dict(warps_per_sm=best["warps_per_sm"], fuse=best["fuse"],
                          warps_per_block=best["warps_per_block"], resident_warps=best["resident_warps"],
                          ms=best["ms"],
                          frames=int(llr_sample.shape[0]), grid=results)
        try:
            save_cache(cache, path)
        except OSError:
            pass
    return (best["warps_per_sm"], best["fuse"], best["warps_per_block"], best["resident_warps"]), True
