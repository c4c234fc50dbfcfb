"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module draws random numbers and applies the channel model the paper's
simulation chain uses (Sec. III: uniform source bits, BPSK 0 -> +1, 1 -> -1,
AWGN, channel LLR = 2y / sigma^2).  It holds none of the decoder's
arithmetic: no encoder, CRC, code construction, f/g/h, metric or selection.
Codewords are always produced by the caller (the oracle's encoder in tests,
the library's encoder in the benchmark) and handed in as bits.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CODES_DIR = os.path.join(os.path.dirname(HERE), "tests", "golden", "codes")


def sigma_for(ebn0_db: float, rate: float) -> float:
    """Noise standard deviation for BPSK at Eb/N0 (dB) and code rate R:
    sigma^2 = 1 / (2 R 10^(EbN0/10))."""
    return math.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0)))


def info_bits(n_frames: int, k_info: int, seed: int) -> np.ndarray:
    """Uniform random information bits, uint8 0/1, shape (n_frames, k_info)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(n_frames, k_info), dtype=np.uint8)


def bpsk_awgn_llr(x_bits: np.ndarray, sigma: float | np.ndarray, seed: int,
                  punct: np.ndarray | None = None) -> np.ndarray:
    """float32 channel LLRs of codewords x (uint8, shape (F, N)) sent with BPSK
    over AWGN; punctured positions are dropped (the receiver never sees them),
    so the result has shape (F, N - P).  sigma may be a scalar or per frame."""
    x = np.asarray(x_bits, dtype=np.uint8)
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(size=x.shape)
    sig = np.asarray(sigma, dtype=np.float64)
    if sig.ndim == 1:
        sig = sig[:, None]
    y = (1.0 - 2.0 * x.astype(np.float64)) + sig * noise
    llr = (2.0 * y / (sig * sig)).astype(np.float32)
    if punct is not None:
        keep = np.asarray(punct, dtype=np.uint8) == 0
        llr = llr[:, keep]
    return np.ascontiguousarray(llr)


def noiseless_llr(x_bits: np.ndarray, magnitude: float = 8.0, punct=None) -> np.ndarray:
    """LLRs of +-magnitude agreeing with x (no noise)."""
    x = np.asarray(x_bits, dtype=np.uint8)
    llr = np.where(x == 0, magnitude, -magnitude).astype(np.float32)
    if punct is not None:
        llr = llr[:, np.asarray(punct, dtype=np.uint8) == 0]
    return np.ascontiguousarray(llr)


def random_llr(n_frames: int, n: int, seed: int, scale: float = 3.0) -> np.ndarray:
    """Gaussian float32 LLRs that belong to no codeword (stress inputs)."""
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal(size=(n_frames, n))).astype(np.float32)


def random_int_llr(n_frames: int, n: int, seed: int, lo: int, hi: int) -> np.ndarray:
    """Integer-valued LLRs drawn uniformly from [lo, hi] (float64 array)."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(n_frames, n)).astype(np.float64)


def torch_bpsk_awgn_llr(x_bits, sigma, generator, punct_keep_idx=None):
    """Device-side twin of bpsk_awgn_llr for the benchmark (same channel model,
    torch's Philox generator).  x_bits: uint8 tensor (F, N); sigma: float or a
    float tensor (F,).  Returns float32 (F, N - P)."""
    import torch
    x = x_bits.to(torch.float32)
    noise = torch.randn(x.shape, generator=generator, device=x.device, dtype=torch.float32)
    if isinstance(sigma, torch.Tensor):
        sig = sigma.to(torch.float32).reshape(-1, 1)
    else:
        sig = torch.full((1, 1), float(sigma), device=x.device)
    y = (1.0 - 2.0 * x) + sig * noise
    llr = 2.0 * y / (sig * sig)
    if punct_keep_idx is not None:
        llr = llr.index_select(1, punct_keep_idx)
    return llr.contiguous()


# ---------------------------------------------------------------------------
# Workload definitions: the code parameters of each benchmark/test workload.
# Frozen sets are stored files written by tests/golden/make_codes.py.

CRC_POLYS = {0: 0, 8: 0x07, 16: 0x1021, 32: 0x04C11DB7}
# further generators, without their top bit: the 6-, 11- and 24-bit CRCs of
# the 5G NR channel coding (D^6+D^5+1, D^11+D^10+D^9+D^5+1, CRC24C)
CUSTOM_CRC_POLYS = {6: 0x21, 11: 0x621, 24: 0xB2B117}

WORKLOADS = {
    # plain CA-SCL, (128, 64 incl. CRC-8), L=4, fp32, unpruned, GA at 2.0 dB
    "c1_cascl_128_64_L4": dict(N=128, K=64, crc_len=8, L=4, design_db=2.0, ebn0_db=2.0, P=0),
    # CA-SCL (2048, 1723 incl. CRC-32), L=32; GA at 4.5 dB
    "c2_2048_1723": dict(N=2048, K=1723, crc_len=32, L=32, design_db=4.5, ebn0_db=4.5, P=0),
    # tree-pruned CA-SCL (1024, 512 incl. CRC-16), L=8
    "c3_1024_512_L8": dict(N=1024, K=512, crc_len=16, L=8, design_db=2.0, ebn0_db=2.0, P=0),
    # serving contexts (N, K, L), CRC-16 for N <= 512, CRC-32 above
    "mcs_128_40": dict(N=128, K=40, crc_len=16, L=8, design_db=2.0, ebn0_db=3.0, P=0),
    "mcs_256_128": dict(N=256, K=128, crc_len=16, L=8, design_db=2.0, ebn0_db=2.5, P=0),
    "mcs_512_256": dict(N=512, K=256, crc_len=16, L=16, design_db=2.0, ebn0_db=2.0, P=0),
    "mcs_1024_512": dict(N=1024, K=512, crc_len=32, L=16, design_db=2.0, ebn0_db=2.0, P=0),
    "mcs_2048_1723": dict(N=2048, K=1723, crc_len=32, L=32, design_db=4.5, ebn0_db=4.0, P=0),
    # list-size sweep (Sec. III-B-1, Fig. 3): (2048, 1024 incl. CRC-32), R = 1/2
    "ls_2048_1024": dict(N=2048, K=1024, crc_len=32, L=32, design_db=2.0, ebn0_db=2.0, P=0),
}

# SPC4+ on/off study (Sec. III-B-2, Table 2): N in {256, 1024, 4096}, rate
# K_info/N in {1/3, 1/2, 2/3}, list sizes 8 and 32; CRC-16 for N = 256 and
# CRC-32 above (the table names no CRC); GA at 2 dB.
for _n in (256, 1024, 4096):
    for _num, _den in ((1, 3), (1, 2), (2, 3)):
        _c = 16 if _n <= 256 else 32
        WORKLOADS[f"spc_{_n}_r{_num}{_den}"] = dict(N=_n, K=round(_n * _num / _den) + _c, crc_len=_c, L=32,
                                                   design_db=2.0, ebn0_db=2.0, P=0)
# custom CRC lengths (Sec. III-A: any CRC can be defined)
for _c in (6, 11, 24):
    WORKLOADS[f"crc{_c}_512_256"] = dict(N=512, K=256, crc_len=_c, L=8, design_db=2.0, ebn0_db=2.0, P=0,
                                        crc_poly=CUSTOM_CRC_POLYS[_c])
# a density-evolution frozen set (Sec. II-A, Tal-Vardy) for the (1024, 512) code
WORKLOADS["de_1024_512"] = dict(N=1024, K=512, crc_len=16, L=8, design_db=2.0, ebn0_db=2.0, P=0,
                                construction="de")
# large codes (Sec. IV-D, Fig. 7: R = 1/2, L = 8)
for _n in (4096, 8192):
    WORKLOADS[f"ln_{_n}_{_n // 2}"] = dict(N=_n, K=_n // 2, crc_len=32, L=8, design_db=2.0, ebn0_db=2.0, P=0)


def uneven_contexts(n_ctx: int = 48, seed: int = 7):
    """Code contexts of the uneven-batch workload: N in {128..2048},
    rate K_info/(N-P) in [1/4, 8/9], CRC-8/16/32, quasi-uniform puncturing of
    0-20 % of the bits, L in {1..32}, design Eb/N0 uniform in [0, 5] dB."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_ctx):
        N = int(rng.choice([128, 256, 512, 1024, 2048]))
        P = int(round(float(rng.uniform(0.0, 0.2)) * N))
        crc_len = int(rng.choice([8, 16, 32]))
        rate = float(rng.uniform(0.25, 8.0 / 9.0))
        k_info = max(1, int(round(rate * (N - P))))
        K = k_info + crc_len
        if K > N - P:
            K = N - P
            k_info = K - crc_len
        L = int(rng.choice([1, 2, 4, 8, 16, 32]))
        ebn0 = float(rng.uniform(0.0, 5.0))
        out.append(dict(name=f"u{i:02d}", N=N, K=K, crc_len=crc_len, L=L, design_db=ebn0,
                        ebn0_db=ebn0, P=P))
    return out


def load_code(name: str) -> dict:
    """A stored code: dict with N, K, crc_len, crc_poly, frozen (uint8 array),
    punct (uint8 array or None) and the workload fields."""
    with open(os.path.join(CODES_DIR, name + ".json")) as fh:
        d = json.load(fh)
    d["frozen"] = np.frombuffer(bytes.fromhex(d["frozen_hex"]), dtype=np.uint8).copy()
    d["punct"] = (np.frombuffer(bytes.fromhex(d["punct_hex"]), dtype=np.uint8).copy()
                  if d.get("punct_hex") else None)
    return d
