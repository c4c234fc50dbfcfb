"""Plain CPU oracle for polar SCL decoding -- TEST INFRASTRUCTURE ONLY.

Loads ``polar_oracle.c`` (compiled with gcc, ``-ffp-contract=off``) through
ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this package; the GPU library never does, and this
package never imports the GPU library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polar_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PRUNE_R0, PRUNE_R1, PRUNE_REP, PRUNE_SPC = 1, 2, 4, 8
NODE_INTERNAL, NODE_R0, NODE_R1, NODE_REP, NODE_SPC = 0, 1, 2, 3, 4
F32, I16, I8, IWIDE, EXACT = 0, 1, 2, 3, 4
SC, CASCL, PA, FA = 0, 1, 2, 3


class _Code(C.Structure):
    _fields_ = [("N", C.c_int), ("K", C.c_int), ("crc_len", C.c_int), ("crc_poly", C.c_uint32),
                ("systematic", C.c_int), ("frozen", C.c_void_p), ("punct", C.c_void_p)]


class _Pruning(C.Structure):
    _fields_ = [("mask", C.c_uint32), ("rep_max", C.c_int), ("spc_max", C.c_int),
                ("r1_t", C.c_int), ("spc_t", C.c_int), ("r1_max", C.c_int), ("node_min", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("fg_elems", C.c_longlong), ("node_steps", C.c_longlong), ("sorts", C.c_longlong),
                ("cand_total", C.c_longlong), ("stages", C.c_longlong)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (plain gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "polar_oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            vp, i, d = C.c_void_p, C.c_int, C.c_double
            L.orc_polar_transform.argtypes = [i, vp]
            L.orc_crc.argtypes = [vp, i, i, C.c_uint32]
            L.orc_crc.restype = C.c_uint32
            L.orc_encode_batch.argtypes = [vp, i, vp, vp, vp]
            L.orc_ga_reliability.argtypes = [i, vp, d, vp]
            L.orc_ga_frozen.argtypes = [i, i, i, vp, d, vp, vp]
            L.orc_qup_pattern.argtypes = [i, i, vp]
            L.orc_de_bms.argtypes = [i, vp, i, vp, vp, i, vp]
            L.orc_de_awgn_channel.argtypes = [d, i, vp, vp]
            L.orc_de_awgn_channel.restype = i
            L.orc_de_reliability.argtypes = [i, vp, d, i, vp]
            L.orc_de_frozen.argtypes = [i, i, i, vp, d, i, vp, vp]
            L.orc_decode.argtypes = [vp, vp, i, i, vp, i, i, d, vp, vp, vp, vp, vp]
            L.orc_decode_batch.argtypes = [vp, vp, i, i, i, vp, i, i, d, vp, vp, vp, vp]
            L.orc_sc_plain.argtypes = [vp, vp, vp, i, i, d, vp]
            L.orc_node_list.argtypes = [vp, vp, vp]
        return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Code:
    """A polar code for the oracle: frozen (N bytes, 1 = frozen), K = |A|
    (CRC included), CRC length/polynomial, optional puncturing pattern."""

    def __init__(self, frozen, crc_len=0, crc_poly=0, punct=None, systematic=True):
        self.frozen = np.ascontiguousarray(np.asarray(frozen, dtype=np.uint8))
        self.N = int(self.frozen.size)
        self.K = int(self.N - self.frozen.sum())
        self.crc_len = int(crc_len)
        self.crc_poly = int(crc_poly)
        self.punct = None if punct is None else np.ascontiguousarray(np.asarray(punct, dtype=np.uint8))
        self.systematic = bool(systematic)
        self.P = 0 if self.punct is None else int(self.punct.sum())
        self.K_info = self.K - self.crc_len
        self._c = _Code(self.N, self.K, self.crc_len, self.crc_poly, int(self.systematic),
                        self.frozen.ctypes.data, None if self.punct is None else self.punct.ctypes.data)

    @property
    def ref(self):
        return C.byref(self._c)


def pruning(mask=0, rep_max=0, spc_max=4, r1_t=2, spc_t=4, r1_max=0, node_min=0):
    return _Pruning(mask, rep_max, spc_max, r1_t, spc_t, r1_max, node_min)


def polar_transform(v):
    v = np.ascontiguousarray(np.asarray(v, dtype=np.uint8).copy())
    lib().orc_polar_transform(v.size, _ptr(v))
    return v


def crc(bits, c, poly):
    b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8))
    return int(lib().orc_crc(_ptr(b), b.size, c, poly))


def encode(code: Code, info):
    info = np.ascontiguousarray(np.asarray(info, dtype=np.uint8).reshape(-1, code.K_info))
    x = np.zeros((info.shape[0], code.N), dtype=np.uint8)
    rc = C.c_int(0)
    lib().orc_encode_batch(code.ref, info.shape[0], _ptr(info), _ptr(x), C.byref(rc))
    if rc.value:
        raise RuntimeError(f"oracle encoder: systematic property failed (rc={rc.value})")
    return x


def ga_reliability(N, sigma2, punct=None):
    z = np.zeros(N, dtype=np.float64)
    p = None if punct is None else np.ascontiguousarray(np.asarray(punct, dtype=np.uint8))
    lib().orc_ga_reliability(N, _ptr(p), float(sigma2), _ptr(z))
    return z


def ga_frozen(N, K, K_info, design_ebn0_db, punct=None):
    fr = np.zeros(N, dtype=np.uint8)
    z = np.zeros(N, dtype=np.float64)
    p = None if punct is None else np.ascontiguousarray(np.asarray(punct, dtype=np.uint8))
    lib().orc_ga_frozen(N, K, K_info, _ptr(p), float(design_ebn0_db), _ptr(fr), _ptr(z))
    return fr, z


def de_bms(N, q, p, mu=64, punct=None):
    """Density-evolution error-probability bounds of the N bit channels for a
    channel given as a mixture of BSCs (weights q, crossovers p)."""
    q = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64))
    pe = np.zeros(N, dtype=np.float64)
    pu = None if punct is None else np.ascontiguousarray(np.asarray(punct, dtype=np.uint8))
    lib().orc_de_bms(N, _ptr(pu), int(q.size), _ptr(q), _ptr(p), int(mu), _ptr(pe))
    return pe


def de_awgn_channel(sigma2, mu=64):
    q = np.zeros(mu, dtype=np.float64)
    p = np.zeros(mu, dtype=np.float64)
    m = lib().orc_de_awgn_channel(float(sigma2), int(mu), _ptr(q), _ptr(p))
    return q[:m], p[:m]


def de_reliability(N, sigma2, mu=64, punct=None):
    pe = np.zeros(N, dtype=np.float64)
    pu = None if punct is None else np.ascontiguousarray(np.asarray(punct, dtype=np.uint8))
    lib().orc_de_reliability(N, _ptr(pu), float(sigma2), int(mu), _ptr(pe))
    return pe


def de_frozen(N, K, K_info, design_ebn0_db, mu=64, punct=None):
    fr = np.zeros(N, dtype=np.uint8)
    pe = np.zeros(N, dtype=np.float64)
    pu = None if punct is None else np.ascontiguousarray(np.asarray(punct, dtype=np.uint8))
    lib().orc_de_frozen(N, K, K_info, _ptr(pu), float(design_ebn0_db), int(mu), _ptr(fr), _ptr(pe))
    return fr, pe


def qup_pattern(N, P):
    p = np.zeros(N, dtype=np.uint8)
    lib().orc_qup_pattern(N, P, _ptr(p))
    return p


def decode(code: Code, llr, L, algo=CASCL, prune=None, mode=F32, wide_frac=0, wide_q=0.0,
           want_paths=False, stats: Stats | None = None):
    """Decode one frame.  llr: the N-P channel LLRs (float64 array holding the
    values given to the decoder).  Returns dict(info, status, pm[, paths])."""
    llr = np.ascontiguousarray(np.asarray(llr, dtype=np.float64))
    assert llr.size == code.N - code.P
    info = np.zeros(max(code.K_info, 1), dtype=np.uint8)
    st = np.zeros(1, dtype=np.int32)
    pm = np.zeros(L, dtype=np.float64)
    paths = np.zeros((L, code.N), dtype=np.uint8) if want_paths else None
    pr = C.byref(prune) if prune is not None else None
    rc = lib().orc_decode(code.ref, _ptr(llr), L, algo, pr, mode, wide_frac, float(wide_q),
                          _ptr(info), _ptr(st), _ptr(pm), _ptr(paths),
                          C.byref(stats) if stats is not None else None)
    if rc:
        raise ValueError(f"oracle decode rejected the arguments (rc={rc})")
    out = dict(info=info[:code.K_info], status=int(st[0]), pm=pm)
    if want_paths:
        out["paths"] = paths
    return out


def decode_batch(code: Code, llr, L, algo=CASCL, prune=None, mode=F32, wide_frac=0, wide_q=0.0,
                 want_pm=True, stats: Stats | None = None):
    llr = np.ascontiguousarray(np.asarray(llr, dtype=np.float64).reshape(-1, code.N - code.P))
    n = llr.shape[0]
    info = np.zeros((n, max(code.K_info, 1)), dtype=np.uint8)
    st = np.zeros(n, dtype=np.int32)
    pm = np.zeros((n, L), dtype=np.float64) if want_pm else None
    pr = C.byref(prune) if prune is not None else None
    rc = lib().orc_decode_batch(code.ref, _ptr(llr), n, L, algo, pr, mode, wide_frac, float(wide_q),
                                _ptr(info), _ptr(st), _ptr(pm),
                                C.byref(stats) if stats is not None else None)
    if rc:
        raise ValueError(f"oracle decode rejected the arguments (rc={rc})")
    return dict(info=info[:, :code.K_info], status=st, pm=pm)


def sc_plain(code: Code, llr, prune=None, mode=F32, wide_frac=0, wide_q=0.0):
    llr = np.ascontiguousarray(np.asarray(llr, dtype=np.float64))
    x = np.zeros(code.N, dtype=np.uint8)
    pr = C.byref(prune) if prune is not None else None
    rc = lib().orc_sc_plain(code.ref, _ptr(llr), pr, mode, wide_frac, float(wide_q), _ptr(x))
    if rc:
        raise ValueError("oracle sc_plain rejected the arguments")
    return x


def node_list(code: Code, prune=None):
    out = np.zeros(3 * code.N, dtype=np.int32)
    pr = C.byref(prune) if prune is not None else None
    n = lib().orc_node_list(code.ref, pr, _ptr(out))
    return out[: 3 * n].reshape(n, 3)
