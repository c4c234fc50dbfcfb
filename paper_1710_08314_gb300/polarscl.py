"""ctypes binding of libpolarscl (include/polarscl.h): same names, argument
marshalling only.  Tensors are passed as device pointers; streams as the raw
cudaStream_t of a torch stream.  There is no CPU fallback: if the library or
CUDA is missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

PSCL_OK, PSCL_EINVAL, PSCL_ENOMEM, PSCL_EUNSUPPORTED, PSCL_ECUDA, PSCL_ETIMEDOUT, PSCL_EAGAIN = 0, -1, -2, -3, -4, -5, -6
PSCL_SC, PSCL_CASCL, PSCL_PASCL, PSCL_FASCL = 0, 1, 2, 3
PSCL_F32, PSCL_I16, PSCL_I8 = 0, 1, 2
PSCL_PRUNE_R0, PSCL_PRUNE_R1, PSCL_PRUNE_REP, PSCL_PRUNE_SPC = 1, 2, 4, 8

ALGOS = {"sc": PSCL_SC, "cascl": PSCL_CASCL, "pascl": PSCL_PASCL, "fascl": PSCL_FASCL}
QUANTS = {"f32": PSCL_F32, "i16": PSCL_I16, "i8": PSCL_I8}


class pscl_pruning(C.Structure):
    _fields_ = [("mask", C.c_uint32), ("rep_max", C.c_int), ("spc_max", C.c_int),
                ("r1_t", C.c_int), ("spc_t", C.c_int), ("r1_max", C.c_int), ("node_min", C.c_int)]


def pruning(mask=0, rep_max=0, spc_max=4, r1_t=2, spc_t=4, r1_max=0, node_min=0) -> pscl_pruning:
    return pscl_pruning(mask, rep_max, spc_max, r1_t, spc_t, r1_max, node_min)


class pscl_work_item(C.Structure):
    _fields_ = [("code", C.c_void_p), ("n_frames", C.c_int), ("L", C.c_int), ("algo", C.c_int),
                ("quant", C.c_int), ("pruning", C.c_void_p), ("llr_offset", C.c_size_t),
                ("info_offset", C.c_size_t), ("status_offset", C.c_size_t)]


class pscl_context(C.Structure):
    _fields_ = [("code", C.c_void_p), ("L", C.c_int), ("pruning", C.c_void_p), ("quant", C.c_int)]


class pscl_server_cfg(C.Structure):
    _fields_ = [("contexts", C.c_void_p), ("n_contexts", C.c_int), ("ring_slots", C.c_int),
                ("max_frames_per_request", C.c_int), ("max_inflight_frames", C.c_longlong),
                ("hbm_budget_bytes", C.c_longlong), ("idle_timeout_ms", C.c_int), ("max_warps", C.c_int)]


class pscl_request(C.Structure):
    _fields_ = [("context", C.c_int), ("n_frames", C.c_int), ("llr", C.c_void_p), ("info_out", C.c_void_p),
                ("status_out", C.c_void_p)]


class pscl_completion(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("status", C.c_int), ("n_frames", C.c_int), ("t_submit_ns", C.c_uint64),
                ("t_done_ns", C.c_uint64), ("device_ns", C.c_uint64)]


class PsclError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"polarscl error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_libs: dict[str, C.CDLL] = {}


def variant() -> str:
    if os.environ.get("PSCL_CHECKED", "0") == "1":
        return "checked"
    return "opprof" if os.environ.get("PSCL_OPPROF", "0") == "1" else "release"


def lib() -> C.CDLL:
    v = variant()
    with _lock:
        if v not in _libs:
            path = _build.lib_path(v)
            if not os.path.exists(path) or os.environ.get("PSCL_AUTOBUILD", "1") == "1":
                path = _build.build(v)
            L = C.CDLL(path)
            vp, i, u32 = C.c_void_p, C.c_int, C.c_uint32
            L.pscl_create_code.argtypes = [i, i, vp, i, u32, vp, i, C.POINTER(vp)]
            L.pscl_destroy_code.argtypes = [vp]
            L.pscl_code_info.argtypes = [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i)]
            L.pscl_prepare.argtypes = [vp, vp]
            L.pscl_decode.argtypes = [vp, vp, i, i, i, vp, i, vp, vp, vp, vp]
            L.pscl_workspace_size.argtypes = [vp, i, i, i, vp, i, C.POINTER(C.c_size_t)]
            L.pscl_decode_ws.argtypes = [vp, vp, i, i, i, vp, i, vp, vp, vp, vp, C.c_size_t, vp]
            L.pscl_encode.argtypes = [vp, vp, i, vp, vp]
            L.pscl_decode_static.argtypes = [vp, vp, i, i, i, vp, i, vp, vp, vp, vp]
            L.pscl_decode_host.argtypes = [vp, vp, i, i, i, vp, i, vp, vp, vp]
            L.pscl_code_tune.argtypes = [vp, i, i, vp, i, i, i, i]
            L.pscl_server_start.argtypes = [vp, C.POINTER(vp)]
            L.pscl_server_submit.argtypes = [vp, vp, C.POINTER(C.c_uint64)]
            L.pscl_server_poll.argtypes = [vp, vp, i, C.POINTER(i)]
            L.pscl_server_status.argtypes = [vp, C.POINTER(i), C.POINTER(i), C.POINTER(C.c_uint64),
                                             C.POINTER(C.c_longlong)]
            L.pscl_server_stop.argtypes = [vp, i]
            L.pscl_debug_server_exit.argtypes = [vp, C.POINTER(i), C.POINTER(C.c_longlong),
                                                 C.POINTER(C.c_ulonglong), vp]
            L.pscl_debug_server_slots.argtypes = [vp, vp, vp, vp, vp]
            L.pscl_server_context_info.argtypes = [vp, i, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t),
                                                   C.POINTER(C.c_size_t)]
            L.pscl_batch_create.argtypes = [vp, i, C.POINTER(vp)]
            L.pscl_batch_destroy.argtypes = [vp]
            L.pscl_batch_run.argtypes = [vp, vp, vp, vp, vp]
            L.pscl_batch_run_plain.argtypes = [vp, vp, vp, vp, vp]
            L.pscl_batch_info.argtypes = [vp, C.POINTER(i), C.POINTER(i), C.POINTER(C.c_size_t)]
            L.pscl_last_error.restype = C.c_char_p
            L.pscl_version.restype = C.c_char_p
            L.pscl_debug_error_word.argtypes = [C.POINTER(u32)]
            L.pscl_debug_step_cycles.argtypes = [vp, i]
            L.pscl_set_tuning.argtypes = [i]
            L.pscl_set_fusion.argtypes = [i]
            L.pscl_set_sc_kernel.argtypes = [i]
            _libs[v] = L
            # optional process-wide tuning overrides (the autotuner sets these per call)
            if os.environ.get("PSCL_WARPS_PER_SM"):
                L.pscl_set_tuning(int(os.environ["PSCL_WARPS_PER_SM"]))
            if os.environ.get("PSCL_FUSE"):
                L.pscl_set_fusion(int(os.environ["PSCL_FUSE"]))
        return _libs[v]


def _check(rc):
    if rc != PSCL_OK:
        raise PsclError(rc, lib().pscl_last_error().decode())
    return rc


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    if hasattr(t, "ctypes"):
        return t.ctypes.data_as(C.c_void_p)
    return C.c_void_p(int(t))


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def pscl_last_error() -> str:
    return lib().pscl_last_error().decode()


def pscl_version() -> str:
    return lib().pscl_version().decode()


def pscl_create_code(N, K, frozen, crc_len, crc_poly, puncture=None, systematic=1):
    """frozen / puncture: host numpy uint8 arrays of N entries."""
    import numpy as np
    fr = np.ascontiguousarray(np.asarray(frozen, dtype=np.uint8))
    pu = None if puncture is None else np.ascontiguousarray(np.asarray(puncture, dtype=np.uint8))
    h = C.c_void_p()
    _check(lib().pscl_create_code(N, K, _ptr(fr), crc_len, crc_poly, _ptr(pu), int(systematic), C.byref(h)))
    return h


def pscl_destroy_code(code):
    return _check(lib().pscl_destroy_code(code))


def pscl_code_info(code):
    N, K, Ki, P = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(lib().pscl_code_info(code, C.byref(N), C.byref(K), C.byref(Ki), C.byref(P)))
    return N.value, K.value, Ki.value, P.value


def pscl_code_tune(code, L, quant, warps_per_sm, fuse_leaves, prune=None, warps_per_block=0, resident_warps=0):
    return _check(lib().pscl_code_tune(code, L, quant, C.byref(prune) if prune is not None else None,
                                       warps_per_sm, fuse_leaves, warps_per_block, resident_warps))


def pscl_prepare(code, prune=None):
    return _check(lib().pscl_prepare(code, C.byref(prune) if prune is not None else None))


def pscl_decode(code, llr, n_frames, L, algo, prune, quant, info_out, status_out, pm_out=None, stream=None):
    return _check(lib().pscl_decode(code, _ptr(llr), n_frames, L, algo,
                                    C.byref(prune) if prune is not None else None, quant,
                                    _ptr(info_out), _ptr(status_out), _ptr(pm_out), _stream(stream)))


def pscl_decode_host(code, llr_host, n_frames, L, algo, prune, quant, info_host, status_host, stream=None):
    """llr_host, info_host, status_host: CPU tensors or numpy arrays (page-locked
    tensors let the copies overlap the decodes); synchronize `stream` before
    reading the outputs."""
    return _check(lib().pscl_decode_host(code, _ptr(llr_host), n_frames, L, algo,
                                         C.byref(prune) if prune is not None else None, quant,
                                         _ptr(info_host), _ptr(status_host), _stream(stream)))


def pscl_workspace_size(code, n_frames, L, algo, prune, quant) -> int:
    b = C.c_size_t()
    _check(lib().pscl_workspace_size(code, n_frames, L, algo, C.byref(prune) if prune is not None else None,
                                     quant, C.byref(b)))
    return b.value


def pscl_decode_ws(code, llr, n_frames, L, algo, prune, quant, info_out, status_out, pm_out, workspace,
                   workspace_bytes, stream=None):
    return _check(lib().pscl_decode_ws(code, _ptr(llr), n_frames, L, algo,
                                       C.byref(prune) if prune is not None else None, quant, _ptr(info_out),
                                       _ptr(status_out), _ptr(pm_out), _ptr(workspace), workspace_bytes,
                                       _stream(stream)))


def pscl_decode_static(code, llr, n_frames, L, algo, prune, quant, info_out, status_out, pm_out=None,
                       stream=None):
    """pscl_decode with the library's static scratch: allocates nothing."""
    return _check(lib().pscl_decode_static(code, _ptr(llr), n_frames, L, algo,
                                           C.byref(prune) if prune is not None else None, quant,
                                           _ptr(info_out), _ptr(status_out), _ptr(pm_out), _stream(stream)))


def pscl_encode(code, info, n_frames, x_out, stream=None):
    return _check(lib().pscl_encode(code, _ptr(info), n_frames, _ptr(x_out), _stream(stream)))


STEP_CATEGORIES = ("f", "g", "leaf", "h", "rsub", "rsub2", "rsub4", "-", "node_r0", "node_r1", "node_rep",
                   "node_spc", "load", "final", "sel2_general", "-")


def pscl_debug_step_cycles(reset=True):
    """Step-profiling build only: {category: (SM cycles, steps)} summed over
    the list kernel's warps since the last reset."""
    out = (C.c_uint64 * 32)()
    _check(lib().pscl_debug_step_cycles(out, 1 if reset else 0))
    return {STEP_CATEGORIES[i]: (out[2 * i], out[2 * i + 1]) for i in range(16) if out[2 * i + 1]}


def pscl_debug_error_word() -> int:
    w = C.c_uint32()
    _check(lib().pscl_debug_error_word(C.byref(w)))
    return w.value


def pscl_debug_last_launches() -> int:
    return lib().pscl_debug_last_launches()


def pscl_set_tuning(target_warps_per_sm: int):
    return _check(lib().pscl_set_tuning(int(target_warps_per_sm)))


def pscl_set_fusion(max_leaves: int):
    return _check(lib().pscl_set_fusion(int(max_leaves)))


def pscl_set_sc_kernel(enable: bool):
    return _check(lib().pscl_set_sc_kernel(1 if enable else 0))


# ---------------------------------------------------------------------------
class Code:
    """Owning wrapper of a pscl_code with torch-allocated outputs."""

    def __init__(self, frozen, crc_len=0, crc_poly=0, puncture=None, systematic=True):
        import numpy as np
        fr = np.asarray(frozen, dtype=np.uint8)
        self.frozen = fr.copy()
        self.puncture = None if puncture is None else np.asarray(puncture, dtype=np.uint8).copy()
        self.N = int(fr.size)
        self.K = int(self.N - (fr != 0).sum())
        self.crc_len = int(crc_len)
        self.handle = pscl_create_code(self.N, self.K, fr, self.crc_len, int(crc_poly), puncture, int(systematic))
        _, _, self.K_info, self.P = pscl_code_info(self.handle)
        self.nbytes = (self.K_info + 7) // 8

    def close(self):
        if self.handle is not None:
            pscl_destroy_code(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def decode(self, llr, L, algo=PSCL_CASCL, prune=None, quant=PSCL_F32, want_pm=False, stream=None):
        import torch
        n = int(llr.shape[0])
        dev = llr.device
        info = torch.empty((n, self.nbytes), dtype=torch.uint8, device=dev)
        status = torch.empty((n,), dtype=torch.int32, device=dev)
        pm = torch.empty((n, L), dtype=torch.float32, device=dev) if want_pm else None
        pscl_decode(self.handle, llr, n, L, algo, prune, quant, info, status, pm, stream)
        return info, status, pm

    def encode(self, info_packed, stream=None):
        import torch
        n = int(info_packed.shape[0])
        x = torch.empty((n, self.N), dtype=torch.uint8, device=info_packed.device)
        pscl_encode(self.handle, info_packed, n, x, stream)
        return x


def pscl_batch_create(items):
    arr = (pscl_work_item * len(items))(*items)
    h = C.c_void_p()
    _check(lib().pscl_batch_create(C.cast(arr, C.c_void_p), len(items), C.byref(h)))
    return h


def pscl_batch_destroy(batch):
    return _check(lib().pscl_batch_destroy(batch))


def pscl_batch_run(batch, llr_pool, info_pool, status_pool, stream=None):
    return _check(lib().pscl_batch_run(batch, _ptr(llr_pool), _ptr(info_pool), _ptr(status_pool), _stream(stream)))


def pscl_batch_run_plain(batch, llr_pool, info_pool, status_pool, stream=None):
    return _check(lib().pscl_batch_run_plain(batch, _ptr(llr_pool), _ptr(info_pool), _ptr(status_pool),
                                             _stream(stream)))


def pscl_batch_info(batch):
    a, b, c = C.c_int(), C.c_int(), C.c_size_t()
    _check(lib().pscl_batch_info(batch, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


class Batch:
    """An uneven batch over torch pools.  parts: list of dicts with keys code
    (Code), llr (cuda float32 tensor, frames x (N-P)), L, algo, quant, prune."""

    def __init__(self, parts):
        import torch
        self.parts = parts
        dev = parts[0]["llr"].device
        llr_off = info_off = st_off = 0
        items, self.slices = [], []
        self._prunes = []
        for p in parts:
            code = p["code"]
            n = int(p["llr"].shape[0])
            pr = p.get("prune")
            self._prunes.append(pr)
            items.append(pscl_work_item(code.handle.value, n, p["L"], p.get("algo", PSCL_CASCL),
                                        p.get("quant", PSCL_F32), C.cast(C.pointer(pr), C.c_void_p) if pr else None,
                                        llr_off, info_off, st_off))
            self.slices.append((llr_off, n * (code.N - code.P), info_off, n * code.nbytes, st_off, n))
            llr_off += n * (code.N - code.P)
            info_off += n * code.nbytes
            st_off += n
        self.llr_pool = torch.cat([p["llr"].reshape(-1) for p in parts]).contiguous()
        self.info_pool = torch.zeros(max(info_off, 1), dtype=torch.uint8, device=dev)
        self.status_pool = torch.zeros(max(st_off, 1), dtype=torch.int32, device=dev)
        self.handle = pscl_batch_create(items)
        self.n_frames = st_off

    def run(self, stream=None):
        pscl_batch_run(self.handle, self.llr_pool, self.info_pool, self.status_pool, stream)

    def run_plain(self, stream=None):
        pscl_batch_run_plain(self.handle, self.llr_pool, self.info_pool, self.status_pool, stream)

    def outputs(self, i):
        lo, ln, io, inn, so, n = self.slices[i]
        code = self.parts[i]["code"]
        return self.info_pool[io:io + inn].reshape(n, code.nbytes), self.status_pool[so:so + n]

    def close(self):
        if self.handle is not None:
            pscl_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pscl_server_start(cfg):
    h = C.c_void_p()
    _check(lib().pscl_server_start(C.byref(cfg), C.byref(h)))
    return h


def pscl_server_submit(server, req):
    """Returns the ticket, or None when the server is full (PSCL_EAGAIN)."""
    t = C.c_uint64()
    rc = lib().pscl_server_submit(server, C.byref(req), C.byref(t))
    if rc == PSCL_EAGAIN:
        return None
    _check(rc)
    return t.value


def pscl_server_poll(server, max_n=256):
    arr = (pscl_completion * max_n)()
    n = C.c_int()
    _check(lib().pscl_server_poll(server, C.cast(arr, C.c_void_p), max_n, C.byref(n)))
    return [arr[k] for k in range(n.value)]


def pscl_server_status(server):
    r, st, done, fl = C.c_int(), C.c_int(), C.c_uint64(), C.c_longlong()
    _check(lib().pscl_server_status(server, C.byref(r), C.byref(st), C.byref(done), C.byref(fl)))
    return dict(running=bool(r.value), device_status=st.value, completed=done.value, in_flight=fl.value)


def pscl_server_stop(server, timeout_ms=5000):
    return _check(lib().pscl_server_stop(server, timeout_ms))


def pscl_server_context_info(server, context):
    a, b, c = C.c_size_t(), C.c_size_t(), C.c_size_t()
    _check(lib().pscl_server_context_info(server, context, C.byref(a), C.byref(b), C.byref(c)))
    return dict(smem_per_warp=a.value, scratch_per_warp=b.value, bytes_per_frame=c.value)


class Server:
    """Serving loop over a list of (Code, L, prune[, quant]) contexts; a
    context without its own number format takes `quant`."""

    def __init__(self, contexts, quant=PSCL_F32, ring_slots=256, max_frames=256, max_inflight=0,
                 idle_timeout_ms=5000, max_warps=0, hbm_budget=0):
        self._ctx_arr = (pscl_context * len(contexts))()
        self._keep = []
        for k, ctx in enumerate(contexts):
            code, L, prune = ctx[:3]
            self._ctx_arr[k].code = code.handle.value
            self._ctx_arr[k].L = L
            self._ctx_arr[k].pruning = C.cast(C.pointer(prune), C.c_void_p) if prune is not None else None
            self._ctx_arr[k].quant = ctx[3] if len(ctx) > 3 else quant
            self._keep.append((code, prune))
        self.cfg = pscl_server_cfg(C.cast(self._ctx_arr, C.c_void_p).value, len(contexts), ring_slots,
                                   max_frames, max_inflight, hbm_budget, idle_timeout_ms, max_warps)
        self.handle = pscl_server_start(self.cfg)

    def debug_exit(self):
        w, i, b = C.c_int(), C.c_longlong(), C.c_ulonglong()
        t = (C.c_uint32 * 4)()
        _check(lib().pscl_debug_server_exit(self.handle, C.byref(w), C.byref(i), C.byref(b), C.cast(t, C.c_void_p)))
        return dict(warp=w.value, idle_ns=i.value, budget_ns=b.value, opened=t[0], head=t[1], opening=t[2],
                    tail=t[3])

    def debug_slots(self):
        R = self.cfg.ring_slots
        cl, dn, nf, tk = (C.c_uint64 * R)(), (C.c_uint32 * R)(), (C.c_int32 * R)(), (C.c_uint64 * R)()
        _check(lib().pscl_debug_server_slots(self.handle, C.cast(cl, C.c_void_p), C.cast(dn, C.c_void_p),
                                             C.cast(nf, C.c_void_p), C.cast(tk, C.c_void_p)))
        return [dict(slot=k, ticket=tk[k], claim_tag=cl[k] >> 32, claim_pos=cl[k] & 0xFFFFFFFF, done=dn[k], n=nf[k])
                for k in range(R) if tk[k] != 2 ** 64 - 1]

    def context_info(self, context):
        return pscl_server_context_info(self.handle, context)

    def submit(self, context, llr, info_out, status_out):
        req = pscl_request(context, int(llr.shape[0]), llr.data_ptr(), info_out.data_ptr(), status_out.data_ptr())
        return pscl_server_submit(self.handle, req)

    def poll(self, max_n=256):
        return pscl_server_poll(self.handle, max_n)

    def status(self):
        return pscl_server_status(self.handle)

    def stop(self, timeout_ms=5000):
        if self.handle is not None:
            pscl_server_stop(self.handle, timeout_ms)
            self.handle = None
