"""Helpers shared by the GPU tests: run the library and the oracle on the same
seeded inputs and compare them element by element."""
import numpy as np

import oracle
import synth

QMAP = {"f32": (0, oracle.F32), "i16": (1, oracle.I16), "i8": (2, oracle.I8)}
AMAP = {"sc": (0, oracle.SC), "cascl": (1, oracle.CASCL), "pascl": (2, oracle.PA), "fascl": (3, oracle.FA)}


def unpack_info(info_bytes, k_info):
    bits = np.unpackbits(np.asarray(info_bytes, dtype=np.uint8), axis=1)
    return bits[:, :k_info]


def make_inputs(d, n_frames, ebn0_db, seed, systematic=True):
    code = oracle.Code(d["frozen"], d["crc_len"], d["crc_poly"], d["punct"], systematic)
    info = synth.info_bits(n_frames, code.K_info, seed)
    x = oracle.encode(code, info)
    rate = code.K_info / (code.N - code.P)
    llr = synth.bpsk_awgn_llr(x, synth.sigma_for(ebn0_db, rate), seed + 1, d["punct"])
    return code, info, llr


def gpu_code(d, systematic=True):
    from paper_1710_08314_gb300 import Code
    return Code(d["frozen"], d["crc_len"], d["crc_poly"], d["punct"], systematic)


def gpu_decode(gcode, llr, L, algo, quant, prune=None):
    import torch
    from paper_1710_08314_gb300 import polarscl as ps
    t = torch.from_numpy(np.ascontiguousarray(llr, dtype=np.float32)).cuda()
    info, status, pm = gcode.decode(t, L, AMAP[algo][0], prune, QMAP[quant][0], want_pm=True)
    torch.cuda.synchronize()
    if ps.variant() == "checked":
        assert ps.pscl_debug_error_word() == 0, "bounds check tripped"
    return (unpack_info(info.cpu().numpy(), gcode.K_info), status.cpu().numpy(), pm.cpu().numpy())


def oracle_decode(code, llr, L, algo, quant, prune=None):
    r = oracle.decode_batch(code, llr.astype(np.float64), L, AMAP[algo][1], prune, QMAP[quant][1])
    return r["info"], r["status"], r["pm"]


def compare(gpu, orc, frames=None):
    gi, gs, gp = gpu
    oi, os_, op = orc
    if frames is not None:
        gi, gs, gp = gi[frames], gs[frames], gp[frames]
    bad = [f for f in range(len(oi)) if not (np.array_equal(gi[f], oi[f]) and gs[f] == os_[f]
                                             and np.array_equal(gp[f].astype(np.float64), op[f]))]
    return bad


def describe(gpu, orc, f, frames=None):
    gi, gs, gp = gpu
    oi, os_, op = orc
    g = f if frames is None else frames[f]
    return (f"frame {g}: status gpu {gs[g]:#x} oracle {os_[f]:#x}; info diff bits "
            f"{np.flatnonzero(gi[g] != oi[f])[:10]}; pm gpu {gp[g][:8]} oracle {op[f][:8]}")
