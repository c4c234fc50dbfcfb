"""The oracle on every host core, for GPU tests that compare hundreds of
full-size frames: a pool of spawned worker processes (spawned, so that no
worker inherits a CUDA context), each decoding a contiguous share of the
frames with the plain CPU oracle."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _worker(args):
    code_args, llr, L, algo, prune, mode = args
    import oracle
    frozen, crc_len, crc_poly, punct, systematic = code_args
    code = oracle.Code(frozen, crc_len, crc_poly, punct, systematic)
    pr = oracle.pruning(**prune) if prune is not None else None
    r = oracle.decode_batch(code, llr, L, algo, pr, mode)
    return r["info"], r["status"], r["pm"]


class OraclePool:
    def __init__(self, processes: int | None = None):
        self.n = processes or max(1, len(os.sched_getaffinity(0)))
        self.pool = mp.get_context("spawn").Pool(self.n)

    def decode(self, code, llr, L, algo, mode, prune: dict | None = None):
        """Same results as oracle.decode_batch(code, llr, ...), frames split
        over the workers.  prune: the keyword arguments of oracle.pruning."""
        llr = np.ascontiguousarray(np.asarray(llr, dtype=np.float64))
        code_args = (code.frozen, code.crc_len, code.crc_poly, code.punct, code.systematic)
        chunks = [c for c in np.array_split(np.arange(llr.shape[0]), self.n) if c.size]
        res = self.pool.map(_worker, [(code_args, llr[c], L, algo, prune, mode) for c in chunks])
        return (np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res]),
                np.concatenate([r[2] for r in res]))

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
