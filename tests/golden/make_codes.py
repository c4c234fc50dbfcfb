"""Write the stored code definitions under tests/golden/codes/.

Calls only the oracle (its Gaussian-approximation construction and its
quasi-uniform puncturing pattern) and the workload parameters of ``synth``.
Run from the repository root:  python tests/golden/make_codes.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def make(name, N, K, crc_len, design_db, P, L, ebn0_db, crc_poly=None, construction="ga", **_):
    punct = oracle.qup_pattern(N, P) if P else None
    k_info = K - crc_len
    if construction == "de":
        frozen, _z = oracle.de_frozen(N, K, k_info, design_db, 64, punct)
        source = "oracle.de_frozen (density evolution, 64-component degrading merges)"
    else:
        frozen, _z = oracle.ga_frozen(N, K, k_info, design_db, punct)
        source = "oracle.ga_frozen (Gaussian approximation) + oracle.qup_pattern"
    poly = synth.CRC_POLYS[crc_len] if crc_poly is None else crc_poly
    systematic = True
    code = oracle.Code(frozen, crc_len, poly, punct, systematic=True)
    try:
        oracle.encode(code, synth.info_bits(4, k_info, 0))
    except RuntimeError:
        systematic = False
    d = dict(name=name, N=N, K=K, crc_len=crc_len, crc_poly=poly, P=P, L=L,
             design_db=design_db, ebn0_db=ebn0_db, systematic=systematic,
             frozen_hex=frozen.astype(np.uint8).tobytes().hex(),
             punct_hex=None if punct is None else punct.astype(np.uint8).tobytes().hex(),
             source=source)
    with open(os.path.join(synth.CODES_DIR, name + ".json"), "w") as fh:
        json.dump(d, fh, indent=1)
        fh.write("\n")
    return d


def main():
    os.makedirs(synth.CODES_DIR, exist_ok=True)
    for name, w in synth.WORKLOADS.items():
        make(name, **w)
    ctx = synth.uneven_contexts()
    for w in ctx:
        make(**w)
    with open(os.path.join(synth.CODES_DIR, "uneven_index.json"), "w") as fh:
        json.dump([w["name"] for w in ctx], fh)
        fh.write("\n")


if __name__ == "__main__":
    main()
