"""Pins of the oracle's list decoder against results the mathematics fixes:
brute-force maximum likelihood, the exact MAP metric, plain SC, the
equivalence of pruned and unpruned trees, float vs fixed point, the
quantiser, and the adaptive schedules (Sec. II-B, III-B, IV)."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth
from test_oracle_basics import kron_F, poly_mod_remainder

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ALL_PRUNE = oracle.pruning(15, rep_max=0, spc_max=4, r1_t=2, spc_t=4)


def stored(name, systematic=True):
    d = synth.load_code(name)
    return oracle.Code(d["frozen"], d["crc_len"], d["crc_poly"], d["punct"], systematic), d


def random_code(N, K, seed, crc_len=0):
    rng = np.random.default_rng(seed)
    fr = np.ones(N, dtype=np.uint8)
    fr[rng.choice(N, K, replace=False)] = 0
    return fr, oracle.Code(fr, crc_len, synth.CRC_POLYS[crc_len], None, systematic=False)


def all_codewords(frozen):
    """Every codeword x = u F with u_{A^c} = 0, by enumeration (with u_A)."""
    N = frozen.size
    F = kron_F(int(np.log2(N)))
    A = np.flatnonzero(frozen == 0)
    out = []
    for bits in itertools.product([0, 1], repeat=A.size):
        u = np.zeros(N, dtype=np.int64)
        u[A] = bits
        out.append((np.array(bits, dtype=np.uint8), ((u @ F) % 2).astype(np.uint8)))
    return out


def discrepancy(x, lam):
    """Min-sum distance D(x) = sum |lambda_i| over bits that disagree with HD."""
    hd = (lam < 0).astype(np.uint8)
    return float(np.abs(lam)[x != hd].sum())


def crc_valid(uA, c, poly):
    k = uA.size - c
    r = poly_mod_remainder(uA[:k], c, poly)
    return all(uA[k + j] == (r >> (c - 1 - j)) & 1 for j in range(c))


# ---------------------------------------------------------------------------
def test_noiseless_round_trip_every_mode():
    for name in ["c1_cascl_128_64_L4", "c3_1024_512_L8", "u04", "u09"]:
        code, d = stored(name)
        info = synth.info_bits(2, code.K_info, 1)
        x = oracle.encode(code, info)
        llr = synth.noiseless_llr(x, 8.0, code.punct)
        for mode in [oracle.F32, oracle.I16, oracle.I8]:
            for algo, L in [(oracle.SC, 1), (oracle.CASCL, 4), (oracle.FA, 8), (oracle.PA, 8)]:
                for pr in [None, ALL_PRUNE]:
                    for f in range(2):
                        r = oracle.decode(code, llr[f], L, algo, pr, mode)
                        assert np.array_equal(r["info"], info[f]), (name, mode, algo, pr)
                        assert r["status"] & 1


def test_noiseless_round_trip_L32_n2048():
    code, _ = stored("c2_2048_1723")
    info = synth.info_bits(1, code.K_info, 2)
    x = oracle.encode(code, info)
    r = oracle.decode(code, synth.noiseless_llr(x)[0], 32, oracle.CASCL, None, oracle.F32)
    assert np.array_equal(r["info"], info[0]) and r["status"] & 1


@pytest.mark.parametrize("mode", [oracle.F32, oracle.I16, oracle.I8])
@pytest.mark.parametrize("prune", [False, True])
def test_list_of_one_is_plain_sc(mode, prune):
    code, d = stored("c3_1024_512_L8")
    pr = ALL_PRUNE if prune else None
    info = synth.info_bits(12, code.K_info, 3)
    x = oracle.encode(code, info)
    llr = synth.bpsk_awgn_llr(x, synth.sigma_for(1.0, 0.5), 4)
    for f in range(12):
        r = oracle.decode(code, llr[f], 1, oracle.CASCL, pr, mode, want_paths=True)
        assert np.array_equal(r["paths"][0], oracle.sc_plain(code, llr[f], pr, mode))


@pytest.mark.parametrize("N,K,crc_len", [(8, 4, 0), (16, 8, 0), (16, 7, 0), (16, 9, 8), (16, 10, 8)])
def test_min_sum_list_equals_brute_force_ml(N, K, crc_len):
    """With L >= 2^|A| nothing is discarded and the min-sum metric of a complete
    path equals the discrepancy D(x) of its codeword (max-log recursion), so the
    decoder returns argmin D over the (CRC-valid) codewords."""
    fr, code = random_code(N, K, seed=N * 100 + K, crc_len=crc_len)
    code = oracle.Code(fr, crc_len, synth.CRC_POLYS[crc_len], None, systematic=False)
    cws = all_codewords(fr)
    rng = np.random.default_rng(K)
    L = 1 << K
    for trial in range(6):
        lam = rng.integers(-(1 << 30), 1 << 30, N).astype(np.float64)
        r = oracle.decode(code, lam, L, oracle.CASCL, None, oracle.IWIDE, 0, float(1 << 50), want_paths=True)
        cand = [(discrepancy(x, lam), uA, x) for uA, x in cws
                if crc_len == 0 or crc_valid(uA, crc_len, code.crc_poly)]
        best = min(cand, key=lambda t: t[0])
        assert sum(1 for t in cand if t[0] == best[0]) == 1
        assert np.array_equal(r["info"], best[1][:K - crc_len])
        # metric invariant on every final path (normalised metrics: differences)
        Ds = np.array([discrepancy(r["paths"][p], lam) for p in range(L)])
        assert np.array_equal(r["pm"] - r["pm"].min(), Ds - Ds.min())


def test_min_sum_float_metric_is_discrepancy_on_integer_llrs():
    fr, code = random_code(16, 6, seed=5)
    rng = np.random.default_rng(6)
    for trial in range(10):
        lam = rng.integers(-40, 41, 16).astype(np.float64)
        r = oracle.decode(code, lam, 64, oracle.CASCL, None, oracle.F32, want_paths=True)
        for p in range(64):
            assert r["pm"][p] == discrepancy(r["paths"][p], lam)


def test_exact_metric_list_is_map():
    """Exact f and PM += ln(1 + e^{-(1-2u) lambda}): a complete path's metric is
    -ln P(x | y) = sum_i ln(1 + e^{-(1-2x_i) lambda_i}), and with L >= 2^|A|
    the chosen codeword maximises sum_i (1 - 2 x_i) lambda_i."""
    fr, code = random_code(16, 7, seed=11)
    cws = all_codewords(fr)
    rng = np.random.default_rng(12)
    for trial in range(8):
        lam = 2.0 * rng.standard_normal(16)
        r = oracle.decode(code, lam, 128, oracle.CASCL, None, oracle.EXACT, want_paths=True)
        for p in range(128):
            x = r["paths"][p].astype(np.float64)
            ref = np.sum(np.logaddexp(0.0, -(1 - 2 * x) * lam))
            assert r["pm"][p] == pytest.approx(ref, rel=1e-9, abs=1e-12)
        corr = [(float(np.sum((1 - 2 * x.astype(np.float64)) * lam)), uA) for uA, x in cws]
        best = max(corr, key=lambda t: t[0])
        assert np.array_equal(r["info"], best[1])


@pytest.mark.parametrize("name,L", [("c1_cascl_128_64_L4", 1), ("c1_cascl_128_64_L4", 4),
                                    ("c1_cascl_128_64_L4", 16), ("mcs_256_128", 8),
                                    ("u27", 2), ("u43", 32)])
def test_pruned_equals_unpruned_with_full_enumeration(name, L):
    """Each pruned node with full candidate enumeration keeps the L best
    (path, sub-codeword) pairs, which is what leaf-by-leaf decoding keeps, so
    decisions and (normalised) metrics agree when no two metrics tie."""
    code, d = stored(name)
    full = oracle.pruning(15, rep_max=0, spc_max=8, r1_t=0, spc_t=0, r1_max=8)
    rng = np.random.default_rng(L)
    for trial in range(4):
        lam = rng.integers(-(1 << 30), 1 << 30, code.N - code.P).astype(np.float64)
        a = oracle.decode(code, lam, L, oracle.CASCL, None, oracle.IWIDE, 0, float(1 << 50))
        b = oracle.decode(code, lam, L, oracle.CASCL, full, oracle.IWIDE, 0, float(1 << 50))
        assert np.array_equal(a["info"], b["info"])
        assert (a["status"] & 1) == (b["status"] & 1)
        assert np.array_equal(np.sort(a["pm"]), np.sort(b["pm"]))


@pytest.mark.parametrize("mode,frac", [(oracle.I8, 2), (oracle.I16, 5)])
@pytest.mark.parametrize("prune", [False, True])
def test_fixed_point_equals_float_without_saturation(mode, frac, prune):
    """When no value can reach the saturation bound, fixed point decides exactly
    like float on the scaled integers (normalisation shifts every metric of a
    step by the same amount, so (PM, c) orders agree, ties included)."""
    fr, code = random_code(16, 8, seed=21, crc_len=0)
    pr = ALL_PRUNE if prune else None
    rng = np.random.default_rng(22)
    for trial in range(40):
        q = np.zeros(16)
        idx = rng.choice(16, 4, replace=False)
        q[idx] = rng.integers(-2, 3, 4)  # sum |q| <= 8: every |LLR| <= 8, PM <= 16*8 = 128
        if np.abs(q).sum() > 7:
            q[idx[0]] = 0
        for L in [1, 2, 4, 8]:
            a = oracle.decode(code, q, L, oracle.CASCL, pr, oracle.F32)
            b = oracle.decode(code, q / 2.0 ** frac, L, oracle.CASCL, pr, mode)
            assert np.array_equal(a["info"], b["info"]) and a["status"] == b["status"]
            act = np.isfinite(a["pm"])
            assert np.array_equal(a["pm"][act] - a["pm"][act].min(), b["pm"][act])


def test_quantiser_and_saturation_pins():
    """Two-bit code, A = {1}: the second leaf's LLR is g(q0, q1, 0) = sat(q0 + q1)
    and with L = 2 the two final metrics are (0, |leaf LLR|), exposing the
    quantised value: q = clamp(rint_half_even(lambda 2^f), -Q, Q)."""
    gold = json.load(open(os.path.join(GOLD, "fixed_point_pins.json")))
    code = oracle.Code(np.array([1, 0], dtype=np.uint8), 0, 0, None, systematic=True)
    modes = {"i8": oracle.I8, "i16": oracle.I16}
    for case in gold["cases"]:
        r = oracle.decode(code, np.array(case["llr"], dtype=np.float64), 2, oracle.CASCL, None,
                          modes[case["mode"]])
        assert sorted(r["pm"].tolist()) == [0.0, float(case["leaf_abs"])], case
        assert int(r["info"][0]) == case["bit"], case


def test_sorted_crc_check_equals_check_all_then_best():
    """Sec. IV-B: checking candidates best-first and stopping at the first valid
    CRC is the same as checking all and taking the best valid one."""
    code, d = stored("c1_cascl_128_64_L4")
    A = np.flatnonzero(d["frozen"] == 0)
    info = synth.info_bits(60, code.K_info, 31)
    x = oracle.encode(code, info)
    llr = synth.bpsk_awgn_llr(x, synth.sigma_for(0.5, 0.5), 32)
    for f in range(60):
        r = oracle.decode(code, llr[f], 8, oracle.CASCL, None, oracle.F32, want_paths=True)
        valid = [p for p in range(8) if np.isfinite(r["pm"][p])
                 and crc_valid(r["paths"][p][A], code.crc_len, code.crc_poly)]
        order = sorted(range(8), key=lambda p: (r["pm"][p], p))
        slot = (r["status"] >> 16) & 0xFF
        if valid:
            assert slot == min(valid, key=lambda p: (r["pm"][p], p)) and r["status"] & 1
        else:
            assert slot == order[0] and not r["status"] & 1
        assert np.array_equal(r["info"], r["paths"][slot][A][:code.K_info])


@pytest.mark.parametrize("prune", [False, True])
def test_adaptive_schedules_equal_their_stages(prune):
    """FA runs L = 1, 2, 4, ..., Lmax and stops at the first CRC pass; PA runs 1
    then Lmax (Sec. II-B).  Each stage is a fresh CA-SCL(L) decode."""
    code, d = stored("c1_cascl_128_64_L4")
    pr = ALL_PRUNE if prune else None
    info = synth.info_bits(40, code.K_info, 41)
    x = oracle.encode(code, info)
    llr = synth.bpsk_awgn_llr(x, synth.sigma_for(1.0, 0.5), 42)
    Lmax = 16
    for f in range(40):
        stages = {L: oracle.decode(code, llr[f], L, oracle.CASCL, pr, oracle.F32) for L in [1, 2, 4, 8, 16]}
        fa = oracle.decode(code, llr[f], Lmax, oracle.FA, pr, oracle.F32)
        Lu = (fa["status"] >> 8) & 0xFF
        passed = [L for L in [1, 2, 4, 8, 16] if stages[L]["status"] & 1]
        assert Lu == (passed[0] if passed else Lmax)
        assert fa["status"] == stages[Lu]["status"] and np.array_equal(fa["info"], stages[Lu]["info"])
        pa = oracle.decode(code, llr[f], Lmax, oracle.PA, pr, oracle.F32)
        Lp = 1 if stages[1]["status"] & 1 else Lmax
        assert pa["status"] == stages[Lp]["status"] and np.array_equal(pa["info"], stages[Lp]["info"])
        sc = oracle.decode(code, llr[f], Lmax, oracle.SC, pr, oracle.F32)
        assert sc["status"] == stages[1]["status"] and np.array_equal(sc["info"], stages[1]["info"])


def test_list_decoding_beats_sc_statistically():
    """Sanity: CA-SCL(4) makes fewer frame errors than SC on the (128, 64) code."""
    code, d = stored("c1_cascl_128_64_L4")
    info = synth.info_bits(400, code.K_info, 51)
    x = oracle.encode(code, info)
    llr = synth.bpsk_awgn_llr(x, synth.sigma_for(2.0, code.K_info / 128), 52)
    e_sc = e_l = 0
    for f in range(400):
        e_sc += not np.array_equal(oracle.decode(code, llr[f], 1, oracle.SC)["info"], info[f])
        e_l += not np.array_equal(oracle.decode(code, llr[f], 4, oracle.CASCL)["info"], info[f])
    assert e_l < e_sc
