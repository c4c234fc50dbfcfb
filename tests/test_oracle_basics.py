"""Pins of the oracle's encoder, CRC, construction and tree classification
against things the paper and the mathematics fix (not against the oracle)."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def kron_F(n):
    """F^{(x)n} from its definition (Sec. II-A footnote) with numpy's Kronecker
    product: F^{(x)1} = [[1,0],[1,1]], F^{(x)n} = F^{(x)1} (x) F^{(x)(n-1)}."""
    F1 = np.array([[1, 0], [1, 1]], dtype=np.int64)
    F = np.array([[1]], dtype=np.int64)
    for _ in range(n):
        F = np.kron(F1, F)
    return F


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_transform_is_u_times_kron(n):
    N = 1 << n
    F = kron_F(n)
    rng = np.random.default_rng(n)
    for _ in range(20):
        u = rng.integers(0, 2, N).astype(np.uint8)
        ref = (u.astype(np.int64) @ F) % 2
        assert np.array_equal(oracle.polar_transform(u), ref.astype(np.uint8))


def test_transform_block_structure_matches_footnote():
    # F^{(x)n} = [[F', 0], [F', F']]
    for n in range(2, 6):
        F, Fp = kron_F(n), kron_F(n - 1)
        h = 1 << (n - 1)
        assert np.array_equal(F[:h, :h], Fp) and not F[:h, h:].any()
        assert np.array_equal(F[h:, :h], Fp) and np.array_equal(F[h:, h:], Fp)


def test_transform_involution():
    rng = np.random.default_rng(3)
    for N in [2, 16, 1024]:
        v = rng.integers(0, 2, N).astype(np.uint8)
        assert np.array_equal(oracle.polar_transform(oracle.polar_transform(v)), v)


def poly_mod_remainder(bits, c, poly):
    """M(x) x^c mod G(x) over GF(2) with Python integers (textbook long
    division on the whole polynomial), G(x) = x^c + poly."""
    m = 0
    for b in bits:
        m = (m << 1) | int(b)
    m <<= c
    g = (1 << c) | poly
    while m.bit_length() > c:
        m ^= g << (m.bit_length() - c - 1)
    return m


def test_crc_catalogue_check_values():
    gold = json.load(open(os.path.join(GOLD, "crc_check_values.json")))
    bits = np.unpackbits(np.frombuffer(gold["message_ascii"].encode(), dtype=np.uint8))
    for case in gold["cases"]:
        assert oracle.crc(bits, case["c"], case["poly"]) == case["check"]


@pytest.mark.parametrize("c", [8, 16, 32])
def test_crc_equals_polynomial_division(c):
    poly = synth.CRC_POLYS[c]
    rng = np.random.default_rng(c)
    for nb in [0, 1, 7, 33, 100, 1691]:
        bits = rng.integers(0, 2, nb).astype(np.uint8)
        assert oracle.crc(bits, c, poly) == poly_mod_remainder(bits, c, poly)


@pytest.mark.parametrize("c", [8, 16, 32])
def test_crc_of_message_and_remainder_is_zero(c):
    poly = synth.CRC_POLYS[c]
    rng = np.random.default_rng(100 + c)
    for nb in [1, 56, 1691]:
        bits = rng.integers(0, 2, nb).astype(np.uint8)
        r = oracle.crc(bits, c, poly)
        rbits = np.array([(r >> (c - 1 - k)) & 1 for k in range(c)], dtype=np.uint8)
        assert oracle.crc(np.concatenate([bits, rbits]), c, poly) == 0


@pytest.mark.parametrize("name", ["c1_cascl_128_64_L4", "c3_1024_512_L8", "c2_2048_1723", "u00", "u09"])
def test_encoder_systematic_and_in_code(name):
    d = synth.load_code(name)
    code = oracle.Code(d["frozen"], d["crc_len"], d["crc_poly"], d["punct"], systematic=True)
    info = synth.info_bits(8, code.K_info, 5)
    x = oracle.encode(code, info)
    A = np.flatnonzero(d["frozen"] == 0)
    for f in range(8):
        # x_A = (info || crc) with the CRC remainder MSB first (Sec. II-A)
        r = poly_mod_remainder(info[f], code.crc_len, code.crc_poly)
        rbits = [(r >> (code.crc_len - 1 - k)) & 1 for k in range(code.crc_len)]
        assert np.array_equal(x[f, A], np.concatenate([info[f], np.array(rbits, dtype=np.uint8)]))
        # x is a codeword: u = x F has zero frozen part
        u = oracle.polar_transform(x[f])
        assert not u[d["frozen"] == 1].any()


def test_encoder_non_systematic_is_uF():
    d = synth.load_code("c1_cascl_128_64_L4")
    code = oracle.Code(d["frozen"], d["crc_len"], d["crc_poly"], None, systematic=False)
    info = synth.info_bits(4, code.K_info, 9)
    x = oracle.encode(code, info)
    F = kron_F(7)
    A = np.flatnonzero(d["frozen"] == 0)
    for f in range(4):
        r = poly_mod_remainder(info[f], code.crc_len, code.crc_poly)
        u = np.zeros(128, dtype=np.int64)
        u[A] = np.concatenate([info[f], [(r >> (7 - k)) & 1 for k in range(8)]])
        assert np.array_equal(x[f], ((u @ F) % 2).astype(np.uint8))


def test_ga_two_channel_closed_form():
    # N = 2: the right (g) channel doubles the mean, the left (f) channel
    # satisfies phi(z0) = 1 - (1 - phi(z))^2 (Trifonov's GA recursion)
    def phi(x):
        if x < 10:
            return min(1.0, np.exp(-0.4527 * x ** 0.86 + 0.0218))
        return np.sqrt(np.pi / x) * np.exp(-x / 4) * (1 - 10 / (7 * x))
    for sigma2 in [0.2, 0.5, 1.0, 4.0]:
        z = 2.0 / sigma2
        zz = oracle.ga_reliability(2, sigma2)
        assert zz[1] == pytest.approx(2 * z, rel=1e-15)
        assert phi(zz[0]) == pytest.approx(1 - (1 - phi(z)) ** 2, rel=1e-9)


def test_ga_bitflip_partial_order():
    # turning a 0 into a 1 in a channel index replaces one check (f) step by a
    # variable (g) step, which can only make the channel better
    N = 256
    z = oracle.ga_reliability(N, 0.7)
    for i in range(N):
        for b in range(8):
            if not (i >> b) & 1:
                assert z[i | (1 << b)] >= z[i] - 1e-9 * abs(z[i])


def test_ga_frozen_count_and_best_channels():
    fr, z = oracle.ga_frozen(1024, 512, 496, 2.0)
    assert int((fr == 0).sum()) == 512
    assert z[fr == 0].min() >= z[fr == 1].max()
    # the last channel (all g steps) is the most reliable, the first the least
    assert fr[1023] == 0 and fr[0] == 1


def test_qup_is_bitreversed_prefix():
    N, P = 64, 13
    p = oracle.qup_pattern(N, P)
    rev = [int(format(i, "06b")[::-1], 2) for i in range(P)]
    assert p.sum() == P and all(p[r] for r in rev)


def test_node_classification_hand_cases():
    gold = json.load(open(os.path.join(GOLD, "node_types_n8.json")))
    for case in gold["cases"]:
        fr = np.zeros(case["N"], dtype=np.uint8)
        fr[case["frozen_idx"]] = 1
        code = oracle.Code(fr)
        pr = oracle.pruning(case["mask"], rep_max=case["rep_max"], spc_max=case["spc_max"])
        got = oracle.node_list(code, pr).tolist()
        assert got == case["nodes"], case
