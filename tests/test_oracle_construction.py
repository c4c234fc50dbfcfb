"""Pins of the oracle's density-evolution construction (Sec. II-A cites Tal
and Vardy) and of CRCs of any length (Sec. III-A: standard and custom CRCs).

Density evolution holds a channel as a mixture of binary symmetric channels
and merges components to stay within mu of them (a degrading operation), so
it returns upper bounds on the bit channels' error probabilities.  What fixes
it from outside:
  - on the binary erasure channel (BSCs of crossover 0 and 1/2) nothing is
    ever merged and the bounds are the exact erasure recursion,
    e- = 1 - (1 - e_a)(1 - e_b), e+ = e_a e_b, with error probability e/2;
  - two uses of a BSC(p): the check channel is a BSC(2p(1-p)) and the
    variable channel's ML error probability is p^2 + p(1 - p) = p;
  - quantising BPSK-AWGN preserves the uncoded error probability Q(1/sigma);
  - a finer merge (mu bins that refine the coarser ones) is less degraded;
  - the union bound: SC's frame error rate is at most the sum of the bounds
    over the information positions.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from test_oracle_basics import poly_mod_remainder


def erasure_tree(N, eps, punct=None):
    """Erasure probabilities of the N bit channels, in the decoder's tree
    order (left child: check combination of channels i and i + N/2)."""
    e = np.full(N, float(eps))
    if punct is not None:
        e[np.asarray(punct) == 1] = 1.0

    def rec(v):
        if v.size == 1:
            return v
        h = v.size // 2
        a, b = v[:h], v[h:]
        return np.concatenate([rec(1.0 - (1.0 - a) * (1.0 - b)), rec(a * b)])

    return rec(e)


@pytest.mark.parametrize("N,eps", [(2, 0.3), (16, 0.5), (256, 0.4), (1024, 0.25)])
def test_de_on_the_erasure_channel_is_exact(N, eps):
    pe = oracle.de_bms(N, [1.0 - eps, eps], [0.0, 0.5], mu=8)
    assert np.allclose(pe, erasure_tree(N, eps) / 2.0, rtol=0, atol=1e-12)


def test_de_punctured_positions_are_erasures():
    N = 64
    punct = oracle.qup_pattern(N, 9)
    pe = oracle.de_bms(N, [0.7, 0.3], [0.0, 0.5], mu=8, punct=punct)
    assert np.allclose(pe, erasure_tree(N, 0.3, punct) / 2.0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("p", [0.01, 0.11, 0.3])
def test_de_two_uses_of_a_bsc(p):
    pe = oracle.de_bms(2, [1.0], [p], mu=64)
    assert pe[0] == pytest.approx(2 * p * (1 - p), abs=1e-15)
    assert pe[1] == pytest.approx(p, abs=1e-15)


@pytest.mark.parametrize("sigma2", [0.25, 0.5, 1.0])
def test_awgn_quantisation_keeps_the_uncoded_error_probability(sigma2):
    q, p = oracle.de_awgn_channel(sigma2, 64)
    assert q.sum() == pytest.approx(1.0, abs=1e-12)
    assert (p >= 0).all() and (p <= 0.5).all()
    pe_uncoded = 0.5 * math.erfc(1.0 / math.sqrt(sigma2) / math.sqrt(2.0))
    assert float((q * p).sum()) == pytest.approx(pe_uncoded, rel=1e-10)
    assert oracle.de_reliability(1, sigma2, 64)[0] == pytest.approx(pe_uncoded, rel=1e-10)


def test_finer_merges_give_smaller_bounds():
    sigma2 = synth.sigma_for(2.0, 0.5) ** 2
    coarse = oracle.de_reliability(256, sigma2, 16)
    fine = oracle.de_reliability(256, sigma2, 256)
    assert (fine <= coarse * (1 + 1e-9) + 1e-300).all()
    assert (fine < coarse).any()


def test_de_frozen_set_and_union_bound():
    N, K = 256, 128
    fr, pe = oracle.de_frozen(N, K, K, 2.0, 64)
    A = fr == 0
    assert int(A.sum()) == K and pe[A].max() <= pe[~A].min()
    # SC frame errors (genie-free, plain SC of the oracle) stay below the union bound
    code = oracle.Code(fr, 0, 0, None, systematic=False)
    info = synth.info_bits(3000, K, 7)
    x = oracle.encode(code, info)
    llr = synth.bpsk_awgn_llr(x, synth.sigma_for(2.0, 0.5), 8)
    errs = sum(not np.array_equal(oracle.sc_plain(code, llr[f]), x[f]) for f in range(3000))
    bound = float(pe[A].sum())
    assert errs / 3000 <= bound + 3 * math.sqrt(bound / 3000) + 1e-3
    # and DE agrees with GA on all but a few positions at this size
    fr_ga, _ = oracle.ga_frozen(N, K, K, 2.0)
    assert int(((fr == 0) & (fr_ga == 0)).sum()) >= K - 4


@pytest.mark.parametrize("c", sorted(synth.CUSTOM_CRC_POLYS))
def test_custom_crc_lengths_equal_polynomial_division(c):
    poly = synth.CUSTOM_CRC_POLYS[c]
    rng = np.random.default_rng(c)
    for nb in [0, 1, 5, 40, 257, 1000]:
        bits = rng.integers(0, 2, nb).astype(np.uint8)
        r = oracle.crc(bits, c, poly)
        assert r == poly_mod_remainder(bits, c, poly) and r < (1 << c)
        # message followed by its remainder divides evenly
        tail = np.array([(r >> (c - 1 - k)) & 1 for k in range(c)], dtype=np.uint8)
        assert oracle.crc(np.concatenate([bits, tail]), c, poly) == 0


@pytest.mark.parametrize("name", ["crc6_512_256", "crc11_512_256", "crc24_512_256"])
def test_custom_crc_codes_decode_noiseless_frames(name):
    d = synth.load_code(name)
    code = oracle.Code(d["frozen"], d["crc_len"], d["crc_poly"], None, d["systematic"])
    info = synth.info_bits(3, code.K_info, 1)
    x = oracle.encode(code, info)
    llr = synth.noiseless_llr(x)
    for f in range(3):
        r = oracle.decode(code, llr[f], 8, oracle.CASCL)
        assert np.array_equal(r["info"], info[f]) and r["status"] & 1
