"""Pins of the oracle's R1 (Chase-t) and SPC node handlers with a flip depth t
smaller than the node size, at list sizes L > 1 (Sec. II-B simplified SCL,
Sec. IV-C sorting of LLRs in R1 and SPC nodes).

The expected lists are built here by brute force from definitions, without
the oracle:
  - the t least reliable positions r_0..r_{t-1} of a node are its positions
    sorted by (|alpha|, index);
  - the candidate words of a path are the words that agree with the hard
    decisions HD(alpha) outside {r_k} (SPC: and have even parity); word w has
    flip index j = sum_k 2^k [w_{r_k} != HD(alpha_{r_k})], R1 candidates are
    ordered by j, SPC candidates by j among the even-parity ones;
  - a candidate's metric is the parent's metric plus the min-sum discrepancy
    of its word, sum of |alpha_i| over positions where it differs from HD;
  - candidate id c = p * M + (rank of the candidate), the min(L, #) smallest
    (metric, c) survive, and survivors take slots in increasing c.
LLRs are small integers, so every float sum is exact.
"""
import itertools

import numpy as np
import pytest

import oracle


def hard(alpha):
    return (alpha < 0).astype(np.uint8)


def discrepancy(word, alpha):
    return float(np.abs(alpha)[word != hard(alpha)].sum())


def least_reliable(alpha, t):
    """Positions of the t smallest |alpha|, ties broken by the smaller index."""
    S = alpha.size
    return sorted(range(S), key=lambda i: (abs(float(alpha[i])), i))[:t]


def chase_words(alpha, t, spc):
    """Candidate words of one path at an R1 (spc=False) or SPC node, in
    candidate order: the words that differ from HD only at the t least
    reliable positions (SPC: of even parity), ranked by flip index."""
    h = hard(alpha)
    r = least_reliable(alpha, t)
    found = []
    # every assignment of the t least reliable positions; the others keep HD
    for bits in itertools.product([0, 1], repeat=t):
        w = h.copy()
        w[r] = bits
        if spc and int(w.sum()) % 2:
            continue
        j = sum(1 << k for k in range(t) if w[r[k]] != h[r[k]])
        found.append((j, w))
    found.sort(key=lambda e: e[0])
    return [w for _, w in found]


def f_minsum(a, b):
    m = np.minimum(np.abs(a), np.abs(b))
    return np.where((a < 0) != (b < 0), -m, m)


def survivors(cands, L):
    """cands: list of (metric, c, payload); keep the min(L, n) smallest
    (metric, c) and return them in increasing c."""
    keep = sorted(cands, key=lambda e: (e[0], e[1]))[:L]
    return sorted(keep, key=lambda e: e[1])


def run_oracle(frozen, llr, L, pr):
    code = oracle.Code(np.asarray(frozen, dtype=np.uint8), 0, 0, None, systematic=False)
    return oracle.decode(code, llr.astype(np.float64), L, oracle.CASCL, pr, oracle.F32, want_paths=True)


def prune_for(kind, t):
    return oracle.pruning(15, rep_max=0, spc_max=0, r1_t=t, spc_t=t, r1_max=0)


def check_list(r, expect, L):
    """The oracle's final list equals the expected survivors slot by slot."""
    assert len(expect) <= L
    for slot, (pm, _, word) in enumerate(expect):
        assert np.array_equal(r["paths"][slot], word), slot
        assert r["pm"][slot] == pm, slot
    assert np.all(np.isinf(r["pm"][len(expect):]))


def distinct_int_llr(rng, n, lo=1, hi=60):
    """Nonzero integers with pairwise distinct magnitudes and random signs."""
    mags = rng.choice(np.arange(lo, hi + 1), size=n, replace=False)
    return (mags * rng.choice([-1, 1], size=n)).astype(np.float64)


# ---------------------------------------------------------------------------
# the whole code is one node: its LLRs are the channel LLRs
@pytest.mark.parametrize("Nv", [4, 8, 16])
@pytest.mark.parametrize("t", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["r1", "spc"])
def test_single_node_candidate_list(Nv, t, kind):
    if t > Nv:
        pytest.skip("t > node size")
    frozen = np.zeros(Nv, dtype=np.uint8)
    if kind == "spc":
        frozen[0] = 1
    pr = prune_for(kind, t)
    rng = np.random.default_rng(1000 * Nv + 10 * t + (kind == "spc"))
    M = (1 << t) if kind == "r1" else (1 << (t - 1))
    for trial in range(6):
        alpha = distinct_int_llr(rng, Nv)
        words = chase_words(alpha, t, kind == "spc")
        assert len(words) == M
        cands = [(discrepancy(w, alpha), c, w) for c, w in enumerate(words)]
        for L in sorted({max(1, M // 2), M, 2 * M if 2 * M <= 32 else M}):
            r = run_oracle(frozen, alpha, L, pr)
            check_list(r, survivors(cands, L), L)


# two paths reach the node: a REP node (the left half: all frozen but its
# last leaf) splits the list before the R1 or SPC node on the right half
@pytest.mark.parametrize("Nv", [4, 8, 16])
@pytest.mark.parametrize("t", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["r1", "spc"])
def test_node_behind_a_rep_split(Nv, t, kind):
    if t > Nv:
        pytest.skip("t > node size")
    frozen = np.ones(2 * Nv, dtype=np.uint8)
    frozen[Nv - 1] = 0
    frozen[Nv:] = 0
    if kind == "spc":
        frozen[Nv] = 1
    pr = prune_for(kind, t)
    rng = np.random.default_rng(7 + 1000 * Nv + 10 * t + (kind == "spc"))
    M = (1 << t) if kind == "r1" else (1 << (t - 1))
    ones = np.ones(Nv, dtype=np.uint8)
    zeros = np.zeros(Nv, dtype=np.uint8)
    for trial in range(6):
        llr = distinct_int_llr(rng, 2 * Nv)
        a, b = llr[:Nv], llr[Nv:]
        # left half: a REP node on f(a, b); the two candidates both survive
        aL = f_minsum(a, b)
        left = [(discrepancy(zeros, aL), zeros), (discrepancy(ones, aL), ones)]
        for L in sorted({2, M, 2 * M} - {1}):
            if L > 32:
                continue
            cands = []
            for p, (pm_p, bl) in enumerate(left):
                aR = np.where(bl == 1, -a, a) + b
                for j, w in enumerate(chase_words(aR, t, kind == "spc")):
                    x = np.concatenate([bl ^ w, w])
                    cands.append((pm_p + discrepancy(w, aR), p * M + j, x))
            r = run_oracle(frozen, llr, L, pr)
            check_list(r, survivors(cands, L), L)


def test_reliability_ties_break_by_index():
    """Equal |alpha| at two positions: the smaller index is the less reliable
    one, so with t = 1 the single R1 flip candidate flips the first of them."""
    frozen = np.zeros(8, dtype=np.uint8)
    pr = prune_for("r1", 1)
    alpha = np.array([9.0, -3.0, 7.0, 3.0, -11.0, 5.0, 13.0, -6.0])
    r = run_oracle(frozen, alpha, 2, pr)
    h = hard(alpha)
    flip = h.copy()
    flip[1] ^= 1  # |alpha_1| = |alpha_3| = 3: position 1 ranks first
    assert np.array_equal(r["paths"][0], h) and r["pm"][0] == 0.0
    assert np.array_equal(r["paths"][1], flip) and r["pm"][1] == 3.0
    # t = 2 flips both tied positions: candidates {}, {1}, {3}, {1, 3}
    r = run_oracle(frozen, alpha, 4, prune_for("r1", 2))
    exp = []
    for j in range(4):
        w = h.copy()
        if j & 1:
            w[1] ^= 1
        if j & 2:
            w[3] ^= 1
        exp.append(w)
    for slot, w in enumerate(exp):
        assert np.array_equal(r["paths"][slot], w)
    assert r["pm"].tolist() == [0.0, 3.0, 3.0, 6.0]


def test_spc_candidates_keep_even_parity_and_rank_order():
    """An SPC node with odd hard-decision parity: every candidate flips an odd
    number of the t least reliable positions; the first one flips r_0 only."""
    frozen = np.zeros(8, dtype=np.uint8)
    frozen[0] = 1
    alpha = np.array([4.0, -9.0, 2.0, 6.0, -1.0, 8.0, 5.0, 7.0])  # HD parity: two negatives -> even
    alpha[3] = -6.0  # three negatives: odd parity
    r = run_oracle(frozen, alpha, 8, prune_for("spc", 4))
    h = hard(alpha)
    order = [4, 2, 0, 6]  # |alpha| = 1, 2, 4, 5
    exp = []
    for j in range(16):
        if bin(j).count("1") % 2 == 1:
            w = h.copy()
            for k in range(4):
                if j >> k & 1:
                    w[order[k]] ^= 1
            exp.append((float(sum(abs(alpha[order[k]]) for k in range(4) if j >> k & 1)), w))
    for slot, (pm, w) in enumerate(exp):
        assert np.array_equal(r["paths"][slot], w)
        assert r["pm"][slot] == pm
        assert int(w.sum()) % 2 == 0
