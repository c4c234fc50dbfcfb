"""Pins of the lower node-size limit of tree pruning (Sec. II-B names node
types by size range: SPC4 is SPC nodes of four leaves only, REP2+ REP nodes
of two or more).  node_min = m leaves every node below m leaves to the
leaf-by-leaf decoder; nothing else about the pruned tree changes."""
import numpy as np
import pytest

import oracle
import synth

R0, R1, REP, SPC = 1, 2, 3, 4


def node_type(fr, o, S, pr):
    """Classification written out from the node definitions (all frozen,
    all information, all frozen but the last, only the first frozen)."""
    leaf = fr[o:o + S]
    nf = int(leaf.sum())
    if S == 1:
        return R0 if nf else R1
    if S < pr["node_min"]:
        return 0
    if nf == S and pr["mask"] & 1:
        return R0
    if nf == 0 and pr["mask"] & 2 and (pr["r1_max"] == 0 or S <= pr["r1_max"]):
        return R1
    if nf == S - 1 and not leaf[-1] and pr["mask"] & 4 and (pr["rep_max"] == 0 or S <= pr["rep_max"]):
        return REP
    if nf == 1 and leaf[0] and S >= 4 and pr["mask"] & 8 and (pr["spc_max"] == 0 or S <= pr["spc_max"]):
        return SPC
    return 0


def walk(fr, pr, o, S, d, out):
    t = node_type(fr, o, S, pr)
    if t:
        out.append([d, o, t])
        return
    walk(fr, pr, o, S // 2, d + 1, out)
    walk(fr, pr, o + S // 2, S // 2, d + 1, out)


def expand_small(nodes, n, m):
    """The node list of node_min = 0 with every pruned node below m leaves
    replaced by its leaves."""
    out = []
    for d, o, t in nodes:
        S = 1 << (n - d)
        if 1 < S < m:
            out.extend([n, o + i, None] for i in range(S))
        else:
            out.append([d, o, t])
    return out


CODES = ["c3_1024_512_L8", "c2_2048_1723", "mcs_256_128", "c1_cascl_128_64_L4"]
PRUNES = [dict(mask=15, rep_max=0, spc_max=4, r1_t=2, spc_t=4, r1_max=0),
          dict(mask=15, rep_max=8, spc_max=0, r1_t=2, spc_t=4, r1_max=0),
          dict(mask=5, rep_max=0, spc_max=4, r1_t=2, spc_t=4, r1_max=0)]


@pytest.mark.parametrize("name", CODES)
@pytest.mark.parametrize("p", range(len(PRUNES)))
@pytest.mark.parametrize("m", [0, 3, 5, 9, 17, 64])
def test_node_list_with_node_min(name, p, m):
    d = synth.load_code(name)
    fr = np.asarray(d["frozen"], dtype=np.uint8)
    N = fr.size
    n = N.bit_length() - 1
    code = oracle.Code(fr, d["crc_len"], d["crc_poly"], d["punct"], d["systematic"])
    pd = dict(PRUNES[p], node_min=m)
    got = oracle.node_list(code, oracle.pruning(**pd)).tolist()
    want = []
    walk(fr, pd, 0, N, 0, want)
    assert got == want
    # the same as the unlimited tree with its small nodes taken apart
    base = oracle.node_list(code, oracle.pruning(**dict(PRUNES[p], node_min=0))).tolist()
    exp = expand_small(base, n, m)
    assert [x[:2] for x in got] == [x[:2] for x in exp]
    for g, e in zip(got, exp):
        if e[2] is not None:
            assert g[2] == e[2]
        else:
            assert g[2] == (R0 if fr[g[1]] else R1)
    assert all(1 << (n - dd) >= m or (1 << (n - dd)) == 1 for dd, _, _ in got)


@pytest.mark.parametrize("mode", [oracle.F32, oracle.I8])
def test_node_min_above_n_decodes_like_the_unpruned_tree(mode):
    d = synth.load_code("mcs_256_128")
    code = oracle.Code(d["frozen"], d["crc_len"], d["crc_poly"], d["punct"], d["systematic"])
    info = synth.info_bits(6, code.K_info, 3)
    x = oracle.encode(code, info)
    llr = synth.bpsk_awgn_llr(x, synth.sigma_for(1.5, code.K_info / code.N), 4)
    pr = oracle.pruning(15, rep_max=0, spc_max=0, r1_t=2, spc_t=4, node_min=code.N + 1)
    for f in range(6):
        a = oracle.decode(code, llr[f], 8, oracle.CASCL, None, mode)
        b = oracle.decode(code, llr[f], 8, oracle.CASCL, pr, mode)
        assert np.array_equal(a["info"], b["info"]) and a["status"] == b["status"]
        assert np.array_equal(a["pm"], b["pm"])
