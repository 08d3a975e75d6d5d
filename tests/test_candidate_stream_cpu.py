"""The row-task grid kernel's candidate stream (query_rows.cu), checked on the CPU.

A warp task's candidates are the slot ranges [rs, re) of its neighbour rows
(one per lane, empty rows allowed).  Each range is widened to whole slot
pairs: its first pair prs = rs >> 1 and np = ((re + 1) >> 1) - prs pairs, and
the rows' pairs are concatenated in lane order into one stream (row l starts
at pp_l, the exclusive prefix sum of np).  An entry is kept as its stream
code 2 * pair + half and resolved after the scan: its row is the last lane
whose pp is <= the pair (a five-step binary search over the 32 lanes), its
slot 2 * (prs + pair - pp) + half, and it is dropped unless rs <= slot < re
(the halves the widening added).  Checked here: over random row sets, every
slot of every range has exactly one code, and exactly the widened halves are
dropped."""
import numpy as np
import pytest


def stream(rs, re):
    prs = rs >> 1
    np_ = np.where(re > rs, ((re + 1) >> 1) - prs, 0)
    pp = np.concatenate([[0], np.cumsum(np_)[:-1]])
    return prs, np_, pp, int(np_.sum())


def resolve(code, pp, prs, rs, re):
    sp = code >> 1
    L = 0
    for st in (16, 8, 4, 2, 1):
        if pp[L + st] <= sp:
            L += st
    slot = 2 * (prs[L] + sp - pp[L]) + (code & 1)
    return L, slot, rs[L] <= slot < re[L]


@pytest.mark.parametrize("seed", range(40))
def test_every_slot_has_exactly_one_code(seed):
    g = np.random.default_rng(4000 + seed)
    nrows = int(g.integers(1, 33))
    # neighbour rows: ascending, disjoint slot ranges, some empty, odd ends
    rs = np.zeros(32, np.int64)
    re = np.zeros(32, np.int64)
    cur = int(g.integers(0, 5))
    for l in range(nrows):
        cur += int(g.integers(0, 7))
        n = 0 if g.random() < 0.25 else int(g.integers(1, 40))
        rs[l], re[l] = cur, cur + n
        cur += n
    # lanes beyond the rows hold empty ranges at 0, like the kernel's
    prs, np_, pp, P = stream(rs, re)
    pp = pp.copy()
    pp[nrows:] = P                 # their prefix is the total
    seen = {}
    dropped = 0
    for code in range(2 * P):
        L, slot, ok = resolve(code, pp, prs, rs, re)
        if not ok:
            dropped += 1
            continue
        assert L < nrows and slot not in seen
        seen[slot] = L
    want = {s: l for l in range(nrows) for s in range(rs[l], re[l])}
    assert seen == want
    widened = sum(int(rs[l] & 1) + int(re[l] & 1) for l in range(nrows) if re[l] > rs[l])
    assert dropped == widened
