"""The grid query kernel's candidate stream, checked on the CPU.

The kernel (query.cu, k_grid_query) takes chunks of 16 cell-sorted query
slots; runs of queries whose cells are equal or follow each other along the
fastest axis of one row form a group.  For each group it enumerates the
(2m+1)^(naxes-1) neighbour rows 32 at a time (lane l of round rr handles row
32 rr + l, whose per-axis offsets are the base-(2m+1) digits of that number:
a per-event table holds each row's linear offset and, for m = 1, bit masks of
the axes whose offset is -1 or +1, tested against the group's grid-edge
bits), looks up each row's slot range over the cells x_first-m .. x_last+m
along the fastest axis (x_first, x_last: the group's first and last cell on
the row), and appends the non-empty ranges with their counts to a
compact list (at most 128 entries; a group that does not fit is rolled back
and opens the next batch); one exclusive scan per batch turns the counts into
stream positions.  The stream is presented either in tiles of 64 candidates
(the lanes holding overlapping ranges copy their parts, and write the
candidates' slots, into one of two ring buffers, a cursor moving to the first
range reaching past the tile) or by rounds of 32 candidates whose slots the
lanes find by binary search over the stream positions; both are re-enacted
and must agree.  Lanes find a candidate's group by a four-step search over
the groups' stream starts.

This file re-enacts those steps lane by lane on random and adversarial grids
and checks: every shared-memory index stays inside its array, every copy's
destination lies inside its ring buffer and its source inside the point set,
and each query is paired with exactly the points of its group's box (each
once): the cells within +-m of its own cell on every gridded axis but the
fastest, and within x_first-m .. x_last+m on that one, a box that holds the
query's own +-m neighbourhood.
"""
import numpy as np
import pytest

KCHUNKQ = 16
TILE = 64
NB = 2
RANGE_CAP = 128
MAX_NBR_ROWS = 128
INT_MAX = 2 ** 31 - 1


def make_grid(pts, naxes, h):
    """Cells of edge h over the last naxes coordinates (the fastest first),
    points sorted by cell: (dims, cell of each slot, cstart over cells + 1)."""
    D = pts.shape[1]
    axes = list(range(D - naxes, D))
    lo = pts[:, axes].min(0)
    ext = pts[:, axes].max(0) - lo
    dims = (np.floor(ext / h) + 1).astype(np.int64)
    c = np.minimum(np.floor((pts[:, axes] - lo) / h).astype(np.int64), dims - 1)
    cid = np.zeros(len(pts), np.int64)
    st = 1
    for a in range(naxes):
        cid += c[:, a] * st
        st *= dims[a]
    order = np.argsort(cid, kind="stable")
    scell = cid[order]
    cstart = np.searchsorted(scell, np.arange(st + 1)).astype(np.int64)
    return dims, scell, cstart


def decode(cell, dims, naxes):
    cc = [0] * 5
    v = cell
    cc[0] = v % dims[0]
    v //= dims[0]
    for a in range(1, naxes):
        cc[a] = v % dims[a]
        v //= dims[a]
    return cc


def run_kernel(dims, scell, cstart, naxes, m):
    """Pairs (query slot, candidate slot) the kernel's stream presents."""
    n = len(scell)
    d5 = [int(x) for x in dims] + [1] * (5 - naxes)
    nrows = (2 * m + 1) ** (naxes - 1)
    assert nrows <= MAX_NBR_ROWS
    side = 2 * m + 1
    rstride = [0, 1, 0, 0, 0]
    for ax in range(2, 5):
        rstride[ax] = rstride[ax - 1] * d5[ax - 1]
    # per-event table of row l = 32 rr + lane: linear offset, and edge bits
    # (m = 1: axes with offset -1 in bits 0-3, +1 in bits 8-11) or digits
    tdelta, tedge = [], []
    for rr in range(MAX_NBR_ROWS // 32):
        dl_row, te_row = [], []
        for lane in range(32):
            l = rr * 32 + lane
            ll, dl, dg, lowm, highm = l, 0, 0, 0, 0
            for ax in range(1, naxes):
                d = ll % side
                ll //= side
                dg |= d << (3 * (ax - 1))
                dl += (d - m) * rstride[ax]
                if d < m:
                    lowm |= 1 << (ax - 1)
                if d > m:
                    highm |= 1 << (ax - 1)
            te = (lowm | (highm << 8)) if m == 1 else dg
            if l >= nrows:
                te |= 1 << 31
            dl_row.append(dl)
            te_row.append(te)
        tdelta.append(dl_row)
        tedge.append(te_row)
    pairs = []
    nchunks = (n + KCHUNKQ - 1) // KCHUNKQ
    for c in range(nchunks):
        s0 = c * KCHUNKQ
        nqc = min(KCHUNKQ, n - s0)
        qc = [int(scell[s0 + l]) if l < nqc else -1 for l in range(32)]
        cc = [decode(qc[l] if l < nqc else 0, d5, naxes) for l in range(32)]
        head = [l < nqc and (l == 0 or not (qc[l - 1] == qc[l] or (qc[l] == qc[l - 1] + 1 and cc[l][0] != 0)))
                for l in range(32)]
        heads = [l for l in range(32) if head[l]]
        ng = len(heads)
        gq = [heads[l] if l < ng else nqc for l in range(32)]

        def fetch(g):
            gc = cc[gq[g]]
            xl = cc[gq[g + 1] - 1][0]
            assert all(cc[q][1:] == gc[1:] for q in range(gq[g], gq[g + 1])), "a group lies on one row"
            x0, x1 = max(gc[0] - m, 0), min(xl + m, d5[0] - 1)
            grow, gedge = 0, 1 << 31
            for ax in range(1, naxes):
                grow += gc[ax] * rstride[ax]
                if gc[ax] == 0:
                    gedge |= 1 << (ax - 1)
                if gc[ax] == d5[ax] - 1:
                    gedge |= 1 << (ax + 7)
            lo = [[0] * 32 for _ in range(MAX_NBR_ROWS // 32)]
            hi = [[0] * 32 for _ in range(MAX_NBR_ROWS // 32)]
            for rr in range(MAX_NBR_ROWS // 32):
                if rr * 32 >= nrows:
                    continue
                for lane in range(32):
                    if m == 1:
                        ok = (tedge[rr][lane] & gedge) == 0
                    else:
                        ok = not (tedge[rr][lane] >> 31)
                        for ax in range(1, naxes):
                            v = gc[ax] + ((tedge[rr][lane] >> (3 * (ax - 1))) & 7) - m
                            ok = ok and 0 <= v < d5[ax]
                    if ok:
                        base = (grow + tdelta[rr][lane]) * d5[0]
                        assert 0 <= base + x0 and base + x1 + 1 < len(cstart)
                        lo[rr][lane] = int(cstart[base + x0])
                        hi[rr][lane] = int(cstart[base + x1 + 1])
            return lo, hi

        g0 = 0
        while g0 < ng:
            nr, g = 0, g0
            gr = [0] * 32
            rlo = [None] * RANGE_CAP
            rpre = [None] * (RANGE_CAP + 1)
            while g < ng:
                nr0 = nr
                clo, chi = fetch(g)
                for rr in range(MAX_NBR_ROWS // 32):
                    if rr * 32 >= nrows:
                        break
                    k = 0
                    for lane in range(32):
                        cnt = chi[rr][lane] - clo[rr][lane]
                        if cnt > 0:
                            pos = nr + k
                            k += 1
                            if pos < RANGE_CAP:
                                rlo[pos] = clo[rr][lane]
                                rpre[pos] = cnt
                    nr += k
                if nr > RANGE_CAP:
                    nr = nr0
                    break
                assert g - g0 < 32
                gr[g - g0] = nr0
                g += 1
            gend = g
            assert gend > g0, "a single group must fit one batch"
            gqb = [gq[min(g0 + lane, 31)] for lane in range(32)]
            assert nr <= RANGE_CAP
            U = 0
            for i in range(nr):
                v = rpre[i]
                rpre[i] = U
                U += v
            rpre[nr] = U
            gsb = [rpre[gr[lane]] if lane < gend - g0 else INT_MAX for lane in range(32)]
            # tiles (bulk staging) / rounds (direct loads) present the same
            # candidates in stream order; the tile logic is re-enacted here
            ring_slot = [[None] * TILE for _ in range(NB)]
            ntiles = (U + TILE - 1) // TILE
            cur = [0]

            def issue(t, b):
                T0, T1 = t * TILE, min(t * TILE + TILE, U)
                copied = 0
                for lane in range(32):
                    i = cur[0] + lane
                    while i < nr:
                        ps = rpre[i]
                        if ps >= T1:
                            break
                        pe = rpre[i + 1]
                        s, e = max(ps, T0), min(pe, T1)
                        if e > s:
                            lo_ = rlo[i] + (s - ps)
                            dst0 = b * TILE + (s - T0)
                            assert b * TILE <= dst0 and dst0 + (e - s) <= (b + 1) * TILE
                            assert 0 <= lo_ and lo_ + (e - s) <= n
                            for j in range(e - s):
                                ring_slot[b][s - T0 + j] = lo_ + j
                            copied += e - s
                        i += 32
                assert copied == T1 - T0, "expected bytes = copied bytes"
                while cur[0] < nr and rpre[cur[0] + 1] <= T1:
                    cur[0] += 1

            def direct_slot(u):
                # the direct-load staging: binary search over the stream positions
                i = 0
                st = RANGE_CAP // 2
                while st > 0:
                    if i + st < nr and rpre[i + st] <= u:
                        i += st
                    st >>= 1
                return rlo[i] + (u - rpre[i])

            for t in range(min(NB, ntiles)):
                issue(t, t)
            for t in range(ntiles):
                b = t % NB
                T0 = t * TILE
                ln = min(TILE, U - T0)
                for k0 in range(0, ln, 32):
                    for lane in range(32):
                        ul = k0 + lane
                        valid = ul < ln
                        u = T0 + ul
                        j = 0
                        for st in (8, 4, 2, 1):
                            assert j + st < 32
                            if gsb[j + st] <= u:
                                j += st
                        qa, qe = gqb[j], gqb[j + 1]
                        nq = qe - qa if valid else 0
                        if valid:
                            assert direct_slot(u) == ring_slot[b][ul]
                        for jq in range(nq):
                            q = qa + jq
                            assert 0 <= q < nqc
                            pairs.append((s0 + q, ring_slot[b][ul]))
                if t + NB < ntiles:
                    issue(t + NB, b)
            g0 = gend
    return pairs


def neighbourhoods(dims, scell, naxes, m):
    """Brute force: for each slot, the slots whose cells are within +-m (its
    own neighbourhood) and the slots of its group's box: chunks of 16 slots,
    a group a maximal run of slots whose cells are equal or next to each
    other along the fastest axis of one row, its box the cells within +-m on
    the other axes and from its first cell's x - m to its last cell's x + m."""
    n = len(scell)
    coords = np.array([decode(int(c), [int(x) for x in dims] + [1] * (5 - naxes), naxes)[:naxes]
                       for c in scell]).reshape(n, naxes)
    own, box = [], [None] * n
    for i in range(n):
        near = np.all(np.abs(coords - coords[i]) <= m, axis=1)
        own.append(set(np.flatnonzero(near).tolist()))
    for s0 in range(0, n, KCHUNKQ):
        runs = []
        for i in range(s0, min(s0 + KCHUNKQ, n)):
            if runs and np.array_equal(coords[i, 1:], coords[runs[-1][-1], 1:]) and \
                    0 <= coords[i, 0] - coords[runs[-1][-1], 0] <= 1:
                runs[-1].append(i)
            else:
                runs.append([i])
        for run in runs:
            xa, xb = coords[run[0], 0], coords[run[-1], 0]
            inb = np.all(np.abs(coords[:, 1:] - coords[run[0], 1:]) <= m, axis=1) & \
                (coords[:, 0] >= xa - m) & (coords[:, 0] <= xb + m)
            for i in run:
                box[i] = set(np.flatnonzero(inb).tolist())
    return own, box


def check(pts, naxes, m, h):
    dims, scell, cstart = make_grid(pts, naxes, h)
    pairs = run_kernel(dims, scell, cstart, naxes, m)
    own, box = neighbourhoods(dims, scell, naxes, m)
    got = [[] for _ in range(len(pts))]
    for q, s in pairs:
        got[q].append(s)
    for i in range(len(pts)):
        assert len(got[i]) == len(set(got[i])), f"slot {i}: a candidate presented twice"
        assert set(got[i]) == box[i], f"slot {i}: stream differs from the group's box"
        assert own[i] <= set(got[i]), f"slot {i}: a neighbour cell missing"


@pytest.mark.parametrize("naxes,m", [(1, 1), (2, 1), (3, 1), (3, 2), (3, 3), (4, 1), (4, 2), (5, 1)])
def test_stream_equals_neighbourhood_clustered(naxes, m):
    g = np.random.default_rng(100 + 10 * naxes + m)
    centres = g.uniform(-1, 1, size=(25, 6))
    pts = np.repeat(centres, 12, axis=0) + g.normal(0, 0.05, size=(300, 6))
    pts = np.concatenate([pts, g.uniform(-1, 1, size=(101, 6))])   # odd count
    check(pts[g.permutation(len(pts))], naxes, m, 0.2 / m)


def test_dense_cells_force_batches():
    # every cell of a 4^5 block occupied several times: each group has 81
    # non-empty rows, so a chunk's groups need several batches (rollback)
    g = np.random.default_rng(7)
    pts = g.integers(0, 4, size=(2000, 5)).astype(np.float64) + g.uniform(0.1, 0.9, size=(2000, 5))
    check(pts, 5, 1, 1.0)


def test_long_ranges_span_tiles():
    # few cells with many points: ranges longer than a tile, tiles spanning ranges
    g = np.random.default_rng(8)
    pts = g.uniform(0, 2.5, size=(700, 3))
    check(pts, 3, 1, 1.0)


@pytest.mark.parametrize("n", [1, 2, 15, 16, 17, 33])
def test_small_sets(n):
    g = np.random.default_rng(n)
    check(g.uniform(0, 1, size=(n, 4)), 4, 1, 0.3)
