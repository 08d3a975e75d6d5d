"""The grid kernels' per-row sort, checked on the CPU lane by lane.

A query row's entries sit in lanes 0 .. n-1 of a warp as 64-bit keys
(d2 bits << 32 | index; a rejected entry is +inf with index 0, so all
rejected entries share one key), the other lanes hold the largest key.  The
kernel sorts them with a bitonic network across the lanes, only as wide as
the row (stages whose half-size reaches n are skipped), one comparison per
step (equal keys are interchangeable).  For D >= 10 two rows of at most 16
entries are sorted at once, one per half-warp, every step taking its
direction from the lane index within the half.  The chunk kernel sorts two
rows at once, their networks' steps interleaved, at the wider row's width
(checked below: a wider network leaves a row's result unchanged).  Checked
here by simulating the 32 lanes for every row length and random keys with
ties."""
import numpy as np
import pytest

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
REJECT = np.uint64(0x7F800000) << np.uint64(32)


def network(key, width, paired):
    """One pass of the kernel's network over 32 lane keys."""
    key = key.copy()
    lane = np.arange(32)
    hl = lane & 15 if paired else lane
    k2 = 2
    while k2 <= 32:
        if (k2 >> 1) >= width:
            break
        j = k2 >> 1
        while j > 0:
            other = key[lane ^ j]
            take_min = ((hl & j) == 0) == ((hl & k2) == 0)
            key = np.where(take_min == (other < key), other, key)
            j >>= 1
        k2 <<= 1
    return key


def row_keys(g, n):
    """n entries: accepted keys (distinct indices) and some rejected ones."""
    d2 = g.choice(np.arange(1, 40, dtype=np.uint64), size=n)   # ties in d2
    idx = g.permutation(10_000)[:n].astype(np.uint64)
    keys = (d2 << np.uint64(32)) | idx
    rej = g.random(n) < 0.2
    keys[rej] = REJECT
    return keys


@pytest.mark.parametrize("n", range(0, 33))
def test_one_row_sorted(n):
    g = np.random.default_rng(1000 + n)
    for _ in range(200):
        keys = np.full(32, EMPTY)
        keys[:n] = row_keys(g, n)
        out = network(keys, n, False)
        assert np.array_equal(out[:n], np.sort(keys[:n]))
        assert (out[n:] == EMPTY).all()


@pytest.mark.parametrize("n0,n1", [(a, b) for a in range(0, 17, 3) for b in range(0, 17, 4)] + [(16, 16), (1, 16), (16, 1)])
def test_two_rows_sorted_per_half_warp(n0, n1):
    g = np.random.default_rng(2000 + 17 * n0 + n1)
    for _ in range(200):
        keys = np.full(32, EMPTY)
        a, b = row_keys(g, n0), row_keys(g, n1)
        keys[:n0] = a
        keys[16:16 + n1] = b
        out = network(keys, max(n0, n1), True)
        assert np.array_equal(out[:n0], np.sort(a))
        assert np.array_equal(out[16:16 + n1], np.sort(b))
        assert (out[n0:16] == EMPTY).all() and (out[16 + n1:] == EMPTY).all()


def test_accepted_keys_precede_rejected_ones():
    # the kernel counts a row's accepted entries as those below the reject key
    g = np.random.default_rng(3000)
    keys = np.full(32, EMPTY)
    keys[:20] = row_keys(g, 20)
    out = network(keys, 20, False)
    acc = int((keys[:20] < REJECT).sum())
    assert (out[:acc] < REJECT).all() and (out[acc:20] == REJECT).all()


def test_two_rows_sorted_at_the_wider_width():
    # the chunk kernel sorts two rows together with the wider row's width:
    # each row ends sorted exactly as alone
    g = np.random.default_rng(4100)
    for _ in range(500):
        rows = []
        for _u in range(2):
            keys = np.full(32, EMPTY)
            n = int(g.integers(0, 33))
            keys[:n] = row_keys(g, n)
            rows.append((keys, n))
        width = max(rows[0][1], rows[1][1])
        for keys, n in rows:
            out = network(keys, width, False)
            assert np.array_equal(out, network(keys, n, False))
            assert np.array_equal(out[:n], np.sort(keys[:n]))
