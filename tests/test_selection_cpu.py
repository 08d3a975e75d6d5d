"""The exact selection kernel's buffer logic (rows longer than the in-kernel
lists), checked on the CPU.

A warp scans a query's candidates 32 at a time; every accepted candidate
below the current threshold appends its key (d2 bits << 32 | index, unique)
to a shared buffer of cap keys (a power of two >= max(64, 2K)).  Whenever
more than cap - 32 are held, the buffer is sorted, cut to its K smallest and
the threshold becomes the K-th key.  At the end the buffer is sorted and the
first K keys are the row.  Checked here: the row equals the K smallest of
all accepted keys, for degrees far above and below K."""
import numpy as np
import pytest

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def select(chunks, K):
    cap = 64
    while cap < 2 * K:
        cap <<= 1
    buf = np.full(cap, EMPTY)
    fill, thr = 0, EMPTY
    for keys in chunks:                     # 32 lane keys, EMPTY = not accepted
        keys = np.where(keys >= thr, EMPTY, keys)
        new = keys[keys != EMPTY]
        assert fill + len(new) <= cap       # the buffer never overflows
        buf[fill:fill + len(new)] = new
        fill += len(new)
        if fill > cap - 32:
            buf = np.sort(buf)
            buf[K:] = EMPTY
            fill, thr = K, buf[K - 1]
    return np.sort(buf)[:K]


@pytest.mark.parametrize("K", [1, 2, 31, 32, 33, 64, 100, 1000, 1024])
@pytest.mark.parametrize("degree", [0, 1, 40, 500, 5000])
def test_row_is_the_k_smallest(K, degree):
    g = np.random.default_rng(5000 + K + degree)
    ncand = degree + int(g.integers(0, 2000))
    d2 = g.integers(1, 1 << 20, size=ncand).astype(np.uint64)       # many ties in d2
    idx = g.permutation(1 << 22)[:ncand].astype(np.uint64)
    keys = (d2 << np.uint64(32)) | idx
    accepted = np.zeros(ncand, bool)
    accepted[g.permutation(ncand)[:degree]] = True
    keys = np.where(accepted, keys, EMPTY)
    pad = (-ncand) % 32
    lanes = np.concatenate([keys, np.full(pad, EMPTY)]).reshape(-1, 32)
    got = select(list(lanes), K)
    want = np.sort(keys[accepted])[:K]
    assert np.array_equal(got[:len(want)], want)
    assert (got[len(want):] == EMPTY).all()
