"""The compact-output gather, checked on the CPU.

Rows are staged 32 entries per query; a warp handles 32 consecutive rows as
one flat range of their entries (rows the selection kernel writes itself, and
empty rows, contribute none): entry t belongs to the last row whose exclusive
prefix within the 32 is <= t (a five-step binary search over the lanes), and
goes from stage slot row * 32 + (t - prefix) to offsets[row] + (t - prefix).
Checked here: over random counts with empty and marked rows, every staged
entry of every unmarked row is copied exactly once to its place."""
import numpy as np
import pytest

STAGE = 32


def gather_warp(cnt, spilled, offsets, r0, M):
    moves = []
    own = np.zeros(32, np.int64)
    for lane in range(32):
        i = r0 + lane
        if i < M and not spilled[i]:
            own[lane] = cnt[i]
    incl = np.cumsum(own)
    excl = incl - own
    T = int(incl[-1])
    for base in range(0, T, 32):
        for lane in range(32):
            t = base + lane
            R = 0
            for st in (16, 8, 4, 2, 1):
                if excl[R + st] <= t:
                    R += st
            e = t - excl[R]
            if t < T:
                moves.append(((r0 + R) * STAGE + e, offsets[r0 + R] + e))
    return moves


@pytest.mark.parametrize("seed", range(30))
def test_every_entry_copied_once(seed):
    g = np.random.default_rng(6000 + seed)
    M = int(g.integers(1, 200))
    cnt = g.integers(0, STAGE + 1, size=M)
    cnt[g.random(M) < 0.3] = 0
    spilled = g.random(M) < 0.1          # written by the selection kernel
    counts = np.where(spilled, g.integers(33, 100, size=M), cnt)
    offsets = np.concatenate([[0], np.cumsum(counts)])
    moves = []
    for r0 in range(0, M, 32):
        moves += gather_warp(cnt, spilled, offsets, r0, M)
    want = sorted((i * STAGE + e, offsets[i] + e) for i in range(M) if not spilled[i]
                  for e in range(cnt[i]))
    assert sorted(moves) == want
