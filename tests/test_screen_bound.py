"""The packed pre-screen's rejection bound, checked on the CPU.

The row-task grid kernel (query_rows.cu) rejects a candidate when a packed float32 partial sum of
squared differences exceeds r2 (1 + 2^-16) (rounded up), whether or not the
assembler fuses its multiply-adds.  The claim: whenever the exact contract
accepts a pair (s <= r2), every such partial sum is <= that bound.  Checked
here with both fused (one rounding per step) and unfused (two roundings)
emulations, for every prefix and for subsets of dimensions, on pairs placed
at and around the radius, including the hand-worked cases of the oracle pins.
"""
import numpy as np
import pytest

U = 2.0 ** -24


def contract(q, p):
    s = np.float32(0)
    for k in range(len(q)):
        d = np.float32(q[k] - p[k])
        s = np.float32(s + np.float32(d * d))
    return s


def screen_partials(q, p, dims, fused):
    s = np.float32(0)
    out = []
    for k in dims:
        d = np.float32(q[k] - p[k])
        if fused:
            s = np.float32(np.float64(s) + np.float64(d) * np.float64(d))
        else:
            s = np.float32(s + np.float32(d * d))
        out.append(s)
    return out


def bound(r2):
    return np.nextafter(np.float32(np.float64(r2) * (1 + 2.0 ** -16)), np.float32(np.inf))


@pytest.mark.parametrize("D", [1, 2, 3, 8, 12, 16])
def test_accepted_pairs_never_exceed_screen_bound(D):
    g = np.random.default_rng(400 + D)
    n = 4000
    q = g.uniform(-1, 1, size=(n, D)).astype(np.float32)
    dirs = g.normal(size=(n, D))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    r = np.float32(0.1)
    r2 = np.float32(r * r)
    scale = 1 + g.uniform(-1e-6, 1e-6, size=n)
    p = (q + dirs * (r * scale)[:, None]).astype(np.float32)
    T = bound(r2)
    accepted = 0
    for i in range(n):
        if contract(q[i], p[i]) > r2:
            continue
        accepted += 1
        orders = [list(range(D)), list(range(D))[::-1], list(g.permutation(D))]
        for dims in orders:
            for fused in (True, False):
                assert max(screen_partials(q[i], p[i], dims, fused)) <= T
    assert accepted > n // 10   # the set really straddles the boundary


def test_worked_boundary_cases_within_bound():
    x = np.zeros(3, np.float32)
    y = np.array([1.0, 2.0 ** -12, 2.0 ** -12], np.float32)
    r2 = np.float32(1.0)
    assert contract(x, y) <= r2
    for fused in (True, False):
        assert max(screen_partials(x, y, range(3), fused)) <= bound(r2)
    x = np.zeros(2, np.float32)
    y = np.array([2.0 ** -12, 1 + 2.0 ** -12], np.float32)
    r = np.float32(1 + 2.0 ** -12)
    r2 = np.float32(r * r)
    assert contract(x, y) <= r2
    fused = screen_partials(x, y, range(2), True)[-1]
    assert fused > r2            # the fused sum itself would wrongly reject ...
    assert fused <= bound(r2)    # ... but never beyond the screen's margin
