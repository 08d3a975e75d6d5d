"""The roundoff-safe grid, checked on the CPU.

The build picks, per gridded axis, lo and hi (the coordinates' extremes) and
one inverse cell edge inv_h: it starts at fl_down(m / fl_up(r (1 + 2^-10)))
and shrinks (times 0.9, rounded down) until an overestimate of
inv_h (rho + 2^-21 E) + 2^-148, every operation in float32 rounded upward
(rho = r (1 + 2^-20), E = hi - lo), is below m - 2^-20, every axis has at
most 1024 cells and the cell count fits the capacity.  A point's cell
coordinate is floor(fl(fl(x' - lo) * inv_h)) clamped to [0, dim - 1],
x' = x clamped to [lo, hi], and an axis has floor(fl(fl(hi - lo) * inv_h)) + 1
cells.  The claim: two points the float32 contract accepts are at most m
cells apart on every gridded axis, so searching +-m cells finds them.
Emulated here with the same steps (the directed roundings exactly, through
rational arithmetic), on pairs placed at the radius and around cell
boundaries, for small and large extents and offsets.
"""
from fractions import Fraction

import numpy as np
import pytest


def f32_dir(x, up):
    """The rational x rounded to float32 upward (up) or downward."""
    x = Fraction(x)
    y = np.float32(float(x))
    inf = np.float32(np.inf)
    if up:
        while Fraction(float(y)) < x:
            y = np.nextafter(y, inf)
        while Fraction(float(np.nextafter(y, -inf))) >= x:
            y = np.nextafter(y, -inf)
    else:
        while Fraction(float(y)) > x:
            y = np.nextafter(y, -inf)
        while Fraction(float(np.nextafter(y, inf))) <= x:
            y = np.nextafter(y, inf)
    return y


def F(v):
    return Fraction(float(v))


def choose_inv_h(lo, hi, r, m, cap):
    """The build's inverse cell edge for float32 extremes lo, hi (per axis)."""
    r = np.float32(r)
    ext = (hi - lo).astype(np.float32)                                 # round to nearest
    ext_up = [f32_dir(F(h) - F(l), True) for l, h in zip(lo, hi)]
    rho_up = f32_dir(F(r) * (1 + Fraction(1, 2 ** 20)), True)
    need = np.float32(m) - np.float32(2.0 ** -20)
    ih = f32_dir(Fraction(m) / F(f32_dir(F(r) * (1 + Fraction(1, 2 ** 10)), True)), False)
    for _ in range(4096):
        ok, cells = True, 1
        for e, eu in zip(ext, ext_up):
            c = np.floor(np.float32(e * ih)) + 1.0
            if c > 1024:
                ok = False
                break
            cells *= int(c)
            t1 = f32_dir(Fraction(1, 2 ** 21) * F(eu), True)
            t2 = f32_dir(F(rho_up) + F(t1), True)
            t3 = f32_dir(F(ih) * F(t2), True)
            bound = f32_dir(F(t3) + Fraction(1, 2 ** 148), True)
            if not bound < need:
                ok = False
        if ok and cells <= cap:
            return ih
        ih = f32_dir(F(ih) * F(np.float32(0.9)), False)
        assert ih > 0
    raise AssertionError("no inv_h")


def cell(x, lo, hi, ih, dim):
    xc = np.minimum(np.maximum(x, lo), hi).astype(np.float32)
    g = ((xc - lo).astype(np.float32) * ih).astype(np.float32)
    return np.clip(np.floor(g).astype(np.int64), 0, dim - 1)


def contract(q, p):
    s = np.zeros(q.shape[0], np.float32)
    for k in range(q.shape[1]):
        d = (q[:, k] - p[:, k]).astype(np.float32)
        s = (s + (d * d).astype(np.float32)).astype(np.float32)
    return s


def check_event(pts, pairs_a, pairs_b, r, m, cap=1 << 24):
    r = np.float32(r)
    r2 = np.float32(r * r)
    lo, hi = pts.min(axis=0), pts.max(axis=0)
    ih = choose_inv_h(lo, hi, r, m, cap)
    dims = np.floor((hi - lo).astype(np.float32) * ih).astype(np.int64) + 1
    ok = contract(pairs_a, pairs_b) <= r2
    for a in range(pts.shape[1]):
        ca = cell(pairs_a[:, a], lo[a], hi[a], ih, dims[a])
        cb = cell(pairs_b[:, a], lo[a], hi[a], ih, dims[a])
        far = np.flatnonzero(ok & (np.abs(ca - cb) > m))
        assert len(far) == 0, (a, far[:5])
    return int(ok.sum()), dims


@pytest.mark.parametrize("m", [1, 2])
@pytest.mark.parametrize("scale,offset", [(1.0, 0.0), (1.0, 1000.0), (50.0, 0.0), (0.01, -3.0)])
def test_accepted_pairs_within_m_cells(m, scale, offset):
    # points in a box; partners at the radius (mostly along one axis, so that
    # one coordinate moves by ~r) and partners nudged onto cell boundaries
    g = np.random.default_rng(int(900 + 10 * m + scale))
    D, n = 4, 20000
    r = np.float32(0.1 * scale)
    pts = (g.uniform(-1, 1, size=(n, D)) * scale + offset).astype(np.float32)
    u = g.normal(size=(n, D)) * np.array([1.0, 0.05, 0.05, 0.05])
    u = np.roll(u, g.integers(0, D), axis=1)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    b = (pts + u * float(r) * (1 - g.uniform(0, 1e-6, size=n))[:, None]).astype(np.float32)
    inside = (b >= pts.min(axis=0)) & (b <= pts.max(axis=0))
    keep = inside.all(axis=1)
    acc, dims = check_event(np.concatenate([pts, b[keep]]), pts[keep], b[keep], r, m)
    assert acc > n // 4


def farthest_partner(x, r2):
    """The largest y > x (float32) with fl(fl(y - x)^2) <= r2: the partner
    the contract still accepts at the greatest distance along one axis."""
    y = (x + np.sqrt(np.float64(r2))).astype(np.float32)
    for _ in range(8):
        up = np.nextafter(y, np.float32(np.inf))
        d = (up - x).astype(np.float32)
        y = np.where((d * d).astype(np.float32) <= r2, up, y)
    for _ in range(8):
        d = (y - x).astype(np.float32)
        y = np.where((d * d).astype(np.float32) > r2, np.nextafter(y, np.float32(-np.inf)), y)
    return y


@pytest.mark.parametrize("m", [1, 2])
@pytest.mark.parametrize("r", [0.05, 0.1, 0.3])
def test_pairs_straddling_cell_boundaries(m, r):
    # x within a few ulps of a cell boundary (as the build computes it), y the
    # farthest point along the axis that the contract still accepts
    g = np.random.default_rng(int(950 + m + 100 * r))
    D, n = 3, 20000
    r = np.float32(r)
    r2 = np.float32(r * r)
    pts = g.uniform(0, 1, size=(n, D)).astype(np.float32)
    lo, hi = pts.min(axis=0), pts.max(axis=0)
    ih = choose_inv_h(lo, hi, r, m, 1 << 24)
    k = g.integers(1, int(np.floor((hi[0] - lo[0]) * ih)), size=n)
    base = (lo[0] + (k / float(ih))).astype(np.float32)       # near a boundary
    for step in range(-3, 4):
        x = pts.copy()
        x[:, 0] = base
        for _ in range(abs(step)):
            x[:, 0] = np.nextafter(x[:, 0], np.float32(np.inf if step > 0 else -np.inf))
        y = x.copy()
        y[:, 0] = farthest_partner(x[:, 0], r2)
        keep = (y[:, 0] <= hi[0]) & (x[:, 0] >= lo[0])
        acc, _ = check_event(np.concatenate([pts, x[keep], y[keep]]), x[keep], y[keep], r, m)
        assert acc == keep.sum() > n // 4


def test_large_extent_near_the_cell_limit():
    # about 1000 cells on an axis: the extent term of the bound matters
    g = np.random.default_rng(970)
    n = 20000
    r = np.float32(0.001)
    pts = g.uniform(0, 1.0, size=(n, 2)).astype(np.float32)
    b = pts.copy()
    b[:, 0] = (pts[:, 0] + r * (1 - g.uniform(0, 1e-6, size=n))).astype(np.float32)
    keep = b[:, 0] <= pts[:, 0].max()
    acc, dims = check_event(np.concatenate([pts, b[keep]]), pts[keep], b[keep], r, 1)
    assert dims.max() > 900 and acc > n // 2
