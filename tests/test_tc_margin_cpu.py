"""The tensor-core pre-filter's margin, checked on the CPU.

The filter (the tensor-core path) passes a candidate when the BF16 dot
product acc = A(x).B(y) ~= x'.y' - n(y)/2, accumulated in float32, is at least
t(x) = (n(x) - Theta)/2 rounded down, with Theta = (R + 2^-14 nu)^2 + 2^-12 nu^2,
R^2 = r2 (1 + 2^-18) and nu^2 the largest n of the event.  The claim: every
pair the exact float32 contract accepts passes, whatever order and rounding
the tensor cores use to accumulate.  Emulated here: the operand preparation
(centring, two-term bf16 split, the fused norm, -n/2 split in two bf16) and
the accumulation of the 3D + 2 exact bf16 products in float32 in several
orders, rounded to nearest or toward zero, or summed exactly and rounded
once; on clustered events and on pairs placed at and just inside the radius.
"""
import numpy as np
import pytest

from paper_2609_31980_gb300 import synth


def bf16(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def f32(x, mode):
    """float64 -> float32, rounded to nearest or toward zero."""
    y = np.asarray(x, np.float64).astype(np.float32)
    if mode == "rz":
        over = np.abs(y.astype(np.float64)) > np.abs(x)
        y = np.where(over, np.nextafter(y, np.float32(0)), y)
    return y


def contract(q, p):
    s = np.zeros(q.shape[0], np.float32)
    for k in range(q.shape[1]):
        d = (q[:, k] - p[:, k]).astype(np.float32)
        s = (s + (d * d).astype(np.float32)).astype(np.float32)
    return s


def operands(x, c):
    """hi, lo and the norm n of each point (rows), as the prep kernel builds them."""
    xc = (x - c).astype(np.float32)
    hi = bf16(xc)
    lo = bf16((xc - hi).astype(np.float32))
    xh = (hi + lo).astype(np.float32)
    n = np.zeros(x.shape[0], np.float32)
    for k in range(x.shape[1]):     # fused multiply-add chain, one rounding per step
        n = f32(xh[:, k].astype(np.float64) ** 2 + n.astype(np.float64), "rn")
    m = (-0.5 * n).astype(np.float32)
    mh = bf16(m)
    ml = bf16((m - mh).astype(np.float32))
    return hi, lo, n, mh, ml


def products(ox, oy):
    """The 3D + 2 products of A(x) = [hi, hi, lo, 1, 1] and B(y) = [hi, lo, hi,
    m_hi, m_lo], each exact in float32 (bf16 x bf16)."""
    hx, lx, _, _, _ = ox
    hy, ly, _, mhy, mly = oy
    t = [hx * hy, hx * ly, lx * hy, mhy[:, None], mly[:, None]]
    return np.concatenate(t, axis=1).astype(np.float32)


def accumulate(terms, order, mode):
    if order == "exact":
        return f32(terms.astype(np.float64).sum(axis=1), mode)
    idx = np.arange(terms.shape[1])
    if order == "reverse":
        idx = idx[::-1]
    elif order == "ascending":
        idx = None
    elif order == "descending":
        idx = None
    if idx is None:
        key = np.argsort(np.abs(terms), axis=1)
        if order == "descending":
            key = key[:, ::-1]
        terms = np.take_along_axis(terms, key, axis=1)
        idx = np.arange(terms.shape[1])
    if order == "tree":
        t = terms.astype(np.float32)
        while t.shape[1] > 1:
            if t.shape[1] % 2:
                t = np.concatenate([t, np.zeros((t.shape[0], 1), np.float32)], axis=1)
            t = f32(t[:, 0::2].astype(np.float64) + t[:, 1::2].astype(np.float64), mode)
        return t[:, 0]
    acc = np.zeros(terms.shape[0], np.float32)
    for j in idx:
        acc = f32(acc.astype(np.float64) + terms[:, j].astype(np.float64), mode)
    return acc


def threshold(n_x, r2, nu2):
    nu = np.sqrt(nu2)
    R = np.sqrt(np.float64(r2) * (1.0 + 2.0 ** -18))
    th = (R + 2.0 ** -14 * nu) ** 2 + 2.0 ** -12 * nu2
    v = (n_x.astype(np.float64) - th) * 0.5
    t = v.astype(np.float32)                                  # then round down
    return np.where(t.astype(np.float64) > v, np.nextafter(t, np.float32(-np.inf)), t)


ORDERS = ("index", "reverse", "ascending", "descending", "tree", "exact")


def check(x, y, r, c, nu2=None):
    r2 = np.float32(np.float32(r) * np.float32(r))
    acc_ok = contract(x, y) <= r2
    ox, oy = operands(x, c), operands(y, c)
    if nu2 is None:
        nu2 = float(max(ox[2].max(), oy[2].max()))
    tx = threshold(ox[2], r2, nu2)
    terms = products(ox, oy)
    for order in ORDERS:
        for mode in ("rn", "rz"):
            passed = accumulate(terms, order, mode) >= tx
            dropped = np.flatnonzero(acc_ok & ~passed)
            assert len(dropped) == 0, (order, mode, dropped[:5])
    return int(acc_ok.sum())


@pytest.mark.parametrize("D", [8, 12, 16])
def test_pairs_at_the_radius_always_pass(D):
    g = np.random.default_rng(800 + D)
    n = 20000
    x = g.uniform(-1, 1, size=(n, D)).astype(np.float32)
    u = g.normal(size=(n, D))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = 0.1 if D == 8 else 0.12
    scale = 1 - g.uniform(0, 1e-6, size=n)     # at and just inside the radius
    y = (x + u * (r * scale)[:, None]).astype(np.float32)
    c = np.zeros(D, np.float32)
    assert check(x, y, r, c) > n // 2


@pytest.mark.parametrize("D", [8, 12])
def test_event_pairs_always_pass(D):
    # candidate pairs of a clustered event (pairs within the same cluster, and
    # the centre of the bounding box as the prep kernel takes it)
    pts = synth.clustered(400, 25, 2000, D, 0.02 if D == 8 else 0.025, seed=810 + D)
    g = np.random.default_rng(820 + D)
    i = g.integers(0, 400 * 25, size=50000)
    j = (i // 25) * 25 + g.integers(0, 25, size=i.size)
    lo, hi = pts.min(axis=0), pts.max(axis=0)
    c = (lo + np.float32(0.5) * (hi - lo)).astype(np.float32)
    ox = operands(pts, c)
    assert check(pts[i], pts[j], 0.1 if D == 8 else 0.12, c, nu2=float(ox[2].max())) > 1000


def test_far_from_the_centre():
    # coordinates of magnitude ~100 (nu large against r): the margin grows
    # with nu, the pairs still pass
    g = np.random.default_rng(830)
    D, n = 12, 20000
    x = (g.uniform(-1, 1, size=(n, D)) * 100).astype(np.float32)
    u = g.normal(size=(n, D))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    y = (x + u * 0.12).astype(np.float32)
    assert check(x, y, 0.12, np.zeros(D, np.float32)) > n // 4
