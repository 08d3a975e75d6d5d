"""Pins of the CPU oracle against values the paper's definition and mathematics fix.

Each test checks the brute-force oracle (oracle/frnn_oracle.c) against
something other than itself: hand-worked fixtures under tests/golden/ (each
with its citation), closed-form lattice shell counts, invariants of Eq. 1
(symmetry, truncation prefix, relabelling, exact power-of-two scaling) and the
float32 rounding-error bound of the FP64 audit.  A plausible slip in the oracle
(a dropped or transposed term, a wrong sign, '<' for '<=', another summation
order, a fused multiply-add, a wrong tie-break, a self-pair kept, the radius
compared unrounded) fails at least one of them; tests/test_oracle_mutants.py
plants such mistakes and checks that.
"""
import json
import os

import numpy as np
import pytest

from conftest import GOLDEN, hexf
from oracle import oracle
from paper_2609_31980_gb300 import synth


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _bits(a):
    return np.asarray(a, np.float32).view(np.uint32)


def test_ex1_line_hand_worked():
    g = _load("ex1_line.json")
    pts = np.array(g["points"], np.float32)
    for case in g["cases"]:
        counts, idx, d2, deg = oracle.self_query(pts, g["r"], case["K"])
        np.testing.assert_array_equal(counts, case["counts"])
        np.testing.assert_array_equal(idx, case["idx"])
        want = np.array([[hexf(v) for v in row] for row in case["dist2"]], np.float32)
        np.testing.assert_array_equal(_bits(d2), _bits(want))
        np.testing.assert_array_equal(deg, [2, 2, 3, 1])


def test_ex1_line_compact_rows_hand_worked():
    g = _load("ex1_line_csr.json")
    pts = np.array(g["points"], np.float32)
    for case in g["cases"]:
        off, idx, d2, deg = oracle.csr(pts, pts, g["r"], case["K"], query_ids=np.arange(len(pts)))
        np.testing.assert_array_equal(off, case["offsets"])
        np.testing.assert_array_equal(idx, case["idx"])
        np.testing.assert_array_equal(_bits(d2), _bits([hexf(v) for v in case["dist2"]]))
        np.testing.assert_array_equal(deg, case["degree"])


def _pair(x, y, r):
    q = np.array([[hexf(v) for v in x]], np.float32)
    p = np.array([[hexf(v) for v in y]], np.float32)
    counts, idx, d2, deg = oracle.frnn(q, p, float(np.float32(r)), 1)
    return bool(counts[0] == 1), d2[0, 0]


def test_ex2_inclusive_boundary():
    g = _load("ex2_boundary.json")
    for case in g["cases"]:
        inside, d2 = _pair(g["x"], g["y"], hexf(case["r"]))
        assert inside == case["inside"]
        if inside:
            assert _bits(d2) == _bits(hexf(case["d2"]))


def test_ex5_radius_enters_as_its_rounded_square():
    from fractions import Fraction
    g = _load("ex5_radius_square.json")
    r, d2_want = hexf(g["r"]), hexf(g["d2"])
    # the fixture's premise, from its hand-worked numbers: fl(r*r) lies above r^2
    assert Fraction(float(d2_want)) == Fraction(10737419, 2 ** 30) > Fraction(float(r)) ** 2
    inside, d2 = _pair(g["x"], g["y"], r)
    assert inside == g["inside"]
    assert _bits(d2) == _bits(d2_want)


def test_fp64_audit_is_inclusive_at_exactly_r():
    # a pair at exactly distance r is inside in both arithmetics, so it is no
    # crossing: ex2 (every value exact) and ex5 (d^2 = r^2 exactly in double)
    for name in ("ex2_boundary.json", "ex5_radius_square.json"):
        g = _load(name)
        q = np.array([[hexf(v) for v in g["x"]]], np.float32)
        p = np.array([[hexf(v) for v in g["y"]]], np.float32)
        r = hexf(g["cases"][0]["r"]) if "cases" in g else hexf(g["r"])
        assert oracle.fp64_audit(q, p, float(r)) == (0, 0, 0)


def test_ex3_index_order_summation_and_audit():
    g = _load("ex3_order.json")
    r = hexf(g["r"])
    for case in g["cases"]:
        inside, d2 = _pair(g["x"], case["y"], r)
        assert inside == case["inside"], case["why"]
        if inside:
            assert _bits(d2) == _bits(hexf(case["d2"]))
        q = np.array([[hexf(v) for v in g["x"]]], np.float32)
        p = np.array([[hexf(v) for v in case["y"]]], np.float32)
        tot, only32, only64 = oracle.fp64_audit(q, p, float(r))
        assert only32 == int(case["inside"] and not case["inside_fp64"])
        assert only64 == int(case["inside_fp64"] and not case["inside"])


def test_ex4_no_fused_multiply_add():
    g = _load("ex4_nofma.json")
    r = hexf(g["r"])
    assert _bits(np.float32(r) * np.float32(r)) == _bits(hexf(g["r2"]))
    inside, d2 = _pair(g["x"], g["y"], r)
    assert inside == g["inside"]
    assert _bits(d2) == _bits(hexf(g["d2"]))
    assert hexf(g["d2_with_fma"]) > hexf(g["r2"])
    q = np.array([[hexf(v) for v in g["x"]]], np.float32)
    p = np.array([[hexf(v) for v in g["y"]]], np.float32)
    assert oracle.fp64_audit(q, p, float(r)) == (1, 1, 0)


def _lattice(side, D, spacing):
    axes = [np.arange(side)] * D
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, D)
    return grid, (grid * spacing).astype(np.float32)


@pytest.mark.parametrize("case", _load("lattice_shells.json")["cases"], ids=lambda c: f"D{c['D']}")
def test_lattice_shell_counts_closed_form(case):
    g = _load("lattice_shells.json")
    spacing = float.fromhex(g["spacing"])
    side, D, ru = g["side"], case["D"], g["r_units"]
    ints, pts = _lattice(side, D, spacing)
    r = ru * spacing
    K = 128
    centre = int(np.flatnonzero((ints == side // 2).all(axis=1))[0])
    counts, idx, d2, deg = oracle.self_query(pts, r, K, rows=[centre])
    assert deg[0] == case["degree_interior"]
    assert counts[0] == case["degree_interior"]
    got = d2[0, :counts[0]] / np.float32(spacing * spacing)
    shells = {int(k): v for k, v in case["shell_counts"].items()}
    vals, cnt = np.unique(got, return_counts=True)
    assert dict(zip(vals.astype(int).tolist(), cnt.tolist())) == shells
    # order: shells ascending, and inside a shell original indices ascending
    nb = idx[0, :counts[0]]
    sq = ((ints[nb] - ints[centre]) ** 2).sum(axis=1)
    assert np.all(np.diff(sq) >= 0)
    for n in shells:
        assert np.all(np.diff(nb[sq == n]) > 0)
    assert centre not in nb
    assert np.all(idx[0, counts[0]:] == -1) and np.all(np.isinf(d2[0, counts[0]:]))


def test_lattice_every_point_degree_matches_integer_count():
    """Whole 7^3 lattice, r = 2 steps: each point's degree equals an exact
    integer count of lattice points within squared distance 4 (boundary points
    included), computed here with integers only."""
    ints, pts = _lattice(7, 3, 0.125)
    deg = oracle.degree(pts, pts, 0.25, query_ids=np.arange(len(pts)))
    diff = ints[:, None, :] - ints[None, :, :]
    want = ((diff ** 2).sum(-1) <= 4).sum(1) - 1
    np.testing.assert_array_equal(deg, want)


def test_self_query_symmetry_bitwise():
    pts = synth.clustered(40, 10, 200, 5, 0.05, seed=11)
    n = len(pts)
    counts, idx, d2, deg = oracle.self_query(pts, 0.3, n)
    assert np.all(deg == counts)
    pairs = {}
    for i in range(n):
        for e in range(counts[i]):
            pairs[(i, int(idx[i, e]))] = int(_bits(d2[i, e]))
    for (i, j), b in pairs.items():
        assert pairs[(j, i)] == b


def test_count_is_min_degree_k_and_truncation_is_prefix():
    pts = synth.clustered(30, 20, 100, 4, 0.04, seed=12)
    full = oracle.self_query(pts, 0.2, len(pts))
    for K in (1, 2, 5, 17, 32):
        counts, idx, d2, deg = oracle.self_query(pts, 0.2, K)
        np.testing.assert_array_equal(counts, np.minimum(full[3], K))
        np.testing.assert_array_equal(deg, full[3])
        np.testing.assert_array_equal(idx, full[1][:, :K])
        np.testing.assert_array_equal(_bits(d2), _bits(full[2][:, :K]))


def test_rows_sorted_by_distance_then_index_and_padded():
    pts = synth.uniform(600, 3, seed=13)
    counts, idx, d2, deg = oracle.self_query(pts, 0.15, 16)
    for i in range(len(pts)):
        c = counts[i]
        key = list(zip(d2[i, :c].tolist(), idx[i, :c].tolist()))
        assert key == sorted(key)
        assert len(set(idx[i, :c].tolist())) == c and i not in idx[i, :c]
        assert np.all(idx[i, c:] == -1) and np.all(np.isinf(d2[i, c:]))


def test_relabelling_permutes_output():
    pts = synth.clustered(20, 15, 60, 6, 0.05, seed=14)
    n = len(pts)
    perm = np.random.default_rng(7).permutation(n)
    a = oracle.self_query(pts, 0.25, n)
    b = oracle.self_query(pts[perm], 0.25, n)
    inv = np.argsort(perm)
    for i in range(n):
        ib = inv[i]
        assert a[0][i] == b[0][ib]
        c = a[0][i]
        # same neighbour set with the same d2 (order may differ where d2 ties)
        sa = sorted(zip(_bits(a[2][i, :c]).tolist(), a[1][i, :c].tolist()))
        sb = sorted(zip(_bits(b[2][ib, :c]).tolist(), perm[b[1][ib, :c]].tolist()))
        assert sa == sb


def test_power_of_two_scaling_is_exact():
    pts = synth.clustered(25, 12, 80, 8, 0.03, seed=15)
    a = oracle.self_query(pts, 0.2, 64)
    b = oracle.self_query(pts * np.float32(8.0), 1.6, 64)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(_bits(a[2] * np.float32(64.0)), _bits(b[2]))


def test_distinct_sets_have_no_self_exclusion():
    pts = synth.uniform(50, 2, seed=16)
    counts, idx, d2, deg = oracle.frnn(pts, pts, 0.2, 50)
    # without query ids every point finds itself at d2 = +0 first
    assert np.all(idx[:, 0] == np.arange(50))
    assert np.all(_bits(d2[:, 0]) == 0)


def test_one_dimension_neighbourhoods_are_contiguous():
    pts = synth.uniform(300, 1, seed=17)
    order = np.argsort(pts[:, 0], kind="stable")
    rank = np.empty(300, np.int64)
    rank[order] = np.arange(300)
    counts, idx, d2, deg = oracle.self_query(pts, 0.02, 300)
    for i in range(300):
        rk = np.sort(np.append(rank[idx[i, :counts[i]]], rank[i]))
        if len(rk) > 1:
            # ties in coordinate may reorder equal points; contiguous in value order
            vals = np.sort(pts[order[rk], 0])
            inside = (pts[:, 0] >= vals[0]) & (pts[:, 0] <= vals[-1])
            assert inside.sum() == len(rk)


def test_fp64_audit_crossings_lie_inside_rounding_band():
    """Crossing pairs can only sit where |s64 - r^2| is within float32's
    rounding error of the D-term sum: |s32 - s| <= (D+1) u s with u = 2^-24
    (standard recursive-summation bound, plus the rounding of each difference
    and square); r2 = fl(r*r) adds u r^2."""
    rng = np.random.default_rng(18)
    D = 6
    pts = synth.clustered(30, 20, 50, D, 0.05, seed=18)
    r = 0.21
    tot, only32, only64 = oracle.fp64_audit(pts, pts, r, query_ids=np.arange(len(pts)))
    # recompute which pairs are near the boundary in float64 and bound the count
    p64 = pts.astype(np.float64)
    s = ((p64[:, None, :] - p64[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(s, np.inf)
    u = 2.0 ** -24
    band = (abs(s - r * r) <= (2 * D + 4) * u * r * r).sum()
    assert tot <= band
    # and a set built to sit on the boundary does produce crossings
    ex = _load("ex3_order.json")
    q = np.zeros((1, 3), np.float32)
    p = np.array([[hexf(v) for v in ex["cases"][0]["y"]]], np.float32)
    assert oracle.fp64_audit(q, p, 1.0)[0] == 1


@pytest.mark.parametrize("D", [5, 12, 16])
def test_cross_polytope_closed_form(D):
    # the origin and the 2D points +-e_k (all values exact in float32): at
    # r = 1 the origin's neighbours are the 2D unit points at d2 = 1 (ordered
    # by index), every unit point's only neighbour is the origin (the nearest
    # other unit points are at d2 = 2, the opposite one at 4); at r = 2 a unit
    # point also reaches the 2D - 2 others at d2 = 2 and its opposite at 4
    pts = np.zeros((2 * D + 1, D), np.float32)
    for k in range(D):
        pts[1 + 2 * k, k] = 1.0
        pts[2 + 2 * k, k] = -1.0
    c, i, d, deg = oracle.self_query(pts, 1.0, 2 * D + 1)
    assert deg[0] == 2 * D and (i[0, :2 * D] == np.arange(1, 2 * D + 1)).all()
    assert (d[0, :2 * D] == 1.0).all()
    assert (deg[1:] == 1).all() and (i[1:, 0] == 0).all() and (d[1:, 0] == 1.0).all()
    c, i, d, deg = oracle.self_query(pts, 2.0, 2 * D + 1)
    assert (deg[1:] == 2 * D).all()
    for q in range(1, 2 * D + 1):
        opposite = q + 1 if q % 2 else q - 1
        assert i[q, 0] == 0 and d[q, 0] == 1.0
        assert (d[q, 1:2 * D - 1] == 2.0).all()
        assert i[q, 2 * D - 1] == opposite and d[q, 2 * D - 1] == 4.0


def test_empty_inputs():
    pts = np.zeros((0, 3), np.float32)
    counts, idx, d2, deg = oracle.frnn(pts, pts, 0.1, 4)
    assert counts.shape == (0,) and idx.shape == (0, 4)
    q = np.zeros((2, 3), np.float32)
    counts, idx, d2, deg = oracle.frnn(q, pts, 0.1, 4)
    assert np.all(counts == 0) and np.all(idx == -1) and np.all(np.isinf(d2))


def test_duplicates_kept_with_index_tiebreak():
    pts = np.zeros((5, 2), np.float32)
    counts, idx, d2, deg = oracle.self_query(pts, 0.0, 3)
    np.testing.assert_array_equal(counts, [3] * 5)
    np.testing.assert_array_equal(idx[0], [1, 2, 3])
    np.testing.assert_array_equal(idx[4], [0, 1, 2])
    assert np.all(_bits(d2) == 0)
