"""Compact (CSR) output against the oracle, through the C ABI
(frnn_query_csr_count + frnn_query_csr_fill): offsets, indices and distances
bit-exact, full degrees equal, on both search paths, with rows that overflow
the in-kernel lists, cross-set queries, empty inputs and the full-size events."""
import numpy as np
import pytest

from oracle import oracle
from paper_2609_31980_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2609_31980_gb300 import frnn
    c = frnn.Context()
    yield c
    c.close()


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _csr(ctx, refs, r, K, path="grid", queries=None):
    tr = _t(refs)
    g = ctx.build_grid(tr, r)
    self_q = queries is None
    tq = tr if self_q else _t(queries)
    off, idx, d2, deg = ctx.query_csr(g, tq, r, K, self_q, path, degree=True)
    ctx.sync()
    out = off.cpu().numpy(), idx.cpu().numpy(), d2.cpu().numpy(), deg.cpu().numpy()
    g.close()
    return out


def _assert_csr_equal(got, want, rows=None):
    go, gi, gd, gdeg = got
    wo, wi, wd, wdeg = want
    if rows is None:
        np.testing.assert_array_equal(go, wo)
        np.testing.assert_array_equal(gi, wi)
        np.testing.assert_array_equal(gd.view(np.uint32), wd.view(np.uint32))
        np.testing.assert_array_equal(gdeg, wdeg)
        return
    # sampled rows: want is the oracle's CSR of those rows only
    for k, i in enumerate(rows):
        a, b = go[i], go[i + 1]
        c, d = wo[k], wo[k + 1]
        assert b - a == d - c, f"row {i}: {b - a} entries vs {d - c}"
        np.testing.assert_array_equal(gi[a:b], wi[c:d])
        np.testing.assert_array_equal(gd[a:b].view(np.uint32), wd[c:d].view(np.uint32))
    np.testing.assert_array_equal(gdeg[rows], wdeg)


@pytest.mark.parametrize("D,path", [(3, "grid"), (8, "grid"), (8, "tc"), (12, "tc")])
@pytest.mark.parametrize("K", [8, 64])
def test_csr_matches_oracle(ctx, D, path, K):
    pts = synth.clustered(300, 30, 4000, D, 0.02, seed=700 + D)
    r = 0.1 * np.sqrt(D / 8.0)
    got = _csr(ctx, pts, r, K, path)
    want = oracle.csr(pts, pts, r, K, query_ids=np.arange(len(pts)))
    _assert_csr_equal(got, want)
    assert got[0][-1] > 0


@pytest.mark.parametrize("path", ["grid", "tc"])
@pytest.mark.parametrize("K", [16, 100, 1024])
def test_csr_rows_beyond_the_lists(ctx, path, K):
    # every point repeated 5x inside tight clusters: degrees far above 32,
    # so rows go through the selection kernel's count and fill passes
    pts = np.repeat(synth.clustered(30, 40, 200, 8, 0.01, seed=701), 5, axis=0)
    got = _csr(ctx, pts, 0.05, K, path)
    want = oracle.csr(pts, pts, 0.05, K, query_ids=np.arange(len(pts)))
    _assert_csr_equal(got, want)
    assert want[3].max() > 32


@pytest.mark.parametrize("D", [10, 12])
@pytest.mark.parametrize("K", [7, 40])
def test_csr_mixed_row_lengths_high_dimensions(ctx, D, K):
    # short rows sorted two at a time next to long and overflowing rows
    pts = synth.mixed_degrees(D, 700 + D)
    got = _csr(ctx, pts, 0.12, K)
    want = oracle.csr(pts, pts, 0.12, K, query_ids=np.arange(len(pts)))
    _assert_csr_equal(got, want)


@pytest.mark.parametrize("path", ["grid", "tc"])
def test_csr_cross_set(ctx, path):
    refs = synth.clustered(200, 25, 3000, 8, 0.03, seed=702)
    qs = synth.clustered(150, 20, 2000, 8, 0.03, seed=703)
    got = _csr(ctx, refs, 0.1, 32, path, queries=qs)
    want = oracle.csr(qs, refs, 0.1, 32)
    _assert_csr_equal(got, want)


def test_csr_empty_inputs_and_no_edges(ctx):
    import torch
    refs = synth.uniform(1000, 3, seed=704)
    g = ctx.build_grid(_t(refs), 0.01)
    off, idx, d2, deg = ctx.query_csr(g, torch.empty((0, 3), dtype=torch.float32, device="cuda"),
                                      0.01, 8, False, "grid", degree=True)
    assert off.cpu().tolist() == [0] and idx.numel() == 0 and deg.numel() == 0
    far = np.full((5, 3), 7.0, np.float32)
    off, idx, d2, deg = ctx.query_csr(g, _t(far), 0.01, 8, False, "grid", degree=True)
    assert off.cpu().tolist() == [0] * 6 and idx.numel() == 0 and deg.cpu().tolist() == [0] * 5
    g.close()


def test_csr_fill_needs_its_count_pass(ctx):
    import ctypes
    import torch
    from paper_2609_31980_gb300 import frnn
    pts = _t(synth.uniform(2000, 3, seed=705))
    g = ctx.build_grid(pts, 0.05)
    # no count pass yet
    assert frnn.frnn_query_csr_fill(ctx.handle, None, None) == -1
    off = torch.empty(len(pts) + 1, dtype=torch.int64, device="cuda")
    ne = ctypes.c_int64(0)
    rc = frnn.frnn_query_csr_count(ctx.handle, g.handle, ctypes.c_void_p(pts.data_ptr()), len(pts),
                                   0.05, 16, frnn.FRNN_SELF_QUERY, ctypes.c_void_p(off.data_ptr()),
                                   None, ctypes.byref(ne))
    assert rc == 0 and ne.value == int(off[-1].item()) > 0
    ctx.query(g, pts, 0.05, 16, True, "grid")       # another call in between
    idx = torch.empty(ne.value, dtype=torch.int32, device="cuda")
    d2 = torch.empty(ne.value, dtype=torch.float32, device="cuda")
    assert frnn.frnn_query_csr_fill(ctx.handle, ctypes.c_void_p(idx.data_ptr()),
                                    ctypes.c_void_p(d2.data_ptr())) == -1
    g.close()


def _sample(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=min(k, n), replace=False))


@pytest.mark.parametrize("path,K", [("grid", 64), ("tc", 64), ("grid", 1024)])
def test_csr_event_300k_x8(ctx, path, K):
    w = synth.config2()
    got = _csr(ctx, w.points, w.r, K, path)
    rows = _sample(len(w.points), 800, 706)
    want = oracle.csr(w.points[rows], w.points, w.r, K, query_ids=rows)
    _assert_csr_equal(got, want, rows)
    # same rows as the dense output of the library, truncated to the counts
    counts, idx, d2 = ctx.self_query(_t(w.points), w.r, min(K, 64), path=path)
    c = counts.cpu().numpy()
    if K <= 64:
        np.testing.assert_array_equal(np.diff(got[0]), c)
        keep = np.arange(K)[None, :] < c[:, None]
        np.testing.assert_array_equal(got[1], idx.cpu().numpy()[keep])
    assert got[0][-1] == np.minimum(got[3], K).sum()


def test_csr_event_500k_x12_k1000(ctx):
    w = synth.config3()
    got = _csr(ctx, w.points, w.r, 1000, "tc")
    rows = _sample(len(w.points), 400, 707)
    want = oracle.csr(w.points[rows], w.points, w.r, 1000, query_ids=rows)
    _assert_csr_equal(got, want, rows)


def test_host_compact_call_matches_oracle_and_reports_capacity(ctx):
    from paper_2609_31980_gb300 import frnn
    pts = synth.clustered(200, 30, 3000, 8, 0.02, seed=720)
    want = oracle.csr(pts, pts, 0.1, 48, query_ids=np.arange(len(pts)))
    off, idx, d2 = ctx.self_query_host_csr(pts, 0.1, 48, "grid")
    np.testing.assert_array_equal(off, want[0])
    np.testing.assert_array_equal(idx, want[1])
    np.testing.assert_array_equal(d2.view(np.uint32), want[2].view(np.uint32))
    # too small a buffer: offsets still written, CAPACITY with the edge count
    import ctypes
    small_i = np.empty(5, np.int32)
    small_d = np.empty(5, np.float32)
    off2 = np.empty(len(pts) + 1, np.int64)
    ne = ctypes.c_int64(0)
    rc = frnn.frnn_self_query_host_csr(ctx.handle, ctypes.c_void_p(pts.ctypes.data), len(pts), 8,
                                       0.1, 48, 0, ctypes.c_void_p(off2.ctypes.data),
                                       ctypes.c_void_p(small_i.ctypes.data),
                                       ctypes.c_void_p(small_d.ctypes.data), 5, ctypes.byref(ne))
    assert rc == frnn.FRNN_ERR_CAPACITY and ne.value == want[0][-1]
    np.testing.assert_array_equal(off2, want[0])
    # the binding retries with a buffer of the right size
    off3, idx3, _ = ctx.self_query_host_csr(pts, 0.1, 48, "grid", (off2, small_i, small_d))
    np.testing.assert_array_equal(idx3, want[1])
    empty = ctx.self_query_host_csr(np.zeros((0, 8), np.float32), 0.1, 48, "grid")
    assert empty[0].tolist() == [0] and len(empty[1]) == 0


def test_host_compact_call_large_capacity_small_budget():
    # the caller's buffers hold N K entries, more than the context's budget
    # allows as device rows: the gather waits for the edge count and sizes
    # the device rows by it (the result is the same); with room, it runs
    # before the count is back, and a capacity just below the count fails
    from paper_2609_31980_gb300 import frnn
    pts = synth.clustered(300, 30, 8000, 8, 0.02, seed=721)
    N, K = len(pts), 1000
    want = oracle.csr(pts, pts, 0.1, K, query_ids=np.arange(N))
    E = int(want[0][-1])
    for budget in (60 * 10 ** 6, 0):
        with frnn.Context(budget_bytes=budget) as c:
            out = (np.empty(N + 1, np.int64), np.empty(N * K, np.int32), np.empty(N * K, np.float32))
            off, idx, d2 = c.self_query_host_csr(pts, 0.1, K, "grid", out)
            np.testing.assert_array_equal(off, want[0])
            np.testing.assert_array_equal(idx, want[1])
            np.testing.assert_array_equal(d2.view(np.uint32), want[2].view(np.uint32))
            import ctypes
            small = (np.empty(N + 1, np.int64), np.empty(E - 1, np.int32), np.empty(E - 1, np.float32))
            ne = ctypes.c_int64(0)
            rc = frnn.frnn_self_query_host_csr(c.handle, ctypes.c_void_p(pts.ctypes.data), N, 8, 0.1,
                                               K, 0, ctypes.c_void_p(small[0].ctypes.data),
                                               ctypes.c_void_p(small[1].ctypes.data),
                                               ctypes.c_void_p(small[2].ctypes.data), E - 1,
                                               ctypes.byref(ne))
            assert rc == frnn.FRNN_ERR_CAPACITY and ne.value == E
            np.testing.assert_array_equal(small[0], want[0])
