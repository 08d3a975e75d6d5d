"""GPU path vs the CPU oracle, element by element (bit-exact).

Counts and indices must be equal; distances must match to 0 ULP (compared as
bit patterns).  Inputs come from the seeded generators; full-size workloads are
compared on sampled rows (the oracle computes each sampled row by brute force
against all N points), smaller ones on every row.
"""
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


def _gpu_self(ctx, pts, r, K, path="grid"):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
    counts, idx, d2 = ctx.self_query(t, r, K, path=path)
    ctx.sync()
    return counts.cpu().numpy(), idx.cpu().numpy(), d2.cpu().numpy()


def _assert_rows_equal(got, want, rows=None):
    gc, gi, gd = got
    wc, wi, wd = want[:3]
    if rows is not None:
        gc, gi, gd = gc[rows], gi[rows], gd[rows]
    bad = np.flatnonzero((gc != wc) | (gi != wi).any(1) |
                         (gd.view(np.uint32) != wd.view(np.uint32)).any(1))
    if len(bad):
        b = bad[0]
        raise AssertionError(
            f"{len(bad)} rows differ; first row {b if rows is None else rows[b]}: "
            f"count {gc[b]} vs {wc[b]}\n gpu idx {gi[b][:12]}\n ora idx {wi[b][:12]}\n"
            f" gpu d2 {gd[b][:6]}\n ora d2 {wd[b][:6]}")


def _sample_rows(n, k, seed):
    g = np.random.default_rng(seed)
    return np.sort(g.choice(n, size=min(k, n), replace=False))


def test_uniform_4096x3_full(ctx):
    w = synth.config1()
    got = _gpu_self(ctx, w.points, w.r, w.K)
    want = oracle.self_query(w.points, w.r, w.K)
    _assert_rows_equal(got, want)
    assert got[0].sum() > 4000


def test_event_30k_x8_full(ctx):
    pts = synth.clustered(800, 30, 6000, 8, 0.02, seed=21)
    got = _gpu_self(ctx, pts, 0.1, 64)
    want = oracle.self_query(pts, 0.1, 64)
    _assert_rows_equal(got, want)


def test_event_300k_x8_sampled(ctx):
    w = synth.config2()
    got = _gpu_self(ctx, w.points, w.r, w.K)
    rows = _sample_rows(len(w.points), 3000, 22)
    want = oracle.self_query(w.points, w.r, w.K, rows=rows)
    _assert_rows_equal(got, want, rows)
    # symmetry holds at any size: j in N(i) <=> i in N(j) with identical bits
    c, i, d = got
    assert c.max() < w.K
    sel = rows[:200]
    for q in sel:
        for e in range(c[q]):
            j = i[q, e]
            pos = np.flatnonzero(i[j, :c[j]] == q)
            assert len(pos) == 1 and d[j, pos[0]].view(np.uint32) == d[q, e].view(np.uint32)


@pytest.mark.slow
def test_event_300k_x8_every_row(ctx):
    # the benchmark's event at full size, every row against the oracle
    # (about 20 s of brute force on 16 host cores)
    w = synth.config2()
    _assert_rows_equal(_gpu_self(ctx, w.points, w.r, w.K), oracle.self_query(w.points, w.r, w.K))


@pytest.mark.slow
def test_event_500k_x12_every_row_both_paths(ctx):
    # the high-dimensional event at full size, every row, grid and
    # tensor-core paths (about 80 s of brute force on 16 host cores)
    w = synth.config3()
    want = oracle.self_query(w.points, w.r, w.K)
    _assert_rows_equal(_gpu_self(ctx, w.points, w.r, w.K, path="grid"), want)
    _assert_rows_equal(_gpu_self(ctx, w.points, w.r, w.K, path="tc"), want)


def test_event_40k_x12_full(ctx):
    pts = synth.clustered(1280, 25, 8000, 12, 0.025, seed=23)
    got = _gpu_self(ctx, pts, 0.12, 128)
    want = oracle.self_query(pts, 0.12, 128)
    _assert_rows_equal(got, want)


def test_event_500k_x12_sampled(ctx):
    w = synth.config3()
    got = _gpu_self(ctx, w.points, w.r, w.K)
    rows = _sample_rows(len(w.points), 1500, 24)
    want = oracle.self_query(w.points, w.r, w.K, rows=rows)
    _assert_rows_equal(got, want, rows)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 8, 12, 16])
def test_dimensions(ctx, D):
    pts = synth.clustered(60, 20, 300, D, 0.03, seed=100 + D)
    r = 0.08 * np.sqrt(D)
    got = _gpu_self(ctx, pts, r, 48)
    _assert_rows_equal(got, oracle.self_query(pts, r, 48))


@pytest.mark.parametrize("N", [0, 1, 2, 31, 32, 33, 65])
def test_small_sizes(ctx, N):
    pts = synth.uniform(N, 3, seed=200 + N) if N else np.zeros((0, 3), np.float32)
    got = _gpu_self(ctx, pts, 0.4, 8)
    want = oracle.self_query(pts, 0.4, 8)
    _assert_rows_equal(got, want)


@pytest.mark.parametrize("K", [1, 2, 31, 32, 33, 64, 128, 129, 1024])
def test_k_values_with_truncation(ctx, K):
    # dense: degrees well above small K, some above 128
    pts = synth.clustered(10, 150, 200, 3, 0.02, seed=300)
    got = _gpu_self(ctx, pts, 0.05, K)
    want = oracle.self_query(pts, 0.05, K)
    assert (want[3] > K).any() or K >= 1024
    _assert_rows_equal(got, want)


@pytest.mark.parametrize("D", [10, 12])
@pytest.mark.parametrize("K", [1, 7, 16, 17, 40])
def test_mixed_row_lengths_high_dimensions(ctx, D, K):
    # rows of at most 16 entries are sorted two at a time (one per half-warp)
    # from D = 10 on; next to them rows of 17 to 32 entries and rows that the
    # selection kernel finishes, for K below, at and above each length
    pts = synth.mixed_degrees(D, 700 + D)
    want = oracle.self_query(pts, 0.12, K)
    deg = want[3]
    assert (deg <= 16).sum() > 1000 and ((deg > 16) & (deg <= 32)).sum() > 100
    assert (deg > 32).sum() > 100
    _assert_rows_equal(_gpu_self(ctx, pts, 0.12, K), want)


def test_all_points_in_one_cell(ctx):
    pts = synth.uniform(3000, 3, seed=301, lo=0.0, hi=0.01)
    got = _gpu_self(ctx, pts, 0.05, 32)
    _assert_rows_equal(got, oracle.self_query(pts, 0.05, 32))


def test_duplicates(ctx):
    base = synth.uniform(50, 4, seed=302)
    pts = np.repeat(base, 7, axis=0)
    got = _gpu_self(ctx, pts, 0.2, 16)
    _assert_rows_equal(got, oracle.self_query(pts, 0.2, 16))
    assert (got[2][:, 0].view(np.uint32) == 0).all()


def test_points_exactly_at_r_and_on_cell_boundaries(ctx):
    """Integer lattice scaled by 2^-3: many pairs at exactly r, and with
    r = 2 steps the cell edge r(1+2^-10) puts lattice planes near cell edges;
    plus copies shifted by +-1 ulp."""
    side = 9
    g = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pts = (g * 0.125).astype(np.float32)
    up = np.nextafter(pts, np.float32(np.inf))
    dn = np.nextafter(pts, np.float32(-np.inf))
    allp = np.concatenate([pts, up[::3], dn[1::3]]).astype(np.float32)
    perm = np.random.default_rng(303).permutation(len(allp))
    allp = allp[perm]
    for r in (0.25, 0.125, float(np.nextafter(np.float32(0.25), np.float32(0)))):
        got = _gpu_self(ctx, allp, r, 128)
        _assert_rows_equal(got, oracle.self_query(allp, r, 128))


def test_cross_set_queries(ctx):
    import torch
    refs = synth.clustered(200, 20, 2000, 8, 0.03, seed=304)
    qs = np.concatenate([synth.clustered(50, 10, 500, 8, 0.03, seed=305),
                         synth.uniform(100, 8, seed=306, lo=-1.5, hi=1.5)])
    tr = torch.from_numpy(refs).cuda()
    tq = torch.from_numpy(qs).cuda()
    g = ctx.build_grid(tr, 0.15)
    c, i, d = ctx.query(g, tq, 0.15, 40, self_query=False, path="grid")
    ctx.sync()
    got = (c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy())
    _assert_rows_equal(got, oracle.frnn(qs, refs, 0.15, 40))
    # a smaller radius on the same grid
    c, i, d = ctx.query(g, tq, 0.07, 40, self_query=False, path="grid")
    ctx.sync()
    _assert_rows_equal((c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy()),
                       oracle.frnn(qs, refs, 0.07, 40))


@pytest.mark.parametrize("m,axes", [(2, 0), (1, 1), (2, 1)])
def test_grid_options_do_not_change_results(ctx, m, axes):
    from paper_2609_31980_gb300 import frnn
    pts = synth.clustered(300, 30, 3000, 8, 0.02, seed=307)
    want = oracle.self_query(pts, 0.1, 64)
    ctx.set_option(frnn.FRNN_OPT_CELL_MULT, m)
    ctx.set_option(frnn.FRNN_OPT_GRID_AXES, axes)
    try:
        _assert_rows_equal(_gpu_self(ctx, pts, 0.1, 64), want)
    finally:
        ctx.set_option(frnn.FRNN_OPT_CELL_MULT, 0)
        ctx.set_option(frnn.FRNN_OPT_GRID_AXES, 0)


@pytest.mark.parametrize("naxes", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("axes", [0, 1])
def test_gridded_axis_counts_do_not_change_results(ctx, naxes, m, axes):
    from paper_2609_31980_gb300 import frnn
    pts = synth.clustered(200, 30, 2000, 8, 0.02, seed=309)
    want = oracle.self_query(pts, 0.1, 48)
    ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, naxes)
    ctx.set_option(frnn.FRNN_OPT_CELL_MULT, m)
    ctx.set_option(frnn.FRNN_OPT_GRID_AXES, axes)
    try:
        _assert_rows_equal(_gpu_self(ctx, pts, 0.1, 48), want)
    finally:
        ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, 0)
        ctx.set_option(frnn.FRNN_OPT_CELL_MULT, 0)
        ctx.set_option(frnn.FRNN_OPT_GRID_AXES, 0)


@pytest.mark.parametrize("staging", [1, 2])
@pytest.mark.parametrize("D,naxes", [(8, 3), (8, 4), (8, 5), (12, 5), (3, 3)])
def test_staging_modes_match_oracle(ctx, staging, D, naxes):
    # candidate rows loaded by the lanes (1) or bulk-copied into shared memory (2)
    from paper_2609_31980_gb300 import frnn
    pts = synth.clustered(500, 25, 4000, D, 0.025, seed=340 + D)
    r = 0.1 * np.sqrt(D / 8.0)
    ctx.set_option(frnn.FRNN_OPT_STAGING, staging)
    ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, naxes)
    try:
        _assert_rows_equal(_gpu_self(ctx, pts, r, 48), oracle.self_query(pts, r, 48))
    finally:
        ctx.set_option(frnn.FRNN_OPT_STAGING, 0)
        ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, 0)


@pytest.mark.parametrize("which", ["config2", "config3"])
def test_staging_modes_equal_at_full_size(ctx, which):
    # the full 300k x 8 and 500k x 12 events: bulk-copy staging equals the
    # default staging bit for bit on every row (the default is compared with
    # the oracle on every row by the tests above)
    from paper_2609_31980_gb300 import frnn
    w = getattr(synth, which)()
    ref = _gpu_self(ctx, w.points, w.r, w.K)
    ctx.set_option(frnn.FRNN_OPT_STAGING, 2)
    try:
        _assert_rows_equal(_gpu_self(ctx, w.points, w.r, w.K), ref)
    finally:
        ctx.set_option(frnn.FRNN_OPT_STAGING, 0)


def test_grid_params_reports_the_build(ctx):
    # frnn_grid_params: the automatic choice for D = 8 is five axes (chunk
    # scan); from D = 9 four axes (row-task scan); an explicit request is kept
    import torch
    from paper_2609_31980_gb300 import frnn
    cases = ((synth.config2().points, 0.1, 5, "chunks"),
             (synth.clustered(400, 25, 3000, 12, 0.025, seed=345), 0.12, 4, "rows"),
             (synth.uniform(4096, 3, seed=346), 0.05, 3, "chunks"))
    for pts, r, naxes, kernel in cases:
        D = pts.shape[1]
        g = ctx.build_grid(torch.from_numpy(pts).cuda(), r)
        p = g.params()
        assert p["naxes"] == naxes and p["kernel"] == kernel, p
        assert p["cells"] == int(np.prod(p["dims"])) and p["valid"]
        assert p["axes"] == list(range(D - naxes, D))
        g.close()
    ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, 3)
    try:
        g = ctx.build_grid(torch.from_numpy(synth.uniform(2000, 8, seed=346)).cuda(), 0.1)
        p = g.params()
        assert p["naxes"] == 3 and p["kernel"] == "rows" and p["cell_mult"] == 2, p
        g.close()
    finally:
        ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, 0)


def test_five_axes_dense_cells_many_ranges(ctx):
    # every cell of a 4^5 block holds several points: each group of a query
    # chunk has 81 non-empty neighbour rows, so a chunk's groups are served in
    # several batches of candidate ranges, and rows exceed the kernel's list
    # (the selection kernel finishes them)
    from paper_2609_31980_gb300 import frnn
    g = np.random.default_rng(330)
    pts = (g.integers(0, 4, size=(6000, 5)) + g.uniform(0.1, 0.9, size=(6000, 5))).astype(np.float32)
    pts *= np.float32(0.1)
    ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, 5)
    try:
        for K in (16, 200):
            _assert_rows_equal(_gpu_self(ctx, pts, 0.1, K), oracle.self_query(pts, 0.1, K))
    finally:
        ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, 0)


@pytest.mark.parametrize("e", [1, 3, 4, 6])
def test_exit_dims_do_not_change_results(ctx, e):
    from paper_2609_31980_gb300 import frnn
    pts = synth.clustered(300, 30, 3000, 8, 0.02, seed=308)
    want = oracle.self_query(pts, 0.1, 64)
    ctx.set_option(frnn.FRNN_OPT_EXIT_DIMS, e)
    try:
        _assert_rows_equal(_gpu_self(ctx, pts, 0.1, 64), want)
    finally:
        ctx.set_option(frnn.FRNN_OPT_EXIT_DIMS, 0)


def test_grid_rebuild_in_place(ctx):
    import torch
    a = synth.uniform(5000, 3, seed=309)
    b = synth.uniform(3000, 3, seed=310)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    g = ctx.build_grid(ta, 0.05)
    g2 = ctx.build_grid(tb, 0.05, grid=g)
    assert g2 is g
    c, i, d = ctx.query(g, tb, 0.05, 16, self_query=True, path="grid")
    ctx.sync()
    _assert_rows_equal((c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy()),
                       oracle.self_query(b, 0.05, 16))


def test_nonfinite_input_is_reported(ctx):
    import torch
    from paper_2609_31980_gb300 import frnn
    pts = synth.uniform(1000, 3, seed=311)
    pts[17, 1] = np.nan
    t = torch.from_numpy(pts).cuda()
    c, i, d = ctx.self_query(t, 0.05, 8, path="grid")
    with pytest.raises(frnn.FrnnError) as ei:
        ctx.sync()
    assert ei.value.status == -5
    assert (c.cpu().numpy() == 0).all()
    ctx.sync()   # status is cleared


def test_host_buffer_path(ctx):
    w = synth.config1()
    c, i, d = ctx.self_query_host(w.points, w.r, w.K, path="grid")
    _assert_rows_equal((c, i, d), oracle.self_query(w.points, w.r, w.K))


def test_host_buffer_paths_with_page_locked_buffers(ctx):
    # page-locked outputs are written by the kernels directly (no copy back)
    import torch
    pts = synth.clustered(300, 30, 4000, 8, 0.02, seed=330)
    N, K = len(pts), 40
    want = oracle.self_query(pts, 0.1, K)
    h_in = torch.from_numpy(pts).pin_memory()
    out = (torch.full((N,), -7, dtype=torch.int32).pin_memory().numpy(),
           torch.full((N, K), -7, dtype=torch.int32).pin_memory().numpy(),
           torch.zeros((N, K), dtype=torch.float32).pin_memory().numpy())
    got = ctx.self_query_host(h_in.numpy(), 0.1, K, "grid", out)
    _assert_rows_equal(got, want)
    wc = oracle.csr(pts, pts, 0.1, K, query_ids=np.arange(N))
    cap = int(wc[0][-1]) + 5
    c_out = (torch.empty(N + 1, dtype=torch.int64).pin_memory().numpy(),
             torch.empty(cap, dtype=torch.int32).pin_memory().numpy(),
             torch.empty(cap, dtype=torch.float32).pin_memory().numpy())
    off, idx, d2 = ctx.self_query_host_csr(h_in.numpy(), 0.1, K, "grid", c_out)
    np.testing.assert_array_equal(off, wc[0])
    np.testing.assert_array_equal(idx, wc[1])
    np.testing.assert_array_equal(d2.view(np.uint32), wc[2].view(np.uint32))


def test_invalid_arguments(ctx):
    import torch
    from paper_2609_31980_gb300 import frnn
    t = torch.zeros((10, 3), device="cuda")
    g = ctx.build_grid(t, 0.1)
    with pytest.raises(frnn.FrnnError):
        ctx.query(g, t, 0.1, 0)            # K = 0
    with pytest.raises(frnn.FrnnError):
        ctx.query(g, t, 0.1, 2000)         # K too large
    with pytest.raises(frnn.FrnnError):
        ctx.query(g, t, 0.2, 4)            # r above the grid's radius
    with pytest.raises(frnn.FrnnError):
        ctx.query(g, t.clone(), 0.1, 4, self_query=True)   # not the grid's own points
    with pytest.raises(frnn.FrnnError):
        ctx.query(g, t, 0.1, 4, path="tc")  # D < 8
    with pytest.raises(frnn.FrnnError):
        ctx.build_grid(torch.zeros((4, 17), device="cuda"), 0.1)
    ctx.sync()


def test_subnormal_squares_gradual_underflow(ctx):
    """Coordinates near 2^-60: many squared differences are subnormal; both
    sides must keep gradual underflow (no flush to zero)."""
    g = np.random.default_rng(312)
    pts = (g.integers(0, 64, size=(400, 4)) * 2.0 ** -66).astype(np.float32)
    r = float(2.0 ** -60)
    got = _gpu_self(ctx, pts, r, 64)
    want = oracle.self_query(pts, r, 64)
    assert (want[2][want[2] < np.inf] < np.finfo(np.float32).tiny).any()
    _assert_rows_equal(got, want)


def test_batched_equals_alone_and_oracle(ctx):
    import torch
    sizes = [0, 1, 33, 2000, 4097, 15000, 777]
    evs = [synth.event_mix(n, 8, (40, e)) if n else np.zeros((0, 8), np.float32)
           for e, n in enumerate(sizes)]
    tev = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in evs]
    for rep in range(2):   # second call replays the captured graph
        outs = ctx.query_batched(tev, 0.1, 64, path="grid")
        ctx.sync()
        for e, (p, (c, i, d)) in enumerate(zip(evs, outs)):
            got = (c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy())
            alone = _gpu_self(ctx, p, 0.1, 64)
            _assert_rows_equal(got, alone)
            if len(p) and e % 2 == 0:
                _assert_rows_equal(got, oracle.self_query(p, 0.1, 64))


def test_batch_64_uneven_events_full_size(ctx):
    # the batched workload at full size (64 events, N ~ U[50k, 350k], 14.1 M
    # points) in the batched launch the benchmark times.  Every row of every
    # event equals the plain single-event path (compared on the device: counts,
    # indices and distance bits), and per event 256 sampled rows equal the
    # oracle's brute force over that event
    import torch
    w = synth.config4()
    evs = [torch.from_numpy(p).cuda() for p in w.events]
    outs = ctx.query_batched(evs, w.r, w.K, path="grid")
    ctx.sync()
    grid = None
    for e, (p, t, (c, i, d)) in enumerate(zip(w.events, evs, outs)):
        grid = ctx.build_grid(t, w.r, grid=grid)
        pc, pi, pd = ctx.query(grid, t, w.r, w.K, True, "grid")
        ctx.sync()
        assert torch.equal(c, pc), f"event {e}: batched counts differ from the plain path"
        assert torch.equal(i, pi), f"event {e}: batched indices differ from the plain path"
        assert torch.equal(d.view(torch.int32), pd.view(torch.int32)), \
            f"event {e}: batched distances differ from the plain path"
        del pc, pi, pd
        rows = _sample_rows(len(p), 256, 900 + e)
        rt = torch.from_numpy(rows).cuda()
        got = (c[rt].cpu().numpy(), i[rt].cpu().numpy(), d[rt].cpu().numpy())
        _assert_rows_equal(got, oracle.self_query(p, w.r, w.K, rows=rows))
    grid.close()


def test_batched_many_events_long_cell_scan(ctx):
    # 70 events: over 1.1 M cell entries, so the build's scans take the path
    # that scans the block partials in a separate pass
    import torch
    g = np.random.default_rng(41)
    sizes = g.integers(50, 3000, size=70)
    evs = [synth.event_mix(int(n), 8, (41, e)) for e, n in enumerate(sizes)]
    outs = ctx.query_batched([torch.from_numpy(p).cuda() for p in evs], 0.1, 32, path="grid")
    ctx.sync()
    for e, (p, (c, i, d)) in enumerate(zip(evs, outs)):
        got = (c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy())
        if e % 7 == 0:
            _assert_rows_equal(got, oracle.self_query(p, 0.1, 32))
        else:
            _assert_rows_equal(got, _gpu_self(ctx, p, 0.1, 32))


def test_single_event_2_5m_points_long_cell_scan(ctx):
    pts = synth.uniform(2_500_000, 3, seed=42)
    got = _gpu_self(ctx, pts, 0.004, 16)
    rows = _sample_rows(len(pts), 200, 43)
    _assert_rows_equal(got, oracle.self_query(pts, 0.004, 16, rows=rows), rows)
    assert got[0].sum() > 0


# ------------------------------------------------------------ tensor-core path

@pytest.mark.parametrize("D", [8, 9, 11, 12, 16])
def test_tc_path_matches_oracle(ctx, D):
    pts = synth.clustered(400, 25, 3000, D, 0.025, seed=500 + D)
    r = 0.1 * np.sqrt(D / 8.0)
    got = _gpu_self(ctx, pts, r, 64, path="tc")
    _assert_rows_equal(got, oracle.self_query(pts, r, 64))


def test_tc_path_event_300k_x8_sampled_and_equal_to_grid(ctx):
    w = synth.config2()
    tc = _gpu_self(ctx, w.points, w.r, w.K, path="tc")
    grid = _gpu_self(ctx, w.points, w.r, w.K, path="grid")
    _assert_rows_equal(tc, grid)
    rows = _sample_rows(len(w.points), 1000, 25)
    _assert_rows_equal(tc, oracle.self_query(w.points, w.r, w.K, rows=rows), rows)


def test_tc_path_event_500k_x12_equal_to_grid(ctx):
    from paper_2609_31980_gb300 import frnn
    w = synth.config3()
    ctx.set_option(frnn.FRNN_OPT_TC_SURVIVORS, 0)
    tc = _gpu_self(ctx, w.points, w.r, w.K, path="tc")
    surv = ctx.get_option(frnn.FRNN_OPT_TC_SURVIVORS)
    acc = ctx.get_option(frnn.FRNN_OPT_TC_ACCEPTED)
    grid = _gpu_self(ctx, w.points, w.r, w.K, path="grid")
    _assert_rows_equal(tc, grid)
    assert acc == int(grid[0].sum()) and surv >= acc
    rows = _sample_rows(len(w.points), 800, 26)
    _assert_rows_equal(tc, oracle.self_query(w.points, w.r, w.K, rows=rows), rows)


@pytest.mark.parametrize("path", ["grid", "tc"])
def test_kernel_timing_records_one_duration_per_query(ctx, path):
    import time
    import torch
    from paper_2609_31980_gb300 import frnn
    pts = torch.from_numpy(synth.clustered(300, 40, 20000, 8, 0.02, seed=510)).cuda()
    K = 32
    counts = torch.empty(len(pts), dtype=torch.int32, device="cuda")
    idx = torch.empty((len(pts), K), dtype=torch.int32, device="cuda")
    d2 = torch.empty((len(pts), K), dtype=torch.float32, device="cuda")
    grid = ctx.build_grid(pts, 0.1)
    ctx.set_option(frnn.FRNN_OPT_KERNEL_TIMING, 1)
    assert ctx.get_option(frnn.FRNN_OPT_KERNEL_TIMING) == 1
    ctx.query(grid, pts, 0.1, K, True, path, (counts, idx, d2))
    ctx.sync()
    t0 = time.perf_counter()
    for _ in range(3):
        ctx.query(grid, pts, 0.1, K, True, path, (counts, idx, d2))
    ctx.sync()
    wall_ms = (time.perf_counter() - t0) * 1e3
    ms = ctx.kernel_times()
    assert len(ms) == 4 and all(0.0 < t for t in ms) and sum(ms[1:]) <= wall_ms
    assert ctx.kernel_times() == []           # the read clears the record
    ctx.set_option(frnn.FRNN_OPT_KERNEL_TIMING, 0)
    ctx.query(grid, pts, 0.1, K, True, path, (counts, idx, d2))
    assert ctx.kernel_times() == []
    grid.close()


def test_tc_path_dense_and_duplicates(ctx):
    pts = np.repeat(synth.clustered(20, 40, 100, 8, 0.01, seed=502), 3, axis=0)
    for K in (8, 32, 100):
        got = _gpu_self(ctx, pts, 0.05, K, path="tc")
        _assert_rows_equal(got, oracle.self_query(pts, 0.05, K))


def test_tc_path_cross_set_and_small_sizes(ctx):
    import torch
    refs = synth.clustered(100, 20, 1000, 8, 0.03, seed=503)
    qs = np.concatenate([synth.clustered(30, 10, 300, 8, 0.03, seed=504),
                         synth.uniform(50, 8, seed=505, lo=-1.5, hi=1.5)])
    g = ctx.build_grid(torch.from_numpy(refs).cuda(), 0.15)
    c, i, d = ctx.query(g, torch.from_numpy(qs).cuda(), 0.15, 40, self_query=False, path="tc")
    ctx.sync()
    _assert_rows_equal((c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy()),
                       oracle.frnn(qs, refs, 0.15, 40))
    for n in (1, 2, 7, 9, 129, 300):
        pts = synth.uniform(n, 8, seed=506 + n) * np.float32(0.3)
        _assert_rows_equal(_gpu_self(ctx, pts, 0.2, 16, path="tc"), oracle.self_query(pts, 0.2, 16))


def test_tc_path_batched_equals_alone(ctx):
    import torch
    sizes = [3000, 1, 0, 5001, 129]
    evs = [synth.event_mix(n, 8, (41, e)) if n else np.zeros((0, 8), np.float32)
           for e, n in enumerate(sizes)]
    tev = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in evs]
    for rep in range(2):
        outs = ctx.query_batched(tev, 0.1, 64, path="tc")
        ctx.sync()
        for p, (c, i, d) in zip(evs, outs):
            got = (c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy())
            _assert_rows_equal(got, _gpu_self(ctx, p, 0.1, 64, path="grid"))


# ------------------------------------------------------------ autotuner

def test_autotune_and_mixed_path_batches(ctx):
    """Tune one size class to the tensor-core path and another to the grid
    path; a batch holding both classes runs one launch per path inside its
    graph, and every event equals its single-event result."""
    import torch
    from paper_2609_31980_gb300 import frnn
    small = synth.event_mix(3000, 8, (42, 0))
    large = synth.event_mix(9000, 8, (42, 1))
    ts, tl = torch.from_numpy(small).cuda(), torch.from_numpy(large).cuda()
    try:
        a = ctx.autotune(ts, 0.1, 64, path="tc")
        b = ctx.autotune(tl, 0.1, 64, path="grid")
        assert a["path"] == "tc" and b["path"] == "grid"
        assert a["cell_mult"] in (1, 2) and a["ms"] > 0
        evs = [small, large, synth.event_mix(2500, 8, (42, 2)), synth.event_mix(12000, 8, (42, 3))]
        tev = [torch.from_numpy(p).cuda() for p in evs]
        wants = [oracle.self_query(p, 0.1, 64) for p in evs]
        for rep in range(2):
            outs = ctx.query_batched(tev, 0.1, 64, path="auto")
            ctx.sync()
            for p, want, (c, i, d) in zip(evs, wants, outs):
                got = (c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy())
                _assert_rows_equal(got, _gpu_self(ctx, p, 0.1, 64, path="grid"))
                _assert_rows_equal(got, want)
        # auto single-event queries follow the tuned class and stay exact
        _assert_rows_equal(_gpu_self(ctx, small, 0.1, 64, path="auto"),
                           oracle.self_query(small, 0.1, 64))
    finally:
        ctx.set_option(frnn.FRNN_OPT_AUTOTUNE, 0)
        ctx.set_option(frnn.FRNN_OPT_AUTOTUNE, 1)


@pytest.mark.parametrize("D,m,r", [(2, 3, 0.03), (3, 2, 0.08), (3, 3, 0.08), (4, 2, 0.15)])
def test_fine_cells_on_automatic_axes(ctx, D, m, r):
    """Cells of r/2 and r/3 on the automatic axis choice at low D: the chunk
    scan's table holds the (2m + 1)^(axes - 1) neighbour rows (up to 125),
    so the grid keeps m, and the rows equal the oracle's."""
    import torch
    from paper_2609_31980_gb300 import frnn
    pts = synth.uniform(6000, D, seed=990 + 10 * D + m)
    ctx.set_option(frnn.FRNN_OPT_CELL_MULT, m)
    try:
        g = ctx.build_grid(torch.from_numpy(pts).cuda(), r)
        p = g.params()
        assert p["kernel"] == "chunks" and p["cell_mult"] == m, p
        g.close()
        _assert_rows_equal(_gpu_self(ctx, pts, r, 32), oracle.self_query(pts, r, 32))
    finally:
        ctx.set_option(frnn.FRNN_OPT_CELL_MULT, 0)


def test_autotune_low_dimension_tries_finer_cells(ctx):
    """At D = 3 the tuner also times cells of r/2 and r/3 on the automatic
    axes; whatever it picks, tuned single and batched queries stay exact."""
    import torch
    from paper_2609_31980_gb300 import frnn
    pts = synth.uniform(20000, 3, seed=995)
    try:
        a = ctx.autotune(torch.from_numpy(pts).cuda(), 0.05, 48, path="grid")
        assert a["path"] == "grid" and a["cell_mult"] in (1, 2, 3) and a["ms"] > 0, a
        want = oracle.self_query(pts, 0.05, 48)
        _assert_rows_equal(_gpu_self(ctx, pts, 0.05, 48, path="auto"), want)
        outs = ctx.query_batched([torch.from_numpy(pts).cuda()], 0.05, 48, path="auto")
        ctx.sync()
        c, i, d = outs[0]
        _assert_rows_equal((c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy()), want)
    finally:
        ctx.set_option(frnn.FRNN_OPT_AUTOTUNE, 0)
        ctx.set_option(frnn.FRNN_OPT_AUTOTUNE, 1)


# ------------------------------------------------------------ serving loop

def test_serving_results_equal_alone_and_overlap(ctx):
    """Continuous batching: requests arriving while others run are admitted
    as slots free up; every result equals the single-event result bit for
    bit, and batches overlapped on the device."""
    import torch
    g = np.random.default_rng(600)
    sizes = g.integers(500, 12000, size=40)
    events = [synth.event_mix(int(n), 8, (60, e)) for e, n in enumerate(sizes)]
    arrivals = np.cumsum(g.exponential(2e-4, size=len(events)))
    outs, lat, st = ctx.serve(events, arrivals, 0.1, 64, budget_bytes=2 * 10 ** 9, slots=4,
                              max_batch=6)
    assert st["completed"] == len(events) and st["rejected"] == 0
    assert np.all(lat > 0) and st["p99_ms"] >= st["p50_ms"] > 0
    assert st["peak_inflight_batches"] >= 2
    for e, (p, (c, i, d)) in enumerate(zip(events, outs)):
        _assert_rows_equal((c, i, d), _gpu_self(ctx, p, 0.1, 64, path="grid"))
        if e % 5 == 0:   # a seeded subset against the oracle, every row
            _assert_rows_equal((c, i, d), oracle.self_query(p, 0.1, 64))
    # a small budget serialises the same stream (no request fits twice)
    big = max(sizes)
    outs2, lat2, st2 = ctx.serve(events[:8], arrivals[:8], 0.1, 64,
                                 budget_bytes=int(big * (8 * 4 + 4 + 64 * 8) * 3.5), slots=4,
                                 max_batch=6)
    assert st2["completed"] == 8
    for e, (p, (c, i, d)) in enumerate(zip(events[:8], outs2)):
        _assert_rows_equal((c, i, d), _gpu_self(ctx, p, 0.1, 64, path="grid"))
        if e % 3 == 0:
            _assert_rows_equal((c, i, d), oracle.self_query(p, 0.1, 64))


def test_serving_rejects_oversized_request(ctx):
    from paper_2609_31980_gb300 import frnn
    events = [synth.event_mix(2000, 8, (61, e)) for e in range(3)]
    with pytest.raises(frnn.FrnnError) as ei:
        ctx.serve(events, [0.0, 0.0, 0.0], 0.1, 64, budget_bytes=1000, slots=2, max_batch=2)
    assert ei.value.status == -4


# ---------------------------------------------------------------- 4 gridded axes

@pytest.fixture
def ctx4(ctx):
    from paper_2609_31980_gb300 import frnn
    ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, 4)
    yield ctx
    ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, 0)


@pytest.mark.parametrize("D,path", [(4, "grid"), (5, "grid"), (8, "grid"), (8, "tc"), (12, "tc"),
                                    (12, "grid")])
def test_four_axes_match_oracle(ctx4, D, path):
    pts = synth.clustered(400, 25, 3000, D, 0.025, seed=800 + D)
    r = 0.1 * np.sqrt(D / 8.0)
    got = _gpu_self(ctx4, pts, r, 48, path=path)
    _assert_rows_equal(got, oracle.self_query(pts, r, 48))


def test_four_axes_with_m2_request_and_dense_rows(ctx4):
    from paper_2609_31980_gb300 import frnn
    ctx4.set_option(frnn.FRNN_OPT_CELL_MULT, 2)   # falls back to m = 1 (27 neighbour rows)
    try:
        pts = np.repeat(synth.clustered(25, 40, 300, 6, 0.01, seed=810), 3, axis=0)
        for K in (8, 100):
            _assert_rows_equal(_gpu_self(ctx4, pts, 0.05, K), oracle.self_query(pts, 0.05, K))
    finally:
        ctx4.set_option(frnn.FRNN_OPT_CELL_MULT, 0)


def test_four_axes_lattice_boundaries(ctx4):
    # points exactly on and one ulp around cell boundaries in every coordinate
    g = np.arange(-3, 4, dtype=np.float32) * np.float32(0.125)
    base = np.stack(np.meshgrid(g, g, g, g, indexing="ij"), -1).reshape(-1, 4)
    jit = np.stack([np.nextafter(base, np.float32(np.inf)), np.nextafter(base, np.float32(-np.inf))])
    pts = np.concatenate([base, jit.reshape(-1, 4)]).astype(np.float32)
    got = _gpu_self(ctx4, pts, 0.125, 96)
    _assert_rows_equal(got, oracle.self_query(pts, 0.125, 96))


@pytest.mark.parametrize("path", ["grid", "tc"])
def test_four_axes_cross_set(ctx4, path):
    import torch
    refs = synth.clustered(100, 20, 1500, 8, 0.03, seed=811)
    qs = synth.clustered(80, 20, 1000, 8, 0.03, seed=812)
    g = ctx4.build_grid(torch.from_numpy(refs).cuda(), 0.1)
    c, i, d = ctx4.query(g, torch.from_numpy(qs).cuda(), 0.1, 32, False, path)
    ctx4.sync()
    _assert_rows_equal((c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy()),
                       oracle.frnn(qs, refs, 0.1, 32))
    g.close()


def test_four_axes_batched(ctx4):
    import torch
    evs = [synth.clustered(50 + 10 * e, 20, 500 + 100 * e, 8, 0.02, seed=(813, e)) for e in range(5)]
    outs = ctx4.query_batched([torch.from_numpy(p).cuda() for p in evs], 0.1, 32, path="grid")
    ctx4.sync()
    for p, (c, i, d) in zip(evs, outs):
        _assert_rows_equal((c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy()),
                           oracle.self_query(p, 0.1, 32))


@pytest.mark.parametrize("path", ["grid", "tc"])
def test_four_axes_event_500k_x12_equal_to_three_axes(ctx, path):
    from paper_2609_31980_gb300 import frnn
    w = synth.config3()
    ref = _gpu_self(ctx, w.points, w.r, w.K, path=path)
    ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, 4)
    try:
        got = _gpu_self(ctx, w.points, w.r, w.K, path=path)
    finally:
        ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, 0)
    _assert_rows_equal(got, ref)
    rows = _sample_rows(len(w.points), 300, 814)
    _assert_rows_equal(got, oracle.self_query(w.points, w.r, w.K, rows=rows), rows)


# ------------------------------------------------------------ randomized sweep

def _random_case(g):
    """One seeded configuration: size, dimension, shape of the data, scale and
    offset of the coordinates, radius relative to the spacing, K."""
    N = int(g.choice([1, 2, 3, 17, 100, 777, 2048, 5000]))
    D = int(g.integers(1, 17))
    kind = g.choice(["uniform", "clusters", "lattice", "duplicates", "line"])
    if kind == "uniform":
        x = g.uniform(-1, 1, size=(N, D))
    elif kind == "clusters":
        c = g.uniform(-1, 1, size=(max(1, N // 20), D))
        x = c[g.integers(0, len(c), size=N)] + g.normal(0, 0.03, size=(N, D))
    elif kind == "lattice":
        x = g.integers(0, 6, size=(N, D)) * 0.125
    elif kind == "duplicates":
        base = g.uniform(-1, 1, size=(max(1, N // 4), D))
        x = base[g.integers(0, len(base), size=N)]
    else:   # points on a line: one long axis, the others constant
        x = np.zeros((N, D))
        x[:, int(g.integers(0, D))] = g.uniform(-3, 3, size=N)
    scale = float(g.choice([1e-3, 1.0, 37.0]))
    offset = float(g.choice([0.0, 1.0, -250.0, 1e4]))
    pts = (x * scale + offset).astype(np.float32)
    spacing = scale * (2.0 / max(N, 1) ** (1.0 / D))
    r = float(np.float32(spacing * g.choice([0.3, 1.0, 2.5, 6.0])))
    if kind == "lattice":
        r = float(np.float32(0.125 * scale * g.choice([1, 2])))   # exactly on lattice distances
    K = int(g.choice([1, 5, 32, 33, 100, 200]))
    return pts, max(r, 1e-6), K, kind


@pytest.mark.parametrize("seed", range(24))
def test_random_configurations_match_oracle(ctx, seed):
    # every row of a seeded random configuration, through the default path
    # and the grid path, against the oracle; plus cross-set queries drawn
    # from the same recipe
    import torch
    g = np.random.default_rng(7000 + seed)
    pts, r, K, kind = _random_case(g)
    want = oracle.self_query(pts, r, K)
    for path in ("auto", "grid"):
        _assert_rows_equal(_gpu_self(ctx, pts, r, K, path=path), want)
    if len(pts) >= 2:
        qs = pts[g.permutation(len(pts))[: max(1, len(pts) // 3)]].copy()
        qs += np.float32(r * 0.5) * g.standard_normal(qs.shape).astype(np.float32)
        gr = ctx.build_grid(torch.from_numpy(pts).cuda(), r)
        c, i, d = ctx.query(gr, torch.from_numpy(qs).cuda(), r, K, self_query=False, path="grid")
        ctx.sync()
        _assert_rows_equal((c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy()),
                           oracle.frnn(qs, pts, r, K))
        gr.close()


def test_random_batches_match_oracle(ctx):
    # batches of random events of mixed sizes and shapes (one D per batch)
    import torch
    g = np.random.default_rng(7100)
    for rep in range(4):
        D = int(g.integers(1, 17))
        evs, rs = [], []
        while len(evs) < 6:
            pts, r, K, kind = _random_case(g)
            if pts.shape[1] != D:
                pts = np.ascontiguousarray(
                    np.resize(pts, (pts.shape[0], D)).astype(np.float32))
            evs.append(pts)
        r = float(np.float32(0.1 * float(np.std(np.concatenate(evs))) + 1e-3))
        K = int(g.choice([8, 64]))
        outs = ctx.query_batched([torch.from_numpy(p).cuda() for p in evs], r, K, path="auto")
        ctx.sync()
        for p, (c, i, d) in zip(evs, outs):
            _assert_rows_equal((c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy()),
                               oracle.self_query(p, r, K))


# ------------------------------------------------------------ workspaces reused across dimensions

def test_context_workspaces_reused_across_dimensions():
    # the context keeps workspaces between calls (the cross-set query grid,
    # the batch grid, the host-buffer grid and the row-task pair copy); a call
    # of a higher dimension with fewer points must not reuse rows carved for a
    # lower one
    import torch
    from paper_2609_31980_gb300 import frnn
    g = np.random.default_rng(7200)
    with frnn.Context() as c:
        for D, n, path in ((3, 20000, "grid"), (16, 3000, "grid"), (4, 12000, "grid"),
                           (12, 2500, "grid"), (2, 9000, "grid"), (15, 1666, "grid")):
            refs = synth.clustered(max(1, n // 30), 25, n - (n // 30) * 25, D, 0.03,
                                   seed=int(g.integers(1 << 30)))
            qs = (refs[g.permutation(len(refs))[: len(refs) // 3]] +
                  np.float32(0.02) * g.standard_normal((len(refs) // 3, D)).astype(np.float32))
            qs = np.ascontiguousarray(qs, np.float32)
            r, K = 0.15, 33
            gr = c.build_grid(torch.from_numpy(refs).cuda(), r)
            cc, ii, dd = c.query(gr, torch.from_numpy(qs).cuda(), r, K, self_query=False, path=path)
            c.sync()
            _assert_rows_equal((cc.cpu().numpy(), ii.cpu().numpy(), dd.cpu().numpy()),
                               oracle.frnn(qs, refs, r, K))
            gr.close()
            # batched: the context's batch grid
            evs = [refs[: len(refs) // 2], refs[len(refs) // 2:]]
            outs = c.query_batched([torch.from_numpy(np.ascontiguousarray(e)).cuda() for e in evs],
                                   r, K, path="auto")
            c.sync()
            for e, (bc, bi, bd) in zip(evs, outs):
                _assert_rows_equal((bc.cpu().numpy(), bi.cpu().numpy(), bd.cpu().numpy()),
                                   oracle.self_query(np.ascontiguousarray(e), r, K))
            # host buffers: the context's host-path grid, dense and compact
            want = oracle.self_query(refs, r, K)
            _assert_rows_equal(c.self_query_host(refs, r, K), want)
            off, idx, d2 = c.self_query_host_csr(refs, r, K)
            assert np.array_equal(np.diff(off), want[0])
            for row in range(0, len(refs), 97):
                n_row = want[0][row]
                assert np.array_equal(idx[off[row]: off[row] + n_row], want[1][row][:n_row])
                assert np.array_equal(d2[off[row]: off[row] + n_row].view(np.uint32),
                                      want[2][row][:n_row].view(np.uint32))


def test_extreme_coordinates(ctx):
    # extents that overflow float32 (the parameter step falls back to fewer
    # or one cell), huge offsets, tiny scales near the subnormal range, and
    # radii at the edges of the accepted range: every row against the oracle
    g = np.random.default_rng(7400)
    cases = []
    x = g.uniform(-3e38, 3e38, size=(600, 4)).astype(np.float32)          # hi - lo overflows
    x[300:] = x[:300]                                                      # duplicates: pairs at 0
    cases.append((x, float(np.float32(2.0 ** 60)), 16))                   # the largest radius
    x = (g.uniform(-1, 1, size=(800, 6)) * 1e3 + 1e30).astype(np.float32)  # offset swamps the spread
    cases.append((x, float(np.float32(1e18)), 16))
    x = (g.uniform(-1, 1, size=(800, 5)) * 1e-17).astype(np.float32)      # squares near the subnormals
    cases.append((x, float(np.float32(3e-18)), 16))
    x = g.uniform(-1, 1, size=(500, 3)).astype(np.float32)
    cases.append((x, float(np.float32(2.0 ** 59)), 8))                     # every pair within r
    cases.append((x, float(np.float32(2.0 ** -59)), 8))                    # no pair within r
    for pts, r, K in cases:
        want = oracle.self_query(pts, r, K)
        for path in ("grid", "auto"):
            _assert_rows_equal(_gpu_self(ctx, pts, r, K, path=path), want)
