"""Seeded random sequences of calls on one context, every result against the
oracle.

The context keeps state between calls: grids rebuilt in place, the cross-set
query grid, the batch grid and its captured graph, the host-buffer grid and
buffers, the compact-output staging, the row-task pair copies, options and
the autotuner's choices per size class (so that batches mix scans).  A
sequence mixes builds (new and in place), self and cross-set queries on
every path, batches, host-buffer calls (dense and compact), device compact
output and option changes (gridded axes, cell multiple, staging), with sizes,
dimensions and K drawn per call, so that each workspace is reused after
calls of other shapes.  Every row of every result is compared with the
oracle (counts, indices, distance bits)."""
import numpy as np
import pytest

from oracle import oracle
from paper_2609_31980_gb300 import synth

pytestmark = pytest.mark.gpu


def _rows_equal(got, want, what):
    gc, gi, gd = (np.asarray(x) for x in got)
    wc, wi, wd = want[:3]
    assert np.array_equal(gc, wc), f"{what}: counts differ"
    assert np.array_equal(gi, wi), f"{what}: indices differ"
    assert np.array_equal(np.ascontiguousarray(gd).view(np.uint32),
                          np.ascontiguousarray(wd).view(np.uint32)), f"{what}: distances differ"


def _csr_equal(off, idx, d2, want, what):
    off, idx, d2 = (np.asarray(x) for x in (off, idx, d2))
    assert np.array_equal(np.diff(off), want[0]), f"{what}: row lengths differ"
    for q in range(len(want[0])):
        n = want[0][q]
        assert np.array_equal(idx[off[q]: off[q] + n], want[1][q][:n]), f"{what}: row {q}"
        assert np.array_equal(d2[off[q]: off[q] + n].view(np.uint32),
                              want[2][q][:n].view(np.uint32)), f"{what}: row {q} distances"


def _points(g, n, D):
    kind = g.choice(["uniform", "clusters", "duplicates"]) if n >= 50 else "uniform"
    if kind == "uniform":
        return synth.uniform(n, D, seed=int(g.integers(1 << 30)))
    if kind == "clusters":
        nc = max(1, n // 25)
        return synth.clustered(nc, 20, n - nc * 20, D, 0.03, seed=int(g.integers(1 << 30)))
    base = synth.uniform(max(1, n // 3), D, seed=int(g.integers(1 << 30)))
    return np.ascontiguousarray(base[g.integers(0, len(base), size=n)])


@pytest.mark.parametrize("seed", range(12))
def test_random_call_sequences(seed):
    import torch
    from paper_2609_31980_gb300 import frnn
    g = np.random.default_rng(7300 + seed)
    dev = torch.device("cuda")
    with frnn.Context() as ctx:
        grid, grid_pts, grid_r = None, None, None
        for step in range(40):
            op = g.choice(["build", "rebuild", "self", "cross", "batch", "batch", "host",
                           "host_csr", "csr", "option", "tune"])
            D = int(g.choice([2, 3, 5, 8, 9, 12, 16]))
            n = int(g.choice([1, 40, 700, 3000]))
            K = int(g.choice([1, 16, 33, 64]))
            r = float(np.float32(g.choice([0.05, 0.1, 0.2])))
            what = f"seed {seed} step {step} {op} D={D} n={n} K={K} r={r}"
            if op == "tune":
                # tune one size class (the scan, axes, cell multiple, staging
                # or the tensor-core path it picks then serve that class in
                # later calls and batches, next to untuned classes)
                pts = _points(g, n, D)
                path = "grid" if D < 8 else str(g.choice(["grid", "tc", "auto"]))
                ctx.autotune(torch.from_numpy(pts).to(dev), r, K, path=path)
                continue
            if op == "option":
                ctx.set_option(frnn.FRNN_OPT_GRID_NAXES, int(g.choice([0, 0, 3, 4, 5])))
                ctx.set_option(frnn.FRNN_OPT_CELL_MULT, int(g.choice([0, 0, 1, 2, 3])))
                ctx.set_option(frnn.FRNN_OPT_STAGING, int(g.choice([0, 1, 2])))
                continue
            pts = _points(g, n, D)
            if op in ("build", "rebuild") or grid is None:
                if op == "rebuild" and grid is not None and grid_pts.shape[1] == D:
                    # in place: same dimension, at most the grid's points
                    pts = pts[: min(len(pts), len(grid_pts))]
                    grid_pts = np.ascontiguousarray(pts)
                    grid_t = torch.from_numpy(grid_pts).to(dev)
                    grid = ctx.build_grid(grid_t, r, grid=grid)
                else:
                    if grid is not None:
                        grid.close()
                    grid_pts = np.ascontiguousarray(pts)
                    grid_t = torch.from_numpy(grid_pts).to(dev)
                    grid = ctx.build_grid(grid_t, r)
                grid_r = r
                path = "grid" if grid_pts.shape[1] < 8 else str(g.choice(["grid", "tc", "auto"]))
                c, i, d = ctx.query(grid, grid_t, grid_r, K, self_query=True, path=path)
                ctx.sync()
                _rows_equal((c.cpu(), i.cpu(), d.cpu()), oracle.self_query(grid_pts, grid_r, K), what)
            elif op == "self":
                path = "grid" if D < 8 else str(g.choice(["grid", "tc", "auto"]))
                t = torch.from_numpy(pts).to(dev)
                c, i, d = ctx.self_query(t, r, K, path=path)
                ctx.sync()
                _rows_equal((c.cpu(), i.cpu(), d.cpu()), oracle.self_query(pts, r, K), what)
            elif op == "cross":
                refs = grid_pts
                qs = _points(g, n, refs.shape[1])
                path = "grid" if refs.shape[1] < 8 else str(g.choice(["grid", "tc"]))
                c, i, d = ctx.query(grid, torch.from_numpy(qs).to(dev), grid_r, K,
                                    self_query=False, path=path)
                ctx.sync()
                _rows_equal((c.cpu(), i.cpu(), d.cpu()), oracle.frnn(qs, refs, grid_r, K), what)
            elif op == "batch":
                evs = [_points(g, int(g.choice([1, 50, 900, 2500])), D) for _ in range(int(g.integers(1, 5)))]
                outs = ctx.query_batched([torch.from_numpy(e).to(dev) for e in evs], r, K, path="auto")
                ctx.sync()
                for k, (e, (c, i, d)) in enumerate(zip(evs, outs)):
                    _rows_equal((c.cpu(), i.cpu(), d.cpu()), oracle.self_query(e, r, K), f"{what} event {k}")
            elif op == "host":
                _rows_equal(ctx.self_query_host(pts, r, K), oracle.self_query(pts, r, K), what)
            elif op == "host_csr":
                off, idx, d2 = ctx.self_query_host_csr(pts, r, K)
                _csr_equal(off, idx, d2, oracle.self_query(pts, r, K), what)
            else:   # device compact output, self or cross-set on the current grid
                if g.random() < 0.5:
                    off, idx, d2, _ = ctx.query_csr(grid, grid_t, grid_r, K, self_query=True, path="grid")
                    want = oracle.self_query(grid_pts, grid_r, K)
                else:
                    qs = _points(g, n, grid_pts.shape[1])
                    off, idx, d2, _ = ctx.query_csr(grid, torch.from_numpy(qs).to(dev), grid_r, K,
                                                    self_query=False, path="grid")
                    want = oracle.frnn(qs, grid_pts, grid_r, K)
                ctx.sync()
                _csr_equal(off.cpu(), idx.cpu(), d2.cpu(), want, what)
        if grid is not None:
            grid.close()
