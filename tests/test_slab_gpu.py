"""Slab sharding on the GPU: the steps of slab_self_query (plan, exchange,
assemble, local library query, remap) for W ranks run one after another in
one process on one GPU (the exchange is a plain re-routing of the planned
parts; no rank waits on another).  Every owned row equals the single-GPU
library result on every row and the oracle on sampled rows, bit for bit."""
import numpy as np
import pytest

from oracle import oracle
from paper_2609_31980_gb300 import synth

pytestmark = pytest.mark.gpu


def _sharded(frnn, slab, pts, r, K, ws, axis=-1):
    import torch
    t = torch.from_numpy(pts).cuda()
    n = len(pts)
    cuts = np.linspace(0, n, ws + 1).astype(int)
    x = t[:, axis]
    lo, hi = float(x.min()), float(x.max())
    plans = [slab.slab_plan(t[cuts[k]:cuts[k + 1]], torch.arange(cuts[k], cuts[k + 1], device="cuda"),
                            axis % pts.shape[1], lo, hi, ws, r) for k in range(ws)]
    q_all, out = [], []
    with frnn.Context() as ctx:
        for j in range(ws):
            p, g, o = slab.assemble([plans[k][j] for k in range(ws)])
            c, i, d = slab.library_query(ctx)(p, r, K)
            qg, c, i, d = slab.remap(c, i, d, g, o)
            q_all.append(qg.cpu().numpy())
            out.append((c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy()))
    return q_all, out


@pytest.mark.parametrize("ws", [2, 3, 5])
def test_slab_sharded_rows_equal_single_gpu_and_oracle(ws):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2609_31980_gb300 import frnn, slab
    pts = synth.clustered(1000, 30, 12000, 8, 0.02, seed=960)
    r, K = 0.1, 64
    with frnn.Context() as ctx:
        c, i, d = ctx.self_query(torch.from_numpy(pts).cuda(), r, K, path="grid")
        ctx.sync()
        whole = (c.cpu().numpy(), i.cpu().numpy(), d.cpu().numpy())
    q_all, out = _sharded(frnn, slab, pts, r, K, ws)
    seen = np.zeros(len(pts), np.int64)
    sample = np.random.default_rng(961).choice(len(pts), 300, replace=False)
    want_s = oracle.self_query(pts, r, K, rows=np.sort(sample))
    pos = {q: k for k, q in enumerate(np.sort(sample))}
    for q, (c, i, d) in zip(q_all, out):
        seen[q] += 1
        np.testing.assert_array_equal(c, whole[0][q])
        np.testing.assert_array_equal(i, whole[1][q].astype(np.int64))
        np.testing.assert_array_equal(d.view(np.uint32), whole[2][q].view(np.uint32))
        for row, qq in enumerate(q):
            if qq in pos:
                k = pos[qq]
                assert c[row] == want_s[0][k]
                assert np.array_equal(i[row], want_s[1][k])
                assert np.array_equal(d[row].view(np.uint32), want_s[2][k].view(np.uint32))
    assert (seen == 1).all()
