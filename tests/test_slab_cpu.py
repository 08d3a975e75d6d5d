"""Slab sharding of one event over ranks (paper_2609_31980_gb300/slab.py), on
CPU ranks with the gloo backend.

Each rank holds an arbitrary block of the event's rows; slab_self_query
exchanges the slab and halo points with all_to_all_single and runs a local
self-query.  Here the local query is the CPU oracle (there is no GPU), so
this checks the partition, the halo and the index bookkeeping: every point
is owned by exactly one rank, and every owned row equals the oracle's row of
the whole event (counts, indices, distance bits), including points placed
exactly on slab boundaries and at the radius across them."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _event(kind):
    sys.path.insert(0, ROOT)
    from paper_2609_31980_gb300 import synth
    if kind == "clustered":
        return synth.clustered(150, 20, 1500, 8, 0.02, seed=950), 0.1, 48
    # points on the boundaries of 2 and 3 equal slabs of [0, 1] along the last
    # coordinate, and partners at the radius and one ulp around it across them
    g = np.random.default_rng(951)
    base = g.uniform(0, 1, size=(1200, 4)).astype(np.float32)
    base[:4, 3] = [0.0, 1.0, 0.0, 1.0]   # fix the extent to [0, 1]
    r = np.float32(0.0625)
    extra = []
    for b in (np.float32(0.5), np.float32(1 / 3), np.float32(2 / 3)):
        for dx in (0.0, r, np.nextafter(r, np.float32(1)), np.nextafter(r, np.float32(0))):
            p = g.uniform(0.2, 0.8, size=4).astype(np.float32)
            p[3] = b
            q = p.copy()
            q[3] = np.float32(b + dx)
            extra += [p, q, p.copy()]   # a duplicate too
            q2 = p.copy()
            q2[3] = np.float32(b - dx)
            extra.append(q2)
    pts = np.concatenate([base, np.array(extra, np.float32)])
    return pts[g.permutation(len(pts))], float(r), 32


def _rank_main(rank, ws, port, kind, out_dir):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import oracle
    from paper_2609_31980_gb300 import slab
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        pts, r, K = _event(kind)
        # this rank's block of the input rows (uneven blocks)
        cuts = np.linspace(0, len(pts), ws + 1).astype(int)
        cuts[1:-1] += 37
        lo, hi = cuts[rank], cuts[rank + 1]
        local = torch.from_numpy(pts[lo:hi].copy())
        gidx = torch.arange(lo, hi, dtype=torch.int64)

        def oracle_query(p, rr, KK):
            c, i, d, _ = oracle.frnn(p.numpy(), p.numpy(), rr, KK,
                                     query_ids=np.arange(len(p), dtype=np.int64))
            return torch.from_numpy(c), torch.from_numpy(i), torch.from_numpy(d)

        q, c, i, d = slab.slab_self_query(local, gidx, r, K, axis=-1, local_query=oracle_query)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), q=q.numpy(), c=c.numpy(), i=i.numpy(),
                 d=d.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,kind", [(2, "clustered"), (3, "clustered"), (2, "boundaries"),
                                     (3, "boundaries")])
def test_slab_rows_equal_whole_event_oracle(tmp_path, ws, kind):
    import torch.multiprocessing as mp
    from oracle import oracle
    port = _free_port()
    mp.start_processes(_rank_main, args=(ws, port, kind, str(tmp_path)), nprocs=ws,
                       start_method="spawn")
    pts, r, K = _event(kind)
    want = oracle.self_query(pts, r, K)
    seen = np.zeros(len(pts), np.int64)
    for rank in range(ws):
        z = np.load(tmp_path / f"r{rank}.npz")
        q = z["q"]
        seen[q] += 1
        np.testing.assert_array_equal(z["c"], want[0][q])
        np.testing.assert_array_equal(z["i"], want[1][q].astype(np.int64))
        np.testing.assert_array_equal(z["d"].view(np.uint32), want[2][q].view(np.uint32))
    assert (seen == 1).all(), "every point is owned by exactly one rank"
    assert want[0].sum() > 0


def test_slab_plan_owner_and_halo():
    # the plan alone: ownership is a partition; a point goes to a rank it does
    # not own only within the halo of that rank's slab
    import torch
    from paper_2609_31980_gb300 import slab
    g = np.random.default_rng(952)
    pts = torch.from_numpy(g.uniform(-1, 1, size=(5000, 3)).astype(np.float32))
    gidx = torch.arange(5000, dtype=torch.int64)
    lo, hi, ws, r = -1.0, 1.0, 4, 0.05
    plan = slab.slab_plan(pts, gidx, 2, lo, hi, ws, r)
    owned = np.concatenate([gi[o.bool()].numpy() for _, gi, o in plan])
    assert np.array_equal(np.sort(owned), np.arange(5000))
    w = (hi - lo) / ws
    rho = slab.halo_width(r, lo, hi)
    for j, (p, gi, o) in enumerate(plan):
        x = p[:, 2].double().numpy()
        guest = ~o.bool().numpy()
        assert ((x[guest] >= lo + j * w - rho) & (x[guest] <= lo + (j + 1) * w + rho)).all()
        assert len(np.unique(gi.numpy())) == len(gi)
