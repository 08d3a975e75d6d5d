"""Slab sharding of one large event over several ranks (one GPU each).

The paper evaluates one event on one GPU and names multi-GPU scaling as
future work (Sec. 5).  Queries are independent, so one event too large (or
too slow) for one GPU splits by space: the ranks agree on W equal-width
slabs along one coordinate (a gridded one by default, the last), each point
is owned by the rank of its slab, and each rank also receives every point
within a halo of width rho = r (1 + 2^-10) of its slab (one exchange step,
received into the rank's own memory).  Each rank then self-queries its local
set with the library and keeps the rows of the points it owns: results come
out partitioned by query, with no further communication.

Why the halo suffices: if the float32 contract accepts (x, y), every rounded
squared difference is at most the sum, which is at most fl(r*r), so
|x_a - y_a| <= r (1 + 2^-20) on every coordinate a (the same bound the
grid's roundoff-safe cell edge rests on).  A query owned by slab j lies in
[b_j, b_{j+1}] (up to the float64 rounding of the owner computation, far
below r 2^-10), so all its neighbours lie within rho of that interval and are
present on rank j.

Why the rows equal the single-GPU rows bit for bit: the local set is ordered
by global index, so the local order of any two points is their global order.
Self-exclusion by local index is then self-exclusion by global index, ties in
d2 are broken in the same order, and truncation to K keeps the same entries;
local indices are mapped back through the sorted global indices.

The steps are plain functions over torch tensors (on the GPU in production,
on the CPU in the multi-process tests): slab_plan (destinations and the
owned flag of every local point), the exchange (torch.distributed
all_to_all_single, NCCL or gloo), assemble (the local set in global-index
order), the local query (the library's build + self-query; a test may pass
its own), and remap (owned rows with global indices).  slab_self_query runs
them under torch.distributed.
"""
from __future__ import annotations

import torch

HALO_FACTOR = 1.0 + 2.0 ** -10


def halo_width(r: float, lo: float, hi: float) -> float:
    """rho = r (1 + 2^-10), plus a bound on the float64 rounding of the
    owner computation relative to the coordinates' magnitude."""
    return float(r) * HALO_FACTOR + 2.0 ** -40 * max(abs(lo), abs(hi), 1e-300)


def slab_plan(points: torch.Tensor, gidx: torch.Tensor, axis: int, lo: float, hi: float,
              world: int, r: float):
    """For each destination rank j: (points, global indices, owned-by-j flag)
    of the local points rank j needs: those of its slab [lo + j w, lo + (j+1) w)
    (w = (hi - lo) / world; the last slab closed) and those within the halo.
    Every point is owned by exactly one rank and sent to each rank at most once."""
    x = points[:, axis].to(torch.float64)
    w = (hi - lo) / world
    if w > 0:
        owner = torch.clamp(torch.floor((x - lo) / w), 0, world - 1).to(torch.int64)
    else:
        owner = torch.zeros_like(gidx)
    rho = halo_width(r, lo, hi)
    out = []
    for j in range(world):
        b0 = lo + j * w if j > 0 else float("-inf")
        b1 = lo + (j + 1) * w if j < world - 1 else float("inf")
        need = (owner == j) | ((x >= b0 - rho) & (x <= b1 + rho))
        sel = torch.nonzero(need).squeeze(1)
        out.append((points.index_select(0, sel), gidx.index_select(0, sel),
                    (owner.index_select(0, sel) == j).to(torch.uint8)))
    return out


def assemble(received):
    """The local set from the received parts: points, global indices and the
    owned flag, ordered by global index."""
    pts = torch.cat([p for p, _, _ in received])
    g = torch.cat([i for _, i, _ in received])
    own = torch.cat([o for _, _, o in received])
    order = torch.argsort(g)
    return pts.index_select(0, order), g.index_select(0, order), own.index_select(0, order)


def remap(counts, idx, dist2, g_sorted, owned):
    """Rows of the owned points with global indices (padding stays -1)."""
    rows = torch.nonzero(owned.to(torch.bool)).squeeze(1)
    c = counts.index_select(0, rows)
    i = idx.index_select(0, rows).to(torch.int64)
    gi = torch.where(i >= 0, g_sorted.index_select(0, torch.clamp(i, min=0).reshape(-1)).reshape(i.shape),
                     torch.full_like(i, -1))
    return g_sorted.index_select(0, rows), c, gi, dist2.index_select(0, rows)


def library_query(ctx=None):
    """Local query through the library: build the grid of the local set and
    self-query it (grid path) on the set's CUDA device."""
    def q(pts, r, K):
        from . import frnn
        c = ctx or frnn.Context()
        counts, idx, d2 = c.self_query(pts.contiguous(), r, K, path="grid")
        c.sync()
        return counts, idx, d2
    return q


def _alltoallv(parts, group, dist):
    """Variable-size all-to-all of per-destination tensors (first dimension
    split), through all_to_all_single (NCCL and gloo)."""
    dev = parts[0].device
    send_n = torch.tensor([p.shape[0] for p in parts], dtype=torch.int64, device=dev)
    recv_n = torch.empty_like(send_n)
    dist.all_to_all_single(recv_n, send_n, group=group)
    inner = parts[0].shape[1:]
    width = 1
    for s in inner:
        width *= s
    flat = torch.cat([p.reshape(-1) for p in parts])
    out = torch.empty(int(recv_n.sum().item()) * width, dtype=flat.dtype, device=dev)
    dist.all_to_all_single(out, flat, output_split_sizes=[int(v) * width for v in recv_n.tolist()],
                           input_split_sizes=[int(v) * width for v in send_n.tolist()], group=group)
    sizes = recv_n.tolist()
    chunks, off = [], 0
    for n in sizes:
        chunks.append(out[off * width:(off + n) * width].reshape((n,) + tuple(inner)))
        off += n
    return chunks


def slab_self_query(points: torch.Tensor, gidx: torch.Tensor, r: float, K: int, axis: int = -1,
                    group=None, local_query=None):
    """Self-query of an event whose rows are spread over the ranks of a
    torch.distributed group (any split: this rank holds `points` with
    original indices `gidx`).  Returns this rank's owned rows:
    (global query indices, counts, neighbour global indices [n, K] int64,
    squared distances [n, K]), each row equal to the single-GPU row."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    D = points.shape[1]
    axis = axis % D
    x = points[:, axis]
    big = float("inf")
    mm = torch.tensor([x.min().item() if x.numel() else big, -(x.max().item() if x.numel() else -big)],
                      dtype=torch.float64, device=points.device)
    dist.all_reduce(mm, op=dist.ReduceOp.MIN, group=group)
    lo, hi = float(mm[0]), -float(mm[1])
    if not (lo <= hi):   # an empty event
        lo = hi = 0.0
    plan = slab_plan(points, gidx, axis, lo, hi, world, r)
    pts_r = _alltoallv([p for p, _, _ in plan], group, dist)
    gid_r = _alltoallv([g for _, g, _ in plan], group, dist)
    own_r = _alltoallv([o for _, _, o in plan], group, dist)
    pts, g_sorted, owned = assemble(list(zip(pts_r, gid_r, own_r)))
    query = local_query or library_query()
    counts, idx, d2 = query(pts, r, K)
    return remap(counts, idx, d2, g_sorted, owned)
