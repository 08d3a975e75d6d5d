"""Seeded synthetic point sets shaped like the paper's tracking events.

This module holds input generators only: no distance, grid or neighbour
arithmetic.  Both the CUDA path's tests and the oracle's tests draw their inputs
from here, so the two sides see the same points.

The paper's real event (271,663 points, D=12, r=0.12, K=1000; Sec. 4.1) is not
available, so the workloads below stand in for it: clusters of points around
uniformly placed centres (track-like groups in the embedding space) plus a
uniform background.  Draws are float64 from NumPy's PCG64, cast to float32,
and the point order is shuffled so that an index says nothing about position.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n: int, d: int, seed, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """``n`` points uniform in ``[lo, hi)^d`` as float32 [n, d]."""
    g = _rng(seed)
    return g.uniform(lo, hi, size=(n, d)).astype(np.float32)


def clustered(n_clusters: int, per_cluster: int, n_background: int, d: int,
              sigma: float, seed, box: float = 1.0) -> np.ndarray:
    """Gaussian clusters plus uniform background, shuffled, float32 [n, d].

    Cluster centres are uniform in ``[-box, box]^d``; each cluster has
    ``per_cluster`` points with independent N(0, sigma^2) offsets per
    coordinate (not clipped).  The background is uniform in ``[-box, box]^d``.
    """
    g = _rng(seed)
    centres = g.uniform(-box, box, size=(n_clusters, d))
    pts = np.repeat(centres, per_cluster, axis=0)
    pts += g.normal(0.0, sigma, size=pts.shape)
    bg = g.uniform(-box, box, size=(n_background, d))
    allp = np.concatenate([pts, bg], axis=0)
    # rows in the order of a Fisher-Yates permutation: the same points and
    # generator state as shuffling the rows in place, about ten times faster
    return allp[g.permutation(len(allp))].astype(np.float32)


def mixed_degrees(d: int, seed, sigma: float = 0.025) -> np.ndarray:
    """2,500 points: 60 clusters of 8, 40 of 20 and 12 of 60 points plus 500
    uniform background points in ``[-1, 1]^d``, shuffled.  At r = 0.12 and
    d = 10 or 12 a query has a few, about ten, or 30 to 60 neighbours (or
    none), so all row lengths a warp handles occur side by side."""
    parts = [clustered(nc, pc, 0, d, sigma, seed=(seed, pc)) for nc, pc in ((60, 8), (40, 20), (12, 60))]
    parts.append(uniform(500, d, seed=(seed, 0), lo=-1.0, hi=1.0))
    pts = np.concatenate(parts)
    return pts[_rng((seed, 1)).permutation(len(pts))]


def event_mix(n: int, d: int, seed, per_cluster: int = 30, frac_clustered: float = 0.8,
              sigma: float = 0.02) -> np.ndarray:
    """One tracking-event-shaped set of ``n`` points: ``frac_clustered`` of
    them in clusters of ``per_cluster`` points, the rest uniform background."""
    n_clusters = int(round(frac_clustered * n / per_cluster))
    n_bg = n - n_clusters * per_cluster
    return clustered(n_clusters, per_cluster, n_bg, d, sigma, seed)


@dataclass
class Workload:
    name: str
    r: float
    K: int
    D: int
    events: list = field(default_factory=list)   # list of float32 [N_e, D]
    arrivals: np.ndarray | None = None           # serving: arrival times (s)
    description: str = ""

    @property
    def points(self) -> np.ndarray:
        return self.events[0]


def config1() -> Workload:
    """4096 points uniform in [0,1)^3, r=0.05, K=32, self-query."""
    return Workload("uniform-4096x3-r0.05-k32", 0.05, 32, 3, [uniform(4096, 3, 1)],
                    description="N=4096, D=3, uniform [0,1)^3, r=0.05, K=32")


def config2(n_clusters: int = 8000, per_cluster: int = 30, n_bg: int = 60000) -> Workload:
    """300k points in D=8: 8000 clusters x 30 (sigma 0.02) + 60k background."""
    pts = clustered(n_clusters, per_cluster, n_bg, 8, 0.02, 2)
    n = pts.shape[0]
    return Workload(f"event-{n}x8-r0.1-k64", 0.1, 64, 8, [pts],
                    description=f"N={n}, D=8, {n_clusters}x{per_cluster} clusters sigma 0.02 "
                                f"+ {n_bg} uniform in [-1,1]^8, r=0.1, K=64")


def config3(n_clusters: int = 16000, per_cluster: int = 25, n_bg: int = 100000) -> Workload:
    """500k points in D=12: 16000 clusters x 25 (sigma 0.025) + 100k background."""
    pts = clustered(n_clusters, per_cluster, n_bg, 12, 0.025, 3)
    n = pts.shape[0]
    return Workload(f"event-{n}x12-r0.12-k128", 0.12, 128, 12, [pts],
                    description=f"N={n}, D=12, {n_clusters}x{per_cluster} clusters sigma 0.025 "
                                f"+ {n_bg} uniform in [-1,1]^12, r=0.12, K=128")


def batch_sizes(n_events: int = 64, lo: int = 50_000, hi: int = 350_000, seed=4) -> np.ndarray:
    """Event sizes drawn uniformly from [lo, hi] (integers)."""
    return _rng(seed).integers(lo, hi + 1, size=n_events)


def config4(n_events: int = 64, lo: int = 50_000, hi: int = 350_000, scale: float = 1.0) -> Workload:
    """64 uneven events, N ~ U[50k, 350k], each mixed as in the 300k event."""
    sizes = batch_sizes(n_events, lo, hi)
    sizes = np.maximum((sizes * scale).astype(np.int64), 1)
    ev = [event_mix(int(n), 8, (4, e)) for e, n in enumerate(sizes)]
    return Workload(f"batch-{n_events}ev-U{lo//1000}k-{hi//1000}k-x8-r0.1-k64", 0.1, 64, 8, ev,
                    description=f"{n_events} events, N~U[{lo},{hi}] (seed 4), D=8, mix as the "
                                f"300k event, r=0.1, K=64")


def serving_sizes(n_events: int = 2000, lo: int = 20_000, hi: int = 400_000, seed=5) -> np.ndarray:
    """Event sizes log-uniform on [lo, hi]."""
    g = _rng(seed)
    return np.exp(g.uniform(np.log(lo), np.log(hi), size=n_events)).astype(np.int64)


def poisson_arrivals(n_events: int, rate_hz: float, seed=5) -> np.ndarray:
    """Arrival times (s, from 0) of a Poisson process with the given rate."""
    g = _rng((seed, 1))
    return np.cumsum(g.exponential(1.0 / rate_hz, size=n_events))


def config5_event(e: int, sizes: np.ndarray) -> np.ndarray:
    """Event ``e`` of the serving stream (drawn on demand: 2000 events do not
    all need to live in memory at once)."""
    return event_mix(int(sizes[e]), 8, (5, e))


def config5_event_args(args) -> np.ndarray:
    """config5_event(*args): one picklable argument, for process pools."""
    return config5_event(*args)
