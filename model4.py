"""Grid over G axes + points sorted inside each cell by one more coordinate:
groups = runs of queries in one cell whose sort-coordinate gaps are <= gap;
candidates = points of the (2m+1)^G neighbour cells with the sort coordinate in
[first - r, last + r] of the group."""
import sys, numpy as np
sys.path.insert(0, "/root/repo")
from paper_2609_31980_gb300 import synth

def run(pts, r, gaxes, sax, gap, maxq=16, label=""):
    lo = pts[:, gaxes].min(0); hi = pts[:, gaxes].max(0)
    h = r * (1 + 2**-10)
    dims = (np.floor((hi - lo) / h) + 1).astype(np.int64)
    c = np.minimum(np.floor((pts[:, gaxes] - lo) / h).astype(np.int64), dims - 1)
    G = len(gaxes)
    cid = np.zeros(len(pts), np.int64); st = 1
    for a in range(G):
        cid += c[:, a] * st; st *= dims[a]
    ncell = st
    x = pts[:, sax]
    order = np.lexsort((x, cid)); scid = cid[order]; sx = x[order]
    cstart = np.searchsorted(scid, np.arange(ncell + 1))
    # groups
    n = len(pts)
    brk = np.r_[True, (scid[1:] != scid[:-1]) | (sx[1:] - sx[:-1] > gap)]
    # also break every maxq queries within a run
    gidx = np.cumsum(brk) - 1
    # split long groups
    first = np.flatnonzero(brk); last = np.r_[first[1:], n] - 1
    fs, ls = [], []
    for a, b in zip(first, last):
        for s in range(a, b + 1, maxq):
            fs.append(s); ls.append(min(s + maxq, b + 1) - 1)
    fs = np.array(fs); ls = np.array(ls)
    nq = ls - fs + 1
    gc = scid[fs]; wlo = sx[fs] - r; whi = sx[ls] + r
    coords = np.zeros((len(fs), G), np.int64); rr = gc.copy()
    for a in range(G):
        coords[:, a] = rr % dims[a]; rr //= dims[a]
    offs = np.array(np.meshgrid(*[np.arange(-1, 2)] * G, indexing="ij")).reshape(G, -1).T
    U = np.zeros(len(fs), np.int64); nonempty = np.zeros(len(fs), np.int64)
    for o in offs:
        cc = coords + o
        ok = np.all((cc >= 0) & (cc < dims), 1)
        lin = np.zeros(len(fs), np.int64); st = 1
        for a in range(G):
            lin += np.clip(cc[:, a], 0, dims[a] - 1) * st; st *= dims[a]
        a0 = cstart[lin]; a1 = cstart[lin + 1]
        # window by binary search in each cell's sorted x
        l = np.searchsorted(sx, wlo, side="left"); hh = np.searchsorted(sx, whi, side="right")
        # searchsorted over the global array is wrong across cells; do per cell:
        v = np.zeros(len(fs), np.int64)
        idx = np.flatnonzero(ok & (a1 > a0))
        for i in idx:
            seg = sx[a0[i]:a1[i]]
            v[i] = np.searchsorted(seg, whi[i], "right") - np.searchsorted(seg, wlo[i], "left")
        U += v; nonempty += (ok & (a1 > a0))
    print(f"{label} G={G} gap={gap}: groups {len(fs)} nq {nq.mean():.2f} U/grp {U.mean():.1f} "
          f"useful {(U*nq).sum()/1e6:.1f}M rounds {(nq*np.ceil(U/32)).sum()/1e6:.2f}M "
          f"nonempty cells/grp {nonempty.mean():.1f} cells {ncell}")

w = synth.config2(); pts = w.points.astype(np.float64)
for gap in (0.1, 0.2, 0.5):
    run(pts, w.r, [4, 5, 6, 7], 3, gap, label="300kx8")
