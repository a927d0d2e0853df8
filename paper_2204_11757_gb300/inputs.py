"""Seeded synthetic graph generators shared by the oracle tests, the CUDA tests and the bench.

This module only builds inputs: vertex positions, mesh/geometric topology, edge weights and the
symmetric CSR layout the coarsener consumes.  It holds none of the coarsening arithmetic (no
degrees, no normalised adjacencies, no scores, no merges, no contraction), so the CPU oracle and
the GPU path can both read the same bytes without sharing any of the method.

The workloads stand in for the paper's two test graphs (Section 3): the Stanford bunny, a nearly
regular surface mesh, and SNAP ego-Facebook, an irregular social graph.  Neither dataset is
available here, so the generators produce

* 2D triangulated grids (each square split by a seeded coin-flip diagonal), optionally with
  jittered vertices and weights 1/edge-length;
* 3D tetrahedral meshes of a cube (every cell split into 6 tetrahedra along its main diagonal,
  Kuhn/Freudenthal split, so neighbouring cells agree on face diagonals);
* random geometric graphs in the unit cube with a radius chosen for a target mean degree and
  weights exp(-d^2/r^2);
* batches of jittered 2D/3D meshes of log-uniform size, laid out as one block-diagonal CSR.

CSR conventions (the input contract of the library):
  rowptr int64[n+1], col int32[2m] strictly ascending inside every row, no self-loops,
  symmetric pattern and weights.  The undirected edge id ``eid`` of {u, v} with u < v is the
  position of the pair in lexicographic (u, v) order, i.e. the order of the upper-triangle
  entries when the CSR is read row by row.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Graph", "Batch", "csr_from_edges", "upper_edges", "tri_mesh_2d", "tet_mesh_3d", "rgg_3d",
    "mesh_batch", "config_graph", "CONFIGS", "path_graph", "cycle_graph", "complete_graph",
    "random_graph", "subsample_batch", "powerlaw_graph", "batch_of",
]


@dataclasses.dataclass
class Graph:
    """A symmetric weighted graph in CSR form plus its undirected edge list in eid order."""
    n: int
    rowptr: np.ndarray  # int64[n+1]
    col: np.ndarray     # int32[2m]
    w: np.ndarray       # int32 / float32 / float64 [2m]
    eu: np.ndarray      # int32[m], eu < ev, lexicographic order == eid order
    ev: np.ndarray      # int32[m]
    w_und: np.ndarray   # weight of each undirected edge, eid order
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.eu.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])


@dataclasses.dataclass
class Batch:
    """B independent graphs stored as one block-diagonal CSR (global node ids)."""
    graph: Graph
    graph_ptr: np.ndarray  # int64[B+1], graph g owns nodes [graph_ptr[g], graph_ptr[g+1])
    kinds: np.ndarray      # int8[B], 2 or 3 (mesh dimension)

    @property
    def B(self) -> int:
        return int(self.graph_ptr.shape[0] - 1)


def csr_from_edges(n: int, eu: np.ndarray, ev: np.ndarray, w: np.ndarray, name: str = "") -> Graph:
    """Build the symmetric CSR of an undirected simple graph.

    ``eu``/``ev``/``w`` list each undirected edge once, in any order and orientation.  Self-loops
    and duplicates are rejected (the coarsener's input contract forbids them).
    """
    eu = np.asarray(eu, dtype=np.int64)
    ev = np.asarray(ev, dtype=np.int64)
    w = np.asarray(w)
    if eu.shape != ev.shape or eu.shape != w.shape:
        raise ValueError("edge arrays must have equal length")
    if np.any(eu == ev):
        raise ValueError("self-loop in edge list")
    lo = np.minimum(eu, ev)
    hi = np.maximum(eu, ev)
    key = lo * n + hi
    order = np.argsort(key, kind="stable")
    key = key[order]
    if key.size > 1 and np.any(key[1:] == key[:-1]):
        raise ValueError("duplicate edge in edge list")
    lo = lo[order]
    hi = hi[order]
    wu = w[order]
    m = lo.shape[0]
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    ww = np.concatenate([wu, wu])
    order2 = np.argsort(rows * n + cols, kind="stable")
    rows = rows[order2]
    col = cols[order2].astype(np.int32)
    wcsr = ww[order2]
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return Graph(n=n, rowptr=rowptr, col=col, w=np.ascontiguousarray(wcsr),
                 eu=lo.astype(np.int32), ev=hi.astype(np.int32), w_und=np.ascontiguousarray(wu),
                 name=name)


def upper_edges(rowptr: np.ndarray, col: np.ndarray, w: np.ndarray | None = None):
    """Undirected edge list (eid order) read off a symmetric CSR."""
    n = rowptr.shape[0] - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    sel = col > rows
    eu = rows[sel].astype(np.int32)
    ev = col[sel].astype(np.int32)
    if w is None:
        return eu, ev
    return eu, ev, w[sel]


def _weights_from_points(pts: np.ndarray, eu: np.ndarray, ev: np.ndarray, kind: str, dtype,
                         radius: float | None = None) -> np.ndarray:
    if kind == "unit":
        return np.ones(eu.shape[0], dtype=dtype)
    diff = pts[eu] - pts[ev]
    d2 = np.einsum("ij,ij->i", diff, diff)
    if kind == "inv_len":
        return (1.0 / np.sqrt(d2)).astype(dtype)
    if kind == "gauss":
        return np.exp(-d2 / (radius * radius)).astype(dtype)
    raise ValueError(kind)


def tri_mesh_2d(nx: int, ny: int, seed: int, jitter: float = 0.0, weight: str = "unit",
                dtype=np.int32, name: str = "") -> Graph:
    """Triangulated nx-by-ny vertex grid; each square gets one diagonal by a seeded coin flip.

    Vertex (i, j) has id j*nx + i.  Random draws, in order: one coin per cell (row-major), then
    the vertex jitter U(-jitter, +jitter) per coordinate (only when jitter > 0).
    m = (nx-1)*ny + nx*(ny-1) + (nx-1)*(ny-1).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    coins = rng.integers(0, 2, size=(ny - 1, nx - 1), dtype=np.int8)
    ii, jj = np.meshgrid(np.arange(nx, dtype=np.int64), np.arange(ny, dtype=np.int64))
    vid = jj * nx + ii
    parts_u, parts_v = [], []
    parts_u.append(vid[:, :-1].ravel()); parts_v.append(vid[:, 1:].ravel())      # horizontal
    parts_u.append(vid[:-1, :].ravel()); parts_v.append(vid[1:, :].ravel())      # vertical
    a = vid[:-1, :-1]; b = vid[:-1, 1:]; c = vid[1:, :-1]; d = vid[1:, 1:]
    diag_u = np.where(coins == 0, a, b).ravel()
    diag_v = np.where(coins == 0, d, c).ravel()
    parts_u.append(diag_u); parts_v.append(diag_v)
    eu = np.concatenate(parts_u); ev = np.concatenate(parts_v)
    n = nx * ny
    pts = np.stack([ii.ravel().astype(np.float64), jj.ravel().astype(np.float64)], axis=1)
    if jitter > 0:
        pts = pts + rng.uniform(-jitter, jitter, size=pts.shape)
    w = _weights_from_points(pts, eu, ev, weight, dtype)
    return csr_from_edges(n, eu, ev, w, name=name or f"tri2d_{nx}x{ny}")


_KUHN_OFFSETS = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [1, 0, 1], [0, 1, 1],
                          [1, 1, 1]], dtype=np.int64)


def tet_mesh_3d(k: int, seed: int, jitter: float = 0.0, weight: str = "unit", dtype=np.int32,
                name: str = "") -> Graph:
    """Tetrahedral mesh of a cube with k vertices per side ((k-1)^3 cells, 6 tets per cell).

    Every cell is split along its (0,0,0)-(1,1,1) diagonal (Kuhn split); the edges are then all
    vertex pairs p, p+o with o in {e_x, e_y, e_z, e_x+e_y, e_x+e_z, e_y+e_z, e_x+e_y+e_z}, so
    m = 3(k-1)k^2 + 3(k-1)^2 k + (k-1)^3.  Vertex (x, y, z) has id (z*k + y)*k + x.  The only
    random draw is the vertex jitter U(-jitter, +jitter) per coordinate.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ax = np.arange(k, dtype=np.int64)
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    xs, ys, zs = xx.ravel(), yy.ravel(), zz.ravel()
    n = k * k * k
    eu_parts, ev_parts = [], []
    for o in _KUHN_OFFSETS:
        ok = (xs + o[0] < k) & (ys + o[1] < k) & (zs + o[2] < k)
        u = ((zs * k + ys) * k + xs)[ok]
        v = (((zs + o[2]) * k + (ys + o[1])) * k + (xs + o[0]))[ok]
        eu_parts.append(u); ev_parts.append(v)
    eu = np.concatenate(eu_parts); ev = np.concatenate(ev_parts)
    pts = np.stack([xs, ys, zs], axis=1).astype(np.float64)
    if jitter > 0:
        pts = pts + rng.uniform(-jitter, jitter, size=pts.shape)
    w = _weights_from_points(pts, eu, ev, weight, dtype)
    return csr_from_edges(n, eu, ev, w, name=name or f"tet3d_{k}")


def rgg_3d(n: int, mean_degree: float, seed: int, dtype=np.float32, name: str = "") -> Graph:
    """Random geometric graph: n points U[0,1)^3, edge iff |x-y| < r, r = (3 d / (4 pi n))^(1/3).

    Non-periodic, so boundary nodes have fewer neighbours.  Weight exp(-|x-y|^2 / r^2) computed in
    float64 and rounded to ``dtype``.  Neighbours are found by bucketing points into cells of side
    >= r and testing the 13 forward neighbour cells plus the cell itself.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.random((n, 3))
    r = (3.0 * mean_degree / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    G = max(1, int(math.floor(1.0 / r)))
    cell3 = np.minimum((pts * G).astype(np.int64), G - 1)
    cid = (cell3[:, 2] * G + cell3[:, 1]) * G + cell3[:, 0]
    order = np.argsort(cid, kind="stable")
    cid_s = cid[order]
    ncell = G * G * G
    cstart = np.searchsorted(cid_s, np.arange(ncell + 1, dtype=np.int64))
    ccount = np.diff(cstart)
    pts_s = pts[order]
    r2 = r * r
    offs = [(0, 0, 0)]
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dz, dy, dx) > (0, 0, 0):
                    offs.append((dx, dy, dz))
    eu_parts, ev_parts, w_parts = [], [], []
    cz, rem = np.divmod(np.arange(ncell, dtype=np.int64), G * G)
    cy, cx = np.divmod(rem, G)
    for (dx, dy, dz) in offs:
        nx_, ny_, nz_ = cx + dx, cy + dy, cz + dz
        ok = (nx_ >= 0) & (nx_ < G) & (ny_ >= 0) & (ny_ < G) & (nz_ >= 0) & (nz_ < G)
        src = np.nonzero(ok & (ccount > 0))[0]
        dst = (nz_[src] * G + ny_[src]) * G + nx_[src]
        keep = ccount[dst] > 0
        src, dst = src[keep], dst[keep]
        # every point i in cell src against every point j in cell dst
        cnt_s = ccount[src]; cnt_d = ccount[dst]
        pts_i = np.repeat(np.arange(src.shape[0]), cnt_s)
        i_idx = cstart[src][pts_i] + (np.arange(pts_i.shape[0]) - np.repeat(np.cumsum(cnt_s) - cnt_s, cnt_s))
        rep = cnt_d[pts_i]
        ii = np.repeat(i_idx, rep)
        base = np.repeat(cstart[dst][pts_i], rep)
        within = np.arange(ii.shape[0]) - np.repeat(np.cumsum(rep) - rep, rep)
        jj = base + within
        if (dx, dy, dz) == (0, 0, 0):
            sel = ii < jj
            ii, jj = ii[sel], jj[sel]
        diff = pts_s[ii] - pts_s[jj]
        d2 = np.einsum("ij,ij->i", diff, diff)
        sel = d2 < r2
        ii, jj, d2 = ii[sel], jj[sel], d2[sel]
        eu_parts.append(order[ii]); ev_parts.append(order[jj])
        w_parts.append(np.exp(-d2 / r2).astype(dtype))
    eu = np.concatenate(eu_parts); ev = np.concatenate(ev_parts); w = np.concatenate(w_parts)
    return csr_from_edges(n, eu, ev, w, name=name or f"rgg3d_{n}")


def mesh_batch(B: int, seed: int, nmin: int = 200, nmax: int = 20000, dtype=np.float32,
               name: str = "") -> Batch:
    """B jittered meshes of log-uniform size laid out as one block-diagonal CSR.

    Draws, in order, from PCG64(seed): B sizes N ~ exp(U(ln nmin, ln nmax)), B coins choosing a
    2D (coin 0) or 3D (coin 1) mesh, and B per-graph seeds.  A 2D graph is a k-by-k triangulated
    grid with k = round(sqrt(N)) and jitter 0.3; a 3D graph is a k^3 tetrahedral cube mesh with
    k = round(cbrt(N)) and jitter 0.25.  Weights are 1/edge-length in ``dtype``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=B))
    coins = rng.integers(0, 2, size=B)
    seeds = rng.integers(0, 2**62, size=B)
    rowptrs, cols, ws, eus, evs, wus, kinds, ns = [], [], [], [], [], [], [], []
    noff = 0
    eoff = 0
    for g in range(B):
        if coins[g] == 0:
            k = max(2, int(round(math.sqrt(sizes[g]))))
            gr = tri_mesh_2d(k, k, int(seeds[g]), jitter=0.3, weight="inv_len", dtype=dtype)
            kinds.append(2)
        else:
            k = max(2, int(round(sizes[g] ** (1.0 / 3.0))))
            gr = tet_mesh_3d(k, int(seeds[g]), jitter=0.25, weight="inv_len", dtype=dtype)
            kinds.append(3)
        rowptrs.append(gr.rowptr[:-1] + eoff)
        cols.append(gr.col + noff)
        ws.append(gr.w)
        eus.append(gr.eu + noff); evs.append(gr.ev + noff); wus.append(gr.w_und)
        ns.append(gr.n)
        noff += gr.n
        eoff += gr.nnz
    rowptr = np.concatenate(rowptrs + [np.array([eoff], dtype=np.int64)])
    graph = Graph(n=noff, rowptr=rowptr, col=np.concatenate(cols).astype(np.int32),
                  w=np.concatenate(ws), eu=np.concatenate(eus).astype(np.int32),
                  ev=np.concatenate(evs).astype(np.int32), w_und=np.concatenate(wus),
                  name=name or f"batch{B}")
    graph_ptr = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(np.array(ns, dtype=np.int64), out=graph_ptr[1:])
    return Batch(graph=graph, graph_ptr=graph_ptr, kinds=np.array(kinds, dtype=np.int8))


def batch_of(graphs, kinds=None, name: str = "") -> Batch:
    """Graphs laid out as one block-diagonal CSR (graph g's node x becomes node x + the nodes of
    the graphs before it); ``kinds`` labels each graph (0 when not given)."""
    rowptrs, cols, ws, eus, evs, wus, ns = [], [], [], [], [], [], []
    noff = 0
    eoff = 0
    for gr in graphs:
        rowptrs.append(gr.rowptr[:-1] + eoff)
        cols.append(gr.col + noff)
        ws.append(gr.w)
        eus.append(gr.eu + noff); evs.append(gr.ev + noff); wus.append(gr.w_und)
        ns.append(gr.n)
        noff += gr.n
        eoff += gr.nnz
    rowptr = np.concatenate(rowptrs + [np.array([eoff], dtype=np.int64)])
    graph = Graph(n=noff, rowptr=rowptr, col=np.concatenate(cols).astype(np.int32),
                  w=np.concatenate(ws), eu=np.concatenate(eus).astype(np.int32),
                  ev=np.concatenate(evs).astype(np.int32), w_und=np.concatenate(wus),
                  name=name or f"batch{len(ns)}")
    graph_ptr = np.zeros(len(ns) + 1, dtype=np.int64)
    np.cumsum(np.array(ns, dtype=np.int64), out=graph_ptr[1:])
    k = np.zeros(len(ns), dtype=np.int8) if kinds is None else np.asarray(kinds, dtype=np.int8)
    return Batch(graph=graph, graph_ptr=graph_ptr, kinds=k)


def subsample_batch(batch: Batch, idx) -> Batch:
    """The sub-batch made of graphs ``idx`` (ascending), renumbered into one block-diagonal CSR."""
    idx = np.asarray(idx, dtype=np.int64)
    g = batch.graph
    rowptrs, cols, ws, eus, evs, wus, ns = [], [], [], [], [], [], []
    noff = 0
    eoff = 0
    eid_ptr = np.searchsorted(g.eu, batch.graph_ptr)
    for b in idx:
        n0, n1 = int(batch.graph_ptr[b]), int(batch.graph_ptr[b + 1])
        p0, p1 = int(g.rowptr[n0]), int(g.rowptr[n1])
        rowptrs.append(g.rowptr[n0:n1] - p0 + eoff)
        cols.append(g.col[p0:p1] - n0 + noff)
        ws.append(g.w[p0:p1])
        e0, e1 = int(eid_ptr[b]), int(eid_ptr[b + 1])
        eus.append(g.eu[e0:e1] - n0 + noff); evs.append(g.ev[e0:e1] - n0 + noff)
        wus.append(g.w_und[e0:e1])
        ns.append(n1 - n0)
        noff += n1 - n0
        eoff += p1 - p0
    rowptr = np.concatenate(rowptrs + [np.array([eoff], dtype=np.int64)])
    graph = Graph(n=noff, rowptr=rowptr, col=np.concatenate(cols).astype(np.int32),
                  w=np.concatenate(ws), eu=np.concatenate(eus).astype(np.int32),
                  ev=np.concatenate(evs).astype(np.int32), w_und=np.concatenate(wus),
                  name=f"{g.name}_sub{len(idx)}")
    graph_ptr = np.zeros(len(idx) + 1, dtype=np.int64)
    np.cumsum(np.array(ns, dtype=np.int64), out=graph_ptr[1:])
    return Batch(graph=graph, graph_ptr=graph_ptr, kinds=batch.kinds[idx])


# ---- tiny graphs with known structure ------------------------------------------------------

def path_graph(n: int, dtype=np.int32) -> Graph:
    u = np.arange(n - 1)
    return csr_from_edges(n, u, u + 1, np.ones(n - 1, dtype=dtype), name=f"path{n}")


def cycle_graph(n: int, dtype=np.int32) -> Graph:
    u = np.arange(n)
    return csr_from_edges(n, u, (u + 1) % n, np.ones(n, dtype=dtype), name=f"cycle{n}")


def complete_graph(n: int, dtype=np.int32) -> Graph:
    iu, iv = np.triu_indices(n, 1)
    return csr_from_edges(n, iu, iv, np.ones(iu.shape[0], dtype=dtype), name=f"K{n}")


def random_graph(n: int, p: float, seed: int, weight: str = "unit", dtype=np.float64,
                 connected: bool = False, name: str = "") -> Graph:
    """Erdos-Renyi G(n, p); weights 1 ('unit'), integers 1..9 ('int') or U(0.1, 2) ('float').

    With ``connected`` a random spanning path over a seeded permutation is added first, so the
    graph is connected.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    iu, iv = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p
    if connected and n > 1:
        perm = rng.permutation(n)
        a = np.minimum(perm[:-1], perm[1:]); b = np.maximum(perm[:-1], perm[1:])
        pos = a * n - a * (a + 1) // 2 + (b - a - 1)
        keep[pos] = True
    iu, iv = iu[keep], iv[keep]
    if weight == "unit":
        w = np.ones(iu.shape[0], dtype=dtype)
    elif weight == "int":
        w = rng.integers(1, 10, size=iu.shape[0]).astype(dtype)
    else:
        w = rng.uniform(0.1, 2.0, size=iu.shape[0]).astype(dtype)
    return csr_from_edges(n, iu, iv, w, name=name or f"gnp{n}_{p}_{seed}")


# ---- the five workloads (plus reduced versions for tests) ----------------------------------

CONFIGS = {
    # name: (builder kwargs, coarsening: (mode, ratio)); mode 'one' = one level straight to
    # n_c = floor(n / ratio), 'halving' = levels with targets floor(n / 2^l) down to n_c.
    "c1_tri64_unit": dict(kind="tri", nx=64, ny=64, jitter=0.0, weight="unit", dtype="int32",
                          seed=1, mode="one", ratio=2),
    "c2_tri2048_f64": dict(kind="tri", nx=2048, ny=2048, jitter=0.3, weight="inv_len",
                           dtype="float64", seed=2, mode="halving", ratio=64),
    "c3_tet129_f64": dict(kind="tet", k=129, jitter=0.25, weight="inv_len", dtype="float64",
                          seed=3, mode="halving", ratio=128),
    "c4_rgg8m_f32": dict(kind="rgg", n=1 << 23, degree=12.0, dtype="float32", seed=4,
                         mode="halving", ratio=256),
    "c4_rgg8m_f32_one": dict(kind="rgg", n=1 << 23, degree=12.0, dtype="float32", seed=4,
                             mode="one", ratio=256),
    "c5_batch10k_f32": dict(kind="batch", B=10000, dtype="float32", seed=5, mode="halving",
                            ratio=8),
    "p2_tri512_f64": dict(kind="tri", nx=512, ny=512, jitter=0.3, weight="inv_len",
                          dtype="float64", seed=2, mode="halving", ratio=64),
    # the c4 construction at 2^21 points (its arrays still larger than L2): profiler captures
    "p4_rgg2m_f32": dict(kind="rgg", n=1 << 21, degree=12.0, dtype="float32", seed=4,
                         mode="halving", ratio=256),
    # reduced versions (same construction, sizes the oracle handles in well under a second)
    "s2_tri256_f64": dict(kind="tri", nx=256, ny=256, jitter=0.3, weight="inv_len",
                          dtype="float64", seed=12, mode="halving", ratio=64),
    "s3_tet33_f64": dict(kind="tet", k=33, jitter=0.25, weight="inv_len", dtype="float64",
                         seed=13, mode="halving", ratio=128),
    "s4_rgg64k_f32": dict(kind="rgg", n=1 << 16, degree=12.0, dtype="float32", seed=14,
                          mode="halving", ratio=256),
    "s4_rgg64k_f32_one": dict(kind="rgg", n=1 << 16, degree=12.0, dtype="float32", seed=14,
                              mode="one", ratio=256),
    "s5_batch40_f32": dict(kind="batch", B=40, dtype="float32", seed=15, mode="halving",
                           ratio=8, nmax=3000),
}


def config_graph(name: str):
    """Build a named workload; returns (Graph or Batch, config dict)."""
    cfg = CONFIGS[name]
    dt = np.dtype(cfg["dtype"])
    if cfg["kind"] == "tri":
        g = tri_mesh_2d(cfg["nx"], cfg["ny"], cfg["seed"], cfg["jitter"], cfg["weight"], dt, name)
    elif cfg["kind"] == "tet":
        g = tet_mesh_3d(cfg["k"], cfg["seed"], cfg["jitter"], cfg["weight"], dt, name)
    elif cfg["kind"] == "rgg":
        g = rgg_3d(cfg["n"], cfg["degree"], cfg["seed"], dt, name)
    elif cfg["kind"] == "batch":
        g = mesh_batch(cfg["B"], cfg["seed"], dtype=dt, nmax=cfg.get("nmax", 20000), name=name)
    else:
        raise ValueError(cfg["kind"])
    return g, cfg


def star_ties(leaves_log2: int = 12, dtype=np.float64, chords: int = 0, seed: int = 0) -> Graph:
    """A star whose hub weights alternate 1 + eps and 1 - eps (eps = 2^-41 in binary64, 2^-12 in
    binary32): the hub's degree is an exact power of two and its normalised weights sit exactly
    half a unit in the last place away from the grid of a running sum in [1, 2), so summing the
    hub row hits exact rounding ties.  `chords` adds seeded leaf-leaf edges (weight 1)."""
    L = 1 << leaves_log2
    eps = 2.0 ** -41 if np.dtype(dtype) == np.float64 else 2.0 ** -12
    w = np.where(np.arange(L) % 2 == 0, 1.0 + eps, 1.0 - eps).astype(dtype)
    eu = np.zeros(L, dtype=np.int64)
    ev = np.arange(1, L + 1, dtype=np.int64)
    if chords:
        rng = np.random.Generator(np.random.PCG64(seed))
        a = rng.integers(1, L + 1, size=chords)
        b = rng.integers(1, L + 1, size=chords)
        keep = a != b
        a, b = np.minimum(a[keep], b[keep]), np.maximum(a[keep], b[keep])
        key = np.unique(a * (L + 1) + b)
        a, b = key // (L + 1), key % (L + 1)
        eu = np.concatenate([eu, a]); ev = np.concatenate([ev, b])
        w = np.concatenate([w, np.ones(a.shape[0], dtype=dtype)])
    return csr_from_edges(L + 1, eu, ev, w, name=f"star_ties_{L}")


def hub_graph(n: int, hub_degrees, seed: int, weight: str = "float", dtype=np.float64,
              base_p: float = 0.002) -> Graph:
    """Sparse random graph plus a few hubs: node h < len(hub_degrees) is joined to
    hub_degrees[h] random nodes (hubs also join each other).  Weights as in random_graph."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m0 = int(base_p * n * (n - 1) / 2)
    a = rng.integers(0, n, size=m0); b = rng.integers(0, n, size=m0)
    us, vs = [a], [b]
    for h, dh in enumerate(hub_degrees):
        t = rng.choice(n, size=min(dh, n - 1), replace=False)
        us.append(np.full(t.shape[0], h)); vs.append(t)
    u = np.concatenate(us); v = np.concatenate(vs)
    keep = u != v
    u, v = np.minimum(u[keep], v[keep]), np.maximum(u[keep], v[keep])
    key = np.unique(u.astype(np.int64) * n + v)
    u, v = key // n, key % n
    if weight == "unit":
        w = np.ones(u.shape[0], dtype=dtype)
    elif weight == "int":
        w = rng.integers(1, 10, size=u.shape[0]).astype(dtype)
    else:
        w = rng.uniform(0.1, 2.0, size=u.shape[0]).astype(dtype)
    return csr_from_edges(n, u, v, w, name=f"hubs{n}")


def clique_ring(B: int, size: int, seed: int, dtype=np.float64) -> Graph:
    """B disjoint cliques K_size with random weights U(1, 1.1), joined into a ring by one edge
    of weight 0.05 between consecutive cliques.  Coarsening to n/size needs every clique merged
    completely, which the lightest few edges alone cannot do (they close cycles)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    iu, iv = np.triu_indices(size, 1)
    off = (np.arange(B) * size)[:, None]
    eu = (off + iu[None, :]).ravel(); ev = (off + iv[None, :]).ravel()
    w = rng.uniform(1.0, 1.1, size=eu.shape[0])
    ru = np.arange(B) * size
    rv = (np.arange(B) * size + size + 1) % (B * size)
    eu = np.concatenate([eu, ru]); ev = np.concatenate([ev, rv])
    w = np.concatenate([w, np.full(B, 0.05)]).astype(dtype)
    return csr_from_edges(B * size, eu, ev, w, name=f"cliques{B}x{size}")


def powerlaw_graph(n: int, k: int, seed: int, weight: str = "float", dtype=np.float64) -> Graph:
    """Preferential attachment: nodes k+1.. each join k distinct earlier nodes drawn with
    probability proportional to degree (nodes 0..k start as a clique).  Heavy-tailed degrees,
    the oldest (smallest) ids the largest: the shape of a social network such as the
    ego-Facebook graph (n = 4039, mean degree about 44) at n = 4039, k = 22.
    Weights as in random_graph."""
    rng = np.random.Generator(np.random.PCG64(seed))
    iu, iv = np.triu_indices(k + 1, 1)
    us, vs = [iu.astype(np.int64)], [iv.astype(np.int64)]
    # every edge end point once: drawing an entry uniformly is drawing a node by degree
    ends = np.empty(2 * (len(iu) + (n - k - 1) * k), dtype=np.int64)
    ne = 2 * len(iu)
    ends[:len(iu)] = iu; ends[len(iu):ne] = iv
    for x in range(k + 1, n):
        chosen = set()
        while len(chosen) < k:
            chosen.add(int(ends[rng.integers(0, ne)]))
        t = np.fromiter(sorted(chosen), dtype=np.int64, count=k)
        us.append(t); vs.append(np.full(k, x, dtype=np.int64))
        ends[ne:ne + k] = t; ends[ne + k:ne + 2 * k] = x
        ne += 2 * k
    u = np.concatenate(us); v = np.concatenate(vs)
    if weight == "unit":
        w = np.ones(u.shape[0], dtype=dtype)
    elif weight == "int":
        w = rng.integers(1, 10, size=u.shape[0]).astype(dtype)
    else:
        w = rng.uniform(0.1, 2.0, size=u.shape[0]).astype(dtype)
    return csr_from_edges(n, u, v, w, name=f"powerlaw{n}k{k}")
