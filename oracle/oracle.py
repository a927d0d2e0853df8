"""CPU oracle for spectral-bound greedy coarsening (arXiv 2204.11757) -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module.  The product path (the CUDA library and its Python binding) never does, and this
module never imports the product path: the two share only the seeded input generators.

The sequential arithmetic lives in ``spc_oracle.c`` (compiled with FMA contraction off); this
module marshals arrays to it, strings one level into the multilevel schedule, loops over the
graphs of a batch, and provides the dense spectral tools used to pin the oracle to the paper:

* ``laplacian_norm``   the normalized Laplacian L = I - D^-1/2 W D^-1/2 (Theorem 1 and the
                       sentence after it, following Chung's definition);
* ``lift_weights``     the lift of Definition 2: w_hat(u, v) = sum_{x in u_c, y in v_c} w(x, y)
                       / (|u_c| |v_c|);
* ``coarse_laplacian`` the normalized Laplacian of C^T W C (super-node graph with its self-mass
                       on the diagonal), whose eigenvalues are eigenvalues of the lift (the
                       remark after Theorem 1);
* ``greedy_literal``   Algorithm 1's merge loop written with explicit super-node sets, no
                       union-find, for brute-force cross-checks on tiny graphs.
* ``with_self_mass``   the multilevel driver's reading of a coarse graph: the graph with its
                       accumulated internal weight on the diagonal (the merged node
                       (w_a + w_b) / (d_a + d_b) of the proof of Theorem 2), used by
                       ``coarsen`` unless ``self_mass_degree=False`` asks for the coarse graph
                       without it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libspc_oracle.so")
SRC = os.path.join(HERE, "spc_oracle.c")

I32, F32, F64 = 0, 1, 2
OK, WARN_TARGET_NOT_REACHED = 0, 1

_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, FMA contraction off, no fast-math)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC)):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp]
    try:  # OpenMP only for the parallel CPU baseline; without it that loop runs on one thread
        subprocess.check_call(base + ["-fopenmp", SRC], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base + [SRC])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.orc_degree.argtypes = [i64, P, P, ctypes.c_int, P]
        L.orc_normalise.argtypes = [i64, P, P, ctypes.c_int, P, P]
        L.orc_score.argtypes = [i64, P, P, P, ctypes.c_int, P]
        L.orc_score.restype = i64
        L.orc_score_parallel.argtypes = [i64, P, P, P, ctypes.c_int, P, P]
        L.orc_score_parallel.restype = i64
        L.orc_sort_fitness.argtypes = [i64, P, ctypes.c_int, P]
        L.orc_greedy_merge.argtypes = [i64, i64, P, P, P, i64, P, P, P]
        L.orc_relabel.argtypes = [i64, P, P, P]
        L.orc_contract.argtypes = [i64, i64, P, P, P, ctypes.c_int, P, i64, P, P, P, P, P, P, P]
        L.orc_contract_backward.argtypes = [i64, P, P, ctypes.c_int, P]
        L.orc_pool_features.argtypes = [i64, P, i64, i64, P, ctypes.c_int, P]
        L.orc_pool_backward.argtypes = [i64, P, i64, i64, P, ctypes.c_int, P]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags.c_contiguous
    return ctypes.c_void_p(a.ctypes.data)


def wtype_of(w: np.ndarray) -> int:
    if w.dtype == np.int32:
        return I32
    if w.dtype == np.float32:
        return F32
    if w.dtype == np.float64:
        return F64
    raise TypeError(f"unsupported weight dtype {w.dtype}")


def score_dtype(w: np.ndarray):
    """Scores are float32 for float32 weights and float64 otherwise."""
    return np.float32 if w.dtype == np.float32 else np.float64


def acc_dtype(w: np.ndarray):
    """Degree / self-mass type: int64 for int32 weights, else the weight type."""
    return np.int64 if w.dtype == np.int32 else w.dtype


# ---- single steps ------------------------------------------------------------------------

def degree(g) -> np.ndarray:
    """S1, d_x = sum_y w_xy in ascending y (Theorem 1: d_x is the degree of x)."""
    d = np.empty(g.n, dtype=acc_dtype(g.w))
    lib().orc_degree(g.n, _ptr(g.rowptr), _ptr(g.w), wtype_of(g.w), _ptr(d))
    return d


def normalise(g, d: np.ndarray) -> np.ndarray:
    """S2, p = w_x / d_x per stored entry (Theorem 1's normalised adjacency vectors)."""
    p = np.empty(g.nnz, dtype=score_dtype(g.w))
    lib().orc_normalise(g.n, _ptr(g.rowptr), _ptr(g.w), wtype_of(g.w), _ptr(d), _ptr(p))
    return p


def score_parallel(g):
    """Scores with the edges split over the host's threads (OpenMP); returns (f, threads).
    Same bits as score(): only the edges are shared out."""
    m = (g.nnz) // 2
    f = np.empty(m, dtype=score_dtype(g.w))
    th = np.zeros(1, dtype=np.int32)
    got = lib().orc_score_parallel(g.n, _ptr(g.rowptr), _ptr(g.col), _ptr(g.w), wtype_of(g.w),
                                   _ptr(f), _ptr(th))
    if got != m:
        raise RuntimeError(f"orc_score_parallel returned {got}, expected {m}")
    return f, int(th[0])


def score(g) -> np.ndarray:
    """S1-S3, f(a, b) = ||w_a/d_a - w_b/d_b||_1 per undirected edge in eid order (Algorithm 1)."""
    m = int(g.eu.shape[0])
    f = np.empty(m, dtype=score_dtype(g.w))
    got = lib().orc_score(g.n, _ptr(g.rowptr), _ptr(g.col), _ptr(g.w), wtype_of(g.w), _ptr(f))
    if got != m:
        raise RuntimeError(f"orc_score returned {got}, expected {m}")
    return f


def sort_fitness(f: np.ndarray) -> np.ndarray:
    """S4, edge ids sorted by (f, eid) ascending (Algorithm 1's sort; ties by node id)."""
    order = np.empty(f.shape[0], dtype=np.int32)
    lib().orc_sort_fitness(f.shape[0], _ptr(f), F32 if f.dtype == np.float32 else F64,
                           _ptr(order))
    return order


def greedy_merge(g, order: np.ndarray, n_c: int):
    """S5, Algorithm 1's merge loop.  Returns (rep, merged flags, super-node count, status)."""
    rep = np.empty(g.n, dtype=np.int32)
    merged = np.empty(max(g.m, 1), dtype=np.uint8)
    s = ctypes.c_int64(0)
    rc = lib().orc_greedy_merge(g.n, g.m, _ptr(g.eu), _ptr(g.ev), _ptr(order), n_c, _ptr(rep),
                                _ptr(merged), ctypes.byref(s))
    if rc < 0:
        raise ValueError(f"orc_greedy_merge failed: {rc}")
    return rep, merged[:g.m].astype(bool), int(s.value), rc


def relabel(rep: np.ndarray):
    """S6, super-node ids by ascending smallest member (Definition 1's super-nodes)."""
    n = rep.shape[0]
    lift = np.empty(n, dtype=np.int32)
    nc = ctypes.c_int64(0)
    lib().orc_relabel(n, _ptr(rep), _ptr(lift), ctypes.byref(nc))
    return lift, int(nc.value)


class Coarse:
    """Output of one contraction: the coarse graph and the maps back to the fine graph."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def contract(g, lift: np.ndarray, n_c: int) -> Coarse:
    """S7, Definition 1 (coarse weights = sums of fine weights between super-nodes)."""
    m = g.m
    emap = np.empty(max(m, 1), dtype=np.int32)
    self_mass = np.empty(max(n_c, 1), dtype=acc_dtype(g.w))
    a_und = np.empty(max(m, 1), dtype=g.w.dtype)
    rowptr_c = np.empty(n_c + 1, dtype=np.int64)
    col_c = np.empty(max(2 * m, 1), dtype=np.int32)
    w_c = np.empty(max(2 * m, 1), dtype=g.w.dtype)
    mc = ctypes.c_int64(0)
    rc = lib().orc_contract(g.n, m, _ptr(g.eu), _ptr(g.ev), _ptr(g.w_und), wtype_of(g.w),
                            _ptr(lift), n_c, _ptr(emap), _ptr(self_mass), _ptr(a_und),
                            _ptr(rowptr_c), _ptr(col_c), _ptr(w_c), ctypes.byref(mc))
    if rc < 0:
        raise OverflowError(f"orc_contract failed: {rc}")
    m_c = int(mc.value)
    col_c = col_c[:2 * m_c].copy()
    w_c = w_c[:2 * m_c].copy()
    rows = np.repeat(np.arange(n_c, dtype=np.int64), np.diff(rowptr_c))
    up = col_c > rows
    gc = _GraphLike(n=n_c, rowptr=rowptr_c, col=col_c, w=w_c, eu=rows[up].astype(np.int32),
                    ev=col_c[up].astype(np.int32), w_und=a_und[:m_c].copy())
    return Coarse(graph=gc, emap=emap[:m].copy(), self_mass=self_mass[:n_c].copy(),
                  a_und=a_und[:m_c].copy(), m_c=m_c)


class _GraphLike:
    """Same fields as the generators' Graph (n, rowptr, col, w, eu, ev, w_und)."""

    def __init__(self, n, rowptr, col, w, eu, ev, w_und):
        self.n, self.rowptr, self.col, self.w = n, rowptr, col, w
        self.eu, self.ev, self.w_und = eu, ev, w_und

    @property
    def m(self):
        return int(self.eu.shape[0])

    @property
    def nnz(self):
        return int(self.col.shape[0])


def contract_backward(emap: np.ndarray, grad_a: np.ndarray) -> np.ndarray:
    """S9 reference: grad_w[e] = grad_a[emap[e]], 0 where emap[e] = -1 (assignment fixed)."""
    grad_w = np.empty(emap.shape[0], dtype=grad_a.dtype)
    lib().orc_contract_backward(emap.shape[0], _ptr(emap), _ptr(grad_a),
                                F32 if grad_a.dtype == np.float32 else F64, _ptr(grad_w))
    return grad_w


def pool_features(lift: np.ndarray, n_c: int, x: np.ndarray) -> np.ndarray:
    """Mean of each super-node's member features (Definition 2's averaging over super-node
    sizes, for node features): the members in ascending id summed by a 256-ary tree (a list of
    at most 256 items is summed left to right from 0; a longer one is replaced by the sums of
    its consecutive chunks of 256, recursively); then one division by the member count.
    x is n-by-F (float32 or float64)."""
    x = np.ascontiguousarray(x)
    n, F = x.shape
    lift = np.ascontiguousarray(lift, dtype=np.int32)
    xc = np.empty((n_c, F), dtype=x.dtype)
    rc = lib().orc_pool_features(n, _ptr(lift), n_c, F, _ptr(x),
                                 F32 if x.dtype == np.float32 else F64, _ptr(xc))
    if rc != 0:
        raise ValueError(f"orc_pool_features: {rc}")
    return xc


def pool_backward(lift: np.ndarray, n_c: int, grad_xc: np.ndarray) -> np.ndarray:
    """Gradient of pool_features with the lift held fixed: grad_x[v] = grad_xc[c(v)] / |c(v)|."""
    grad_xc = np.ascontiguousarray(grad_xc)
    F = grad_xc.shape[1]
    lift = np.ascontiguousarray(lift, dtype=np.int32)
    gx = np.empty((lift.shape[0], F), dtype=grad_xc.dtype)
    rc = lib().orc_pool_backward(lift.shape[0], _ptr(lift), n_c, F, _ptr(grad_xc),
                                 F32 if grad_xc.dtype == np.float32 else F64, _ptr(gx))
    if rc != 0:
        raise ValueError(f"orc_pool_backward: {rc}")
    return gx


# ---- one level, multilevel, batch --------------------------------------------------------

class Level:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def coarsen_level(g, n_c: int) -> Level:
    """One pass of Algorithm 1 (score, sort, merge loop) followed by the contraction."""
    if n_c < 1:
        raise ValueError("n_c must be >= 1")
    f = score(g)
    order = sort_fitness(f)
    rep, merged, s, rc = greedy_merge(g, order, n_c)
    lift, nca = relabel(rep)
    assert nca == s
    co = contract(g, lift, nca)
    return Level(f=f, order=order, merged=merged, lift=lift, n_c=nca, status=rc, coarse=co,
                 target=n_c)


def level_targets(n: int, ratio: int, mode: str):
    """Level targets.  'one': a single level to floor(n / ratio).  'halving': targets
    floor(n / 2^l) for l = 1 .. log2(ratio) (ratio a power of two), the last one being
    floor(n / ratio); Section 4 recomputes the norms after partial coarsening."""
    if mode == "one":
        return [max(1, n // ratio)]
    L = int(round(np.log2(ratio)))
    if 2 ** L != ratio:
        raise ValueError("halving schedule needs a power-of-two ratio")
    return [max(1, n // (2 ** l)) for l in range(1, L + 1)]


def with_self_mass(g, mass: np.ndarray):
    """The graph g with twice each node's accumulated internal weight on its diagonal: entry
    (x, x) = 2 mass[x], stored in its ascending-column place, for every x with mass[x] != 0.
    The undirected edge list (eu, ev, w_und) and so the edge ids are unchanged.

    This is the merged node of the proof of Theorem 2: merging a and b gives the normalized
    adjacency vector (w_a + w_b) / (d_a + d_b), whose own coordinate holds w_ab + w_ba and whose
    degree keeps the internal weight.  Degrees (ascending columns) and scores (the sorted union
    of the two rows, which then contains the diagonal entries) follow with no other change."""
    mass = np.asarray(mass)
    diag = 2 * mass.astype(acc_dtype(g.w))
    if g.w.dtype == np.int32:
        if diag.size and int(diag.max()) > np.iinfo(np.int32).max:
            raise OverflowError("2 x self-mass does not fit the int32 weights")
    nodes = np.nonzero(diag)[0]
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    r = np.concatenate([rows, nodes.astype(np.int64)])
    c = np.concatenate([g.col.astype(np.int64), nodes.astype(np.int64)])
    w = np.concatenate([g.w, diag[nodes].astype(g.w.dtype)])
    o = np.lexsort((c, r))
    rowptr = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=g.n), out=rowptr[1:])
    return _GraphLike(n=g.n, rowptr=rowptr, col=np.ascontiguousarray(c[o].astype(np.int32)),
                      w=np.ascontiguousarray(w[o]), eu=g.eu, ev=g.ev, w_und=g.w_und)


def carry_self_mass(mass: np.ndarray, lift: np.ndarray, n_c: int,
                    new_mass: np.ndarray) -> np.ndarray:
    """Accumulated internal weight of each super-node of the next level: its members' masses in
    ascending member id, then the weight of this level's edges inside it (the contraction's
    self-mass), summed left to right from 0."""
    out = np.zeros(n_c, dtype=new_mass.dtype)
    np.add.at(out, lift, mass.astype(new_mass.dtype))   # unbuffered, in ascending x
    out += new_mass
    return out


def coarsen(g, ratio: int, mode: str, self_mass_degree: bool = True):
    """The multilevel driver: repeat one level on the previous coarse graph with the targets of
    ``level_targets``; returns (levels, composed lift).

    With ``self_mass_degree`` (the default) each level scores the coarse graph with its
    accumulated internal weight on the diagonal (``with_self_mass``): the merged node of the
    proof of Theorem 2, which keeps w_ab + w_ba in its own coordinate and the internal weight in
    its degree.  Each level then records ``mass``, the accumulated internal weight of its
    super-nodes.  With ``self_mass_degree=False`` each level scores the coarse graph without
    it.  The first level is the same either way."""
    levels = []
    cur = g
    total = np.arange(g.n, dtype=np.int32)
    mass = np.zeros(g.n, dtype=acc_dtype(g.w))
    for t in level_targets(g.n, ratio, mode):
        lv = coarsen_level(with_self_mass(cur, mass) if self_mass_degree else cur, t)
        levels.append(lv)
        total = lv.lift[total]
        if self_mass_degree:
            mass = carry_self_mass(mass, lv.lift, lv.n_c, lv.coarse.self_mass)
            lv.mass = mass
        cur = lv.coarse.graph
    return levels, total


# The adjacency-reordering option's order (the paper's closing section suggests graph adjacency
# reordering for memory locality; which order is this library's choice).
REORDER_HOPS = 8  # the cluster label: the smallest node id within this many hops
REORDER_SUB = 2   # the sub-cluster label, the same within fewer hops


def hop_min_labels(g, k: int):
    """L_0 .. L_k, where L_i(x) is the smallest node id within i hops of x (x included):
    L_0(x) = x and L_{i+1}(x) = min(L_i(x), min over the neighbours y of x of L_i(y)), one
    synchronous round per hop (a node with no neighbour keeps its own id)."""
    n = g.n
    L = np.arange(n, dtype=np.int64)
    out = [L]
    deg = np.diff(g.rowptr)
    for _ in range(k):
        nb = np.full(n, n, dtype=np.int64)
        has = deg > 0
        if g.nnz > 0:
            nb[has] = np.minimum.reduceat(L[g.col], g.rowptr[:-1][has])
        L = np.minimum(L, nb)
        out.append(L)
    return out


def cluster_order(g, hops: int = REORDER_HOPS, sub: int = REORDER_SUB) -> np.ndarray:
    """The locality order of the adjacency-reordering option: nodes renumbered by
    (L_hops(x), L_sub(x), x) with the labels of hop_min_labels.  Nodes sharing the smallest id
    within `hops` hops form clusters of nearby nodes; inside a cluster the `sub`-hop label
    groups nearer ones.  Returns perm, perm[x] = the new id of node x."""
    n = g.n
    labels = hop_min_labels(g, hops)
    key = np.lexsort((np.arange(n), labels[sub], labels[hops]))
    perm = np.empty(n, dtype=np.int32)
    perm[key] = np.arange(n, dtype=np.int32)
    return perm


def permute(g, perm: np.ndarray):
    """The graph with node x renamed perm[x]: rows in new-id order, columns ascending, every
    weight carried with its entry; edge ids follow the new upper triangle."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    r = perm[rows].astype(np.int64)
    c = perm[g.col].astype(np.int64)
    o = np.lexsort((c, r))
    rowptr = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=g.n), out=rowptr[1:])
    col = np.ascontiguousarray(c[o].astype(np.int32))
    w = np.ascontiguousarray(g.w[o])
    rr = r[o]
    up = col > rr
    return _GraphLike(n=g.n, rowptr=rowptr, col=col, w=w, eu=rr[up].astype(np.int32),
                      ev=col[up], w_und=w[up])


def coarsen_reordered(g, ratio: int, mode: str, self_mass_degree: bool = True):
    """The adjacency-reordering option: the multilevel driver on permute(g, cluster_order(g)).
    Returns (levels of the renumbered graph, composed lift of the original nodes, perm); the
    lift of node x is the renumbered graph's lift of node perm[x]."""
    perm = cluster_order(g)
    levels, total = coarsen(permute(g, perm), ratio, mode, self_mass_degree)
    return levels, total[perm], perm


def coarsen_batch(batch, ratio: int, mode: str, self_mass_degree: bool = True):
    """Each graph of the batch coarsened on its own (its targets from its own size), results
    concatenated with global ids.  Returns per-graph level lists and the global outputs.
    ``self_mass_degree`` selects the multilevel reading as in ``coarsen``."""
    g = batch.graph
    gp = batch.graph_ptr
    eptr = np.searchsorted(g.eu, gp).astype(np.int64)
    per_graph = []
    for b in range(batch.B):
        n0, n1 = int(gp[b]), int(gp[b + 1])
        p0, p1 = int(g.rowptr[n0]), int(g.rowptr[n1])
        e0, e1 = int(eptr[b]), int(eptr[b + 1])
        sub = _GraphLike(n=n1 - n0, rowptr=g.rowptr[n0:n1 + 1] - p0,
                         col=np.ascontiguousarray(g.col[p0:p1] - n0), w=g.w[p0:p1],
                         eu=np.ascontiguousarray(g.eu[e0:e1] - n0),
                         ev=np.ascontiguousarray(g.ev[e0:e1] - n0), w_und=g.w_und[e0:e1])
        per_graph.append(coarsen(sub, ratio, mode, self_mass_degree))
    return per_graph


def compose_emaps(levels) -> np.ndarray:
    """Fine edge -> final coarse edge (-1 once an edge falls inside a super-node)."""
    em = levels[0].coarse.emap.astype(np.int64)
    for lv in levels[1:]:
        nxt = lv.coarse.emap
        em = np.where(em >= 0, nxt[np.maximum(em, 0)], -1)
    return em.astype(np.int32)


# ---- dense spectral tools (Theorem 1, Definition 2) --------------------------------------

def dense_weights(g) -> np.ndarray:
    W = np.zeros((g.n, g.n), dtype=np.float64)
    W[g.eu, g.ev] = g.w_und
    W[g.ev, g.eu] = g.w_und
    return W


def laplacian_norm(W: np.ndarray) -> np.ndarray:
    """L = I - D^-1/2 W D^-1/2 with D the row sums of W (diagonal entries included)."""
    d = W.sum(axis=1)
    s = 1.0 / np.sqrt(d)
    return np.eye(W.shape[0]) - (s[:, None] * W) * s[None, :]


def membership(lift: np.ndarray, n_c: int) -> np.ndarray:
    C = np.zeros((lift.shape[0], n_c), dtype=np.float64)
    C[np.arange(lift.shape[0]), lift] = 1.0
    return C


def lift_weights(W: np.ndarray, lift: np.ndarray, n_c: int) -> np.ndarray:
    """Definition 2 written out: w_hat(u,v) = sum_{x in u_c, y in v_c} w(x,y) / (|u_c||v_c|)."""
    n = W.shape[0]
    sizes = np.bincount(lift, minlength=n_c).astype(np.float64)
    block = np.zeros((n_c, n_c))
    for x in range(n):
        for y in range(n):
            if W[x, y] != 0.0:
                block[lift[x], lift[y]] += W[x, y]
    What = np.empty((n, n))
    for u in range(n):
        for v in range(n):
            What[u, v] = block[lift[u], lift[v]] / (sizes[lift[u]] * sizes[lift[v]])
    return What


def coarse_laplacian(W: np.ndarray, lift: np.ndarray, n_c: int) -> np.ndarray:
    """Normalized Laplacian of A_c = C^T W C (Definition 1's super-node weights; the diagonal
    holds twice each super-node's self-mass)."""
    C = membership(lift, n_c)
    return laplacian_norm(C.T @ W @ C)


# ---- literal Algorithm 1 with explicit super-node sets (tiny graphs only) ----------------

def greedy_literal(n: int, edges, fitness, n_c: int):
    """Algorithm 1's merge loop with super-nodes held as explicit Python sets.

    ``edges`` is a list of (a, b); ``fitness`` their scores.  The list is sorted by (fitness,
    position); each merge replaces the two sets by their union; an edge whose ends already
    share a set is passed over without counting; the loop stops when n_c sets remain.
    Returns the canonical lift (ids by ascending smallest member)."""
    owner = {x: frozenset([x]) for x in range(n)}
    order = sorted(range(len(edges)), key=lambda i: (fitness[i], i))
    s = n
    for i in order:
        if s <= n_c:
            break
        a, b = edges[i]
        if owner[a] is owner[b] or owner[a] == owner[b]:
            continue
        merged = owner[a] | owner[b]
        for x in merged:
            owner[x] = merged
        s -= 1
    sets = sorted({owner[x] for x in range(n)}, key=min)
    ids = {st: k for k, st in enumerate(sets)}
    return np.array([ids[owner[x]] for x in range(n)], dtype=np.int32), len(sets)
