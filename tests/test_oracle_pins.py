"""Pins for the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each test names what it pins.  The oracle is test infrastructure; these tests are what make it
trustworthy before any GPU result is compared with it.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components, minimum_spanning_tree

from oracle import oracle as O
from paper_2204_11757_gb300 import inputs as I

import golden_io



# ---- hand-worked examples (tests/golden/hand_*.txt) -----------------------------------------

@pytest.mark.parametrize("name", golden_io.FILES)
def test_golden_hand_example(name):
    """Scores, sort, merges and contraction of small examples worked by hand: a 4-node graph
    with distinct scores, and a 5-cycle whose equal scores leave every merge to the edge id."""
    rows, ncs = golden_io.parse(name)
    n, eu, ev, w = golden_io.edges(rows)
    g = I.csr_from_edges(n, eu, ev, w)
    assert list(g.eu) == list(eu) and list(g.ev) == list(ev)   # listed in edge-id order
    assert list(O.degree(g)) == golden_io.ints(rows, "degree")
    f = O.score(g)
    exact = [Fraction(s) for s in rows["score_num_den"].split()]
    assert [int(x) for x in f.view(np.uint64)] == golden_io.ints(rows, "score_f64_bits")
    for fi, ex in zip(f, exact):
        assert abs(Fraction(float(fi)) - ex) <= Fraction(1, 2 ** 50)
    order = O.sort_fitness(f)
    assert list(order) == golden_io.ints(rows, "order")
    for nc, (lift, emap, sm, rp, cc, wc) in ncs.items():
        lv = O.coarsen_level(g, nc)
        assert list(lv.lift) == lift, nc
        assert list(lv.coarse.emap) == emap, nc
        assert list(lv.coarse.self_mass) == sm, nc
        assert list(lv.coarse.graph.rowptr) == rp, nc
        assert list(lv.coarse.graph.col) == cc, nc
        assert list(lv.coarse.graph.w) == wc, nc


# ---- score closed forms -------------------------------------------------------------------

@pytest.mark.parametrize("n", [4, 5, 9, 30])
def test_cycle_score_is_two(n):
    """k-regular with t common neighbours: f = 2(k - t)/k; a cycle (k=2, t=0) gives 2."""
    f = O.score(I.cycle_graph(n))
    assert np.all(f == 2.0)


@pytest.mark.parametrize("n", [3, 4, 7, 12])
def test_complete_graph_score(n):
    """K_n (k = n-1, t = n-2): f = 2/(n-1) (the a and b coordinates are the only terms)."""
    f = O.score(I.complete_graph(n))
    np.testing.assert_allclose(f, 2.0 / (n - 1), rtol=1e-15)


def test_regular_triangulation_interior_is_four_thirds():
    """Interior edges of a regular triangulation: degree 6, 2 common neighbours -> 4/3."""
    nx = 12
    g = I.tri_mesh_2d(nx, nx, seed=0)
    # rebuild with every diagonal in the same direction (coin 0 everywhere)
    ii, jj = np.meshgrid(np.arange(nx), np.arange(nx))
    vid = jj * nx + ii
    eu = np.concatenate([vid[:, :-1].ravel(), vid[:-1, :].ravel(), vid[:-1, :-1].ravel()])
    ev = np.concatenate([vid[:, 1:].ravel(), vid[1:, :].ravel(), vid[1:, 1:].ravel()])
    g = I.csr_from_edges(nx * nx, eu, ev, np.ones(eu.shape[0], np.int32))
    f = O.score(g)
    deg = np.diff(g.rowptr)
    interior = (deg[g.eu] == 6) & (deg[g.ev] == 6)
    W = O.dense_weights(g) > 0
    common = (W[g.eu] & W[g.ev]).sum(axis=1)
    sel = interior & (common == 2)
    assert sel.sum() > 50
    np.testing.assert_allclose(f[sel], 4.0 / 3.0, rtol=1e-15)


def _score_identity(g):
    """||p - q||_1 = 2 - 2 sum_x min(p_x, q_x) for probability vectors p, q; the common
    coordinates of rows a and b are N(a) n N(b) (a is not in N(a), no self-loops)."""
    W = O.dense_weights(g)
    d = W.sum(axis=1)
    P = W / d[:, None]
    out = np.empty(g.m)
    for e in range(g.m):
        a, b = g.eu[e], g.ev[e]
        out[e] = 2.0 - 2.0 * np.minimum(P[a], P[b]).sum()
    return out


@pytest.mark.parametrize("seed,weight", [(0, "float"), (1, "int"), (2, "float"), (3, "unit")])
def test_score_identity_random_weighted(seed, weight):
    """Pins the weighted degree, the p_ax orientation and the a/b coordinates at once."""
    dt = np.int32 if weight in ("int", "unit") else np.float64
    g = I.random_graph(40, 0.2, seed, weight=weight, dtype=dt, connected=True)
    np.testing.assert_allclose(O.score(g), _score_identity(g), rtol=0, atol=1e-13)


def test_score_identity_float32():
    g = I.random_graph(30, 0.3, 7, weight="float", dtype=np.float32, connected=True)
    f = O.score(g)
    assert f.dtype == np.float32
    np.testing.assert_allclose(f, _score_identity(g), rtol=0, atol=2e-6)


def test_score_exact_rational():
    """The binary64 score is within a few ulps of the exact rational value (int weights)."""
    g = I.random_graph(14, 0.4, 11, weight="int", dtype=np.int32, connected=True)
    f = O.score(g)
    W = O.dense_weights(g).astype(np.int64)
    d = W.sum(axis=1)
    for e in range(g.m):
        a, b = int(g.eu[e]), int(g.ev[e])
        ex = sum(abs(Fraction(int(W[a, x]), int(d[a])) - Fraction(int(W[b, x]), int(d[b])))
                 for x in range(g.n))
        assert abs(Fraction(float(f[e])) - ex) <= ex * Fraction(g.n, 2 ** 52)


def test_degree_and_normalise_definitions():
    g = I.random_graph(25, 0.3, 5, weight="int", dtype=np.int32, connected=True)
    d = O.degree(g)
    assert np.array_equal(d, O.dense_weights(g).sum(axis=1).astype(np.int64))
    p = O.normalise(g, d)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    assert np.array_equal(p, g.w.astype(np.float64) / d[rows].astype(np.float64))


def test_score_range():
    """0 <= f <= 2 (a difference of two probability vectors)."""
    g, _ = I.config_graph("s2_tri256_f64")
    f = O.score(g)
    assert np.all(f >= 0) and np.all(f <= 2.0 + 1e-12)


# ---- sort ------------------------------------------------------------------------------

def test_sort_fitness_is_the_definition():
    g = I.random_graph(60, 0.15, 3, weight="unit", dtype=np.int32, connected=True)
    f = O.score(g)
    order = O.sort_fitness(f)
    ref = sorted(range(g.m), key=lambda e: (f[e], e))
    assert list(order) == ref
    f32 = f.astype(np.float32)
    assert list(O.sort_fitness(f32)) == sorted(range(g.m), key=lambda e: (f32[e], e))


# ---- greedy merge: brute force (P2) --------------------------------------------------------

def _threshold_partition(n, eu, ev, order, n_c):
    """Components of the shortest prefix of the sorted list that leaves n_c components (all
    edges if none does), by plain graph search on each prefix."""
    m = len(order)
    best = None
    for T in range(0, m + 1):
        sel = np.asarray(order[:T], dtype=np.int64)
        A = coo_matrix((np.ones(T), (eu[sel], ev[sel])), shape=(n, n))
        k, lab = connected_components(A, directed=False)
        best = lab
        if k <= n_c:
            break
    return _canonical(best)


def _canonical(lab):
    first = {}
    out = np.empty(len(lab), dtype=np.int32)
    for x, l in enumerate(lab):
        if l not in first:
            first[l] = len(first)
        out[x] = first[l]
    return out


def _msf_partition(n, eu, ev, order, n_c):
    """Components of the n - n_c lightest minimum-spanning-forest edges (rank as weight)."""
    m = len(order)
    rank = np.empty(m, dtype=np.int64)
    rank[np.asarray(order)] = np.arange(m)
    A = coo_matrix((rank + 1.0, (eu, ev)), shape=(n, n)).tocsr()
    T = minimum_spanning_tree(A).tocoo()
    r = np.sort((T.data - 1).astype(np.int64))
    k = max(0, n - n_c)
    keep = r[:k]
    inv = np.asarray(order)[keep]
    B = coo_matrix((np.ones(len(inv)), (eu[inv], ev[inv])), shape=(n, n))
    _, lab = connected_components(B, directed=False)
    return _canonical(lab)


def test_greedy_bruteforce_small_graphs():
    """Oracle loop == literal set-based loop == threshold components == lightest-MSF components,
    for every target n_c, on random and exhaustive tiny graphs."""
    cases = []
    for seed in range(60):
        n = 3 + seed % 7
        wt = ["unit", "int", "float"][seed % 3]
        dt = np.float64 if wt == "float" else np.int32
        cases.append(I.random_graph(n, 0.5, seed, weight=wt, dtype=dt))
    # every graph on 5 nodes with unit weights, sampled every 7th edge subset
    iu, iv = np.triu_indices(5, 1)
    for mask in range(1, 1 << len(iu), 7):
        sel = np.array([(mask >> i) & 1 for i in range(len(iu))], dtype=bool)
        cases.append(I.csr_from_edges(5, iu[sel], iv[sel], np.ones(sel.sum(), np.int32)))
    checked = 0
    for g in cases:
        if g.m == 0:
            continue
        f = O.score(g)
        order = O.sort_fitness(f)
        edges = list(zip(g.eu.tolist(), g.ev.tolist()))
        for n_c in range(1, g.n + 1):
            rep, merged, s, rc = O.greedy_merge(g, order, n_c)
            lift, nca = O.relabel(rep)
            lit, nlit = O.greedy_literal(g.n, edges, f.tolist(), n_c)
            assert nca == nlit and np.array_equal(lift, lit)
            thr = _threshold_partition(g.n, g.eu, g.ev, order, n_c)
            assert np.array_equal(lift, thr)
            msf = _msf_partition(g.n, g.eu, g.ev, order, n_c)
            assert np.array_equal(lift, msf)
            ncc = connected_components(coo_matrix((np.ones(g.m), (g.eu, g.ev)),
                                                  shape=(g.n, g.n)), directed=False)[0]
            assert nca == max(n_c, ncc)
            assert (rc == O.WARN_TARGET_NOT_REACHED) == (ncc > n_c)
            assert merged.sum() == g.n - nca
            checked += 1
    assert checked > 300


def _prefix_forest(n, eu, ev, order, ids):
    """Edge ids of the minimum spanning forest of the edges `ids` (rank in `order` as weight),
    by plain Kruskal: ascending rank, union-find with no other structure."""
    rank = np.empty(len(order), dtype=np.int64)
    rank[np.asarray(order)] = np.arange(len(order))
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    out = []
    for e in sorted(ids, key=lambda e: rank[e]):
        a, b = find(int(eu[e])), find(int(ev[e]))
        if a != b:
            parent[max(a, b)] = min(a, b)
            out.append(int(e))
    return out


def test_prefix_forest_gives_the_merges_and_extends_by_slabs():
    """Kruskal's view of Algorithm 1's merge loop, on prefixes of the sorted (f, eid) list:
    (1) for every prefix whose spanning forest holds at least k = n - n_c edges, the k
    lightest of them give the loop's partition; (2) the forest of a longer prefix is the
    forest of the shorter one plus the next slab of edges, so a selection can resume slab by
    slab instead of starting over.  Checked against the oracle's loop, not against itself."""
    cases = [I.random_graph(24 + s, 0.25, 70 + s, weight="float", dtype=np.float64,
                            connected=(s % 2 == 0)) for s in range(6)]
    cases.append(I.clique_ring(12, 4, 3, np.float64))
    cases.append(I.rgg_3d(256, 8.0, 5, np.float32))
    checked = resumed = 0
    for g in cases:
        f = O.score(g)
        order = O.sort_fitness(f)
        m = len(order)
        for n_c in (1, g.n // 8, g.n // 4, g.n // 2, g.n - 1):
            k = g.n - max(1, n_c)
            if k <= 0:
                continue
            _, merged, _, _ = O.greedy_merge(g, order, max(1, n_c))
            want = sorted(np.nonzero(merged)[0].tolist())
            rank = np.empty(m, dtype=np.int64)
            rank[order] = np.arange(m)
            for P in sorted({k, (3 * k) // 2, 2 * k, (5 * m) // 8, m}):
                P = min(P, m)
                forest = _prefix_forest(g.n, g.eu, g.ev, order, order[:P])
                if len(forest) >= k:
                    lightest = sorted(forest, key=lambda e: rank[e])[:k]
                    assert sorted(lightest) == want
                    checked += 1
                for P2 in (min(m, P + max(1, P // 2)), m):
                    whole = _prefix_forest(g.n, g.eu, g.ev, order, order[:P2])
                    slab = forest + [int(e) for e in order[P:P2]]
                    assert sorted(_prefix_forest(g.n, g.eu, g.ev, order, slab)) == sorted(whole)
                    resumed += 1
    assert checked > 60 and resumed > 100


def test_relabel_is_first_occurrence_order():
    g = I.random_graph(50, 0.1, 9, weight="float", dtype=np.float64, connected=True)
    lv = O.coarsen_level(g, 17)
    # ids appear in increasing order of first occurrence when scanning nodes 0..n-1
    seen = -1
    for x in range(g.n):
        if lv.lift[x] > seen:
            assert lv.lift[x] == seen + 1
            seen = lv.lift[x]
    assert seen + 1 == lv.n_c == 17


# ---- contraction (P5) ----------------------------------------------------------------------

def _check_contraction(g, lv):
    co = lv.coarse
    C = O.membership(lv.lift, lv.n_c)
    A = C.T @ O.dense_weights(g) @ C          # Definition 1 summed over super-node pairs
    off = A - np.diag(np.diag(A))
    Gc = O.dense_weights(co.graph)
    np.testing.assert_allclose(Gc, off, rtol=1e-12, atol=0)
    np.testing.assert_allclose(2.0 * co.self_mass.astype(np.float64), np.diag(A), rtol=1e-12)
    # weight conservation
    tot = g.w_und.astype(np.float64).sum()
    np.testing.assert_allclose(co.a_und.astype(np.float64).sum()
                               + co.self_mass.astype(np.float64).sum(), tot, rtol=1e-12)
    # emap: fine edge -> coarse edge with matching endpoints
    U = lv.lift[g.eu]; V = lv.lift[g.ev]
    inter = U != V
    assert np.all((co.emap >= 0) == inter)
    ce = co.emap[inter]
    assert np.array_equal(co.graph.eu[ce], np.minimum(U, V)[inter])
    assert np.array_equal(co.graph.ev[ce], np.maximum(U, V)[inter])
    # every super-node induces a connected subgraph of G
    for s in range(lv.n_c):
        mem = np.nonzero(lv.lift == s)[0]
        if len(mem) > 1:
            sub = O.dense_weights(g)[np.ix_(mem, mem)] > 0
            assert connected_components(sub, directed=False)[0] == 1
    # symmetric coarse CSR with sorted rows
    rows = np.repeat(np.arange(lv.n_c), np.diff(co.graph.rowptr))
    for r in range(lv.n_c):
        seg = co.graph.col[co.graph.rowptr[r]:co.graph.rowptr[r + 1]]
        assert np.all(np.diff(seg) > 0)
    assert not np.any(co.graph.col == rows)


@pytest.mark.parametrize("seed,weight,nc", [(0, "int", 10), (1, "float", 5), (2, "unit", 25),
                                            (3, "float", 1), (4, "int", 30)])
def test_contraction_matches_dense_definition(seed, weight, nc):
    dt = np.float64 if weight == "float" else np.int32
    g = I.random_graph(30, 0.15, seed, weight=weight, dtype=dt, connected=(seed % 2 == 0))
    lv = O.coarsen_level(g, nc)
    _check_contraction(g, lv)


def test_contraction_float32_order():
    """F32 coarse weights are sums in ascending fine edge id (checked by replaying them)."""
    g = I.random_graph(40, 0.2, 21, weight="float", dtype=np.float32, connected=True)
    lv = O.coarsen_level(g, 6)
    co = lv.coarse
    for k in range(co.m_c):
        es = np.nonzero(co.emap == k)[0]
        s = np.float32(0)
        for e in es:
            s = np.float32(s + g.w_und[e])
        assert s == co.a_und[k]


def test_int_overflow_is_reported():
    g = I.csr_from_edges(3, np.array([0, 1]), np.array([1, 2]),
                         np.array([2 ** 31 - 1, 2 ** 31 - 1], dtype=np.int32))
    lift = np.array([0, 1, 1], dtype=np.int32)
    O.contract(g, lift, 2)  # one fine edge per coarse edge: fits
    g2 = I.csr_from_edges(3, np.array([0, 0]), np.array([1, 2]),
                          np.array([2 ** 31 - 1, 2 ** 31 - 1], dtype=np.int32))
    with pytest.raises(OverflowError):
        O.contract(g2, lift, 2)


# ---- spectral pins: Theorem 1 (P1) and the lift invariant (P3) ----------------------------

def _lift_eigs(W, lift, n_c):
    return np.linalg.eigvalsh(O.laplacian_norm(O.lift_weights(W, lift, n_c)))


def test_theorem1_single_merges():
    """||Lambda - Lambda_hat||_inf <= f(a, b) for every single-edge merge (Theorem 1)."""
    checked = 0
    for seed in range(40):
        n = 4 + seed % 5
        wt = ["float", "int", "unit"][seed % 3]
        dt = np.float64 if wt == "float" else np.int32
        g = I.random_graph(n, 0.6, 100 + seed, weight=wt, dtype=dt, connected=True)
        W = O.dense_weights(g)
        lam = np.linalg.eigvalsh(O.laplacian_norm(W))
        f = O.score(g)
        for e in range(g.m):
            a, b = int(g.eu[e]), int(g.ev[e])
            rep = np.arange(n, dtype=np.int32)
            rep[b] = a
            lift, nc = O.relabel(rep)
            lam_hat = _lift_eigs(W, lift, nc)
            assert np.max(np.abs(lam - lam_hat)) <= f[e] + 1e-12
            checked += 1
    assert checked > 200


def test_theorem2_multi_merges():
    """s merges whose scores are all <= eps move eigenvalues by at most s(s+1)/2 eps."""
    for seed in range(20):
        g = I.random_graph(8, 0.5, 300 + seed, weight="float", dtype=np.float64, connected=True)
        W = O.dense_weights(g)
        lam = np.linalg.eigvalsh(O.laplacian_norm(W))
        for n_c in range(2, 8):
            lv = O.coarsen_level(g, n_c)
            s = int(lv.merged.sum())
            eps = float(lv.f[lv.merged].max())
            lam_hat = _lift_eigs(W, lv.lift, lv.n_c)
            assert np.max(np.abs(lam - lam_hat)) <= s * (s + 1) / 2 * eps + 1e-12


def test_lift_invariant_small():
    """eig(L(G_hat)) = eig(L_c) plus (n - n_c) eigenvalues equal to 1, where L_c is the
    normalized Laplacian of C^T W C built from the oracle's coarse graph and self-mass."""
    for seed in range(12):
        g = I.random_graph(9, 0.4, 500 + seed, weight="float", dtype=np.float64,
                           connected=True)
        W = O.dense_weights(g)
        for n_c in (2, 4, 7):
            lv = O.coarsen_level(g, n_c)
            Ac = O.dense_weights(lv.coarse.graph) + 2.0 * np.diag(lv.coarse.self_mass)
            lc = np.linalg.eigvalsh(O.laplacian_norm(Ac))
            lh = _lift_eigs(W, lv.lift, lv.n_c)
            ref = np.sort(np.concatenate([lc, np.ones(g.n - lv.n_c)]))
            np.testing.assert_allclose(lh, ref, atol=1e-10)


def test_lift_matrix_form_matches_definition():
    """C S^-1 (C^T W C) S^-1 C^T equals Definition 2's double sum (used for large checks)."""
    g = I.random_graph(12, 0.4, 77, weight="float", dtype=np.float64, connected=True)
    lv = O.coarsen_level(g, 5)
    W = O.dense_weights(g)
    C = O.membership(lv.lift, lv.n_c)
    Sinv = np.diag(1.0 / C.sum(axis=0))
    np.testing.assert_allclose(C @ Sinv @ (C.T @ W @ C) @ Sinv @ C.T,
                               O.lift_weights(W, lv.lift, lv.n_c), rtol=1e-13)


@pytest.mark.slow
def test_c1_mesh_eigen_check():
    """64x64 triangle mesh, one level to 2048: the lift invariant by dense FP64 eigensolves
    (4096^2 and 2048^2), and the 10 smallest eigenvalues of G against the lift."""
    g, cfg = I.config_graph("c1_tri64_unit")
    lv = O.coarsen_level(g, 2048)
    assert lv.n_c == 2048 and lv.status == O.OK
    W = O.dense_weights(g)
    C = O.membership(lv.lift, lv.n_c)
    A = C.T @ W @ C
    Ac = O.dense_weights(lv.coarse.graph) + 2.0 * np.diag(lv.coarse.self_mass.astype(float))
    np.testing.assert_array_equal(A, Ac)
    lc = np.linalg.eigvalsh(O.laplacian_norm(Ac))
    sizes = C.sum(axis=0)
    What = (C / sizes) @ A @ (C / sizes).T
    lh = np.linalg.eigvalsh(O.laplacian_norm(What))
    ref = np.sort(np.concatenate([lc, np.ones(g.n - lv.n_c)]))
    np.testing.assert_allclose(lh, ref, atol=1e-10)
    lam = np.linalg.eigvalsh(O.laplacian_norm(W))
    # smallest eigenvalue is the trivial 0 for both; the lift's spectrum stays in [0, 2]
    assert abs(lam[0]) < 1e-10 and abs(lh[0]) < 1e-10
    assert lh[-1] <= 2.0 + 1e-10
    assert np.all(np.abs(lam[:10] - lh[:10]) <= 2.0)


# ---- backward (P6) --------------------------------------------------------------------------

def test_contract_backward_adjoint_and_fd():
    g = I.random_graph(30, 0.2, 41, weight="float", dtype=np.float64, connected=True)
    lv = O.coarsen_level(g, 8)
    co = lv.coarse
    S = np.zeros((co.m_c, g.m))
    for e in range(g.m):
        if co.emap[e] >= 0:
            S[co.emap[e], e] = 1.0
    rng = np.random.default_rng(0)
    gw = rng.standard_normal(co.m_c)
    gr = O.contract_backward(co.emap, gw)
    np.testing.assert_array_equal(gr, S.T @ gw)
    # adjoint identity <S w, g> = <w, S^T g>
    w = g.w_und
    np.testing.assert_allclose(np.dot(co.a_und, gw), np.dot(w, gr), rtol=1e-12)
    # central differences of L(w) = sum_k a_k(w) g_k with the assignment held fixed
    h = 1e-3
    for e in rng.choice(g.m, 10, replace=False):
        wp = w.copy(); wp[e] += h
        wm = w.copy(); wm[e] -= h
        ap = O.contract(_with_weights(g, wp), lv.lift, lv.n_c).a_und
        am = O.contract(_with_weights(g, wm), lv.lift, lv.n_c).a_und
        fd = (np.dot(ap, gw) - np.dot(am, gw)) / (2 * h)
        assert abs(fd - gr[e]) < 1e-9


def _with_weights(g, w_und):
    return I.csr_from_edges(g.n, g.eu, g.ev, w_und)


# ---- multilevel and batch drivers -------------------------------------------------------------

def test_multilevel_composition():
    g, _ = I.config_graph("s2_tri256_f64")
    levels, total = O.coarsen(g, 64, "halving")
    assert [lv.n_c for lv in levels] == [g.n // 2 ** l for l in range(1, 7)]
    # the composed map is onto [0, n_c) and the final coarse graph conserves weight
    assert set(np.unique(total)) == set(range(levels[-1].n_c))
    sm = 0.0
    for lv in levels:
        sm += lv.coarse.self_mass.sum()
    np.testing.assert_allclose(levels[-1].coarse.a_und.sum() + sm, g.w_und.sum(), rtol=1e-11)
    em = O.compose_emaps(levels)
    fin = levels[-1].coarse.graph
    U = total[g.eu]; V = total[g.ev]
    assert np.all((em >= 0) == (U != V))
    sel = em >= 0
    assert np.array_equal(fin.eu[em[sel]], np.minimum(U, V)[sel])


def test_batch_oracle_is_per_graph():
    b, _ = I.config_graph("s5_batch40_f32")
    res = O.coarsen_batch(b, 8, "halving")
    for gi, (levels, total) in enumerate(res):
        n = int(b.graph_ptr[gi + 1] - b.graph_ptr[gi])
        assert levels[-1].n_c == n // 8


def test_parallel_score_is_the_sequential_score():
    """The edge-partitioned parallel score (the CPU baseline) only shares out the edges: the
    same bits as the sequential score on a mesh, a binary32 random graph, integer weights and
    a heavy-tailed graph."""
    graphs = [I.tri_mesh_2d(40, 30, 1, jitter=0.3, weight="inv_len", dtype=np.float64),
              I.random_graph(300, 0.05, 2, weight="float", dtype=np.float32, connected=True),
              I.random_graph(200, 0.08, 3, weight="int", dtype=np.int32, connected=True),
              I.powerlaw_graph(800, 6, 4, "float", np.float64)]
    for g in graphs:
        f = O.score(g)
        fp, threads = O.score_parallel(g)
        assert threads >= 1
        bits = np.uint64 if f.dtype.itemsize == 8 else np.uint32
        assert fp.dtype == f.dtype and np.array_equal(f.view(bits), fp.view(bits))


# ---- node-feature pooling (mean over super-node members) ----------------------------------------

def _round_f32(q: Fraction) -> np.float32:
    """The binary32 value nearest to q (ties to even), found from exact comparisons."""
    c = np.float32(float(q))
    best = None
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        d = abs(Fraction(float(cand)) - q)
        even = (int(np.array(cand).view(np.uint32)) & 1) == 0
        if best is None or d < best[0] or (d == best[0] and even):
            best = (d, cand)
    return best[1]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_pool_features_exact_means(dtype):
    """Dyadic features (exact sums): every pooled value is the correctly rounded quotient of
    the exact member sum by the member count, computed with rationals."""
    rng = np.random.default_rng(11)
    n, n_c, F = 500, 37, 5
    lift = np.sort(rng.integers(0, n_c, size=n)).astype(np.int32)
    lift[:n_c] = np.arange(n_c)  # every super-node used
    rng.shuffle(lift)
    x = (rng.integers(-1000, 1000, size=(n, F)) / 256.0).astype(dtype)
    xc = O.pool_features(lift, n_c, x)
    for u in range(n_c):
        mem = np.nonzero(lift == u)[0]
        for f in range(F):
            q = sum(Fraction(float(x[v, f])) for v in mem) / len(mem)
            want = float(q) if dtype == np.float64 else _round_f32(q)
            assert xc[u, f] == want, (u, f)


def test_pool_features_sums_in_ascending_member_order():
    """Members 3 < 8 < 20 hold 1e16, 1, -1e16: in ascending order 1e16 + 1 rounds back to
    1e16 and the mean is 0; any other order that adds the 1 last gives 1/3."""
    lift = np.zeros(25, dtype=np.int32)
    lift[[3, 8, 20]] = 1
    x = np.zeros((25, 1))
    x[3, 0], x[8, 0], x[20, 0] = 1e16, 1.0, -1e16
    xc = O.pool_features(lift, 2, x)
    assert xc[1, 0] == 0.0 and xc[0, 0] == 0.0


def test_pool_backward_is_the_adjoint():
    """<pool(x), g> = <x, pool_backward(g)>: exact for dyadic values and power-of-two member
    counts; and the pooled-then-lifted features keep the total mass."""
    rng = np.random.default_rng(12)
    n_c, F = 16, 3
    sizes = 2 ** rng.integers(0, 5, size=n_c)
    lift = np.repeat(np.arange(n_c), sizes).astype(np.int32)
    rng.shuffle(lift)
    n = lift.shape[0]
    x = rng.integers(-64, 64, size=(n, F)) / 8.0
    g = rng.integers(-64, 64, size=(n_c, F)) / 8.0
    xc = O.pool_features(lift, n_c, x)
    gx = O.pool_backward(lift, n_c, g)
    assert float(np.sum(xc * g)) == float(np.sum(x * gx))
    assert np.array_equal((xc * sizes[:, None]).sum(0), x.sum(0))


def test_pool_features_tree_order():
    """258 members: 1e16, 255 zeros, 1, 1.  Chunks of 256: (1e16) + (1 + 1) = 1e16 + 2 exactly,
    so the mean is (1e16 + 2) / 258 correctly rounded; a plain left-to-right sum would lose both
    ones (1e16 + 1 rounds to 1e16) and give 1e16 / 258."""
    lift = np.zeros(300, dtype=np.int32)
    mem = np.arange(20, 278)
    lift[mem] = 1
    x = np.zeros((300, 1))
    x[mem[0], 0] = 1e16
    x[mem[-2], 0] = 1.0
    x[mem[-1], 0] = 1.0
    xc = O.pool_features(lift, 2, x)
    assert xc[1, 0] == float(Fraction(10 ** 16 + 2, 258))
    assert xc[1, 0] != float(Fraction(10 ** 16, 258))


def test_pool_features_three_tree_levels():
    """258 * 256 members: 1e16 first, a 1 at the start of chunks 256 and 257, zeros elsewhere.
    The 258 chunk sums exceed 256, so they are summed in two groups: (1e16 + 0 ...) and
    (1 + 1), then 1e16 + 2 exactly.  Adding the 258 chunk sums left to right instead would
    round both ones away."""
    L = 258 * 256
    lift = np.ones(L + 5, dtype=np.int32)
    lift[:5] = 0
    x = np.zeros((L + 5, 1))
    x[5, 0] = 1e16
    x[5 + 256 * 256, 0] = 1.0
    x[5 + 257 * 256, 0] = 1.0
    xc = O.pool_features(lift, 2, x)
    assert xc[1, 0] == float(Fraction(10 ** 16 + 2, L))
    assert xc[0, 0] == 0.0


# ---- the self-mass reading of the multilevel driver (the merged node of Theorem 2's proof) ----

def _dense_rows(g):
    """Dense weight matrix of a CSR that may hold diagonal entries."""
    M = np.zeros((g.n, g.n))
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    M[rows, g.col] = g.w
    return M


def test_self_mass_scores_are_the_merged_node_definition():
    """With the self-mass on the diagonal, the next level's score of super-nodes (U, X) equals,
    in exact rationals, || sum_{x in U} w_x / sum_{x in U} d_x - (the same for X) ||_1 with the
    fine rows aggregated into super-node coordinates: the merged node (w_a + w_b) / (d_a + d_b)
    of the proof of Theorem 2, repeated.  Without it, some scores differ."""
    differs = 0
    for seed in range(12):
        g = I.random_graph(10, 0.45, 1200 + seed, weight="int", dtype=np.int32, connected=True)
        lv = O.coarsen_level(g, 5)
        co = lv.coarse
        g2 = O.with_self_mass(co.graph, co.self_mass)
        f2 = O.score(g2)
        f_r7 = O.score(co.graph)
        W = O.dense_weights(g).astype(np.int64)
        d = W.sum(axis=1)
        agg = np.zeros((lv.n_c, lv.n_c), dtype=np.int64)      # C^T W C, diagonal included
        for x in range(g.n):
            for y in range(g.n):
                agg[lv.lift[x], lv.lift[y]] += W[x, y]
        D = np.zeros(lv.n_c, dtype=np.int64)
        for x in range(g.n):
            D[lv.lift[x]] += d[x]
        for e in range(co.graph.m):
            U, X = int(co.graph.eu[e]), int(co.graph.ev[e])
            exact = sum(abs(Fraction(int(agg[U, y]), int(D[U])) - Fraction(int(agg[X, y]), int(D[X])))
                        for y in range(lv.n_c))
            assert abs(Fraction(float(f2[e])) - exact) <= Fraction(1, 2 ** 48)
            differs += f_r7[e] != f2[e]
    assert differs > 0


def test_theorem2_proof_inequality_needs_the_self_mass():
    """The proof of Theorem 2 bounds the merged node's distance from a member:
    || w_a/d_a - (w_a + w_b)/(d_a + d_b) ||_1 <= f(a, b) / (d_a/d_b + 1).  Merging one edge and
    reading the merged row from the next level's graph (in super-node coordinates, where the
    distance can only shrink) satisfies it for every edge with the self-mass on the diagonal;
    the graph without self-mass breaks it."""
    broken = 0
    checked = 0
    for seed in range(25):
        g = I.random_graph(9, 0.5, 1300 + seed, weight="float", dtype=np.float64,
                           connected=True)
        W = O.dense_weights(g)
        d = W.sum(axis=1)
        f = O.score(g)
        for e in range(g.m):
            a, b = int(g.eu[e]), int(g.ev[e])
            rep = np.arange(g.n, dtype=np.int32)
            rep[b] = a
            lift, nc = O.relabel(rep)
            co = O.contract(g, lift, nc)
            C = O.membership(lift, nc)
            member = (W[a] @ C) / d[a]                 # w_a / d_a in super-node coordinates
            U = int(lift[a])
            bound = float(f[e]) / (d[a] / d[b] + 1.0)
            for gg, with_mass in ((O.with_self_mass(co.graph, co.self_mass), True),
                                  (co.graph, False)):
                M = _dense_rows(gg)
                merged = M[U] / O.degree(gg)[U]
                dist = float(np.abs(member - merged).sum())
                if with_mass:
                    assert dist <= bound + 1e-12, (seed, e)
                else:
                    broken += dist > bound + 1e-12
            checked += 1
    assert checked > 300 and broken > 0


def test_self_mass_accumulates_internal_weight():
    """For integer weights the carried mass of every super-node is exactly the total weight of
    the original edges inside it, at every level; the first level does not depend on the
    reading."""
    g = I.random_graph(200, 0.04, 7, weight="int", dtype=np.int32, connected=True)
    ref, _ = O.coarsen(g, 8, "halving", self_mass_degree=False)
    levels, total = O.coarsen(g, 8, "halving")
    assert np.array_equal(levels[0].lift, ref[0].lift)
    comp = np.arange(g.n)
    for lv in levels:
        comp = lv.lift[comp]
        inside = comp[g.eu] == comp[g.ev]
        want = np.bincount(comp[g.eu][inside], weights=g.w_und[inside].astype(np.float64),
                           minlength=lv.n_c).astype(np.int64)
        assert np.array_equal(lv.mass, want)
    assert np.array_equal(comp, total)


def test_self_mass_reading_keeps_the_mesh_spectrum():
    """A 128 x 128 mesh halved four times (n/16): without the self-mass one super-node takes
    most of the graph and the lift loses the low spectrum; with it the super-nodes stay small
    and the first 20 eigenvectors stay aligned (the Figure 2 comparison)."""
    torch = pytest.importorskip("torch")
    from paper_2204_11757_gb300 import spectral as S
    g = I.tri_mesh_2d(128, 128, 7, jitter=0.3, weight="inv_len", dtype=np.float64)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    out = {}
    for sm in (False, True):
        levels, lift = O.coarsen(g, 16, "halving", self_mass_degree=sm)
        n_c = levels[-1].n_c
        rep = S.spectral_alignment_sparse(g.n, t(g.rowptr), t(g.col), t(g.w), t(lift), n_c,
                                          k=20)
        out[sm] = (np.bincount(lift).max() / g.n, float(rep.alignment.mean()),
                   rep.max_eig_diff)
    assert out[False][0] > 0.5 and out[False][1] < 0.5
    assert out[True][0] < 0.05 and out[True][1] > 0.85
    assert out[True][2] < out[False][2] / 5


def test_with_self_mass_edge_cases():
    """Zero mass leaves the CSR as it was; a diagonal that does not fit int32 weights is an
    error; diagonal entries sit in ascending-column order and leave the edge ids alone."""
    g = I.random_graph(30, 0.2, 5, weight="int", dtype=np.int32, connected=True)
    z = O.with_self_mass(g, np.zeros(g.n, dtype=np.int64))
    assert np.array_equal(z.rowptr, g.rowptr) and np.array_equal(z.col, g.col)
    assert np.array_equal(z.w, g.w)
    mass = np.zeros(g.n, dtype=np.int64)
    mass[[0, 7, g.n - 1]] = [3, 1, 5]
    h = O.with_self_mass(g, mass)
    assert h.rowptr[-1] == g.rowptr[-1] + 3
    for x in range(g.n):
        row = h.col[h.rowptr[x]:h.rowptr[x + 1]]
        assert np.all(np.diff(row) > 0)
        if mass[x]:
            assert h.w[h.rowptr[x] + np.searchsorted(row, x)] == 2 * mass[x]
    # a diagonal entry lies in its own row only: edges away from the massed nodes keep their bits
    f, fh = O.score(g), O.score(h)
    away = (mass[g.eu] == 0) & (mass[g.ev] == 0)
    assert np.array_equal(f[away].view(np.uint64), fh[away].view(np.uint64))
    assert np.all(f[~away] != fh[~away])
    big = np.zeros(g.n, dtype=np.int64)
    big[3] = 2 ** 30
    with pytest.raises(OverflowError):
        O.with_self_mass(g, big)


def test_batch_oracle_self_mass_reading_is_per_graph():
    """The batch oracle takes the self-mass reading graph by graph: each graph reaches its own
    target and carries a non-negative finite mass."""
    batch = I.mesh_batch(4, 3, nmin=200, nmax=600, dtype=np.float64)
    per = O.coarsen_batch(batch, 8, "halving", self_mass_degree=True)
    gp = batch.graph_ptr
    for b, (levels, total) in enumerate(per):
        n0, n1 = int(gp[b]), int(gp[b + 1])
        assert total.shape[0] == n1 - n0
        assert levels[-1].n_c == max(1, (n1 - n0) // 8)
        assert np.all(np.isfinite(levels[-1].mass)) and levels[-1].mass.min() >= 0


def test_carried_mass_order_is_ascending_members_then_self_mass():
    """The carried mass of a super-node is its members' masses in ascending member id, summed
    left to right from 0, then this level's self-mass.  In binary32 the order shows: 2^24 + 1 + 1
    stays 2^24 left to right (each 1 is a tie to even), while 1 + 1 + 2^24 would give 2^24 + 2."""
    big = np.float32(2 ** 24)
    mass = np.array([big, 5, 1, 7, 1], dtype=np.float32)
    lift = np.array([0, 1, 0, 1, 0], dtype=np.int32)
    self_mass = np.array([1, 3], dtype=np.float32)
    got = O.carry_self_mass(mass, lift, 2, self_mass)
    want = np.zeros(2, dtype=np.float32)
    for x in range(5):                      # ascending member id
        want[lift[x]] = np.float32(want[lift[x]] + mass[x])
    want = (want + self_mass).astype(np.float32)
    assert got.dtype == np.float32
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert got[0] == big and got[1] == np.float32(15)
    # the reverse member order would have kept the two ones
    assert np.float32(np.float32(1 + 1) + big) + 1 != got[0]


def _hop_dists_bruteforce(g):
    """All-pairs hop distances by a textbook queue BFS from every node (None: unreachable)."""
    from collections import deque
    adj = [g.col[g.rowptr[x]:g.rowptr[x + 1]].tolist() for x in range(g.n)]
    out = []
    for s in range(g.n):
        dist = [None] * g.n
        dist[s] = 0
        q = deque([s])
        while q:
            x = q.popleft()
            for y in adj[x]:
                if dist[y] is None:
                    dist[y] = dist[x] + 1
                    q.append(y)
        out.append(dist)
    return out


def test_cluster_order_is_hop_min_label_then_id():
    """The reordering's order against its definition by brute force: L_k(x) is the smallest id
    among the nodes within k hops of x (all-pairs BFS), and new ids ascend with
    (L_8(x), L_2(x), x); every round of the oracle's label propagation equals L_k."""
    graphs = [I.path_graph(19), I.cycle_graph(24), I.complete_graph(5)]
    for seed in range(6):
        graphs.append(I.random_graph(60, 0.05, 40 + seed, weight="float", dtype=np.float64,
                                     connected=seed % 2 == 0))
    graphs.append(I.tri_mesh_2d(9, 7, 3, jitter=0.3, weight="inv_len", dtype=np.float64))
    for g in graphs:
        d = _hop_dists_bruteforce(g)
        lab = lambda x, k: min(y for y in range(g.n) if d[x][y] is not None and d[x][y] <= k)
        labels = O.hop_min_labels(g, O.REORDER_HOPS)
        for k in range(O.REORDER_HOPS + 1):
            assert labels[k].tolist() == [lab(x, k) for x in range(g.n)]
        perm = O.cluster_order(g)
        assert sorted(perm.tolist()) == list(range(g.n))
        want = sorted(range(g.n), key=lambda x: (lab(x, O.REORDER_HOPS), lab(x, O.REORDER_SUB), x))
        assert [int(np.nonzero(perm == i)[0][0]) for i in range(g.n)] == want
    # a path 0 - 1 - ... - 18 renumbered: node x's 8-hop label is max(0, x - 8), so the nodes
    # within 8 hops of 0 come first, then one node per label
    g = I.path_graph(19)
    assert O.hop_min_labels(g, 8)[8].tolist() == [max(0, x - 8) for x in range(19)]


def test_permuted_graph_is_the_same_graph():
    """permute() renames nodes only: the renamed weighted adjacency matrix equals the
    original's, rows stay sorted, and the undirected edge list follows the new upper triangle."""
    g = I.random_graph(80, 0.06, 9, weight="float", dtype=np.float64, connected=True)
    perm = O.cluster_order(g)
    h = O.permute(g, perm)
    W, H = O.dense_weights(g), O.dense_weights(h)
    assert np.array_equal(H[np.ix_(perm, perm)], W)
    for x in range(h.n):
        assert np.all(np.diff(h.col[h.rowptr[x]:h.rowptr[x + 1]]) > 0)
    assert h.m == g.m and np.all(h.eu < h.ev)
    assert np.all(np.diff(h.eu.astype(np.int64) * h.n + h.ev) > 0)


def test_reordered_coarsening_is_a_coarsening_of_the_input():
    """The reordering option coarsens an isomorphic copy: its lift, read on the input graph, is
    a partition of the target size whose super-nodes are connected, and its coarse graph's total
    weight plus the carried mass equals the input's total weight."""
    g = I.tri_mesh_2d(30, 20, 4, jitter=0.3, weight="inv_len", dtype=np.float64)
    levels, lift, perm = O.coarsen_reordered(g, 8, "halving")
    assert lift.max() + 1 == levels[-1].n_c == g.n // 8
    for U in range(levels[-1].n_c):
        members = set(np.nonzero(lift == U)[0].tolist())
        seen, stack = set(), [next(iter(members))]
        while stack:
            x = stack.pop()
            if x in seen:
                continue
            seen.add(x)
            stack.extend(int(y) for y in g.col[g.rowptr[x]:g.rowptr[x + 1]] if y in members)
        assert seen == members
    last = levels[-1]
    np.testing.assert_allclose(last.coarse.a_und.sum() + last.mass.sum(), g.w_und.sum(),
                               rtol=1e-12)
