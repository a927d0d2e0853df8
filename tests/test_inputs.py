"""The seeded input generators match the structure their recipes state (CPU only): closed-form
edge counts of the meshes, the random geometric graph's edge rule by brute force over all point
pairs, canonical symmetric CSR, and block-diagonal batches whose blocks are the standalone
generators' graphs."""
import math

import numpy as np
import pytest

from paper_2204_11757_gb300 import inputs as I


def _check_canonical(g):
    """Symmetric CSR with strictly ascending columns, no self-loops, and an undirected edge list
    (eu < ev) in lexicographic order whose weights are the CSR's."""
    n = g.n
    assert g.rowptr[0] == 0 and g.rowptr[-1] == g.nnz and np.all(np.diff(g.rowptr) >= 0)
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    assert np.all(g.col >= 0) and np.all(g.col < n) and not np.any(g.col == rows)
    for x in range(0, n, max(1, n // 97)):
        c = g.col[g.rowptr[x]:g.rowptr[x + 1]]
        assert np.all(np.diff(c) > 0)
    dense = {}
    for r, c, w in zip(rows.tolist(), g.col.tolist(), g.w.tolist()):
        dense[(r, c)] = w
    for (r, c), w in dense.items():
        assert dense[(c, r)] == w
    assert g.nnz == 2 * g.m
    assert np.all(g.eu < g.ev)
    key = g.eu.astype(np.int64) * n + g.ev
    assert np.all(np.diff(key) > 0)
    for e in range(g.m):
        assert dense[(int(g.eu[e]), int(g.ev[e]))] == g.w_und[e]


@pytest.mark.parametrize("nx,ny", [(2, 2), (5, 3), (17, 11)])
def test_tri_mesh_edge_count_and_one_diagonal_per_cell(nx, ny):
    g = I.tri_mesh_2d(nx, ny, seed=nx * ny, jitter=0.3, weight="inv_len", dtype=np.float64)
    assert g.n == nx * ny
    assert g.m == (nx - 1) * ny + nx * (ny - 1) + (nx - 1) * (ny - 1)
    _check_canonical(g)
    edges = set(zip(g.eu.tolist(), g.ev.tolist()))
    for j in range(ny - 1):
        for i in range(nx - 1):
            a, b, c, d = j * nx + i, j * nx + i + 1, (j + 1) * nx + i, (j + 1) * nx + i + 1
            assert ((a, d) in edges) != ((b, c) in edges)  # exactly one diagonal
    # a triangulated grid is planar: m <= 3n - 6
    assert g.m <= 3 * g.n - 6 or g.n < 3


@pytest.mark.parametrize("k", [2, 3, 6])
def test_tet_mesh_edge_count_and_kuhn_diagonals(k):
    g = I.tet_mesh_3d(k, seed=k, jitter=0.25, weight="inv_len", dtype=np.float64)
    assert g.n == k ** 3
    assert g.m == 3 * (k - 1) * k * k + 3 * (k - 1) ** 2 * k + (k - 1) ** 3
    _check_canonical(g)
    # every cell holds its (0,0,0)-(1,1,1) diagonal and not the other three body diagonals
    edges = set(zip(g.eu.tolist(), g.ev.tolist()))
    vid = lambda x, y, z: (z * k + y) * k + x
    for z in range(k - 1):
        for y in range(k - 1):
            for x in range(k - 1):
                assert (vid(x, y, z), vid(x + 1, y + 1, z + 1)) in edges
                assert (vid(x + 1, y, z), vid(x, y + 1, z + 1)) not in edges


def test_mesh_weights_are_inverse_lengths():
    g = I.tri_mesh_2d(6, 5, seed=3, jitter=0.3, weight="inv_len", dtype=np.float64)
    # the jitter is the second draw of the generator's stream (after one coin per cell)
    rng = np.random.Generator(np.random.PCG64(3))
    rng.integers(0, 2, size=(4, 5), dtype=np.int8)
    ii, jj = np.meshgrid(np.arange(6.0), np.arange(5.0))
    pts = np.stack([ii.ravel(), jj.ravel()], axis=1) + rng.uniform(-0.3, 0.3, size=(30, 2))
    d = np.linalg.norm(pts[g.eu] - pts[g.ev], axis=1)
    assert np.allclose(g.w_und, 1.0 / d, rtol=1e-14, atol=0.0)


@pytest.mark.parametrize("n,deg,dt", [(1500, 12.0, np.float32), (700, 6.0, np.float64)])
def test_rgg_is_every_pair_within_the_radius(n, deg, dt):
    """The cell-bucketed search finds exactly the pairs that brute force over all n(n-1)/2 pairs
    finds, with weight exp(-d^2/r^2) rounded once to the weight type."""
    g = I.rgg_3d(n, deg, seed=11, dtype=dt)
    _check_canonical(g)
    pts = np.random.Generator(np.random.PCG64(11)).random((n, 3))
    r = (3.0 * deg / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    iu, iv = np.triu_indices(n, 1)
    diff = pts[iu] - pts[iv]
    d2 = np.einsum("ij,ij->i", diff, diff)
    sel = d2 < r * r
    assert g.m == int(sel.sum())
    assert np.array_equal(g.eu, iu[sel]) and np.array_equal(g.ev, iv[sel])
    assert np.array_equal(g.w_und, np.exp(-d2[sel] / (r * r)).astype(dt))
    # mean degree near the target (boundary nodes have fewer neighbours)
    assert 0.6 * deg < 2 * g.m / n < 1.05 * deg


def test_batch_blocks_are_the_standalone_graphs():
    b = I.mesh_batch(12, seed=7, nmin=20, nmax=400, dtype=np.float32)
    assert b.B == 12 and b.graph_ptr[0] == 0 and b.graph_ptr[-1] == b.graph.n
    _check_canonical(b.graph)
    g = b.graph
    # no edge leaves its graph's node range
    owner = np.searchsorted(b.graph_ptr, np.arange(g.n), side="right") - 1
    assert np.array_equal(owner[g.eu], owner[g.ev])
    # each block equals the generator's graph for that block's draws
    rng = np.random.Generator(np.random.PCG64(7))
    sizes = np.exp(rng.uniform(math.log(20), math.log(400), size=12))
    coins = rng.integers(0, 2, size=12)
    seeds = rng.integers(0, 2**62, size=12)
    for k in range(12):
        lo, hi = int(b.graph_ptr[k]), int(b.graph_ptr[k + 1])
        if coins[k] == 0:
            s = max(2, int(round(math.sqrt(sizes[k]))))
            ref = I.tri_mesh_2d(s, s, int(seeds[k]), 0.3, "inv_len", np.float32)
        else:
            s = max(2, int(round(sizes[k] ** (1.0 / 3.0))))
            ref = I.tet_mesh_3d(s, int(seeds[k]), 0.25, "inv_len", np.float32)
        assert b.kinds[k] == (2 if coins[k] == 0 else 3)
        assert hi - lo == ref.n
        sel = owner[g.eu] == k
        assert np.array_equal(g.eu[sel] - lo, ref.eu) and np.array_equal(g.ev[sel] - lo, ref.ev)
        assert np.array_equal(g.w_und[sel], ref.w_und)


def test_csr_from_edges_rejects_loops_and_duplicates():
    with pytest.raises(ValueError):
        I.csr_from_edges(3, np.array([0, 1]), np.array([1, 1]), np.ones(2))
    with pytest.raises(ValueError):
        I.csr_from_edges(3, np.array([0, 1]), np.array([1, 0]), np.ones(2))
