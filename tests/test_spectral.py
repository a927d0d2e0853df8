"""The spectral-quality diagnostic (eigenvalues and eigenvector overlaps of L(G) and of the
lift of G_c) against the oracle's dense definitions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2204_11757_gb300 import inputs as I
from paper_2204_11757_gb300 import spectral as S


def _case():
    g = I.tri_mesh_2d(20, 18, 3, jitter=0.3, weight="inv_len", dtype=np.float64)
    levels, lift = O.coarsen(g, 4, "halving")
    return g, lift, levels[-1].n_c


def _tensors(g, device="cpu"):
    return (torch.from_numpy(g.rowptr).to(device), torch.from_numpy(g.col).to(device),
            torch.from_numpy(g.w).to(device))


def test_spectral_alignment_matches_dense_definitions():
    """Eigenvalues of both Laplacians equal numpy's on the oracle's dense matrices; the lift's
    spectrum is the coarse Laplacian's plus ones (the lift invariant)."""
    g, lift, n_c = _case()
    rp, col, w = _tensors(g)
    rep = S.spectral_alignment(g.n, rp, col, w, torch.from_numpy(lift), n_c, k=40)
    W = O.dense_weights(g)
    eg = np.linalg.eigvalsh(O.laplacian_norm(W))[:40]
    el = np.linalg.eigvalsh(O.laplacian_norm(O.lift_weights(W, lift, n_c)))[:40]
    assert np.allclose(rep.eig_graph.numpy(), eg, atol=1e-10)
    assert np.allclose(rep.eig_lift.numpy(), el, atol=1e-10)
    ec = np.linalg.eigvalsh(O.coarse_laplacian(W, lift, n_c))
    want = np.sort(np.concatenate([ec, np.ones(g.n - n_c)]))[:40]
    assert np.allclose(rep.eig_lift.numpy(), want, atol=1e-9)
    assert rep.max_eig_diff == pytest.approx(float(np.max(np.abs(eg - el))), abs=1e-10)
    # overlaps of orthonormal bases: every alignment is at most 1
    assert float(rep.alignment.max()) <= 1.0 + 1e-9
    assert float(np.linalg.norm(rep.overlap.numpy())) <= np.sqrt(40) + 1e-9
    # the null vectors D^1/2 1 differ (the lift averages degrees over each super-node)
    u0 = np.linalg.eigh(O.laplacian_norm(W))[1][:, 0]
    v0 = np.linalg.eigh(O.laplacian_norm(O.lift_weights(W, lift, n_c)))[1][:, 0]
    assert float(rep.overlap[0, 0]) == pytest.approx(abs(float(u0 @ v0)), abs=1e-8)


def test_identity_coarsening_is_perfectly_aligned():
    g, _, _ = _case()
    rp, col, w = _tensors(g)
    rep = S.spectral_alignment(g.n, rp, col, w, torch.arange(g.n), g.n, k=20)
    assert rep.max_eig_diff < 1e-12
    assert np.allclose(rep.alignment.numpy(), 1.0, atol=1e-8)


@pytest.mark.gpu
def test_spectral_alignment_on_gpu_coarsening():
    """The 64x64 unit mesh coarsened on the GPU to 2048 nodes: the diagnostic on the GPU
    (cuSOLVER) agrees with the CPU computation of the same report."""
    import __graft_entry__ as ge
    ge.build()
    from paper_2204_11757_gb300 import api
    g, cfg = I.config_graph("c1_tri64_unit")
    ctx = api.Context()
    try:
        lift, n_c, _ = ctx.coarsen(api.CSR.from_graph(g), g.n // cfg["ratio"], levels=1)
        rp, col, w = _tensors(g, "cuda")
        rep = S.spectral_alignment(g.n, rp, col, w, lift, n_c, k=50)
        cpu = S.spectral_alignment(g.n, *_tensors(g), lift.cpu(), n_c, k=50)
        assert np.allclose(rep.eig_graph.cpu().numpy(), cpu.eig_graph.numpy(), atol=1e-9)
        assert np.allclose(rep.eig_lift.cpu().numpy(), cpu.eig_lift.numpy(), atol=1e-9)
        assert rep.max_eig_diff < 0.5
    finally:
        ctx.close()


# ---- the sparse variant ---------------------------------------------------------------------

@pytest.mark.parametrize("dense_max", [4096, 0])
def test_sparse_alignment_equals_dense(dense_max):
    """Both routes of the sparse variant (dense LAPACK below dense_max, shift-invert Lanczos
    above) give the dense report: the mesh is jittered, so its eigenvalues are simple and the
    overlaps are unique."""
    g, lift, n_c = _case()
    rp, col, w = _tensors(g)
    d = S.spectral_alignment(g.n, rp, col, w, torch.from_numpy(lift), n_c, k=40)
    s = S.spectral_alignment_sparse(g.n, rp, col, w, torch.from_numpy(lift), n_c, k=40,
                                    dense_max=dense_max)
    assert s.lifted == 40
    assert np.allclose(s.eig_graph.numpy(), d.eig_graph.numpy(), atol=1e-10)
    assert np.allclose(s.eig_lift.numpy(), d.eig_lift.numpy(), atol=1e-10)
    assert np.allclose(s.overlap.numpy(), d.overlap.numpy(), atol=1e-9)
    assert np.allclose(s.alignment.numpy(), d.alignment.numpy(), atol=1e-9)
    assert s.max_eig_diff == pytest.approx(d.max_eig_diff, abs=1e-10)


def test_sparse_alignment_mixes_in_the_lift_ones():
    """Coarsening 12 nodes to 6 with k = 12: the lift's spectrum is the 6 coarse eigenvalues
    and six 1s, and only the coarse eigenvalues at or below 1 give overlap columns."""
    g = I.tri_mesh_2d(4, 3, 1, jitter=0.3, weight="inv_len", dtype=np.float64)
    levels, lift = O.coarsen(g, 2, "halving")
    n_c = levels[-1].n_c
    rp, col, w = _tensors(g)
    s = S.spectral_alignment_sparse(g.n, rp, col, w, torch.from_numpy(lift), n_c, k=g.n)
    W = O.dense_weights(g)
    ec = np.linalg.eigvalsh(O.coarse_laplacian(W, lift, n_c))
    el = np.linalg.eigvalsh(O.laplacian_norm(O.lift_weights(W, lift, n_c)))
    assert np.allclose(s.eig_lift.numpy(), el, atol=1e-10)
    assert s.lifted == int(np.count_nonzero(ec <= 1.0))
    assert s.overlap.shape == (g.n, s.lifted)


def _rows(g):
    return np.repeat(np.arange(g.n), np.diff(g.rowptr))


def test_sparse_alignment_residuals_on_a_16k_mesh():
    """A 128 x 128 mesh coarsened 4x: each returned eigenpair satisfies L u = lambda u for L(G)
    and for the lift's Laplacian applied matrix-free from Definition 2 (block sums over
    super-nodes, divided by |u_c| |v_c|), without the coarse factorisation.  The null vectors
    are sqrt(d) and sqrt(d_hat), so overlap[0, 0] has a closed form."""
    g = I.tri_mesh_2d(128, 128, 5, jitter=0.3, weight="inv_len", dtype=np.float64)
    levels, lift = O.coarsen(g, 4, "halving")
    n_c = levels[-1].n_c
    rp, col, w = _tensors(g)
    k = 12
    s = S.spectral_alignment_sparse(g.n, rp, col, w, torch.from_numpy(lift), n_c, k=k,
                                    dense_max=0, vectors=True)
    assert s.lifted == k
    r, c = _rows(g), g.col.astype(np.int64)
    d = np.bincount(r, weights=g.w, minlength=g.n)

    def L_graph(y):        # y - D^-1/2 W D^-1/2 y, entry by entry
        z = np.zeros_like(y)
        np.add.at(z, r, (g.w / np.sqrt(d[r] * d[c]))[:, None] * y[c])
        return y - z

    sizes = np.bincount(lift, minlength=n_c).astype(np.float64)
    block = np.zeros((n_c, n_c))
    np.add.at(block, (lift[r], lift[c]), g.w)
    # d_hat(u) = sum_v w_hat(u, v) = sum_{v_c} block[u_c, v_c] |v_c| / (|u_c| |v_c|)
    d_hat = block.sum(axis=1)[lift] / sizes[lift]

    def L_lift(y):         # y - D_hat^-1/2 W_hat D_hat^-1/2 y with W_hat from Definition 2
        t = y / np.sqrt(d_hat)[:, None]
        per = np.zeros((n_c, y.shape[1]))
        np.add.at(per, lift, t)                          # sum of t over each super-node v_c
        z = (block / sizes[None, :]) @ per               # sum_{v_c} block[u_c, v_c] per / |v_c|
        z = z[lift] / sizes[lift][:, None]               # ... / |u_c|
        return y - z / np.sqrt(d_hat)[:, None]

    U = s.vec_graph.numpy()
    V = s.vec_lift.numpy()
    lg, ll = s.eig_graph.numpy(), s.eig_lift.numpy()
    assert np.abs(L_graph(U) - U * lg).max() < 1e-9
    assert np.abs(L_lift(V) - V * ll).max() < 1e-9
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-9)
    assert np.allclose(V.T @ V, np.eye(k), atol=1e-9)
    assert abs(lg[0]) < 1e-10 and abs(ll[0]) < 1e-10
    u0 = np.sqrt(d) / np.linalg.norm(np.sqrt(d))
    v0 = np.sqrt(d_hat) / np.linalg.norm(np.sqrt(d_hat))
    assert float(s.overlap[0, 0]) == pytest.approx(abs(float(u0 @ v0)), abs=1e-8)
    # both spectra lie in [0, 2], and every alignment is at most 1
    assert lg.min() > -1e-10 and ll.max() < 2.0
    assert float(s.alignment.max()) <= 1.0 + 1e-9


@pytest.mark.gpu
@pytest.mark.parametrize("ratio", [8, 32])
def test_spectral_quality_of_gpu_lifts(ratio):
    """Figure 2's comparison on the 256^2 jittered mesh from the GPU's multilevel lift (the
    self-mass reading, the default): the lift equals the oracle's, its report equals the one
    from the oracle's lift, and the coarsening stays spectrally close (no giant super-node:
    the mean alignment of the 50 leading eigenvectors stays above 0.9 even at 32x)."""
    import __graft_entry__ as ge
    ge.build()
    from paper_2204_11757_gb300 import api
    g, _ = I.config_graph("s2_tri256_f64")
    levels, total = O.coarsen(g, ratio, "halving")
    ctx = api.Context()
    try:
        lift, n_c, _ = ctx.coarsen(api.CSR.from_graph(g), levels[-1].target,
                                   levels=int(round(np.log2(ratio))))
        lift = lift.cpu()
    finally:
        ctx.close()
    assert n_c == levels[-1].n_c and np.array_equal(lift.numpy(), total)
    rp, col, w = _tensors(g)
    rep = S.spectral_alignment_sparse(g.n, rp, col, w, lift, n_c, k=50)
    ref = S.spectral_alignment_sparse(g.n, rp, col, w, torch.from_numpy(total), n_c, k=50)
    assert rep.max_eig_diff == pytest.approx(ref.max_eig_diff, rel=1e-9)
    assert np.allclose(rep.alignment.numpy(), ref.alignment.numpy(), atol=1e-9)
    assert np.bincount(total).max() < 0.02 * g.n
    assert float(rep.alignment.mean()) > 0.9 and rep.max_eig_diff < 0.05
