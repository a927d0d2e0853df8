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
