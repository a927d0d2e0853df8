"""Spectral quality of a coarsening: the eigenvalue and eigenvector comparison of Section 3.2.

The paper assesses a coarsening by the smallest eigenvalues and the eigenvectors of the
normalized Laplacian of G against those of the lift of G_c (Definition 2: a graph on the n
original nodes whose weight between u and v is the total weight between their super-nodes
divided by |u_c| |v_c|).  Theorem 1 bounds the eigenvalue change of one merge; Figure 2 shows
how the leading eigenvectors of the two Laplacians align.  This module computes both for
graphs small enough for a dense eigensolve (a few thousand nodes), on the GPU through
torch.linalg.eigh:

* the k smallest eigenvalues of L(G) and of L(lift), and their largest difference,
* the k-by-k matrix |U_G^T U_lift| of eigenvector overlaps (1 on the diagonal for a perfect
  coarsening), with per-vector alignment ||U_G^T u_j|| for every lift eigenvector u_j.

L = I - D^-1/2 W D^-1/2 with D the row sums of W, diagonal entries included (the lift has
them: pairs inside one super-node).  Everything is binary64.

`spectral_alignment_sparse` gives the same report for graphs of up to about a million nodes on
the host: a shift-invert Lanczos solve for L(G), and the lift's eigenpairs from its n_c-node
coarse Laplacian without forming the n-by-n lift.
"""
from __future__ import annotations

import dataclasses

import torch


def _dense(n: int, rowptr: torch.Tensor, col: torch.Tensor, w: torch.Tensor,
           device) -> torch.Tensor:
    rows = torch.repeat_interleave(torch.arange(n, device=device),
                                   (rowptr[1:] - rowptr[:-1]).to(device))
    W = torch.zeros((n, n), dtype=torch.float64, device=device)
    W[rows, col.to(device).long()] = w.to(device, torch.float64)
    return W


def normalized_laplacian(W: torch.Tensor) -> torch.Tensor:
    """I - D^-1/2 W D^-1/2, D the row sums of W (diagonal entries included)."""
    s = W.sum(dim=1).rsqrt()
    return torch.eye(W.shape[0], dtype=W.dtype, device=W.device) - s[:, None] * W * s[None, :]


def lift_weights(W: torch.Tensor, lift: torch.Tensor, n_c: int) -> torch.Tensor:
    """Definition 2: w_hat(u, v) = sum over x in u_c, y in v_c of w(x, y), over |u_c| |v_c|."""
    n = W.shape[0]
    lift = lift.to(W.device).long()
    C = torch.zeros((n, n_c), dtype=W.dtype, device=W.device)
    C[torch.arange(n, device=W.device), lift] = 1.0
    block = C.T @ W @ C                       # total weight between super-nodes
    sizes = C.sum(dim=0)
    return block[lift][:, lift] / (sizes[lift][:, None] * sizes[lift][None, :])


@dataclasses.dataclass
class SpectralReport:
    eig_graph: torch.Tensor     # k smallest eigenvalues of L(G)
    eig_lift: torch.Tensor      # k smallest eigenvalues of L(lift)
    max_eig_diff: float         # max_i |eig_graph[i] - eig_lift[i]|
    overlap: torch.Tensor       # |U_G^T U_lift|, k x k
    alignment: torch.Tensor     # ||U_G^T u_j|| for each lift eigenvector j < k


def spectral_alignment(n: int, rowptr: torch.Tensor, col: torch.Tensor, w: torch.Tensor,
                       lift: torch.Tensor, n_c: int, k: int = 50,
                       device=None) -> SpectralReport:
    """Compare the k smallest eigenpairs of L(G) and L(lift of G_c) for the coarsening given by
    `lift` (node -> super-node in [0, n_c)).  Dense: meant for n up to a few thousand."""
    device = device or (w.device if w.is_cuda else "cpu")
    W = _dense(n, rowptr, col, w, device)
    ev_g, U = torch.linalg.eigh(normalized_laplacian(W))
    ev_l, V = torch.linalg.eigh(normalized_laplacian(lift_weights(W, lift, n_c)))
    k = min(k, n)
    G = (U[:, :k].T @ V[:, :k]).abs()
    return SpectralReport(eig_graph=ev_g[:k], eig_lift=ev_l[:k],
                          max_eig_diff=float((ev_g[:k] - ev_l[:k]).abs().max()),
                          overlap=G, alignment=torch.linalg.vector_norm(G, dim=0))


# ---- sparse variant: graphs beyond a dense eigensolve ------------------------------------------
#
# The lift never needs to be formed.  With C the n-by-n_c membership matrix, S = diag(|u_c|) and
# A_c = C^T W C (Definition 1's super-node weights, diagonal included), the lift's degree at u is
# d_c(u_c) / |u_c|, so D_hat^-1/2 W_hat D_hat^-1/2 = Q (D_c^-1/2 A_c D_c^-1/2) Q^T with
# Q = C S^-1/2, whose columns are orthonormal.  Hence L(lift) = Q L_c Q^T + (I - Q Q^T): every
# eigenpair (lambda, x) of L_c lifts to (lambda, Q x), and the n - n_c directions orthogonal to
# range(Q) have eigenvalue 1.  Only the n_c-node coarse problem is solved, and the overlaps are
# U_G^T Q X = (C^T U_G)^T S^-1/2 X, a sum of U_G's rows over each super-node.


def _csr_host(n: int, rowptr, col, w):
    import numpy as np
    import scipy.sparse as sp
    rp = rowptr.detach().cpu().numpy().astype(np.int64)
    c = col.detach().cpu().numpy().astype(np.int64)
    v = w.detach().cpu().numpy().astype(np.float64)
    return sp.csr_matrix((v, c, rp), shape=(n, n))


def _laplacian_host(A):
    """I - D^-1/2 A D^-1/2 for a scipy sparse A (every node of positive degree)."""
    import numpy as np
    import scipy.sparse as sp
    s = 1.0 / np.sqrt(np.asarray(A.sum(axis=1)).ravel())
    S = sp.diags(s)
    return (sp.identity(A.shape[0], format="csr") - S @ A @ S).tocsr()


def _smallest_eigpairs(L, k: int, dense_max: int, shift: float):
    """The k smallest eigenpairs of the symmetric sparse L, ascending.  Dense LAPACK up to
    dense_max rows; above that ARPACK's Lanczos in shift-invert mode about -shift (L + shift I
    is positive definite for a Laplacian, so its sparse LU factorisation is well posed)."""
    import numpy as np
    n = L.shape[0]
    if n <= dense_max or k >= n - 1:
        ev, U = np.linalg.eigh(L.toarray())
        return ev[:k], U[:, :k]
    from scipy.sparse.linalg import eigsh
    ev, U = eigsh(L.tocsc(), k=k, sigma=-shift, which="LM", tol=0.0)
    order = np.argsort(ev)
    return ev[order], U[:, order]


@dataclasses.dataclass
class SparseSpectralReport:
    eig_graph: torch.Tensor     # k smallest eigenvalues of L(G)
    eig_lift: torch.Tensor      # k smallest eigenvalues of L(lift), the 1s included
    max_eig_diff: float         # max_i |eig_graph[i] - eig_lift[i]|
    lifted: int                 # kc: how many of eig_lift come from lifted coarse eigenvectors
    overlap: torch.Tensor       # |U_G^T (Q X)|, k x kc, for those lifted eigenvectors
    alignment: torch.Tensor     # ||U_G^T Q x_j|| for each of them
    vec_graph: torch.Tensor | None = None   # n x k eigenvectors of L(G), if asked for
    vec_lift: torch.Tensor | None = None    # n x kc lifted eigenvectors Q x_j, if asked for


def spectral_alignment_sparse(n: int, rowptr: torch.Tensor, col: torch.Tensor,
                              w: torch.Tensor, lift: torch.Tensor, n_c: int, k: int = 50,
                              dense_max: int = 4096, shift: float = 1e-3,
                              vectors: bool = False) -> SparseSpectralReport:
    """The comparison of `spectral_alignment` for graphs of up to about a million nodes: L(G)
    through a sparse eigensolver, the lift through its n_c-node coarse Laplacian (the
    factorisation above).  Computed on the host in binary64 (scipy).

    The lift's k smallest eigenvalues merge the coarse ones with n - n_c ones.  Eigenvalue-1
    directions orthogonal to range(Q) have no preferred basis, so `overlap` and `alignment`
    cover only the kc lifted coarse eigenvectors that lie among the k smallest (all k whenever
    the k smallest coarse eigenvalues are below 1, as they are for meshes coarsened by small
    ratios).  Every node must have positive weighted degree.  `vectors` also returns both sets
    of eigenvectors (n x k and n x kc, binary64)."""
    import numpy as np
    import scipy.sparse as sp
    k = min(k, n)
    W = _csr_host(n, rowptr, col, w)
    lf = lift.detach().cpu().numpy().astype(np.int64)
    if lf.shape[0] != n or (n > 0 and (lf.min() < 0 or lf.max() >= n_c)):
        raise ValueError("lift must map each of the n nodes into [0, n_c)")
    C = sp.csr_matrix((np.ones(n), lf, np.arange(n + 1)), shape=(n, n_c))
    A_c = (C.T @ W @ C).tocsr()
    ev_g, U = _smallest_eigpairs(_laplacian_host(W), k, dense_max, shift)
    kc_max = min(k, n_c)
    ev_c, X = _smallest_eigpairs(_laplacian_host(A_c), kc_max, dense_max, shift)
    ones = min(k, n - n_c)
    # coarse eigenvalues at or below 1 come first; a tie with the ones goes to the coarse side
    kc = kc_max if ones == 0 else int(np.count_nonzero(ev_c <= 1.0))
    kc = min(kc, k)
    ev_l = np.sort(np.concatenate([ev_c, np.ones(ones)]))[:k]
    sizes = np.bincount(lf, minlength=n_c).astype(np.float64)
    UC = C.T @ U                                   # n_c x k: U_G's rows summed per super-node
    Xs = X[:, :kc] / np.sqrt(sizes)[:, None]       # S^-1/2 X: Q X is Xs[lift]
    G = np.abs(UC.T @ Xs)
    return SparseSpectralReport(
        eig_graph=torch.from_numpy(ev_g), eig_lift=torch.from_numpy(ev_l),
        max_eig_diff=float(np.max(np.abs(ev_g - ev_l))) if k else 0.0, lifted=kc,
        overlap=torch.from_numpy(G), alignment=torch.from_numpy(np.linalg.norm(G, axis=0)),
        vec_graph=torch.from_numpy(U) if vectors else None,
        vec_lift=torch.from_numpy(Xs[lf]) if vectors else None)
