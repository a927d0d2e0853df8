"""Spectral quality of a coarsening: the eigenvalue and eigenvector comparison of Section 3.2.

The paper judges a coarsening by the smallest eigenvalues and the eigenvectors of the
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
