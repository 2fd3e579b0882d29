"""FP64 reference gradient of the truncated POD computed by ISMA with frozen
draws (plain PyTorch CPU autograd).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only ``tests/`` may call it.  It shares no code with the CUDA library.

The forward map is Algorithm 1 with the index sets I_0, I_1, ... fixed (the
draws are discrete, so the derivative is that of the map for fixed draws):
each round merges the scaled factor U Sigma with the sampled columns
D = A[:, I_t] by the SVD of [U Sigma, D] truncated to r (Algorithm 2, Eqs.
8-9, direct merge), dropping singular values at the oracle's threshold; the
closing refinement takes the SVD of U^T A (equivalently QR(A^T U), SVD(R)).
The SVD steps are torch.linalg.svd, whose adjoint couples singular vectors
through 1 / (sigma_j^2 - sigma_i^2); that is the reference for a
hand-written adjoint.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np
import torch


def forward(A: torch.Tensor, index_sets: Sequence[np.ndarray], k: int, r: int, refine: bool = True):
    """(U_k, sigma_k) of ISMA with frozen draws; differentiable in A (FP64)."""
    m = A.shape[0]
    U = A.new_zeros((m, 0))
    s = A.new_zeros((0,))
    for I in index_sets:
        D = A[:, torch.as_tensor(np.asarray(I, dtype=np.int64))]
        X = torch.cat([U * s[None, :], D], dim=1)
        Ux, sx, _ = torch.linalg.svd(X, full_matrices=False)
        thr = max(X.shape) * np.finfo(np.float64).eps * float(sx[0].detach()) if sx.numel() else 0.0
        keep = min(r, int((sx > thr).sum()))
        U, s = Ux[:, :keep], sx[:keep]
    if refine and U.shape[1] > 0:
        W, S, _ = torch.linalg.svd(U.T @ A, full_matrices=False)
        U, s = U @ W, S
    kk = min(k, U.shape[1])
    return U[:, :kk], s[:kk]


def loss(U: torch.Tensor, s: torch.Tensor, w: torch.Tensor, g: torch.Tensor, ws: torch.Tensor = None):
    """L = sum_i w_i (u_i^T g)^2 (+ sum_i ws_i sigma_i); invariant to mode signs."""
    val = (w * (U.T @ g) ** 2).sum()
    if ws is not None:
        val = val + (ws * s).sum()
    return val


def gradient(A_np: np.ndarray, index_sets, k: int, r: int, w, g, ws=None, refine: bool = True):
    """dL/dA (FP64 NumPy array) and L."""
    A = torch.tensor(np.asarray(A_np, dtype=np.float64), requires_grad=True)
    U, s = forward(A, index_sets, k, r, refine)
    wt = torch.as_tensor(np.asarray(w, dtype=np.float64))
    gt = torch.as_tensor(np.asarray(g, dtype=np.float64))
    wst = None if ws is None else torch.as_tensor(np.asarray(ws, dtype=np.float64))
    L = loss(U, s, wt, gt, wst)
    L.backward()
    return A.grad.numpy(), float(L.detach())
