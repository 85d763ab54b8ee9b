"""Randomized low-rank sketch of J at fixed rank (oracle).

Test infrastructure only (see the package docstring).

Appendix A.1 (alg:randsvd, after Halko, Martinsson & Tropp 2011) at a fixed
target rank r with oversampling p:
  1. Y = A Omega with Omega [n, r+p] i.i.d. N(0, 1);
  2. an orthonormal basis Q of range(Y) (the paper takes the leading left
     singular vectors of Y; here all r+p of them);
  3. B = Q^T A;
  4. SVD of B: B = U_B S V^T, and U = Q U_B;
  5. truncate to rank r (the final recompression of Section 4.4).
The merge across source-detector blocks (Section 4.2, agglomeration) is the
row-block sum B = sum_blocks Q_blk^T A_blk, which this unblocked restatement
computes in one product.

``truncated_svd`` is the optimum the sketch is judged against: the best rank-r
approximation error in the 2-norm is sigma_{r+1} (Section 4.2).
"""
from __future__ import annotations

import numpy as np


def randsvd_fixed(A: np.ndarray, Omega: np.ndarray, rank: int):
    """(U [m, rank], S [rank], V [n, rank]) with A ~ U diag(S) V^T."""
    Y = A @ Omega
    Qy, _, _ = np.linalg.svd(Y, full_matrices=False)
    B = Qy.T @ A
    Ub, S, Vt = np.linalg.svd(B, full_matrices=False)
    U = Qy @ Ub
    return U[:, :rank], S[:rank], Vt[:rank].T


def truncated_svd(A: np.ndarray, rank: int):
    U, S, Vt = np.linalg.svd(A, full_matrices=False)
    return U[:, :rank], S[:rank], Vt[:rank].T, S


def probe_error(A: np.ndarray, U: np.ndarray, S: np.ndarray, V: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Relative error ||A x - U S V^T x|| / ||A x|| for each probe column of X."""
    ax = A @ X
    lx = U @ (S[:, None] * (V.T @ X))
    return np.linalg.norm(ax - lx, axis=0) / np.linalg.norm(ax, axis=0)
