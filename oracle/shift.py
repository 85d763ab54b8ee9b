"""Shift-invariant initial guesses from one Krylov space per optode (oracle).

Test infrastructure only (see the package docstring).

Section 3 of the paper starts the shifted systems of all wavelengths from a Krylov space built once
on a base operator -- the operator at the mean shift, Section 6.1 -- and keeps the projected
matrices up to date per shift from quantities computed once (Section 3.2), so that every
wavelength gets a Galerkin initial guess without new products with its own operator. For one
optode cell c this is, written out plainly:

    Ahat_j = A_j / (D_j h)                  the operator with unit couplings between cells
    Ahat_0 = mean over j of Ahat_j          = Lg + mean(sigma) I + sum_f mean(bhat_f) B_f
    V      = an orthonormal basis of the Krylov space K_m(Ahat_0, e_c)
    x_j    = V (V^T Ahat_j V)^{-1} V^T e_c  the Galerkin projection of Ahat_j x = e_c
    phi_j  = x_j / (D_j h)                  the guess in field units (Ahat_j x = e_c <=> A_j phi = e_c)

The guess depends on the subspace only, not on the basis chosen for it. Here V comes from Lanczos
with full reorthogonalisation (twice per step) in FP64; when the Krylov space is invariant before
m steps (the recurrence breaks down) the smaller space is used and contains the exact solution.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np
import scipy.sparse as sp

from . import model


def scaled_operator(problem, j: int) -> sp.csr_matrix:
    """Ahat_j = A_j / (D_j h)."""
    _, D = model.wavelength_coefficients(problem)
    return (model.operator(problem, j) / (float(D[j]) * problem.grid.h)).tocsr()


def base_operator(problem) -> sp.csr_matrix:
    """Ahat_0: the mean of Ahat_j over the problem's wavelengths (mean shift, mean boundary terms)."""
    acc = None
    for j in range(problem.n_lambda):
        a = scaled_operator(problem, j)
        acc = a if acc is None else acc + a
    return (acc / problem.n_lambda).tocsr()


def krylov_basis(A: sp.csr_matrix, b: np.ndarray, m: int) -> np.ndarray:
    """Orthonormal basis [N][m'] of K_m(A, b), m' <= m (smaller when the space is invariant)."""
    N = b.shape[0]
    V = np.zeros((N, m))
    V[:, 0] = b / np.linalg.norm(b)
    for k in range(1, m):
        w = A @ V[:, k - 1]
        scale = np.linalg.norm(w)
        for _ in range(2):
            w = w - V[:, :k] @ (V[:, :k].T @ w)
        nw = np.linalg.norm(w)
        if nw <= 1e-12 * scale:
            return V[:, :k]
        V[:, k] = w / nw
    return V


def shift_guess(problem, j: int, cell: int, m: int, V: Optional[np.ndarray] = None,
                A0: Optional[sp.csr_matrix] = None) -> np.ndarray:
    """phi_j for the optode in `cell` (field units), from K_m(Ahat_0, e_cell)."""
    N = problem.grid.N
    e = np.zeros(N)
    e[cell] = 1.0
    if V is None:
        V = krylov_basis(base_operator(problem) if A0 is None else A0, e, m)
    Aj = scaled_operator(problem, j)
    G = V.T @ (Aj @ V)
    y = np.linalg.solve(G, V.T @ e)
    _, D = model.wavelength_coefficients(problem)
    return (V @ y) / (float(D[j]) * problem.grid.h)


def shift_guess_fields(problem, m: int, lams: Optional[Sequence[int]] = None):
    """The guesses for every source and detector field: ([nl][n_src][N], [nl][n_det][N])."""
    lams = list(range(problem.n_lambda)) if lams is None else [int(j) for j in lams]
    A0 = base_operator(problem)
    N = problem.grid.N
    out = []
    for cells in (problem.src_voxels(), problem.det_voxels()):
        arr = np.empty((len(lams), len(cells), N))
        for a, c in enumerate(cells):
            e = np.zeros(N)
            e[c] = 1.0
            V = krylov_basis(A0, e, m)
            for q, j in enumerate(lams):
                arr[q, a] = shift_guess(problem, j, int(c), m, V=V)
        out.append(arr)
    return out[0], out[1]
