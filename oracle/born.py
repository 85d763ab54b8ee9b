"""Born operator J, J x and J^T y (oracle).

Test infrastructure only (see the package docstring).

Eqn:lippschwin gives the scattered field at detector d as minus the integral of
phi_d * Delta mu_a * phi_s; eqn:perturbation writes Delta mu_a = sum_c eps_c(lambda)
c_c chi(r); eqn:measurement stacks the rows per source, detector and wavelength
(E_k = I_Ns (x) I_Nd (x) diag(eps_k), so wavelength is the fastest row index) and
the blocks per source (Section 4.1). With cells of volume h^3 the discrete row is

    J[(s, d, lambda), (c, x)] = -h^3 * eps_c(lambda) * phi_s(x; lambda) * phi_d(x; lambda)

row r = (s*N_d + d)*N_lambda + lambda, column c*N + x (chromophore-major).
This equals the exact derivative of the discrete forward value e_d^T A^{-1} e_s
with respect to the concentration c_c in cell x, since A contains mu_a*h^3 on its
diagonal and A is symmetric.

For a wavelength slice lams = [l0, l0+nl) the row index inside the slice is
(s*N_d + d)*nl + (lambda - l0).
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from . import solve as osolve


def _slice(problem, lams):
    return list(range(problem.n_lambda)) if lams is None else [int(j) for j in lams]


def born_matrix(problem, phis: np.ndarray, phid: np.ndarray, lams: Optional[Sequence[int]] = None) -> np.ndarray:
    """Explicit J for the wavelength slice; phis/phid are [len(lams), n, N] fields of that slice."""
    lams = _slice(problem, lams)
    h3 = problem.grid.h ** 3
    ns, nd, nl, nc, N = problem.n_src, problem.n_det, len(lams), problem.n_chrom, problem.grid.N
    J = np.empty((ns * nd * nl, nc * N), dtype=np.result_type(phis, phid))
    for s in range(ns):
        for d in range(nd):
            for a, lam in enumerate(lams):
                r = (s * nd + d) * nl + a
                H = phis[a, s] * phid[a, d]  # one row of H, eqn:lippschwin discretised
                for c in range(nc):
                    J[r, c * N:(c + 1) * N] = -h3 * problem.eps[lam, c] * H
    return J


def born_rows(problem, phis, phid, rows: Sequence[int], lams: Optional[Sequence[int]] = None) -> np.ndarray:
    """Selected rows of J (slice-local row indices), without forming the whole matrix."""
    lams = _slice(problem, lams)
    h3 = problem.grid.h ** 3
    nd, nl, nc, N = problem.n_det, len(lams), problem.n_chrom, problem.grid.N
    out = np.empty((len(rows), nc * N), dtype=np.result_type(phis, phid))
    for i, r in enumerate(rows):
        sd, a = divmod(int(r), nl)
        s, d = divmod(sd, nd)
        H = phis[a, s] * phid[a, d]
        for c in range(nc):
            out[i, c * N:(c + 1) * N] = -h3 * problem.eps[lams[a], c] * H
    return out


def apply(problem, phis, phid, x: np.ndarray, lams: Optional[Sequence[int]] = None) -> np.ndarray:
    """y = J x, row by row from the definition (no blocking): y_r = sum_{c,x} J[r,(c,x)] x[(c,x)]."""
    lams = _slice(problem, lams)
    ns, nd, nl = problem.n_src, problem.n_det, len(lams)
    y = np.empty(ns * nd * nl, dtype=np.result_type(phis, phid, x))
    for s in range(ns):
        for d in range(nd):
            rows = [(s * nd + d) * nl + a for a in range(nl)]
            y[rows] = born_rows(problem, phis, phid, rows, lams) @ x
    return y


def apply_T(problem, phis, phid, y: np.ndarray, lams: Optional[Sequence[int]] = None) -> np.ndarray:
    """g = J^T y (plain transpose), accumulated row by row: g += y_r * J[r, :]."""
    lams = _slice(problem, lams)
    ns, nd, nl, nc, N = problem.n_src, problem.n_det, len(lams), problem.n_chrom, problem.grid.N
    g = np.zeros(nc * N, dtype=np.result_type(phis, phid, y))
    for s in range(ns):
        for d in range(nd):
            rows = [(s * nd + d) * nl + a for a in range(nl)]
            g += born_rows(problem, phis, phid, rows, lams).T @ y[rows]
    return g


def apply_T_adjoint_solve(problem, phis, y: np.ndarray, lams: Optional[Sequence[int]] = None,
                          solver=osolve.solve_splu) -> np.ndarray:
    """J^T y by one extra solve per source and wavelength instead of stored detector fields.

    Since phi_d = A^{-1} e_d, sum_d y[s,d,lambda] phi_d = A^{-1} (sum_d y[s,d,lambda] e_d) =: psi_s
    (A symmetric), so g[(c,x)] = -h^3 sum_lambda eps_c(lambda) sum_s phi_s(x) psi_s(x)."""
    lams = _slice(problem, lams)
    h3 = problem.grid.h ** 3
    ns, nd, nl, nc, N = problem.n_src, problem.n_det, len(lams), problem.n_chrom, problem.grid.N
    Dv = problem.det_voxels()
    g = np.zeros(nc * N, dtype=np.result_type(phis, y))
    for a, lam in enumerate(lams):
        rhs = np.zeros((ns, N), dtype=np.result_type(phis, y))
        for s in range(ns):
            for d in range(nd):
                rhs[s, Dv[d]] += y[(s * nd + d) * nl + a]
        psi = solver(problem, lam, rhs)
        t = np.zeros(N, dtype=g.dtype)
        for s in range(ns):
            t += phis[a, s] * psi[s]
        for c in range(nc):
            g[c * N:(c + 1) * N] += -h3 * problem.eps[lam, c] * t
    return g


def forward_value(problem, j: int, dmua_voxel: Optional[np.ndarray] = None) -> np.ndarray:
    """Nonlinear discrete forward model: phi(r_d) = e_d^T (A_j + h^3 diag(dmua))^{-1} e_s for all (s, d).

    Used to pin J by finite differences (eqn:born without the Born approximation)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    from . import model

    A = model.operator(problem, j)
    if dmua_voxel is not None:
        A = A + sp.diags(problem.grid.h ** 3 * dmua_voxel)
    lu = spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A")
    N = problem.grid.N
    out = np.empty((problem.n_src, problem.n_det), dtype=A.dtype)
    Dv = problem.det_voxels()
    for a, s in enumerate(problem.src_voxels()):
        e = np.zeros(N, dtype=A.dtype)
        e[s] = 1.0
        out[a] = lu.solve(e)[Dv]
    return out
