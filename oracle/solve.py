"""Incident and adjoint fields (oracle).

Test infrastructure only (see the package docstring).

The fields are the solutions of the discretised diffusion problem with a point
source: phi_s = A_j^{-1} e_s for each source s and phi_d = A_j^{-1} e_d for
each detector d (the adjoint field by reciprocity, Section 2.1 after
eqn:lippschwin), at every wavelength j (eqn:discincident, eqn:multipleshifted).
The recycled-Krylov machinery of Section 3 only reaches these same fields
faster, so the oracle solves directly:

* ``fields_splu``: sparse LU (SuperLU) -- the definition of record. The operator
  is a symmetric M-matrix, so elimination adds only like-signed terms off the
  diagonal and the triangular solves with a non-negative right-hand side add
  only non-negative terms: the result is accurate entry by entry, also where the
  field has decayed by many orders of magnitude.
* ``fields_separable``: an independent solver for the uniform box. The operator
  is a Kronecker sum T_x (+) T_y (+) T_z + m I of three symmetric tridiagonal
  matrices (one per axis, Robin terms on their end rows), so it is diagonalised
  by the tensor product of their eigenvectors (fast diagonalisation, Lynch,
  Rice & Thomas 1964). The diagonalisation alone is accurate in norm only: its
  absolute rounding errors (~1e-16 of the field's peak) swamp the far field, down
  to negative values. Two steps of residual correction in FP64 with the assembled
  operator, x += A^-1 (b - A x), make it accurate entry by entry (componentwise
  backward error ~1e-11 on the benchmark grids).
* ``fields_dense``: numpy.linalg.solve on the dense matrix, for tiny grids.
"""
from __future__ import annotations

import os
from typing import Optional, Sequence

import numpy as np
import scipy.sparse.linalg as spla

from . import model


def _lams(problem, lams: Optional[Sequence[int]]):
    return list(range(problem.n_lambda)) if lams is None else [int(j) for j in lams]


def _unit(N: int, idx: int, dtype) -> np.ndarray:
    e = np.zeros(N, dtype=dtype)
    e[idx] = 1.0
    return e


def fields_splu(problem, lams: Optional[Sequence[int]] = None):
    """(phi_src [n_l, n_src, N], phi_det [n_l, n_det, N]) by sparse LU, one factorisation per wavelength."""
    lams = _lams(problem, lams)
    N = problem.grid.N
    dtype = np.complex128 if problem.omega != 0.0 else np.float64
    S = problem.src_voxels()
    Dv = problem.det_voxels()
    phis = np.empty((len(lams), len(S), N), dtype=dtype)
    phid = np.empty((len(lams), len(Dv), N), dtype=dtype)
    for a, j in enumerate(lams):
        lu = spla.splu(model.operator(problem, j).tocsc(), permc_spec="MMD_AT_PLUS_A")
        for b, s in enumerate(S):
            phis[a, b] = lu.solve(_unit(N, s, dtype))
        for b, d in enumerate(Dv):
            phid[a, b] = lu.solve(_unit(N, d, dtype))
    return phis, phid


def solve_splu(problem, j: int, rhs: np.ndarray) -> np.ndarray:
    """A_j^{-1} rhs for a general right-hand side block rhs [n_rhs, N]."""
    lu = spla.splu(model.operator(problem, j).tocsc(), permc_spec="MMD_AT_PLUS_A")
    return np.stack([lu.solve(np.ascontiguousarray(b)) for b in rhs])


def _axis_matrix(n: int, a: float, beta_lo: float, beta_hi: float) -> np.ndarray:
    """1-D part of the operator along one axis: a*(number of neighbours) on the
    diagonal, -a off the diagonal, and the two boundary-face terms on the end rows."""
    T = np.zeros((n, n))
    for i in range(n):
        if i > 0:
            T[i, i - 1] = -a
            T[i, i] += a
        if i < n - 1:
            T[i, i + 1] = -a
            T[i, i] += a
    T[0, 0] += beta_lo
    T[n - 1, n - 1] += beta_hi
    return T


def separable_factors(problem, j: int):
    """Eigen-decompositions (Q, lam) of T_x, T_y, T_z and the diagonal shift m at wavelength j."""
    mua, D = model.wavelength_coefficients(problem)
    g = problem.grid
    h = g.h
    Dj = float(D[j])
    a = Dj * h
    beta = [model.face_coefficient(Dj, h, float(A)) for A in problem.robin_A]
    facs = []
    for n, (lo, hi) in ((g.nx, (beta[0], beta[1])), (g.ny, (beta[2], beta[3])), (g.nz, (beta[4], beta[5]))):
        lam, Q = np.linalg.eigh(_axis_matrix(n, a, lo, hi))
        facs.append((Q, lam))
    m = float(mua[j]) * h ** 3 + (1j * problem.omega * h ** 3 / problem.c_medium if problem.omega else 0.0)
    return facs, m


def solve_separable(problem, j: int, rhs: np.ndarray, refine: int = 2) -> np.ndarray:
    """A_j^{-1} rhs [n_rhs, N] by fast diagonalisation followed by `refine` steps of residual
    correction with the assembled sparse operator (the residual b - A x in FP64)."""
    x = _diagonalised_solve(problem, j, rhs)
    if refine:
        A = model.operator(problem, j)
        for _ in range(refine):
            x = x + _diagonalised_solve(problem, j, rhs - (A @ x.T).T)
    return x


def _diagonalised_solve(problem, j: int, rhs: np.ndarray) -> np.ndarray:
    """A_j^{-1} rhs [n_rhs, N] by fast diagonalisation alone (accurate in norm)."""
    facs, m = separable_factors(problem, j)
    (Qx, lx), (Qy, ly), (Qz, lz) = facs
    g = problem.grid
    denom = lz[:, None, None] + ly[None, :, None] + lx[None, None, :] + m
    out = []
    for b in rhs:
        B = b.reshape(g.nz, g.ny, g.nx)
        Bh = np.einsum("kc,jb,ia,cba->kji", Qz.T, Qy.T, Qx.T, B, optimize=True)
        Xh = Bh / denom
        out.append(np.einsum("kc,jb,ia,cba->kji", Qz, Qy, Qx, Xh, optimize=True).reshape(-1))
    return np.stack(out)


def fields_separable(problem, lams: Optional[Sequence[int]] = None, src: Optional[Sequence[int]] = None,
                     det: Optional[Sequence[int]] = None):
    """Fields by fast diagonalisation. src/det select subsets (default: all)."""
    lams = _lams(problem, lams)
    N = problem.grid.N
    dtype = np.complex128 if problem.omega != 0.0 else np.float64
    S = problem.src_voxels() if src is None else problem.src_voxels()[list(src)]
    Dv = problem.det_voxels() if det is None else problem.det_voxels()[list(det)]
    phis = np.empty((len(lams), len(S), N), dtype=dtype)
    phid = np.empty((len(lams), len(Dv), N), dtype=dtype)
    for a, j in enumerate(lams):
        if len(S):
            phis[a] = solve_separable(problem, j, np.stack([_unit(N, s, dtype) for s in S]))
        if len(Dv):
            phid[a] = solve_separable(problem, j, np.stack([_unit(N, d, dtype) for d in Dv]))
    return phis, phid


def fields_dense(problem, lams: Optional[Sequence[int]] = None):
    """Fields by dense LAPACK solve (tiny grids only)."""
    lams = _lams(problem, lams)
    N = problem.grid.N
    dtype = np.complex128 if problem.omega != 0.0 else np.float64
    E = np.eye(N, dtype=dtype)
    S = problem.src_voxels()
    Dv = problem.det_voxels()
    phis = np.empty((len(lams), len(S), N), dtype=dtype)
    phid = np.empty((len(lams), len(Dv), N), dtype=dtype)
    for a, j in enumerate(lams):
        A = model.operator(problem, j).toarray()
        phis[a] = np.linalg.solve(A, E[:, S]).T
        phid[a] = np.linalg.solve(A, E[:, Dv]).T
    return phis, phid


def _worker(args):
    problem, j = args
    return fields_splu(problem, [j])


def fields_splu_parallel(problem, lams: Optional[Sequence[int]] = None, workers: Optional[int] = None):
    """fields_splu spread over processes (one wavelength per task, BLAS threads 1).

    The pool is started with the 'spawn' method so it is safe after CUDA was initialised."""
    import multiprocessing as mp

    lams = _lams(problem, lams)
    if workers is None:
        workers = len(os.sched_getaffinity(0))
    workers = max(1, min(workers, len(lams)))
    if workers == 1:
        return fields_splu(problem, lams)
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with ctx.Pool(workers) as pool:
            parts = pool.map(_worker, [(problem, j) for j in lams])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]))
