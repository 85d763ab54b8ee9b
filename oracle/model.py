"""Background optical coefficients and the discrete diffusion operator (oracle).

Test infrastructure only (see the package docstring).

Continuous model (Section 2.1, eqn:diffusion, eqn:dirichlet, eqn:robin):
    -div(D grad phi) + mu_a phi = S            in the box
    phi = 0                                   on Dirichlet faces
    phi + 2 A D d(phi)/dn = 0                 on Robin faces
with D and mu_a constant in space (the paper's Delta D = 0 assumption,
Section 2.1) and S a point source. The propagation speed nu is dropped for the
continuous-wave case; the frequency-domain case adds i*omega/c_m to mu_a.

Discretisation: the paper's Galerkin FEM (eqn:discincident, eqn:matrices) is
restated on a box as cell-centred finite volumes with cells of side h. Each
unknown is a cell average, every cell has volume h^3:
  * interior face between cells i and j: flux D*h*(phi_i - phi_j)
    (face area h^2 over centre distance h)  -- the stiffness K;
  * absorption: mu_a*h^3*phi_i               -- the lumped mass M;
  * Robin face: the face value phi_b follows from
    phi_b + 2AD (phi_b - phi_i)/(h/2) = 0, so phi_b = phi_i*4AD/(h+4AD) and the
    outward flux D*(phi_i - phi_b)/(h/2)*h^2 = 2*D*h^2/(h + 4*A*D) * phi_i
    -- the boundary matrix R; A = 0 gives the Dirichlet face, 2*D*h;
  * source: b = e_cell (unit power into one cell).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def mu_a(eps: np.ndarray, c_bg: np.ndarray) -> np.ndarray:
    """Background absorption per wavelength: mu_a(lambda) = sum_l eps_l(lambda) c_l
    (eqn:perturbation applied to the background concentrations). eps [n_lambda, n_chrom]."""
    n_lambda, n_chrom = eps.shape
    out = np.zeros(n_lambda)
    for j in range(n_lambda):
        for l in range(n_chrom):
            out[j] += eps[j, l] * c_bg[l]
    return out


def diffusion(mua: np.ndarray, mus_prime: np.ndarray) -> np.ndarray:
    """D(lambda) = 1 / (3 (mu_a + mu_s')), in mm (nu factored out)."""
    return 1.0 / (3.0 * (mua + mus_prime))


def face_coefficient(D: float, h: float, A: float) -> float:
    """Diagonal contribution of one boundary face: 2 D h^2 / (h + 4 A D); A = 0 is Dirichlet."""
    return 2.0 * D * h * h / (h + 4.0 * A * D)


def assemble(nx: int, ny: int, nz: int, h: float, D: float, mua: float, robin_A,
             omega: float = 0.0, c_medium: float = 1.0) -> sp.csr_matrix:
    """Sparse FV matrix of the diffusion operator (one wavelength), voxel index (k*ny+j)*nx+i.

    Built face by face: every interior face adds D*h to both diagonals and -D*h to
    both off-diagonals; every boundary face adds face_coefficient(...) to its cell;
    every cell adds mu_a*h^3 (+ i*omega*h^3/c_m when omega != 0)."""
    N = nx * ny * nz
    cplx = omega != 0.0
    dtype = np.complex128 if cplx else np.float64
    idx = np.arange(N).reshape(nz, ny, nx)
    diag = np.full(N, mua * h ** 3, dtype=dtype)
    if cplx:
        diag += 1j * omega * h ** 3 / c_medium
    rows, cols, vals = [], [], []
    a = D * h
    # interior faces along each axis
    for axis in (2, 1, 0):  # x, y, z in array axes (nz, ny, nx)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(0, -1)
        hi[axis] = slice(1, None)
        p = idx[tuple(lo)].reshape(-1)
        q = idx[tuple(hi)].reshape(-1)
        np.add.at(diag, p, a)
        np.add.at(diag, q, a)
        rows += [p, q]
        cols += [q, p]
        vals += [np.full(p.shape, -a), np.full(q.shape, -a)]
    # boundary faces: -x, +x, -y, +y, -z, +z
    faces = [(2, 0), (2, -1), (1, 0), (1, -1), (0, 0), (0, -1)]
    for f, (axis, end) in enumerate(faces):
        sl = [slice(None)] * 3
        sl[axis] = end
        cells = idx[tuple(sl)].reshape(-1)
        np.add.at(diag, cells, face_coefficient(D, h, float(robin_A[f])))
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(diag)
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate([np.asarray(x, dtype=dtype) for x in vals])
    return sp.csr_matrix((v, (r, c)), shape=(N, N))


def wavelength_coefficients(problem):
    """(mu_a[n_lambda], D[n_lambda]) for a workloads.Problem."""
    mua = mu_a(problem.eps, problem.c_bg)
    return mua, diffusion(mua, problem.mus_prime)


def operator(problem, j: int) -> sp.csr_matrix:
    """The FV operator A_j at wavelength index j of a workloads.Problem."""
    mua, D = wavelength_coefficients(problem)
    g = problem.grid
    return assemble(g.nx, g.ny, g.nz, g.h, float(D[j]), float(mua[j]), problem.robin_A,
                    problem.omega, problem.c_medium)
