"""Shape reconstruction with parametric level sets and Levenberg-Marquardt (oracle).

Test infrastructure only (see the package docstring).

Section 5 of the paper (eqn:pals, eqn:minimization, Algorithm alg:opt), written out in FP64:

* Shape (eqn:pals): mu(r) = H_eps(phi(r) - tau), phi(r) = sum_k alpha_k psi(beta_k |r - chi_k|_nu)
  with |v|_nu = sqrt(|v|^2 + nu^2). The paper names compactly supported radial basis functions and a
  smooth Heaviside without fixing them; this project takes Wendland's C2 function
  psi(t) = (1 - t)_+^4 (4t + 1) and H_eps(t) = 1/2 + arctan(pi t / eps) / pi, whose derivative is
  delta_eps(t) = (1/eps) / (1 + (pi t / eps)^2). Parameters p = [alpha, beta, chi_x, chi_y, chi_z]
  (N_p = 5 n_p); positions in mm at the voxel centres ((i + 1/2) h, ...).
* Data (eqn:measurement): y = sum_c c_c E_c H mu + eta, i.e. y = J (c (x) mu) with the Born matrix
  J of this project (columns chromophore-major), W = I / sigma.
* Reconstruction with the compressed operator J ~ U diag(S) V^T (U with orthonormal columns,
  Section 5 "compressed low-rank representation"): the columns of D(p) are E_c H mu = U S V_c^T mu,
  where V_c are the rows of V of chromophore c. Everything then lives in rank-r coordinates:
  with yh = U^T y, |y - D c|^2 = (|y|^2 - |yh|^2) + |yh - S M c|^2, M[:, c] = V_c^T mu, and the
  Jacobian of the residual is -S sum_c c_c V_c^T dmu/dp (the paper's J = -W Ebar H dmu/dp).
* Algorithm alg:opt: alternate the linear least-squares step for c and Levenberg-Marquardt steps
  (J^T J + nu I) dp = -J^T eps on p, until the residual meets the discrepancy principle
  |eps| <= gamma |eta| (the paper's loop conditions are printed with the inequality reversed; the
  stopping rule stated in the text is followed). nu follows the usual rule: divided by 3 after an
  accepted step, multiplied by 4 after a rejected one.
* Metrics (Section 6.2): relative L2 error |mu - mu_hat| / |mu| of the shapes and the Dice
  coefficient 2 |A and B| / (|A| + |B|) of the voxel sets where mu > 1/2.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


@dataclasses.dataclass
class PalsModel:
    tau: float = 0.5     # level of phi that bounds the anomaly
    eps: float = 0.1     # width of the smoothed Heaviside
    nu: float = 0.02     # smoothing of |r| (mm)


def voxel_centres(grid) -> np.ndarray:
    """[N][3] voxel centres in mm, voxel x = (k*ny + j)*nx + i."""
    k, j, i = np.meshgrid(np.arange(grid.nz), np.arange(grid.ny), np.arange(grid.nx), indexing="ij")
    return np.stack([(i.ravel() + 0.5) * grid.h, (j.ravel() + 0.5) * grid.h, (k.ravel() + 0.5) * grid.h], axis=1)


def split(p: np.ndarray):
    n = p.size // 5
    return p[:n], p[n:2 * n], np.stack([p[2 * n:3 * n], p[3 * n:4 * n], p[4 * n:5 * n]], axis=1)


def wendland(t):
    return np.where(t < 1.0, (1.0 - t) ** 4 * (4.0 * t + 1.0), 0.0)


def wendland_d(t):
    return np.where(t < 1.0, -20.0 * t * (1.0 - t) ** 3, 0.0)


def heaviside(t, eps):
    return 0.5 + np.arctan(np.pi * t / eps) / np.pi


def delta(t, eps):
    return (1.0 / eps) / (1.0 + (np.pi * t / eps) ** 2)


def level_function(p, X, model: PalsModel):
    alpha, beta, chi = split(p)
    d = X[:, None, :] - chi[None, :, :]
    rn = np.sqrt((d ** 2).sum(-1) + model.nu ** 2)
    return (alpha[None, :] * wendland(beta[None, :] * rn)).sum(1)


def shape(p, X, model: PalsModel):
    """mu(r) of eqn:pals at the points X [N][3]."""
    return heaviside(level_function(p, X, model) - model.tau, model.eps)


def shape_jacobian(p, X, model: PalsModel):
    """(mu [N], dmu/dp [N][5 n_p]) by the chain rule through H_eps, psi and |.|_nu."""
    alpha, beta, chi = split(p)
    d = X[:, None, :] - chi[None, :, :]                       # [N][n][3]
    rn = np.sqrt((d ** 2).sum(-1) + model.nu ** 2)            # [N][n]
    t = beta[None, :] * rn
    psi, dpsi = wendland(t), wendland_d(t)
    phi = (alpha[None, :] * psi).sum(1)
    mu = heaviside(phi - model.tau, model.eps)
    de = delta(phi - model.tau, model.eps)[:, None]
    d_alpha = de * psi
    d_beta = de * alpha[None, :] * dpsi * rn
    # d rn / d chi = -(r - chi) / rn
    g = de * alpha[None, :] * dpsi * beta[None, :] / rn       # [N][n]
    d_chi = [-g * d[:, :, a] for a in range(3)]
    return mu, np.concatenate([d_alpha, d_beta] + d_chi, axis=1)


def project(Vc: np.ndarray, mu: np.ndarray, dmu: np.ndarray) -> np.ndarray:
    """A[c] = V_c^T [mu, dmu/dp]: Vc [n_c][N][r] -> [n_c][r][1 + N_p]."""
    F = np.concatenate([mu[:, None], dmu], axis=1)
    return np.einsum("cxr,xq->crq", Vc, F)


def reduced_terms(A, S, yh, c):
    """(M = [V_c^T mu], residual eps_h = yh - S M c, Jacobian -S sum_c c_c V_c^T dmu/dp)."""
    M = A[:, :, 0].T                                           # [r][n_c]
    eps_h = yh - S * (M @ c)
    Jp = -S[:, None] * np.einsum("c,crq->rq", c, A[:, :, 1:])
    return M, eps_h, Jp


def solve_c(A, S, yh):
    """The linear least-squares step of alg:opt: c = argmin |yh - S M c|."""
    D = S[:, None] * A[:, :, 0].T
    return np.linalg.lstsq(D, yh, rcond=None)[0]


def reconstruct(Vc, U_T_y, y_norm2, S, p0, X, model: PalsModel, c0, noise_norm, gamma=1.05,
                fix_c=False, max_outer=10, max_inner=20, nu0=1e-2):
    """Algorithm alg:opt. Vc [n_c][N][r], U_T_y = U^T y [r], y_norm2 = |y|^2, S [r], p0 [5 n_p].
    Returns (p, c, |eps| history of accepted steps, evaluations)."""
    yh = np.asarray(U_T_y, float)
    out2 = max(y_norm2 - float(yh @ yh), 0.0)                  # part of y outside range(U)
    p = np.array(p0, float)
    c = np.array(c0, float)
    evals = 0

    def evaluate(pp, cc):
        nonlocal evals
        evals += 1
        mu, dmu = shape_jacobian(pp, X, model)
        A = project(Vc, mu, dmu)
        M, e, Jp = reduced_terms(A, S, yh, cc)
        return A, e, Jp, float(np.sqrt(out2 + e @ e))

    A, e, Jp, res = evaluate(p, c)
    hist = [res]
    target = gamma * noise_norm
    for _ in range(max_outer):
        if res <= target:
            break
        outer_start = res
        if not fix_c:
            c = solve_c(A, S, yh)
            A, e, Jp, res = evaluate(p, c)
            hist.append(res)
        nu = nu0 * float(np.max(np.einsum("rq,rq->q", Jp, Jp)))
        for _ in range(max_inner):
            if res <= target:
                break
            G = Jp.T @ Jp
            dp = np.linalg.solve(G + nu * np.eye(G.shape[0]), -(Jp.T @ e))
            A2, e2, Jp2, res2 = evaluate(p + dp, c)
            if res2 < res:
                p, A, e, Jp, res = p + dp, A2, e2, Jp2, res2
                hist.append(res)
                nu /= 3.0
                if np.linalg.norm(dp) <= 1e-10 * (1.0 + np.linalg.norm(p)):
                    break
            else:
                nu *= 4.0
        if res >= outer_start * (1.0 - 1e-6):
            break
    return p, c, hist, evals


def rel_l2(mu, mu_hat):
    return float(np.linalg.norm(mu - mu_hat) / np.linalg.norm(mu))


def dice(mu, mu_hat, level=0.5):
    a, b = mu > level, mu_hat > level
    return float(2.0 * np.logical_and(a, b).sum() / (a.sum() + b.sum()))
