"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test fixes part of the oracle by a closed form, a conservation law, a
finite difference of the nonlinear forward model, brute force, a second
independent solver, or an algebraic identity, so that a dropped term, a wrong
sign or index, or a transposed operand fails at least one of them.
"""
import dataclasses
import math

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse.linalg as spla

import workloads
from oracle import born, model, sketch, solve


# ---------------------------------------------------------------- operator (Section 2.2)

def test_operator_is_symmetric_m_matrix():
    p = workloads.small(nx=7, ny=6, nz=5)
    A = model.operator(p, 0).toarray()
    assert np.array_equal(A, A.T)
    off = A - np.diag(np.diag(A))
    assert (off <= 0).all()
    # strictly diagonally dominant rows (absorption and boundary terms) -> SPD M-matrix
    assert (np.diag(A) - np.abs(off).sum(axis=1) > 0).all()
    assert np.linalg.eigvalsh(A).min() > 0


def test_operator_stencil_counts():
    """Interior cell: 6 neighbours at -D h, diagonal 6 D h + mu_a h^3 (no boundary term)."""
    p = workloads.small(nx=5, ny=5, nz=5)
    mua, D = model.wavelength_coefficients(p)
    A = model.operator(p, 1).tocsr()
    h = p.grid.h
    c = p.grid.voxel(2, 2, 2)
    row = A.getrow(c)
    assert row.nnz == 7
    assert math.isclose(A[c, c], 6 * D[1] * h + mua[1] * h ** 3, rel_tol=1e-14)
    for nb in (c - 1, c + 1, c - 5, c + 5, c - 25, c + 25):
        assert math.isclose(A[c, nb], -D[1] * h, rel_tol=1e-14)


def test_robin_dirichlet_limit_and_corner_cell():
    """A = 0 gives the Dirichlet face 2 D h; a corner cell has three boundary faces."""
    assert math.isclose(model.face_coefficient(0.5, 2.0, 0.0), 2 * 0.5 * 2.0)
    p = workloads.small(nx=4, ny=4, nz=4, n_src=1, n_det=1, robin_A=(0.0, 1.0, 2.0, 3.0, 4.0, 5.0))
    mua, D = model.wavelength_coefficients(p)
    A = model.operator(p, 0)
    h, d = p.grid.h, D[0]
    beta = [2 * d * h * h / (h + 4 * a * d) for a in (0.0, 1.0, 2.0, 3.0, 4.0, 5.0)]
    # corner (0,0,0): faces -x, -y, -z; three interior neighbours
    expect = 3 * d * h + mua[0] * h ** 3 + beta[0] + beta[2] + beta[4]
    assert math.isclose(A[0, 0], expect, rel_tol=1e-14)
    last = p.grid.N - 1  # corner (3,3,3): faces +x, +y, +z
    expect = 3 * d * h + mua[0] * h ** 3 + beta[1] + beta[3] + beta[5]
    assert math.isclose(A[last, last], expect, rel_tol=1e-14)


def test_manufactured_solution_second_order():
    """phi* = f(x) f(y) f(z), f = cos(k (t - L/2)) with k chosen so that phi* + 2AD dphi*/dn = 0
    on every face (eqn:robin); q = (3 D k^2 + mu_a) phi*. The FV solution must converge to phi*
    at second order: this pins the interior stencil, the h^3 absorption and the Robin face term."""
    D, mua, Arob, L = 0.5, 0.03, 3.0, 24.0
    k = so.brentq(lambda k: math.cos(k * L / 2) - 2 * Arob * D * k * math.sin(k * L / 2), 1e-6, math.pi / L - 1e-9)
    errs = []
    for n in (6, 12, 24):
        h = L / n
        c = (np.arange(n) + 0.5) * h
        f = np.cos(k * (c - L / 2))
        phi = np.einsum("k,j,i->kji", f, f, f).reshape(-1)
        q = (3 * D * k * k + mua) * phi
        A = model.assemble(n, n, n, h, D, mua, [Arob] * 6)
        ph = spla.spsolve(A.tocsc(), h ** 3 * q)
        errs.append(np.abs(ph - phi).max() / np.abs(phi).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(orders) > 1.9, (errs, orders)
    assert errs[-1] < 5e-4


def test_photon_conservation():
    """Sum over cells of (A phi) = 1: absorbed mu_a h^3 sum(phi) plus what leaves through the
    boundary faces equals the unit source, because interior fluxes cancel pairwise."""
    p = workloads.small(nx=9, ny=8, nz=7, robin_A=(3.0, 1.0, 0.0, 3.0, 2.0, 3.0))
    mua, D = model.wavelength_coefficients(p)
    phis, _ = solve.fields_splu(p, [2])
    g = p.grid
    h = g.h
    for f in phis[0]:
        F = f.reshape(g.nz, g.ny, g.nx)
        absorbed = mua[2] * h ** 3 * f.sum()
        out = 0.0
        for face, sl in enumerate(((slice(None), slice(None), 0), (slice(None), slice(None), -1),
                                   (slice(None), 0, slice(None)), (slice(None), -1, slice(None)),
                                   (0, slice(None), slice(None)), (-1, slice(None), slice(None)))):
            A_f = p.robin_A[face]
            # outward flux through a face from the Robin condition with the half-cell gradient
            phi_b = F[sl] * 4 * A_f * D[2] / (h + 4 * A_f * D[2])
            out += (D[2] * (F[sl] - phi_b) / (h / 2) * h * h).sum()
        assert math.isclose(absorbed + out, 1.0, rel_tol=1e-11)


def test_infinite_medium_green_function():
    """Far from the boundary the field of a unit source is e^{-mu_eff r}/(4 pi D r),
    mu_eff = sqrt(mu_a / D); the lattice value converges at O(h^2)."""
    diffs = []
    for n, h in ((32, 1.5), (64, 0.75)):
        p = workloads.make_problem(workloads.Grid(n, n, n, h), 1, 1, 1, seed=3)
        p.src_ijk = np.array([[n // 2, n // 2, n // 2]])
        mua, D = model.wavelength_coefficients(p)
        mu = math.sqrt(mua[0] / D[0])
        phis, _ = solve.fields_separable(p, [0], det=[])
        F = phis[0, 0].reshape(n, n, n)
        r = 6.0
        off = int(round(r / h))
        G = math.exp(-mu * r) / (4 * math.pi * D[0] * r)
        diffs.append(abs(F[n // 2, n // 2, n // 2 + off] - G) / G)
    assert diffs[0] < 0.1 and diffs[1] < 0.02
    assert diffs[0] / diffs[1] > 3.0


@pytest.mark.parametrize("mua_t,musp_t", [(0.1, 0.5), (0.03, 1.2)])
def test_green_function_written_in_mua_and_musp(mua_t, musp_t):
    """The diffusion coefficient of the medium (Section 2.1, the reduced-scattering form of D in the
    workload definitions) pinned by the continuum: with one chromophore and mu_a, mu_s' given, the
    lattice field of a unit source far from the boundary must converge at second order in h to
        3 (mu_a + mu_s') / (4 pi r) * exp(-sqrt(3 mu_a (mu_a + mu_s')) r),
    the infinite-medium Green's function written in mu_a and mu_s' only (no D from the oracle).
    A slip such as D = 1/(3 mu_s') moves the amplitude and the decay rate by tens of per cent."""
    diffs = []
    r = 6.0
    for n, h in ((32, 1.5), (64, 0.75)):
        p = workloads.make_problem(workloads.Grid(n, n, n, h), 1, 1, 1, seed=5, n_chrom=1)
        p.c_bg = np.array([0.05])
        p.eps = np.array([[mua_t / 0.05]])
        p.mus_prime = np.array([musp_t])
        p.src_ijk = np.array([[n // 2, n // 2, n // 2]])
        phis, _ = solve.fields_separable(p, [0], det=[])
        F = phis[0, 0].reshape(n, n, n)
        G = 3.0 * (mua_t + musp_t) / (4.0 * math.pi * r) * math.exp(-math.sqrt(3.0 * mua_t * (mua_t + musp_t)) * r)
        off = int(round(r / h))
        diffs.append(F[n // 2, n // 2, n // 2 + off] / G - 1.0)
    # second order in h (ratio ~4 under halving); Richardson's extrapolation of the two lattice
    # values removes the h^2 term and must land within 1.5 % of the closed form
    assert abs(diffs[0]) < 0.15 and abs(diffs[1]) < 0.03, diffs
    assert abs(diffs[0] / diffs[1]) > 3.5, diffs
    assert abs((4.0 * diffs[1] - diffs[0]) / 3.0) < 0.015, diffs


def test_mu_a_is_the_concentration_slope_of_the_forward_model():
    """eqn:perturbation: mu_a(lambda) = sum_c eps_c(lambda) c_c, so d mu_a / d c_c = eps_c(lambda).
    Central differences of the discrete forward value e_d^T A^-1 e_s in the background concentration
    c_bg[c], with D held at its background value (the Born model's medium), must equal the row sum
    of J's chromophore-c block, sum_x J[(s,d,lambda), c N + x] (J pinned above by differences of the
    nonlinear model); and mu_a itself must equal sum_c c_c times the measured slope d mu_a / d c_c,
    each slope read off the forward model as the ratio of its c_c derivative to its derivative in a
    uniform mu_a. n_lambda != n_chrom, so a transposed eps cannot pass."""
    import scipy.sparse.linalg as spla

    p = workloads.small(nx=6, ny=5, nz=4, n_src=2, n_det=2, n_lambda=3)
    g = p.grid
    mua0, D0 = model.wavelength_coefficients(p)
    phis, phid = solve.fields_splu(p)
    J = born.born_matrix(p, phis, phid)
    N, nd, nl = g.N, p.n_det, p.n_lambda

    def fwd(cb, lam):
        A = model.assemble(g.nx, g.ny, g.nz, g.h, float(D0[lam]), float(model.mu_a(p.eps, cb)[lam]), p.robin_A)
        lu = spla.splu(A.tocsc())
        out = np.empty((p.n_src, nd))
        for a, s in enumerate(p.src_voxels()):
            e = np.zeros(N)
            e[s] = 1.0
            out[a] = lu.solve(e)[p.det_voxels()]
        return out

    delta = 1e-6
    for lam in range(nl):
        du = (born.forward_value(p, lam, delta * np.ones(N)) - born.forward_value(p, lam, -delta * np.ones(N))) / (2 * delta)
        mua_rebuilt = 0.0
        for c in range(p.n_chrom):
            cp, cm = p.c_bg.copy(), p.c_bg.copy()
            cp[c] += delta
            cm[c] -= delta
            fd = (fwd(cp, lam) - fwd(cm, lam)) / (2 * delta)
            for s in range(p.n_src):
                for d in range(nd):
                    r = (s * nd + d) * nl + lam
                    row_sum = J[r, c * N:(c + 1) * N].sum()
                    assert abs(fd[s, d] - row_sum) <= 1e-6 * abs(row_sum), (lam, c, s, d)
            mua_rebuilt += p.c_bg[c] * float(np.median(fd / du))
        assert math.isclose(mua_rebuilt, mua0[lam], rel_tol=1e-6), (lam, mua_rebuilt, mua0[lam])


# ---------------------------------------------------------------- fields (Section 3 target)

def test_dense_brute_force_matches_splu():
    p = workloads.small(nx=6, ny=5, nz=4, n_src=2, n_det=2, n_lambda=3)
    a, b = solve.fields_splu(p)
    c, d = solve.fields_dense(p)
    assert np.abs(a - c).max() <= 1e-13 * np.abs(a).max()
    assert np.abs(b - d).max() <= 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("freq", [0.0, 100.0])
def test_separable_solver_matches_splu(freq):
    p = workloads.small(nx=13, ny=11, nz=9, freq_mhz=freq)
    a, b = solve.fields_splu(p)
    c, d = solve.fields_separable(p)
    for x, y in ((a, c), (b, d)):
        rel = np.linalg.norm(x - y, axis=-1) / np.linalg.norm(x, axis=-1)
        assert rel.max() < 1e-13


def test_splu_componentwise_backward_error():
    """Oettli-Prager: |b - A phi| <= w (|A||phi| + |b|) entry by entry with w at rounding level.
    For an M-matrix this bounds the entrywise error of phi also in the decayed far field."""
    p = workloads.make_problem(workloads.Grid(16, 16, 24, 2.0), 2, 2, 2, seed=11, geometry="transmission")
    phis, _ = solve.fields_splu(p, [1])
    A = model.operator(p, 1).tocsr()
    absA = abs(A)
    for s, f in zip(p.src_voxels(), phis[0]):
        b = np.zeros(p.grid.N)
        b[s] = 1.0
        r = np.abs(b - A @ f)
        w = r / (absA @ np.abs(f) + b)
        assert w.max() < 1e-14
        assert f.min() > 0  # positive inverse of an M-matrix


def test_separable_solver_entrywise_in_the_far_field():
    """The fast-diagonalisation solve with its residual correction is accurate entry by entry:
    positive everywhere (inverse of an M-matrix applied to a unit source), componentwise backward
    error at rounding level against the assembled operator, and equal to SuperLU entry by entry
    where the transmission field has decayed by 16 orders of magnitude. Without the correction the
    same solve is accurate in norm but off by ~1e-3 relative in the far field."""
    p = workloads.make_problem(workloads.Grid(32, 32, 40, 3.0), 2, 2, 1, seed=12, geometry="transmission")
    A = model.operator(p, 0).tocsr()
    absA = abs(A)
    b = np.zeros((2, p.grid.N))
    b[np.arange(2), p.src_voxels()] = 1.0
    plain = solve.solve_separable(p, 0, b, refine=0)
    fixed = solve.solve_separable(p, 0, b)
    ref, _ = solve.fields_splu(p)
    assert fixed.min() < 1e-15 * fixed.max()  # the far field really has decayed
    assert np.abs(plain / ref[0] - 1.0).max() > 1e-5  # uncorrected: accurate in norm only
    assert fixed.min() > 0
    w = np.abs(b - (A @ fixed.T).T) / ((absA @ np.abs(fixed).T).T + b)
    assert w.max() < 1e-12
    assert np.abs(fixed / ref[0] - 1.0).max() < 1e-12


def test_reciprocity():
    """phi_s(r_d) = phi_d(r_s): A is symmetric (Section 2.1, adjoint field)."""
    for freq in (0.0, 100.0):
        p = workloads.small(nx=10, ny=9, nz=8, n_src=3, n_det=4, freq_mhz=freq)
        phis, phid = solve.fields_splu(p)
        S, Dv = p.src_voxels(), p.det_voxels()
        a = phis[:, :, Dv]  # [l, s, d]
        b = np.transpose(phid[:, :, S], (0, 2, 1))
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_frequency_domain_limits():
    """omega -> 0 recovers the CW field; the FD operator is complex symmetric, not Hermitian."""
    p0 = workloads.small(nx=8, ny=7, nz=6)
    p1 = workloads.small(nx=8, ny=7, nz=6, freq_mhz=1e-6)
    a, _ = solve.fields_splu(p0, [0])
    b, _ = solve.fields_splu(p1, [0])
    assert np.abs(b.real - a).max() < 1e-9 * np.abs(a).max()
    p2 = workloads.small(nx=8, ny=7, nz=6, freq_mhz=100.0)
    A = model.operator(p2, 0).toarray()
    assert np.array_equal(A, A.T) and not np.allclose(A, A.conj().T)



@pytest.mark.parametrize("freq", [100.0, 400.0])
def test_frequency_domain_inverse_bounded_by_the_continuous_wave_inverse(freq):
    """The bound behind the componentwise floor for complex fields: the modulation adds the same
    imaginary shift to every diagonal entry, so |A^-1| <= (Re A)^-1 entrywise, and Re A is the
    continuous-wave operator (an M-matrix with (Re A) 1 >= mu_a h^3 entrywise, so the row sums of
    (Re A)^-1 are at most 1 / (mu_a h^3)). Dense inverses on a small grid, all faces Robin and one
    Dirichlet face."""
    p = workloads.small(nx=7, ny=6, nz=5, freq_mhz=freq, robin_A=(0.0, 3.0, 3.0, 3.0, 3.0, 3.0))
    A = model.operator(p, 0).toarray()
    Ar = A.real
    assert np.allclose(A.imag, np.diag(np.diag(A.imag))) and np.ptp(np.diag(A.imag)) == 0.0
    assert np.diag(A.imag)[0] > 0.0
    ia, ir = np.abs(np.linalg.inv(A)), np.linalg.inv(Ar)
    assert ir.min() > 0.0
    assert (ia <= ir * (1 + 1e-12)).all()
    # strictly below where the modulation matters (its shift is not negligible here)
    assert (ia < ir).mean() > 0.99
    mua, _ = model.wavelength_coefficients(p)
    assert (ir.sum(axis=1) <= 1.0 / (mua[0] * p.grid.h ** 3) * (1 + 1e-12)).all()


# ---------------------------------------------------------------- Born rows (eqn:lippschwin)

def test_born_entries_are_fd_of_nonlinear_forward_model():
    """J[(s,d,l),(c,x)] = d phi_s(r_d) / d c_c(x): central differences of the nonlinear discrete
    forward model (eqn:born without the Born approximation) for every voxel and chromophore of a
    tiny grid. Pins sign, the h^3 factor, the eps_c(lambda) index and the row/column order."""
    p = workloads.small(nx=4, ny=4, nz=3, n_src=2, n_det=2, n_lambda=2, h=2.0)
    # keep sources/detectors inside a 4x4 face: draw positions by hand
    p.src_ijk = np.array([[1, 1, 2], [2, 2, 2]])
    p.det_ijk = np.array([[2, 1, 2], [1, 2, 2]])
    phis, phid = solve.fields_splu(p)
    J = born.born_matrix(p, phis, phid)
    N, nc, nl, nd = p.grid.N, p.n_chrom, p.n_lambda, p.n_det
    delta = 1e-5
    for lam in range(nl):
        for x in range(N):
            e = np.zeros(N)
            e[x] = delta
            for c in range(nc):
                dmua = e * p.eps[lam, c]
                fp = born.forward_value(p, lam, dmua)
                fm = born.forward_value(p, lam, -dmua)
                fd = (fp - fm) / (2 * delta)
                for s in range(p.n_src):
                    for d in range(nd):
                        r = (s * nd + d) * nl + lam
                        assert abs(J[r, c * N + x] - fd[s, d]) <= 1e-6 * abs(fd[s, d]) + 1e-14


def test_born_row_sum_is_uniform_mua_derivative():
    """sum_x H[(s,d,l),x] = -d phi_s(r_d)/d mu_a(uniform), by central FD on a config-1-like grid."""
    p = workloads.config(1)
    lam = 5
    phis, phid = solve.fields_splu(p, [lam])
    J = born.born_rows(p, phis, phid, rows=range(p.n_src * p.n_det), lams=[lam])
    N = p.grid.N
    H = J[:, :N] / (-(p.grid.h ** 3) * p.eps[lam, 0])
    delta = 1e-6
    ones = np.ones(N)
    fd = (born.forward_value(p, lam, delta * ones) - born.forward_value(p, lam, -delta * ones)) / (2 * delta)
    lhs = -(p.grid.h ** 3) * H.sum(axis=1)
    assert np.abs(lhs - fd.reshape(-1)).max() <= 1e-6 * np.abs(fd).max()


def test_apply_and_transpose_match_explicit_matrix():
    p = workloads.small(nx=7, ny=6, nz=5, n_src=3, n_det=2, n_lambda=5)
    lams = [1, 2, 3]
    phis, phid = solve.fields_splu(p, lams)
    J = born.born_matrix(p, phis, phid, lams)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(J.shape[1])
    y = rng.standard_normal(J.shape[0])
    jx = born.apply(p, phis, phid, x, lams)
    jty = born.apply_T(p, phis, phid, y, lams)
    assert np.allclose(jx, J @ x, rtol=1e-13, atol=1e-13 * np.abs(J @ x).max())
    assert np.allclose(jty, J.T @ y, rtol=1e-13, atol=1e-13 * np.abs(J.T @ y).max())
    assert math.isclose(jx @ y, x @ jty, rel_tol=1e-12)


def test_apply_T_adjoint_solve_form_agrees():
    """J^T y from stored detector fields equals J^T y from one extra solve per source."""
    p = workloads.small(nx=9, ny=8, nz=6, n_src=3, n_det=4, n_lambda=3)
    phis, phid = solve.fields_splu(p)
    y = np.random.default_rng(1).standard_normal(p.M)
    g1 = born.apply_T(p, phis, phid, y)
    g2 = born.apply_T_adjoint_solve(p, phis, y)
    assert np.abs(g1 - g2).max() <= 1e-12 * np.abs(g1).max()


def test_born_symmetry_source_detector_swap():
    """Swapping the roles of sources and detectors transposes the (s, d) index of H."""
    p = workloads.small(nx=8, ny=8, nz=6, n_src=3, n_det=3, n_lambda=2)
    phis, phid = solve.fields_splu(p)
    J = born.born_matrix(p, phis, phid)
    q = workloads.small(nx=8, ny=8, nz=6, n_src=3, n_det=3, n_lambda=2)
    q.src_ijk, q.det_ijk = p.det_ijk.copy(), p.src_ijk.copy()
    Jq = born.born_matrix(q, phid, phis)
    nd, nl = 3, 2
    for s in range(3):
        for d in range(3):
            for lam in range(nl):
                assert np.array_equal(J[(s * nd + d) * nl + lam], Jq[(d * nd + s) * nl + lam])


# ---------------------------------------------------------------- sketch (Appendix A.1)

def test_randsvd_recovers_exact_low_rank():
    rng = np.random.default_rng(2)
    m, n, r = 120, 300, 12
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    U, S, V = sketch.randsvd_fixed(A, rng.standard_normal((n, r + 5)), r)
    assert np.linalg.norm(A - U @ np.diag(S) @ V.T, 2) <= 1e-12 * np.linalg.norm(A, 2)
    assert np.allclose(U.T @ U, np.eye(r), atol=1e-12) and np.allclose(V.T @ V, np.eye(r), atol=1e-12)


def test_randsvd_near_optimal_on_decaying_spectrum():
    """Error within a small factor of the optimum sigma_{r+1} (Halko et al. bound with p = 20)."""
    rng = np.random.default_rng(3)
    m, n, r = 200, 500, 20
    Qa, _ = np.linalg.qr(rng.standard_normal((m, m)))
    Qb, _ = np.linalg.qr(rng.standard_normal((n, m)))
    s = 0.7 ** np.arange(m)
    A = Qa @ np.diag(s) @ Qb.T
    U, S, V = sketch.randsvd_fixed(A, rng.standard_normal((n, r + 20)), r)
    _, _, _, sall = sketch.truncated_svd(A, r)
    assert math.isclose(sall[r], s[r], rel_tol=1e-10)
    err = np.linalg.norm(A - U @ np.diag(S) @ V.T, 2)
    assert s[r] <= err * (1 + 1e-9) and err <= 1.5 * s[r]
    X = rng.standard_normal((n, 8))
    assert sketch.probe_error(A, U, S, V, X).max() < 10 * s[r] / s[0]


def _random_points(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 10.0, size=(n, 2))


def test_geometric_bisection_follows_the_split_rule():
    """Every leaf has at most two points, the leaves partition the points, and at every inner node
    the two sides are separated by the centre of the node box's widest side."""
    from oracle import sketch as osk

    pts = _random_points(37, 1)
    tree = osk.geometric_bisection(pts, (0.0, 0.0), (10.0, 10.0))
    leaves = osk.tree_leaves(tree)
    assert all(1 <= len(l) <= 2 for l in leaves)
    assert sorted(i for l in leaves for i in l) == list(range(37))

    def check(t, lo, hi):
        if osk.tree_is_leaf(t):
            return
        low = [i for l in osk.tree_leaves(t[0]) for i in l]
        high = [i for l in osk.tree_leaves(t[1]) for i in l]
        members = low + high
        lo, hi = list(lo), list(hi)
        while True:  # cuts that leave every point on one side only shrink the box
            ax = int(np.argmax(np.subtract(hi, lo)))
            cut = (lo[ax] + hi[ax]) / 2.0
            below = pts[members, ax] <= cut
            if below.all():
                hi[ax] = cut
            elif not below.any():
                lo[ax] = cut
            else:
                break
        assert pts[low, ax].max() <= cut < pts[high, ax].min()
        hi1, lo2 = list(hi), list(lo)
        hi1[ax] = cut
        lo2[ax] = cut
        check(t[0], lo, hi1)
        check(t[1], lo2, hi)

    check(tree, (0.0, 0.0), (10.0, 10.0))
    assert osk.tree_depth(tree) >= 4


def test_recursive_lowrank_exact_and_within_the_section_bound():
    """With eps at rounding level the recursion reproduces H; at a moderate eps its Frobenius error
    is inside 2^(L/2) (L+1) eps ||H||_F, the merges never exceed the sum of their children's ranks,
    and merging two exact SVDs without truncation gives the stacked matrix's singular values."""
    from oracle import sketch as osk

    p = workloads.make_problem(workloads.Grid(10, 9, 8, 2.0), 6, 4, 2, seed=13, geometry="transmission", margin=0)
    rs, rd = solve.fields_splu(p)
    J = born.born_matrix(p, rs, rd)
    nd, nl = p.n_det, p.n_lambda
    blocks = {s: J[[(s * nd + d) * nl + a for d in range(nd) for a in range(nl)]] for s in range(p.n_src)}
    xy = np.asarray(p.src_ijk, float)[:, :2] + 0.5
    tree = osk.geometric_bisection(xy, (0.0, 0.0), (float(p.grid.nx), float(p.grid.ny)))
    order = [i for l in osk.tree_leaves(tree) for i in l]
    H = np.vstack([blocks[i] for i in order])
    U, S, V, _ = osk.recursive_lowrank(blocks, tree, 1e-15)
    assert np.abs(U @ (S[:, None] * V.T) - H).max() <= 1e-10 * np.abs(H).max()
    L = osk.tree_depth(tree)
    for eps in (1e-2, 1e-3, 1e-5):
        U, S, V, ranks = osk.recursive_lowrank(blocks, tree, eps)
        err = np.linalg.norm(H - U @ (S[:, None] * V.T))
        assert err <= osk.recursive_error_bound(eps, L, np.linalg.norm(H))
        if eps >= 1e-3:
            assert S.size < min(H.shape)  # the truncation compresses
    A = blocks[order[0]]
    B = blocks[order[1]]
    f = [np.linalg.svd(X, full_matrices=False) for X in (A, B)]
    W = np.vstack([s[:, None] * vt for (_, s, vt) in f])
    assert np.allclose(np.linalg.svd(W, compute_uv=False), np.linalg.svd(np.vstack([A, B]), compute_uv=False),
                       rtol=1e-10, atol=1e-14 * np.abs(A).max())


@pytest.mark.parametrize("depth", [1, 2, 3, 5])
def test_recursive_error_bound_is_the_leaf_sum_bound_at_its_equality_case(depth):
    """Section 4.5 first bounds the error by (L + 1) eps sum_b ||H_b||_F over the leaf blocks, then
    uses Cauchy-Schwarz over the (at most 2^L) leaves: sum_b ||H_b||_F <= 2^(L/2) ||H||_F, with
    equality when a full binary tree of depth L has 2^L leaves of equal norm. For such a tree the
    leaf-sum form, computed from the blocks themselves, must equal recursive_error_bound; for
    leaves of unequal norm it must stay below it. A 2^L or an L in place of L + 1 fails."""
    from oracle import sketch as osk

    eps = 1e-3
    rng = np.random.default_rng(depth)
    nleaf = 2 ** depth
    blocks = [rng.standard_normal((3, 7)) for _ in range(nleaf)]
    blocks = [b / np.linalg.norm(b) * 2.5 for b in blocks]  # equal Frobenius norms
    H = np.vstack(blocks)
    leaf_sum = (depth + 1) * eps * sum(np.linalg.norm(b) for b in blocks)
    assert math.isclose(osk.recursive_error_bound(eps, depth, np.linalg.norm(H)), leaf_sum, rel_tol=1e-12)
    uneven = [b * (1.0 + i) for i, b in enumerate(blocks)]
    leaf_sum_u = (depth + 1) * eps * sum(np.linalg.norm(b) for b in uneven)
    assert leaf_sum_u <= osk.recursive_error_bound(eps, depth, np.linalg.norm(np.vstack(uneven))) * (1 + 1e-12)


def test_recursive_error_bound_literal_values():
    """2^(L/2) (L + 1) eps ||H||_F at two depths, by hand: L = 2, eps = 1e-3, ||H|| = 1 gives
    2 * 3 * 1e-3 = 6e-3; L = 4, eps = 1e-2, ||H|| = 2 gives 4 * 5 * 1e-2 * 2 = 0.4."""
    from oracle import sketch as osk

    assert math.isclose(osk.recursive_error_bound(1e-3, 2, 1.0), 6e-3, rel_tol=1e-15)
    assert math.isclose(osk.recursive_error_bound(1e-2, 4, 2.0), 0.4, rel_tol=1e-15)


# --------------------------------------------------------------------------- shift-invariant guess
def _cg_iterates(A, b, m):
    """m steps of plain (unpreconditioned) conjugate gradients from zero."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    for _ in range(m):
        q = A @ p
        a = rr / (p @ q)
        x += a * p
        r -= a * q
        rr2 = r @ r
        p = r + (rr2 / rr) * p
        rr = rr2
    return x


def test_shift_guess_is_cg_iterate_when_shifts_are_pure():
    """With Dirichlet faces the boundary term of Ahat_j does not depend on the wavelength, so Ahat_j =
    Ahat_0 + (sigma_j - mean sigma) I and K_m(Ahat_0, e) = K_m(Ahat_j, e): the Galerkin guess is then
    the m-th conjugate-gradient iterate of Ahat_j x = e (the CG iterate is the Galerkin solution over
    the Krylov space), computed here by a separate recurrence."""
    from oracle import shift

    p = workloads.small(seed=71, nx=9, ny=8, nz=7, n_src=2, n_det=2, n_lambda=5)
    p = dataclasses.replace(p, robin_A=np.zeros(6))
    mua, D = model.wavelength_coefficients(p)
    cell = int(p.src_voxels()[0])
    e = np.zeros(p.grid.N)
    e[cell] = 1.0
    for m in (6, 15):
        for j in (0, 4):
            g = shift.shift_guess(p, j, cell, m)
            x = _cg_iterates(shift.scaled_operator(p, j), e, m) / (D[j] * p.grid.h)
            assert np.abs(g - x).max() <= 1e-9 * np.abs(x).max()


def test_shift_guess_exact_when_the_krylov_space_is_invariant():
    """On a tiny grid m = N steps exhaust the Krylov space, or Lanczos stops early where the space is
    invariant (here for the optode on the grid's mirror plane j = 1 of ny = 3). With pure shifts
    (Dirichlet faces) a space invariant under Ahat_0 is invariant under every Ahat_j and holds
    Ahat_j^-1 e: the guess is then the solution itself."""
    from oracle import shift

    p = workloads.small(seed=72, nx=4, ny=3, nz=3, n_src=1, n_det=1, n_lambda=3)
    p = dataclasses.replace(p, robin_A=np.zeros(6))
    assert int(p.det_ijk[0][1]) == 1  # on the mirror plane: an invariant space smaller than N
    for j in range(p.n_lambda):
        for cell in (int(p.src_voxels()[0]), int(p.det_voxels()[0])):
            e = np.zeros(p.grid.N)
            e[cell] = 1.0
            exact = solve.solve_splu(p, j, e[None])[0]
            g = shift.shift_guess(p, j, cell, p.grid.N)
            assert np.abs(g - exact).max() <= 1e-10 * np.abs(exact).max()


def test_shift_guess_energy_error_decreases_with_m():
    """The Galerkin guess minimises the Ahat_j-norm of the error over the Krylov space, and the spaces
    are nested, so that error cannot grow with m (Robin faces: the shifts are not pure here)."""
    from oracle import shift

    p = workloads.small(seed=73, nx=10, ny=9, nz=8, n_src=1, n_det=1, n_lambda=4)
    _, D = model.wavelength_coefficients(p)
    cell = int(p.src_voxels()[0])
    e = np.zeros(p.grid.N)
    e[cell] = 1.0
    for j in (0, 3):
        A = shift.scaled_operator(p, j)
        xs = solve.solve_splu(p, j, e[None])[0] * (D[j] * p.grid.h)
        errs = []
        for m in (2, 5, 10, 20, 40):
            g = shift.shift_guess(p, j, cell, m) * (D[j] * p.grid.h)
            d = xs - g
            errs.append(float(d @ (A @ d)))
        assert all(b <= a * (1 + 1e-9) for a, b in zip(errs, errs[1:]))
        assert errs[-1] < 1e-3 * errs[0]


# --------------------------------------------------------------------------- PaLS reconstruction
def _pals_case(seed=75, n_basis=2):
    from oracle import recon

    p = workloads.make_problem(workloads.Grid(14, 12, 10, 2.0), 3, 3, 4, seed=seed, geometry="transmission",
                               margin=2)
    X = recon.voxel_centres(p.grid)
    rng = np.random.default_rng(seed)
    L = np.array([p.grid.nx, p.grid.ny, p.grid.nz]) * p.grid.h
    chi = L * (0.35 + 0.3 * rng.random((n_basis, 3)))
    ptrue = np.concatenate([1.0 + 0.5 * rng.random(n_basis), 1.0 / (8.0 + 4.0 * rng.random(n_basis)),
                            chi[:, 0], chi[:, 1], chi[:, 2]])
    return p, X, ptrue


def test_pals_jacobian_matches_central_differences():
    from oracle import recon

    _, X, p0 = _pals_case(n_basis=3)
    model = recon.PalsModel()
    mu, dmu = recon.shape_jacobian(p0, X, model)
    assert np.abs(mu - recon.shape(p0, X, model)).max() == 0.0
    for q in range(p0.size):
        step = 1e-6 * max(1.0, abs(p0[q]))
        e = np.zeros_like(p0)
        e[q] = step
        fd = (recon.shape(p0 + e, X, model) - recon.shape(p0 - e, X, model)) / (2 * step)
        assert np.abs(fd - dmu[:, q]).max() <= 1e-5 * max(1e-12, np.abs(dmu[:, q]).max()) + 1e-9


def test_wendland_function_is_c2_with_compact_support():
    from oracle import recon

    t = np.array([0.0, 1.0, 1.5])
    assert np.allclose(recon.wendland(t), [1.0, 0.0, 0.0])
    assert np.allclose(recon.wendland_d(t), [0.0, 0.0, 0.0])
    # the derivative is the difference quotient of the function, and the second derivative is
    # continuous across the support radius (zero on both sides of t = 1)
    h = 1e-5
    for t0 in (0.2, 0.5, 0.9):
        assert abs((recon.wendland(t0 + h) - recon.wendland(t0 - h)) / (2 * h) - recon.wendland_d(t0)) < 1e-8
    d2 = lambda t0: (recon.wendland_d(t0 + h) - recon.wendland_d(t0 - h)) / (2 * h)
    assert abs(d2(1.0 - 1e-3)) < 1e-3 and abs(d2(1.0 + 1e-3)) == 0.0


def test_reduced_residual_equals_the_truncated_operator_residual():
    """|y - U S V^T (c (x) mu)|^2 computed directly equals (|y|^2 - |U^T y|^2) + |U^T y - S M c|^2
    of the rank-r formulation, for a rank below the number of measurements."""
    from oracle import born, recon
    from oracle import solve as osolve

    p, X, ptrue = _pals_case()
    rs, rd = osolve.fields_splu(p)
    J = born.born_matrix(p, rs, rd)
    Uf, Sf, Vt = np.linalg.svd(J, full_matrices=False)
    r = 20
    U, S, V = Uf[:, :r], Sf[:r], Vt[:r].T
    N, nc = p.grid.N, p.n_chrom
    model = recon.PalsModel()
    c = np.array([0.05, 0.02, 0.03, 0.01])
    y = workloads.gaussian(76, J.shape[0])
    mu, dmu = recon.shape_jacobian(ptrue, X, model)
    Vc = V.reshape(nc, N, r)
    A = recon.project(Vc, mu, dmu)
    _, e, _ = recon.reduced_terms(A, S, U.T @ y, c)
    direct = y - U @ (S * (V.T @ np.kron(c, mu)))
    yh = U.T @ y
    assert abs((y @ y - yh @ yh + e @ e) - direct @ direct) <= 1e-10 * (y @ y)


def test_noiseless_reconstruction_drives_the_residual_to_zero():
    from oracle import born, recon
    from oracle import solve as osolve

    p, X, ptrue = _pals_case()
    rs, rd = osolve.fields_splu(p)
    J = born.born_matrix(p, rs, rd)
    U, S, Vt = np.linalg.svd(J, full_matrices=False)
    N, nc = p.grid.N, p.n_chrom
    model = recon.PalsModel()
    c = np.array([0.05, 0.02, 0.03, 0.01])
    mu_true = recon.shape(ptrue, X, model)
    y = J @ np.kron(c, mu_true)
    rng = np.random.default_rng(77)
    p0 = ptrue + np.concatenate([0.05 * rng.standard_normal(2), 0.01 * rng.standard_normal(2),
                                 0.8 * rng.standard_normal(6)])
    pr, cr, hist, _ = recon.reconstruct(Vt.T.reshape(nc, N, -1), U.T @ y, float(y @ y), S, p0, X, model, c,
                                        noise_norm=0.0, fix_c=True, max_outer=3, max_inner=100)
    assert hist[-1] <= 1e-3 * hist[0]
    assert recon.dice(mu_true, recon.shape(pr, X, model)) >= 0.9


def test_dice_and_l2_definitions():
    from oracle import recon

    a = np.array([1.0, 1.0, 0.0, 0.0])
    b = np.array([1.0, 0.0, 1.0, 0.0])
    assert recon.dice(a, a) == 1.0 and recon.rel_l2(a, a) == 0.0
    assert recon.dice(a, b) == 0.5
    assert recon.dice(a, 1.0 - a) == 0.0
    assert abs(recon.rel_l2(a, b) - 1.0) < 1e-15
