"""Parity of the Born kernels (rows, J x, J^T y, autograd) with the CPU FP64 oracle.

The kernels are fed the oracle's fields (rounded to the kernel's precision), so these
tests isolate the Born arithmetic from the solver; the solver-to-Born path is covered
in test_gpu_fields.py.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import born as oborn
from oracle import solve as osolve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    # ragged: N = 13*11*9 = 1287 is odd, so the vector path's tail code runs too
    p = workloads.small(seed=11, nx=13, ny=11, nz=9, n_src=3, n_det=5, n_lambda=4)
    rs, rd = osolve.fields_splu(p)
    return p, rs, rd


@pytest.fixture(scope="module")
def case_even():
    p = workloads.small(seed=12, nx=16, ny=12, nz=10, n_src=34, n_det=33, n_lambda=3, margin=0)
    rs, rd = osolve.fields_separable(p)
    return p, rs, rd


def _ctx(hd, p, precision):
    return hd.Context.from_problem(p, precision=precision, tol=1e-10, tol_cw=0.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("which", ["case", "case_even"])
def test_born_rows_elementwise(lib, request, precision, which):
    p, rs, rd = request.getfixturevalue(which)
    dt = torch.float64 if precision == "fp64" else torch.float32
    with _ctx(lib, p, precision) as ctx:
        ps = torch.tensor(rs, dtype=dt, device="cuda")
        pd = torch.tensor(rd, dtype=dt, device="cuda")
        J = ctx.born_assemble(ps, pd, 0, p.n_lambda).cpu().numpy()
    Jr = oborn.born_matrix(p, ps.cpu().double().numpy(), pd.cpu().double().numpy())
    if precision == "fp64":
        assert np.array_equal(J, Jr)  # same operation order -> same bits
    else:
        assert np.all(np.abs(J - Jr) <= 4e-7 * np.abs(Jr) + 1e-45)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_born_row_ranges_and_leading_dimension(lib, case, precision):
    p, rs, rd = case
    dt = torch.float64 if precision == "fp64" else torch.float32
    lams = [1, 2, 3]
    with _ctx(lib, p, precision) as ctx:
        ps = torch.tensor(rs[1:], dtype=dt, device="cuda")
        pd = torch.tensor(rd[1:], dtype=dt, device="cuda")
        cols = p.n_chrom * p.grid.N
        M = p.n_src * p.n_det * 3
        full = ctx.born_assemble(ps, pd, 1, 3).cpu().numpy()
        for row0, nrows in ((0, 1), (5, 17), (M - 7, 7), (13, M - 13)):
            Jp = ctx.born_assemble(ps, pd, 1, 3, row0, nrows, ldJ=cols + 5)
            Jp = Jp.cpu().numpy()
            assert np.array_equal(Jp[:, :cols], full[row0:row0 + nrows])
        with pytest.raises(lib.HydotError):
            ctx.born_assemble(ps, pd, 1, 3, M - 2, 3)
    Jr = oborn.born_matrix(p, ps.cpu().double().numpy(), pd.cpu().double().numpy(), lams)
    assert np.allclose(full, Jr, rtol=4e-7 if precision == "mixed" else 0, atol=0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("which", ["case", "case_even"])
def test_apply_and_apply_T(lib, request, precision, which):
    p, rs, rd = request.getfixturevalue(which)
    dt = torch.float64 if precision == "fp64" else torch.float32
    tol = 1e-12 if precision == "fp64" else 2e-5
    rng = np.random.default_rng(4)
    x = rng.standard_normal(p.n_chrom * p.grid.N)
    y = rng.standard_normal(p.M)
    with _ctx(lib, p, precision) as ctx:
        ps = torch.tensor(rs, dtype=dt, device="cuda")
        pd = torch.tensor(rd, dtype=dt, device="cuda")
        jx = ctx.born_apply(ps, pd, 0, p.n_lambda, torch.tensor(x, dtype=dt, device="cuda")).cpu().numpy()
        g0 = torch.full((p.n_chrom * p.grid.N,), 0.5, dtype=dt, device="cuda")
        jty = ctx.born_apply_T(ps, pd, 0, p.n_lambda, torch.tensor(y, dtype=dt, device="cuda"), g0).cpu().numpy()
    fs, fd = ps.cpu().double().numpy(), pd.cpu().double().numpy()
    Jr = oborn.born_matrix(p, fs, fd)
    assert np.abs(jx - Jr @ x).max() <= tol * np.abs(Jr @ x).max()
    ref = Jr.T @ y + 0.5  # accumulates into g
    assert np.abs(jty - ref).max() <= tol * np.abs(Jr.T @ y).max()
    # adjoint identity on the GPU results
    lhs = float(jx @ y)
    rhs = float(x @ (jty - 0.5))
    assert abs(lhs - rhs) <= 10 * tol * abs(lhs) + 1e-30


def test_apply_T_matches_adjoint_solve_form(lib, case):
    """g = J^T y from stored detector fields equals the oracle's one-solve-per-source form."""
    p, rs, rd = case
    y = np.random.default_rng(5).standard_normal(p.M)
    with _ctx(lib, p, "fp64") as ctx:
        g = ctx.born_apply_T(torch.tensor(rs, device="cuda"), torch.tensor(rd, device="cuda"), 0, p.n_lambda,
                             torch.tensor(y, device="cuda")).cpu().numpy()
    g2 = oborn.apply_T_adjoint_solve(p, rs, y)
    assert np.abs(g - g2).max() <= 1e-11 * np.abs(g2).max()


def test_apply_T_accumulates_over_slices(lib, case):
    p, rs, rd = case
    y = np.random.default_rng(6).standard_normal(p.M)
    with _ctx(lib, p, "fp64") as ctx:
        ps, pd = torch.tensor(rs, device="cuda"), torch.tensor(rd, device="cuda")
        full = ctx.born_apply_T(ps, pd, 0, 4, torch.tensor(y, device="cuda")).cpu().numpy()
        # the same product as two slices [0,1) and [1,4): rows of a slice are (s, d, lambda - lam0)
        Y = y.reshape(p.n_src, p.n_det, 4)
        g = torch.zeros(p.n_chrom * p.grid.N, dtype=torch.float64, device="cuda")
        ctx.born_apply_T(ps[:1].contiguous(), pd[:1].contiguous(), 0, 1,
                         torch.tensor(Y[:, :, :1].reshape(-1).copy(), device="cuda"), g)
        ctx.born_apply_T(ps[1:].contiguous(), pd[1:].contiguous(), 1, 3,
                         torch.tensor(Y[:, :, 1:].reshape(-1).copy(), device="cuda"), g)
    assert np.abs(g.cpu().numpy() - full).max() <= 1e-12 * np.abs(full).max()


def test_autograd_gradcheck(lib):
    from paper_1410_0986_gb300 import born_apply

    p = workloads.small(seed=13, nx=6, ny=5, nz=4, n_src=2, n_det=2, n_lambda=2)
    rs, rd = osolve.fields_dense(p)
    with _ctx(lib, p, "fp64") as ctx:
        ps, pd = torch.tensor(rs, device="cuda"), torch.tensor(rd, device="cuda")
        x = torch.randn(p.n_chrom * p.grid.N, dtype=torch.float64, device="cuda", requires_grad=True)
        assert torch.autograd.gradcheck(lambda v: born_apply(v, ctx, ps, pd, 0, 2), (x,), eps=1e-6, atol=1e-9)


def test_misfit_gradient_vs_central_differences(lib):
    """Config-3-style check on a reduced grid: misfit 0.5||J dc - y||^2 with an ellipsoidal
    anomaly; autograd gradient (mixed-precision fields, FP32 adjoint kernel) against central
    differences (step 1e-6, FP64 forward) at 64 seeded coordinates, relative 1e-4."""
    from paper_1410_0986_gb300 import born_apply

    p = workloads.make_problem(workloads.Grid(32, 32, 20, 1.5), 4, 4, 6, seed=17, margin=2)
    dc = workloads.ellipsoid_anomaly(p.grid, seed=18)
    dc_true = workloads.ellipsoid_anomaly(p.grid, seed=19)
    with lib.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8) as cm, \
            lib.Context.from_problem(p, precision="fp64", tol=1e-13, tol_cw=1e-11) as cd:
        ps, pd, _ = cm.solve_fields(0, p.n_lambda)
        qs, qd, _ = cd.solve_fields(0, p.n_lambda)
        ytrue = cd.born_apply(qs, qd, 0, p.n_lambda, torch.tensor(dc_true, device="cuda"))
        noise = torch.tensor(workloads.gaussian(20, p.M), device="cuda")
        y = ytrue + noise * (ytrue.norm() / p.M ** 0.5) * 10 ** (-30 / 20)
        x = torch.tensor(dc, dtype=torch.float32, device="cuda", requires_grad=True)
        r = born_apply(x, cm, ps, pd, 0, p.n_lambda) - y.float()
        (0.5 * (r * r).sum()).backward()
        grad = x.grad.double()

        def f(v):
            rr = cd.born_apply(qs, qd, 0, p.n_lambda, v) - y
            return 0.5 * float((rr * rr).sum())

        idx = np.random.default_rng(21).choice(p.n_chrom * p.grid.N, size=64, replace=False)
        base = torch.tensor(dc, device="cuda")
        h = 1e-6
        fd = []
        for i in idx:
            e = torch.zeros_like(base)
            e[i] = h
            fd.append((f(base + e) - f(base - e)) / (2 * h))
        fd = np.array(fd)
    g = grad.cpu().numpy()[idx]
    scale = np.abs(grad.cpu().numpy()).max()
    assert np.abs(g - fd).max() <= 1e-4 * scale


@pytest.mark.parametrize("ns,nd,grid", [(32, 32, (16, 16, 12)), (64, 32, (16, 16, 12)), (40, 100, (16, 16, 12)),
                                        (3, 5, (16, 16, 12)), (24, 24, (20, 14, 9)), (16, 7, (20, 14, 9))])
def test_apply_and_apply_T_optode_blocks(lib, ns, nd, grid):
    """J x and J^T y in FP32 against the FP64 oracle for optode counts that fill whole 32-wide
    blocks (the guard-free path) and ones that leave partial blocks (40 x 100: several detector
    blocks, the last one partial); the 20 x 14 x 9 grid (N = 2520) ends in a partial 256-voxel
    chunk of the register-tiled J^T y kernel, with 24 sources (tiles of 24) and 16 (tiles of 16)."""
    p = workloads.make_problem(workloads.Grid(*grid, 2.0), ns, nd, 3, seed=51, geometry="transmission", margin=0)
    rs, rd = osolve.fields_separable(p)
    y = workloads.gaussian(52, p.M)
    xv = workloads.gaussian(53, p.n_chrom * p.grid.N)
    g_ref = oborn.apply_T(p, rs, rd, y)
    y_ref = oborn.apply(p, rs, rd, xv)
    with lib.Context.from_problem(p, precision="mixed", tol=1e-8, tol_cw=0.0) as ctx:
        ps = torch.tensor(rs, dtype=torch.float32, device="cuda")
        pd = torch.tensor(rd, dtype=torch.float32, device="cuda")
        g = torch.zeros(p.n_chrom * p.grid.N, device="cuda")
        ctx.born_apply_T(ps, pd, 0, p.n_lambda, torch.tensor(y, dtype=torch.float32, device="cuda"), g)
        yy = ctx.born_apply(ps, pd, 0, p.n_lambda, torch.tensor(xv, dtype=torch.float32, device="cuda"))
    assert np.abs(g.double().cpu().numpy() - g_ref).max() <= 2e-5 * np.abs(g_ref).max()
    assert np.abs(yy.double().cpu().numpy() - y_ref).max() <= 2e-5 * np.abs(y_ref).max()


def test_apply_T_tiled_and_per_voxel_kernels_agree(lib, monkeypatch):
    """The register-tiled J^T y kernel and the per-voxel one (taken when HYDOT_NO_TILE_T is set, and
    for FP64, more than 4 chromophores or N not a multiple of 4) give the same gradient to FP32
    rounding, on a case with two source tiles, two detector chunks and a partial voxel chunk."""
    p = workloads.make_problem(workloads.Grid(20, 14, 9, 2.0), 40, 36, 5, seed=54, geometry="transmission", margin=0)
    gen = torch.Generator(device="cuda").manual_seed(5)
    N = p.grid.N
    ps = torch.rand(p.n_lambda, p.n_src, N, device="cuda", generator=gen)
    pd = torch.rand(p.n_lambda, p.n_det, N, device="cuda", generator=gen)
    y = torch.randn(p.M, device="cuda", generator=gen)
    out = []
    with lib.Context.from_problem(p, precision="mixed", tol=1e-8, tol_cw=0.0) as ctx:
        for flag in (None, "1"):
            if flag:
                monkeypatch.setenv("HYDOT_NO_TILE_T", flag)
            g = torch.zeros(p.n_chrom * N, device="cuda")
            ctx.born_apply_T(ps, pd, 0, p.n_lambda, y, g)
            out.append(g.double().cpu())
    scale = out[1].abs().max()
    assert (out[0] - out[1]).abs().max() <= 1e-5 * scale


def _perturbed_fields_oracle(p, dc):
    """Oracle fields of the perturbed medium: sparse LU of A_lambda + h^3 diag(dmu_a)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from oracle import model

    N = p.grid.N
    nc = p.n_chrom
    out_s = np.empty((p.n_lambda, p.n_src, N))
    out_d = np.empty((p.n_lambda, p.n_det, N))
    for lam in range(p.n_lambda):
        dmua = sum(p.eps[lam, c] * dc[c * N:(c + 1) * N] for c in range(nc))
        lu = spla.splu((model.operator(p, lam) + sp.diags(p.grid.h ** 3 * dmua)).tocsc())
        for out, cells in ((out_s, p.src_voxels()), (out_d, p.det_voxels())):
            for a, v in enumerate(cells):
                e = np.zeros(N)
                e[v] = 1.0
                out[lam, a] = lu.solve(e)
    return out_s, out_d


@pytest.mark.parametrize("grid,precision", [((17, 12, 10), "mixed"), ((20, 16, 12), "mixed"), ((17, 12, 10), "fp64")])
def test_absorption_perturbation_fields(lib, grid, precision):
    """hydot_set_absorption: fields of the perturbed medium (the nonlinear forward model) against
    the oracle's sparse LU; 20 x 16 x 12 would take the TMA inner kernels without the perturbation."""
    p = workloads.make_problem(workloads.Grid(*grid, 2.0), 2, 3, 2, seed=81, geometry="transmission", margin=1)
    dc = workloads.ellipsoid_anomaly(p.grid, seed=82, contrast=0.5)
    rs, rd = _perturbed_fields_oracle(p, dc)
    kw = dict(tol=1e-13, tol_cw=0.0) if precision == "fp64" else dict(tol=1e-10, tol_cw=1e-8)
    with lib.Context.from_problem(p, precision=precision, **kw) as ctx:
        ctx.set_absorption(dc)
        ps, pd, st = ctx.solve_fields(0, p.n_lambda)
        ctx.set_absorption(None)
        qs, _, _ = ctx.solve_fields(0, p.n_lambda)
    tol = 1e-10 if precision == "fp64" else 1e-6
    for got, ref in ((ps, rs), (pd, rd)):
        g = got.double().cpu().numpy()
        assert (np.linalg.norm(g - ref, axis=-1) / np.linalg.norm(ref, axis=-1)).max() <= tol
    # the perturbation absorbs: removing it raises every field
    assert (qs.double() - ps.double()).min() >= -1e-6 * float(qs.abs().max())


def test_born_error_is_first_order_in_the_contrast(lib):
    """The Born model y(0) + t J dc against the nonlinear forward model y(t) (the perturbed fields
    at the detector cells): the relative error vanishes with t and grows linearly (halving t halves
    it), as the remainder of the first-order expansion must."""
    p = workloads.make_problem(workloads.Grid(24, 24, 16, 2.0), 3, 3, 2, seed=83, geometry="transmission")
    dc = workloads.ellipsoid_anomaly(p.grid, seed=84, contrast=0.005)
    det = torch.tensor(p.det_voxels(), device="cuda")
    with lib.Context.from_problem(p, precision="fp64", tol=1e-13, tol_cw=0.0) as ctx:
        ps, pd, _ = ctx.solve_fields(0, p.n_lambda)
        y0 = ps[:, :, det].permute(1, 2, 0).reshape(-1)  # rows (s, d, lambda)
        jdc = ctx.born_apply(ps, pd, 0, p.n_lambda, torch.tensor(dc, device="cuda"))
        errs = []
        for t in (2.0, 1.0, 0.5, 0.25):
            ctx.set_absorption(t * dc)
            qs, _, _ = ctx.solve_fields(0, p.n_lambda, detectors=False)
            yt = qs[:, :, det].permute(1, 2, 0).reshape(-1)
            errs.append(float((yt - y0 - t * jdc).norm() / (yt - y0).norm()))
        ctx.set_absorption(None)
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert errs[-1] < 0.05, errs
    assert all(1.7 < r < 2.3 for r in ratios), (errs, ratios)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_solve_form_of_the_gradient(lib, precision):
    """Section 5's gradient needs J^T y. Its second form solves one extra system per source and
    wavelength, psi_s = A^-1 sum_d y[s,d,lambda] e_d (A symmetric, so this equals sum_d y phi_d), and
    forms g = -h^3 sum_lambda eps_c sum_s phi_s psi_s without the detector fields. The adjoint fields
    match the oracle's sparse-LU solves of the same right-hand sides (1e-10 FP64, 1e-6 mixed,
    norm-wise per field); g matches the oracle's adjoint-solve form and the stored-field product
    (1e-10 / 2e-5 of the largest entry). The data of one source are all zero: its field is zero."""
    p = workloads.small(seed=31, nx=16, ny=12, nz=9, n_src=3, n_det=5, n_lambda=3)
    rs, rd = osolve.fields_splu(p)
    nl, ns, nd, N = p.n_lambda, p.n_src, p.n_det, p.grid.N
    y = np.random.default_rng(2).standard_normal(p.M)
    y[(1 * nd) * nl:(2 * nd) * nl] = 0.0  # source 1 has no data
    Dv = p.det_voxels()
    psi_ref = np.empty((nl, ns, N))
    for a in range(nl):
        rhs = np.zeros((ns, N))
        for s in range(ns):
            for d in range(nd):
                rhs[s, Dv[d]] += y[(s * nd + d) * nl + a]
        psi_ref[a] = osolve.solve_splu(p, a, rhs)
    g_ref = oborn.apply_T_adjoint_solve(p, rs, y)
    dt = torch.float64 if precision == "fp64" else torch.float32
    kw = dict(tol=1e-13, tol_cw=0.0) if precision == "fp64" else dict(tol=1e-10, tol_cw=1e-8, cw_floor=100.0)
    tf, tg = (1e-10, 1e-10) if precision == "fp64" else (1e-6, 2e-5)
    with lib.Context.from_problem(p, precision=precision, **kw) as ctx:
        ps, pd, _ = ctx.solve_fields(0, nl)
        yt = torch.tensor(y, dtype=dt, device="cuda")
        psi, st = ctx.solve_adjoint(0, nl, yt)
        assert st["n_not_converged"] == 0 and st["n_fields"] == nl * ns
        g = ctx.born_apply_T_adjoint(ps, psi, 0, nl).double().cpu().numpy()
        g2 = ctx.born_apply_T(ps, pd, 0, nl, yt).double().cpu().numpy()
    got = psi.double().cpu().numpy()
    for a in range(nl):
        for s in range(ns):
            if s == 1:
                assert not got[a, s].any()
                continue
            assert np.linalg.norm(got[a, s] - psi_ref[a, s]) <= tf * np.linalg.norm(psi_ref[a, s])
    assert np.abs(g - g_ref).max() <= tg * np.abs(g_ref).max()
    assert np.abs(g - g2).max() <= tg * np.abs(g_ref).max()
