"""Full-size parity at the benchmark's launch configuration (64x64x48 grid, 32 + 32 optodes,
16-wavelength chunks, FP32 PCG with FP64 refinement to a componentwise backward error <= 1e-8).

Expected values are the oracle's sparse-direct fields at sampled voxels and at every optode
cell, and its J x (every row) and J^T y (sampled voxels) on one-wavelength slices, written by
tests/golden/make_golden.py (oracle only). Born entries are checked at the sampled voxels against
the row maximum of the oracle's H row; J x and J^T y element by element against the oracle's
products of its own FP64 fields, and by the adjoint identity.
"""
import os

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cw_mixed_64x64x48.npz")
CHUNK = 16
CW_FLOOR = 100.0  # the benchmark's setting: Born entries within ~1e-6 of their row maximum


@pytest.fixture(scope="module")
def solved(lib):
    gold = np.load(GOLD)
    p = workloads.config(2)
    ctx = lib.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, max_lambda_per_call=CHUNK,
                                  cw_floor=CW_FLOOR)
    ctx.set_shift_guess(40)  # the benchmark's setting: solves start from the shift-invariant guesses
    out = {}
    for a, lam in enumerate(gold["lams"]):
        lam0 = (int(lam) // CHUNK) * CHUNK
        ps, pd, st = ctx.solve_fields(lam0, CHUNK)
        out[int(lam)] = (lam0, ps, pd, st, a)
    yield p, gold, ctx, out
    ctx.close()


def test_fields_at_sampled_voxels(solved):
    p, gold, ctx, out = solved
    vox = torch.tensor(gold["vox"], device="cuda")
    for lam, (lam0, ps, pd, st, a) in out.items():
        assert st["n_not_converged"] == 0
        gs = ps[lam - lam0][:, vox].double().cpu().numpy()
        gd = pd[lam - lam0][:, vox].double().cpu().numpy()
        for got, ref, nrm in ((gs, gold["phis"][a], gold["norms_s"][a]), (gd, gold["phid"][a], gold["norms_d"][a])):
            # entrywise error against the field norm (bounds the 1e-6 norm-wise criterion from below)
            assert (np.abs(got - ref).max(axis=1) / nrm).max() <= 1e-6
            # far field: entry-by-entry relative accuracy at the optode cells (the Born rows need it)
            n_opt = p.n_src + p.n_det
            rel = np.abs(got[:, -n_opt:] - ref[:, -n_opt:]) / np.abs(ref[:, -n_opt:])
            assert rel.max() <= 1e-5, rel.max()


def test_born_rows_at_sampled_voxels(solved, lib):
    p, gold, ctx, out = solved
    N, nc, nd = p.grid.N, p.n_chrom, p.n_det
    h3 = p.grid.h ** 3
    vox = gold["vox"]
    cols = torch.tensor(np.concatenate([c * N + vox for c in range(nc)]), device="cuda")
    for lam, (lam0, ps, pd, st, a) in out.items():
        s_list = (0, 13, 31)
        for s in s_list:
            row0 = s * nd * CHUNK
            J = ctx.born_assemble(ps, pd, lam0, CHUNK, row0, nd * CHUNK)
            rows = torch.arange(nd, device="cuda") * CHUNK + (lam - lam0)  # (s, d, lam) for d = 0..nd-1
            Jr = J[rows]
            got = Jr[:, cols].double().cpu().numpy().reshape(nd, nc, -1)
            rowmax_gpu = Jr.abs().max(dim=1).values.double().cpu().numpy()
            del J, Jr
            eps = p.eps[lam]
            ref_h = gold["phis"][a][s][None, :] * gold["phid"][a]  # [nd, vox]
            ref = -h3 * eps[None, :, None] * ref_h[:, None, :]
            rowmax = h3 * np.abs(eps).max() * gold["hmax"][a][s]  # [nd]
            err = np.abs(got - ref).max(axis=(1, 2)) / rowmax
            assert err.max() <= 1e-5, err.max()
            assert np.abs(rowmax_gpu - rowmax).max() <= 1e-5 * rowmax.max()
            assert (np.abs(rowmax_gpu - rowmax) / rowmax).max() <= 1e-5


def test_apply_and_transpose_elementwise_full_size(solved):
    """eqn:measurement and its transpose on one-wavelength slices of the solved chunks, against the
    oracle's products of its sparse-direct fields: y = J x at all 1,024 (s, d) rows and g = J^T y at
    the sampled voxels of every chromophore, each within 2e-5 of the largest entry. The probe vectors
    are positive (x = 0.05 |gaussian|, y = |gaussian|, the recipe make_golden.py stores)."""
    p, gold, ctx, out = solved
    N, nc = p.grid.N, p.n_chrom
    x = torch.tensor(0.05 * np.abs(workloads.gaussian(20141010, nc * N)), dtype=torch.float32, device="cuda")
    y = torch.tensor(np.abs(workloads.gaussian(20141011, p.n_src * p.n_det)), dtype=torch.float32, device="cuda")
    vox = torch.tensor(gold["vox"], device="cuda")
    for lam, (lam0, ps, pd, st, a) in out.items():
        k = lam - lam0
        psl, pdl = ps[k:k + 1].contiguous(), pd[k:k + 1].contiguous()
        jx = ctx.born_apply(psl, pdl, lam, 1, x).double().cpu().numpy()
        ref = gold["jx"][a]
        assert np.abs(jx - ref).max() <= 2e-5 * np.abs(ref).max(), np.abs(jx - ref).max() / np.abs(ref).max()
        g = ctx.born_apply_T(psl, pdl, lam, 1, y).view(nc, N)[:, vox].double().cpu().numpy()
        refg = gold["jty"][a]
        assert np.abs(g - refg).max() <= 2e-5 * gold["jty_max"][a], np.abs(g - refg).max() / gold["jty_max"][a]


def test_apply_adjoint_identity_full_size(solved):
    p, gold, ctx, out = solved
    lam0, ps, pd, st, a = next(iter(out.values()))
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randn(p.n_chrom * p.grid.N, device="cuda", generator=g)
    y = torch.randn(p.n_src * p.n_det * CHUNK, device="cuda", generator=g)
    jx = ctx.born_apply(ps, pd, lam0, CHUNK, x)
    jty = ctx.born_apply_T(ps, pd, lam0, CHUNK, y)
    lhs = float((jx.double() * y.double()).sum())
    rhs = float((x.double() * jty.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), 1e-300) + 1e-5 * float(jx.double().abs().sum() * y.abs().max())


def test_config3_misfit_gradient_on_a_wavelength_slice(lib):
    """The gradient workload at full grid size (96x96x64, h = 1.5 mm, 24 + 24 optodes) on wavelengths 0-3:
    misfit 0.5 ||J dc - y||^2 with the seeded ellipsoidal anomaly, y = J dc_true + noise at 30 dB;
    the autograd gradient (mixed-precision fields, FP32 adjoint kernel) against the oracle's
    J^T (J dc - y) from its own FP64 fields, at 64 seeded coordinates, relative 1e-4 of the largest
    component. The misfit is quadratic in dc, so this component equals the central difference of
    the FP64 misfit up to rounding."""
    from oracle import born as oborn
    from oracle import solve as osolve
    from paper_1410_0986_gb300 import born_apply

    p = workloads.config(3)
    lams = [0, 1, 2, 3]
    nl = len(lams)
    dc = workloads.ellipsoid_anomaly(p.grid, seed=301)
    dc_true = workloads.ellipsoid_anomaly(p.grid, seed=302)
    rs, rd = osolve.fields_separable(p, lams)
    y_true = oborn.apply(p, rs, rd, dc_true, lams)
    M = y_true.size
    y = y_true + workloads.gaussian(303, M) * (np.linalg.norm(y_true) / M ** 0.5) * 10 ** (-30 / 20)
    g_ref = oborn.apply_T(p, rs, rd, oborn.apply(p, rs, rd, dc, lams) - y, lams)
    del rs, rd
    with lib.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=CW_FLOOR,
                                  max_lambda_per_call=nl) as ctx:
        ctx.set_shift_guess(40)  # as in the benchmark's gradient workload
        ps, pd, st = ctx.solve_fields(0, nl)
        x = torch.tensor(dc, dtype=torch.float32, device="cuda", requires_grad=True)
        r = born_apply(x, ctx, ps, pd, 0, nl) - torch.tensor(y, dtype=torch.float32, device="cuda")
        (0.5 * (r * r).sum()).backward()
        g = x.grad.double().cpu().numpy()
    idx = np.random.default_rng(304).choice(g.size, size=64, replace=False)
    scale = np.abs(g_ref).max()
    assert np.abs(g[idx] - g_ref[idx]).max() <= 1e-4 * scale
    # all 2.36 M components, norm-wise (the components at optode cells carry products with the
    # far field of the other optodes, which the oracle's fields resolve entry by entry)
    assert np.linalg.norm(g - g_ref) <= 1e-5 * np.linalg.norm(g_ref)


def test_config5_fields_at_the_sketch_configuration(lib):
    """The large hyperspectral workload at full size (128x128x96, h = 1 mm, 1.57 M voxels, 64 + 64 optodes) on wavelengths
    0-3, solved as the benchmark's sketch phase solves them (512 fields in one call): sources 0 and
    63 and detectors 0 and 63 at wavelengths 0 and 3 against the oracle's separable FP64 fields, at
    2,000 sampled voxels and every optode cell (entrywise against the field norm <= 1e-6, optode
    cells entry by entry <= 1e-5), and their Born products within 1e-5 of the row maximum."""
    from oracle import solve as osolve

    p = workloads.config(5)
    lams, src, det = [0, 3], [0, p.n_src - 1], [0, p.n_det - 1]
    rs, rd = osolve.fields_separable(p, lams, src=src, det=det)
    with lib.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=CW_FLOOR,
                                  max_lambda_per_call=4) as ctx:
        ps, pd, st = ctx.solve_fields(0, 4)
    assert st["n_not_converged"] == 0 and st["n_fields"] == 4 * (p.n_src + p.n_det)
    n_opt = p.n_src + p.n_det
    vox = np.concatenate([np.random.default_rng(501).choice(p.grid.N, 2000, replace=False),
                          p.src_voxels(), p.det_voxels()])
    vt = torch.tensor(vox, device="cuda")
    for a, lam in enumerate(lams):
        gs = ps[lam][src][:, vt].double().cpu().numpy()
        gd = pd[lam][det][:, vt].double().cpu().numpy()
        for got, full in ((gs, rs[a]), (gd, rd[a])):
            ref = full[:, vox]
            nrm = np.linalg.norm(full, axis=1)
            assert (np.abs(got - ref).max(axis=1) / nrm).max() <= 1e-6
            rel = np.abs(got[:, -n_opt:] - ref[:, -n_opt:]) / np.abs(ref[:, -n_opt:])
            assert rel.max() <= 1e-5, rel.max()
        for i in range(len(src)):
            for j in range(len(det)):
                Hr = rs[a][i, vox] * rd[a][j, vox]
                Hg = gs[i] * gd[j]
                # the row maximum of H over all voxels, from the oracle's full fields
                hmax = np.abs(rs[a][i] * rd[a][j]).max()
                assert np.abs(Hg - Hr).max() <= 1e-5 * hmax


@pytest.mark.parametrize("which", [0, 1])
def test_config4_frequency_domain_phantoms(lib, which):
    """The uneven batch of frequency-domain phantoms (100 MHz, complex-symmetric COCG in complex64 with
    complex128 refinement), the two smallest grids of the uneven batch on wavelengths 0-1: fields at
    every optode cell and 2,000 sampled voxels against the oracle's complex128 fields."""
    from oracle import solve as osolve

    p = workloads.config4_batch()[which]
    lams = [0, 1]
    rs, rd = osolve.fields_separable(p, lams)
    with lib.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, max_lambda_per_call=2) as ctx:
        ps, pd, st = ctx.solve_fields(0, 2)
    assert ps.dtype == torch.complex64 and st["n_not_converged"] == 0
    vox = np.unique(np.concatenate([np.random.default_rng(401 + which).choice(p.grid.N, 2000, replace=False),
                                    p.src_voxels(), p.det_voxels()]))
    for got, ref in ((ps, rs), (pd, rd)):
        g = got.cpu().numpy()[:, :, vox].astype(np.complex128)
        rr = ref[:, :, vox]
        rel = np.linalg.norm(g - rr, axis=-1) / np.linalg.norm(rr, axis=-1)
        assert rel.max() <= 1e-6, rel.max()
