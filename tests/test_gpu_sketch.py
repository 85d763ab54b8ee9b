"""Parity of the tensor-core sketch passes (Appendix A.1) with the CPU oracle.

Pass 1 computes Y = J Omega and pass 2 B^T = J^T Q on the tcgen05 tensor cores with BF16
operands and FP32 accumulation. Two references: (i) the same products with the operands rounded
to BF16 the way the kernels round them, evaluated in FP64 -- this checks the tensor-core data path
(layout, swizzle, descriptors, accumulation) to FP32 accumulation accuracy; (ii) the oracle's FP64
J times the FP64 Omega / Q -- the end-to-end error, bounded by BF16's 2^-9 relative rounding.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import born as oborn
from oracle import solve as osolve

pytestmark = pytest.mark.gpu


def bf16_round(a):
    """Round float32 values to bfloat16 (round to nearest even), returned as float64."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def case():
    # 40 sources x 36 detectors: 1,440 pairs per wavelength -> 12 row tiles, the last one partial
    p = workloads.small(seed=21, nx=16, ny=12, nz=10, n_src=40, n_det=36, n_lambda=3, margin=0)
    rs, rd = osolve.fields_separable(p)
    return p, rs.astype(np.float32), rd.astype(np.float32)


def test_sketch_range_pass(lib, case):
    p, rs, rd = case
    N, nc, ncols = p.grid.N, p.n_chrom, 200
    om = workloads.gaussian(31, (nc, ncols, N)).astype(np.float32)
    om_b = bf16_round(om)
    with lib.Context.from_problem(p, precision="mixed", tol=1e-8, tol_cw=0.0) as ctx:
        Y = ctx.sketch_range(torch.tensor(rs, device="cuda"), torch.tensor(rd, device="cuda"), 0, p.n_lambda,
                             torch.tensor(om, device="cuda").to(torch.bfloat16), ncols).cpu().double().numpy()
    assert np.all(Y[:, ncols:] == 0.0)
    Y = Y[:, :ncols]
    h3 = p.grid.h ** 3
    # (i) emulate the kernels' operand rounding: A = bf16(fp32(phi_s * phi_d)), M = bf16(sum_c eps_c Omega_c)
    nd, nl = p.n_det, p.n_lambda
    ref_i = np.empty_like(Y)
    for lam in range(nl):
        M = bf16_round(np.einsum("c,ckx->kx", p.eps[lam].astype(np.float32), om_b.astype(np.float32)).astype(np.float32))
        for s in range(p.n_src):
            A = bf16_round(rs[lam, s][None, :] * rd[lam])  # [nd, N]
            rows = [(s * nd + d) * nl + lam for d in range(nd)]
            ref_i[rows] = -h3 * A @ M.T
    err_i = np.abs(Y - ref_i).max(axis=1) / np.abs(ref_i).max(axis=1)
    assert err_i.max() <= 2e-3, err_i.max()
    # (ii) end to end against the FP64 oracle
    J = oborn.born_matrix(p, rs.astype(np.float64), rd.astype(np.float64))
    Omega = np.concatenate([om[c].T for c in range(nc)], axis=0).astype(np.float64)  # [(c,x), k]
    ref = J @ Omega
    rel = np.linalg.norm(Y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= 2e-2, rel.max()


def test_sketch_project_pass_accumulates_over_slices(lib, case):
    p, rs, rd = case
    N, nc, ncols = p.grid.N, p.n_chrom, 200
    M = p.M
    Q = workloads.gaussian(32, (M, ncols)).astype(np.float32)
    Qp = np.zeros((M, 224), dtype=np.float32)
    Qp[:, :ncols] = Q
    nd, nl = p.n_det, p.n_lambda
    with lib.Context.from_problem(p, precision="mixed", tol=1e-8, tol_cw=0.0) as ctx:
        ps, pd = torch.tensor(rs, device="cuda"), torch.tensor(rd, device="cuda")
        Bt = torch.zeros(nc * N, 224, device="cuda")
        # two slices [0,1) and [1,3): rows of a slice are (s, d, lambda - lam0)
        for lam0, nlam in ((0, 1), (1, 2)):
            rows = [(s * nd + d) * nl + lam for s in range(p.n_src) for d in range(nd) for lam in range(lam0, lam0 + nlam)]
            Qs = torch.tensor(Qp[rows], device="cuda")
            ctx.sketch_project(ps[lam0:lam0 + nlam].contiguous(), pd[lam0:lam0 + nlam].contiguous(), lam0, nlam, Qs,
                               ncols, Bt)
        Bt = Bt.cpu().double().numpy()
    assert np.all(Bt[:, ncols:] == 0.0)
    Bt = Bt[:, :ncols]
    J = oborn.born_matrix(p, rs.astype(np.float64), rd.astype(np.float64))
    ref = J.T @ Q.astype(np.float64)
    rel = np.linalg.norm(Bt - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert rel.max() <= 2e-2, rel.max()
    # exact operand emulation: A = bf16(phi_s phi_d), B = bf16(eps_c * Q)
    h3 = p.grid.h ** 3
    ref_i = np.zeros_like(ref)
    for lam in range(nl):
        for s in range(p.n_src):
            A = bf16_round(rs[lam, s][None, :] * rd[lam])  # [nd, N]
            rows = [(s * nd + d) * nl + lam for d in range(nd)]
            for c in range(nc):
                Bq = bf16_round((np.float32(p.eps[lam, c]) * Q[rows]).astype(np.float32))
                ref_i[c * N:(c + 1) * N] += -h3 * A.T @ Bq
    err_i = np.abs(Bt - ref_i).max(axis=0) / np.abs(ref_i).max(axis=0)
    assert err_i.max() <= 2e-3, err_i.max()


def test_sketch_project_double_buffered_fields(lib):
    """n_src + n_det <= 64: the projection keeps two wavelengths' field blocks in shared memory (the
    next one loads while the current one is formed); five wavelengths cycle both buffers, and three
    chromophores leave the second accumulator of the last chromophore pair empty. Compared with the
    exact emulation of the BF16 operands."""
    p = workloads.make_problem(workloads.Grid(20, 16, 12, 2.0), 6, 10, 5, seed=45, n_chrom=3,
                               geometry="transmission", margin=0)
    rs, rd = osolve.fields_separable(p)
    rs, rd = rs.astype(np.float32), rd.astype(np.float32)
    N, nc, ncols = p.grid.N, p.n_chrom, 200
    nd, nl = p.n_det, p.n_lambda
    Q = workloads.gaussian(46, (p.M, ncols)).astype(np.float32)
    Qp = np.zeros((p.M, 224), dtype=np.float32)
    Qp[:, :ncols] = Q
    with lib.Context.from_problem(p, precision="mixed", tol=1e-8, tol_cw=0.0) as ctx:
        Bt = torch.zeros(nc * N, 224, device="cuda")
        ctx.sketch_project(torch.tensor(rs, device="cuda"), torch.tensor(rd, device="cuda"), 0, nl,
                           torch.tensor(Qp, device="cuda"), ncols, Bt)
        Bt = Bt.cpu().double().numpy()
    assert np.all(Bt[:, ncols:] == 0.0)
    Bt = Bt[:, :ncols]
    h3 = p.grid.h ** 3
    ref_i = np.zeros((nc * N, ncols))
    for lam in range(nl):
        for s in range(p.n_src):
            A = bf16_round(rs[lam, s][None, :] * rd[lam])
            rows = [(s * nd + d) * nl + lam for d in range(nd)]
            for c in range(nc):
                Bq = bf16_round((np.float32(p.eps[lam, c]) * Q[rows]).astype(np.float32))
                ref_i[c * N:(c + 1) * N] += -h3 * A.T @ Bq
    err_i = np.abs(Bt - ref_i).max(axis=0) / np.abs(ref_i).max(axis=0)
    assert err_i.max() <= 2e-3, err_i.max()


def test_rank_r_factorisation_near_optimal(lib, case):
    """Full pipeline (range, orthonormalisation, projection over two row blocks, recompression):
    the error of U S V^T is within a small factor of the exact optimum sigma_(r+1) plus the BF16
    floor, the factors are orthonormal, and the leading singular values match J's."""
    from paper_1410_0986_gb300.sketch import born_sketch, chunk_rows

    p, rs, rd = case
    N, nc = p.grid.N, p.n_chrom
    rank, over = 200, 20
    om = workloads.gaussian(33, (nc, rank + over, N)).astype(np.float32)
    chunks = [(0, 1), (1, 2)]
    with lib.Context.from_problem(p, precision="mixed", tol=1e-8, tol_cw=0.0) as ctx:
        ps, pd = torch.tensor(rs, device="cuda"), torch.tensor(rd, device="cuda")
        U, S, V, kept = born_sketch(ctx, chunks, torch.tensor(om, device="cuda").to(torch.bfloat16), rank, over,
                                    lambda l0, nl: (ps[l0:l0 + nl].contiguous(), pd[l0:l0 + nl].contiguous()))
        rows = chunk_rows(ctx, chunks)
        U, V = U.cpu().double().numpy(), V.cpu().double().numpy()
    J = oborn.born_matrix(p, rs.astype(np.float64), rd.astype(np.float64))[rows]
    sig = np.linalg.svd(J, compute_uv=False)
    assert kept == rank + over
    assert np.abs(U.T @ U - np.eye(rank)).max() < 1e-3
    assert np.abs(V.T @ V - np.eye(rank)).max() < 1e-2
    assert np.abs(S[:20] / sig[:20] - 1).max() < 1e-2
    err = np.linalg.norm(J - (U * S) @ V.T, 2)
    assert err <= 10 * sig[rank] + 1e-2 * sig[0], (err / sig[0], sig[rank] / sig[0])


def _range_ref_bf16(p, rs, rd, om_b, rows_sel):
    """-h^3 bf16(phi_s phi_d) @ bf16(sum_c eps_c Omega_c)^T for the selected rows (s, d, lambda)."""
    nd, nl, h3 = p.n_det, p.n_lambda, p.grid.h ** 3
    out = {}
    Ms = {}
    for r in rows_sel:
        lam = r % nl
        s, d = divmod(r // nl, nd)
        if lam not in Ms:
            Ms[lam] = bf16_round(np.einsum("c,ckx->kx", p.eps[lam].astype(np.float32),
                                           om_b.astype(np.float32)).astype(np.float32))
        a = bf16_round(rs[lam, s] * rd[lam, d])
        out[r] = -h3 * Ms[lam] @ a
    return out


@pytest.mark.parametrize("shape", [
    # (grid, n_src, n_det, n_lambda): K split over CTAs (long K, few items)
    ((48, 40, 32), 8, 8, 2),
    # detectors per block below 64 and not a power of two; partial source blocks
    ((24, 20, 16), 30, 24, 2),
    # more than 64 detectors: two detector blocks, the second partial
    ((16, 16, 12), 6, 100, 1),
    # five detectors: 25 sources per accumulator, 400 former work units (two per former thread)
    ((16, 12, 10), 60, 5, 1),
])
def test_sketch_range_shapes(lib, shape):
    (nx, ny, nz), ns, nd, nl = shape
    p = workloads.make_problem(workloads.Grid(nx, ny, nz, 2.0), ns, nd, nl, seed=41, geometry="transmission", margin=0)
    rs, rd = osolve.fields_separable(p)
    rs, rd = rs.astype(np.float32), rd.astype(np.float32)
    N, nc, ncols = p.grid.N, p.n_chrom, 220
    om = workloads.gaussian(43, (nc, ncols, N)).astype(np.float32)
    om_b = bf16_round(om)
    with lib.Context.from_problem(p, precision="mixed", tol=1e-8, tol_cw=0.0) as ctx:
        Y = ctx.sketch_range(torch.tensor(rs, device="cuda"), torch.tensor(rd, device="cuda"), 0, nl,
                             torch.tensor(om, device="cuda").to(torch.bfloat16), ncols).cpu().double().numpy()
    assert np.all(Y[:, ncols:] == 0.0)
    rng = np.random.default_rng(5)
    rows = sorted(set(rng.choice(p.M, size=min(p.M, 48), replace=False).tolist()) | {0, p.M - 1})
    ref = _range_ref_bf16(p, rs, rd, om_b, rows)
    for r in rows:
        err = np.abs(Y[r, :ncols] - ref[r]).max() / np.abs(ref[r]).max()
        assert err <= 2e-3, (r, err)


def test_sketch_project_general_shape_fallback(lib):
    """n_src + n_det > 128: the projection takes the general kernel; same emulated reference."""
    p = workloads.make_problem(workloads.Grid(12, 12, 4, 2.0), 72, 64, 1, seed=44, geometry="transmission", margin=0)
    rs, rd = osolve.fields_separable(p)
    rs, rd = rs.astype(np.float32), rd.astype(np.float32)
    N, nc, ncols, nd = p.grid.N, p.n_chrom, 200, p.n_det
    Q = workloads.gaussian(45, (p.M, ncols)).astype(np.float32)
    with lib.Context.from_problem(p, precision="mixed", tol=1e-8, tol_cw=0.0) as ctx:
        Bt = torch.zeros(nc * N, 224, device="cuda")
        Qp = torch.zeros(p.M, 224, device="cuda")
        Qp[:, :ncols] = torch.tensor(Q, device="cuda")
        ctx.sketch_project(torch.tensor(rs, device="cuda"), torch.tensor(rd, device="cuda"), 0, 1, Qp, ncols, Bt)
        Bt = Bt.cpu().double().numpy()[:, :ncols]
    h3 = p.grid.h ** 3
    ref = np.zeros_like(Bt)
    for s in range(p.n_src):
        A = bf16_round(rs[0, s][None, :] * rd[0])
        rows = [s * nd + d for d in range(nd)]
        for c in range(nc):
            ref[c * N:(c + 1) * N] += -h3 * A.T @ bf16_round((np.float32(p.eps[0, c]) * Q[rows]).astype(np.float32))
    err = np.abs(Bt - ref).max(axis=0) / np.abs(ref).max(axis=0)
    assert err.max() <= 2e-3, err.max()


def test_recursive_compression_against_exact_recursion(lib):
    """Algorithm alg:recursive on the GPU (randomised leaves with the adaptive-rank estimator,
    tensor-core passes, agglomeration by hydot_sketch_merge) against the oracle's recursion with
    exact SVDs on the same source tree: the error of U S V^T stays inside the Section 4.5 bound
    (plus the BF16 floor of the passes), and the ranks kept at the leaves and at the root are close
    to the exact ones."""
    from oracle import sketch as osk
    from paper_1410_0986_gb300 import tree

    p0 = workloads.make_problem(workloads.Grid(16, 16, 12, 2.0), 8, 6, 2, seed=71, geometry="transmission", margin=0)
    p, order, root = tree.order_problem(p0)
    rs, rd = osolve.fields_separable(p)
    J = oborn.born_matrix(p, rs, rd)  # rows (s, d, lambda) with sources in tree order
    nd, nl, N, nc = p.n_det, p.n_lambda, p.grid.N, p.n_chrom
    eps = 1e-2
    blocks = {s: J[[(s * nd + d) * nl + a for d in range(nd) for a in range(nl)]] for s in range(p.n_src)}
    ref_tree = osk.geometric_bisection(np.asarray(p.src_ijk, float)[:, :2] + 0.5, (0.0, 0.0),
                                       (float(p.grid.nx), float(p.grid.ny)))
    assert [i for l in osk.tree_leaves(ref_tree) for i in l] == list(range(p.n_src))  # already in tree order
    Ur, Sr, Vr, ranks_ref = osk.recursive_lowrank(blocks, ref_tree, eps)
    om = workloads.gaussian(72, (nc, 220, N)).astype(np.float32)
    ranks = []
    with lib.Context.from_problem(p, precision="mixed", tol=1e-8, tol_cw=0.0) as ctx:
        ps = torch.tensor(rs, dtype=torch.float32, device="cuda")
        pd = torch.tensor(rd, dtype=torch.float32, device="cuda")
        U, S, V = tree.compress(ctx, root, ps, pd, 0, nl, torch.tensor(om, device="cuda").to(torch.bfloat16), eps,
                                log=lambda kind, node, r: ranks.append((kind, node.lo, node.hi, r)))
        U, V = U.double().cpu().numpy(), V.double().cpu().numpy()
    Jhat = U @ (S[:, None] * V.T)
    L = root.depth()
    fro = np.linalg.norm(J)
    err = np.linalg.norm(J - Jhat)
    assert err <= osk.recursive_error_bound(eps, L, fro) + 1e-2 * fro, (err / fro)
    assert np.linalg.norm(J - Jhat, 2) <= 3 * eps * np.linalg.norm(J, 2) + 1e-2 * np.linalg.norm(J, 2)
    r_root = S.size
    assert abs(r_root - Sr.size) <= max(3, Sr.size // 4), (r_root, Sr.size)
    assert np.abs(S[:5] / Sr[:5] - 1).max() < 2e-2
