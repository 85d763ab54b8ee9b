"""Field solves of several independent problems of uneven size from one call (hydot_solve_batch):
each context's fields are the ones a call of its own gives (bit for bit: the solver's reductions
are in a fixed order and the contexts share no workspace) and match the oracle to the mixed
path's 1e-6 relative 2-norm. Covers the uneven frequency-domain batch (the two smallest of the six
100 MHz phantoms), real fields of ragged sizes, per-context wavelength slices, and the errors.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import solve as osolve

pytestmark = pytest.mark.gpu


def _ctx(lib, p, nlam):
    return lib.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, max_lambda_per_call=nlam)


def _rel(got, ref):
    g = got.cpu().numpy().astype(ref.dtype)
    return (np.linalg.norm(g - ref, axis=-1) / np.linalg.norm(ref, axis=-1)).max()


def test_uneven_real_batch_matches_single_calls_and_oracle(lib):
    probs = [workloads.small(seed=31, nx=13, ny=11, nz=9, n_src=3, n_det=2, n_lambda=3),
             workloads.make_problem(workloads.Grid(36, 19, 21, 2.0), 3, 3, 3, seed=32, geometry="transmission",
                                    margin=1),
             workloads.make_problem(workloads.Grid(24, 24, 16, 2.0), 2, 4, 3, seed=33, geometry="transmission",
                                    margin=1)]
    lam0, nlam = [0, 1, 2], [2, 2, 1]
    ctxs = [_ctx(lib, p, 2) for p in probs]
    try:
        out = lib.solve_batch(ctxs, lam0, nlam)
        for i, (p, c) in enumerate(zip(probs, ctxs)):
            ps, pd, st = out[i]
            assert st["n_fields"] == nlam[i] * (p.n_src + p.n_det) and st["n_not_converged"] == 0
            qs, qd, _ = c.solve_fields(lam0[i], nlam[i])
            assert torch.equal(ps, qs) and torch.equal(pd, qd)
            lams = list(range(lam0[i], lam0[i] + nlam[i]))
            rs, rd = osolve.fields_splu(p, lams)
            assert _rel(ps, rs) <= 1e-6 and _rel(pd, rd) <= 1e-6
    finally:
        for c in ctxs:
            c.close()


def test_frequency_domain_phantoms_batch(lib):
    """The two smallest 100 MHz phantoms (32x32x24 and 48x48x32, 16 + 16 optodes), wavelength 0,
    complex64 COCG with complex128 refinement, solved together: every optode cell and 2,000
    sampled voxels against the oracle's complex128 fields."""
    probs = workloads.config4_batch()[:2]
    ctxs = [_ctx(lib, p, 1) for p in probs]
    try:
        out = lib.solve_batch(ctxs, 0, 1)
        for i, (p, c) in enumerate(zip(probs, ctxs)):
            ps, pd, st = out[i]
            assert ps.dtype == torch.complex64 and st["n_not_converged"] == 0
            qs, qd, _ = c.solve_fields(0, 1)
            assert torch.equal(ps, qs) and torch.equal(pd, qd)
            rs, rd = osolve.fields_separable(p, [0])
            vox = np.unique(np.concatenate([np.random.default_rng(501 + i).choice(p.grid.N, 2000, replace=False),
                                            p.src_voxels(), p.det_voxels()]))
            for got, ref in ((ps, rs), (pd, rd)):
                g = got.cpu().numpy()[:, :, vox].astype(np.complex128)
                rr = ref[:, :, vox]
                assert (np.linalg.norm(g - rr, axis=-1) / np.linalg.norm(rr, axis=-1)).max() <= 1e-6
    finally:
        for c in ctxs:
            c.close()


def test_batch_errors(lib):
    p = workloads.small(seed=34, nx=12, ny=10, nz=8, n_src=2, n_det=2, n_lambda=3)
    a, b = _ctx(lib, p, 1), _ctx(lib, p, 1)
    try:
        assert lib.solve_batch([], 0, 1) == []
        with pytest.raises(lib.HydotError) as e:  # one context twice would share its workspace
            lib.solve_batch([a, a], 0, 1)
        assert e.value.code == -1 and "twice" in str(e.value)
        # the second context's slice exceeds its workspace: it alone fails, with its own message,
        # and the first one's fields are still solved
        with pytest.raises(lib.HydotError) as e:
            lib.solve_batch([a, b], [0, 0], [1, 2])
        assert e.value.code == -1 and "context 1" in str(e.value) and "max_lambda_per_call" in str(e.value)
        with pytest.raises(ValueError):
            lib.solve_batch([a, b], [0], 1)
        (ps, pd, st), = lib.solve_batch([b], 2, 1)  # the contexts stay usable
        rs, rd = osolve.fields_splu(p, [2])
        assert _rel(ps, rs) <= 1e-6 and _rel(pd, rd) <= 1e-6
    finally:
        a.close()
        b.close()


def test_config4_all_six_phantoms_in_one_call(lib):
    """All six 100 MHz phantoms (32x32x24 ... 112x96x64, 16 + 16 optodes) at the last of the 64
    wavelengths from one hydot_solve_batch call, with the benchmark's stopping rule (tol 1e-10,
    tol_cw 1e-8, Born-aware floor 100): sampled fields (sources 0 and 15, detector 7) of every
    phantom against the oracle's complex128 fields to 1e-6, and their Born products phi_s phi_d
    within 1e-5 of the product's maximum."""
    probs = workloads.config4_batch()
    lam = probs[0].n_lambda - 1
    ctxs = [lib.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=100.0,
                                     max_lambda_per_call=1) for p in probs]
    try:
        out = lib.solve_batch(ctxs, lam, 1)
    finally:
        for c in ctxs:
            c.close()
    for p, (ps, pd, st) in zip(probs, out):
        assert st["n_not_converged"] == 0 and ps.dtype == torch.complex64
        src, det = [0, p.n_src - 1], [7]
        rs, rd = osolve.fields_separable(p, [lam], src=src, det=det)
        gs = ps[0, src].cpu().numpy().astype(np.complex128)
        gd = pd[0, det].cpu().numpy().astype(np.complex128)
        for g, r in ((gs, rs[0]), (gd, rd[0])):
            assert (np.linalg.norm(g - r, axis=-1) / np.linalg.norm(r, axis=-1)).max() <= 1e-6, p.name
        for a in range(len(src)):
            Hr, Hg = rs[0, a] * rd[0, 0], gs[a] * gd[0]
            assert np.abs(Hg - Hr).max() <= 1e-5 * np.abs(Hr).max(), p.name


def _perturbed_oracle(p, dc):
    """Fields of the medium with a per-voxel absorption change: sparse LU of A_lambda + h^3 diag(dmu_a)
    (complex when the problem is modulated)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    from oracle import model

    N, nc = p.grid.N, p.n_chrom
    outs = []
    for lam in range(p.n_lambda):
        dmua = sum(p.eps[lam, c] * dc[c * N:(c + 1) * N] for c in range(nc))
        lu = spla.splu((model.operator(p, lam) + sp.diags(p.grid.h ** 3 * dmua)).tocsc())
        cells = list(p.src_voxels()) + list(p.det_voxels())
        B = np.zeros((N, len(cells)), dtype=lu.L.dtype)
        B[cells, np.arange(len(cells))] = 1.0
        outs.append(lu.solve(B).T)
    out = np.stack(outs)
    return out[:, :p.n_src], out[:, p.n_src:]


def test_batch_of_mixed_kinds(lib):
    """One call over contexts that take different paths: FP64 real, mixed real with an absorption
    perturbation (generic kernels), mixed complex with odd nx and a perturbation (generic complex
    kernels, double-float complex residual with the per-voxel term), and mixed real with
    shift-invariant guesses (TMA passes). Each equals its own single call bit for bit and meets the
    oracle (1e-10 FP64, 1e-6 mixed)."""
    pa = workloads.small(seed=61, nx=13, ny=11, nz=9, n_src=2, n_det=2, n_lambda=2)
    pb = workloads.make_problem(workloads.Grid(20, 16, 12, 2.0), 2, 3, 2, seed=62, geometry="transmission", margin=1)
    pc = workloads.small(seed=63, nx=15, ny=12, nz=9, n_src=2, n_det=2, n_lambda=2, freq_mhz=100.0)
    pdd = workloads.make_problem(workloads.Grid(24, 24, 16, 2.0), 3, 3, 2, seed=64, geometry="transmission", margin=1)
    dcb = workloads.ellipsoid_anomaly(pb.grid, seed=65, contrast=0.5)
    dcc = workloads.ellipsoid_anomaly(pc.grid, seed=66, contrast=0.5)
    ctxs = [lib.Context.from_problem(pa, precision="fp64", tol=1e-13, tol_cw=0.0),
            lib.Context.from_problem(pb, precision="mixed", tol=1e-10, tol_cw=1e-8),
            lib.Context.from_problem(pc, precision="mixed", tol=1e-10, tol_cw=1e-8),
            lib.Context.from_problem(pdd, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=100.0)]
    try:
        ctxs[1].set_absorption(dcb)
        ctxs[2].set_absorption(dcc)
        ctxs[3].set_shift_guess(16)
        out = lib.solve_batch(ctxs, 0, 2)
        single = [c.solve_fields(0, 2) for c in ctxs]
    finally:
        for c in ctxs:
            c.close()
    refs = [osolve.fields_splu(pa), _perturbed_oracle(pb, dcb), _perturbed_oracle(pc, dcc), osolve.fields_splu(pdd)]
    for q, ((ps, pd, st), (qs, qd, _), (rs, rd)) in enumerate(zip(out, single, refs)):
        assert st["n_not_converged"] == 0, q
        assert torch.equal(ps, qs) and torch.equal(pd, qd), q
        tol = 1e-10 if q == 0 else 1e-6
        assert _rel(ps, rs) <= tol and _rel(pd, rd) <= tol, q
