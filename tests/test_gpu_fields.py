"""Parity of the CUDA field solves with the CPU FP64 oracle (sparse-direct fields).

Tolerances (stated by the project's target): field relative 2-norm error <= 1e-10 for the
FP64 path and <= 1e-6 for the mixed FP32/FP64-refinement path; Born entries within 1e-5 of
the row maximum, which needs the fields accurate entry by entry far from their source: the
mixed path reaches it by refining until the componentwise backward error is <= tol_cw.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import born as oborn
from oracle import solve as osolve

pytestmark = pytest.mark.gpu


def rel_err(got, ref):
    g = got.detach().cpu().numpy().astype(ref.dtype)
    return (np.linalg.norm(g - ref, axis=-1) / np.linalg.norm(ref, axis=-1)).max()


def born_rowmax_err(p, gs, gd, rs, rd, lams=None):
    """max over rows of max_x |H_gpu - H_ref| / max_x |H_ref| (H = phi_s phi_d, J = -h^3 eps H)."""
    gs = gs.detach().cpu().numpy().astype(rs.dtype)
    gd = gd.detach().cpu().numpy().astype(rd.dtype)
    worst = 0.0
    for a in range(rs.shape[0]):
        for s in range(rs.shape[1]):
            Hr = rs[a, s][None, :] * rd[a]
            Hg = gs[a, s][None, :] * gd[a]
            worst = max(worst, (np.abs(Hg - Hr).max(axis=1) / np.abs(Hr).max(axis=1)).max())
    return worst


@pytest.fixture(scope="module")
def hd(lib):
    return lib


CASES = {
    # name: (problem factory, lams)
    "reflection-13x11x9": (lambda: workloads.small(seed=5, nx=13, ny=11, nz=9, n_src=3, n_det=3, n_lambda=3), None),
    "transmission-ragged-37x19x21": (lambda: workloads.make_problem(workloads.Grid(37, 19, 21, 2.0), 3, 4, 3, seed=9,
                                                                    geometry="transmission", margin=1), None),
    "mixed-faces-17x12x10": (lambda: workloads.small(seed=6, nx=17, ny=12, nz=10, n_src=2, n_det=2, n_lambda=2,
                                                     robin_A=(0.0, 3.0, 1.0, 3.0, 0.5, 3.0)), None),
    # nx % 4 == 0: the FP32 path takes the TMA tile kernels; ragged tiles in x, y and z
    "tma-ragged-36x19x21": (lambda: workloads.make_problem(workloads.Grid(36, 19, 21, 2.0), 3, 3, 3, seed=10,
                                                           geometry="transmission", margin=1), None),
    "tma-faces-40x16x9": (lambda: workloads.small(seed=14, nx=40, ny=16, nz=9, n_src=2, n_det=3, n_lambda=2,
                                                  robin_A=(0.0, 3.0, 1.0, 3.0, 0.5, 2.0)), None),
}


@pytest.fixture(scope="module")
def oracle_fields():
    out = {}
    for name, (mk, lams) in CASES.items():
        p = mk()
        out[name] = (p, osolve.fields_splu(p, lams))
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_fields_fp64(hd, oracle_fields, name):
    p, (rs, rd) = oracle_fields[name]
    with hd.Context.from_problem(p, precision="fp64", tol=1e-13, tol_cw=0.0) as ctx:
        ps, pd, st = ctx.solve_fields(0, p.n_lambda)
    assert rel_err(ps, rs) <= 1e-10 and rel_err(pd, rd) <= 1e-10
    assert st["n_not_converged"] == 0


@pytest.mark.parametrize("name", list(CASES))
def test_fields_mixed_and_born_rows(hd, oracle_fields, name):
    p, (rs, rd) = oracle_fields[name]
    with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8) as ctx:
        ps, pd, st = ctx.solve_fields(0, p.n_lambda)
    assert rel_err(ps, rs) <= 1e-6 and rel_err(pd, rd) <= 1e-6
    assert born_rowmax_err(p, ps, pd, rs, rd) <= 1e-5
    assert st["cycles_max"] >= 2 and st["cw_max"] <= 1e-8


@pytest.mark.parametrize("name", ["transmission-ragged-37x19x21", "tma-ragged-36x19x21", "reflection-13x11x9"])
def test_born_aware_floor(hd, oracle_fields, name):
    """cw_floor = 1e-6 / tol_cw: cells far from every optode stop driving refinement, yet every Born
    entry stays within 1e-5 of its row maximum and the fields within 1e-6 (norm-wise)."""
    p, (rs, rd) = oracle_fields[name]
    cyc = []
    for floor in (0.0, 100.0):
        with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=floor) as ctx:
            ps, pd, st = ctx.solve_fields(0, p.n_lambda)
        assert rel_err(ps, rs) <= 1e-6 and rel_err(pd, rd) <= 1e-6
        assert born_rowmax_err(p, ps, pd, rs, rd) <= 1e-5
        cyc.append(st["cycles_max"])
    assert cyc[1] <= cyc[0]


@pytest.mark.parametrize("name,precision", [("tma-ragged-36x19x21", "mixed"), ("transmission-ragged-37x19x21", "mixed"),
                                            ("reflection-13x11x9", "fp64")])
def test_recycled_deflation(hd, oracle_fields, name, precision):
    """Fields from the deflated start (W from Lanczos on the mean-shift operator, per-wavelength
    Galerkin matrices from shift-independent k x k blocks) meet the same tolerances."""
    p, (rs, rd) = oracle_fields[name]
    kw = dict(tol=1e-13, tol_cw=0.0) if precision == "fp64" else dict(tol=1e-10, tol_cw=1e-8, cw_floor=100.0)
    with hd.Context.from_problem(p, precision=precision, deflation_k=8, **kw) as ctx:
        ps, pd, st = ctx.solve_fields(0, p.n_lambda)
    tol = 1e-10 if precision == "fp64" else 1e-6
    assert rel_err(ps, rs) <= tol and rel_err(pd, rd) <= tol
    assert born_rowmax_err(p, ps, pd, rs, rd) <= 1e-5
    assert st["n_not_converged"] == 0


def test_tma_and_generic_kernels_agree(hd, oracle_fields, monkeypatch):
    """The TMA tile kernels and the generic kernels solve the same systems to the same tolerance."""
    p, (rs, rd) = oracle_fields["tma-ragged-36x19x21"]
    out = []
    for flag in ("0", "1"):
        monkeypatch.setenv("HYDOT_NO_TMA", flag)
        with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8) as ctx:
            ps, pd, st = ctx.solve_fields(0, p.n_lambda)
        out.append((ps, pd))
        assert rel_err(ps, rs) <= 1e-6 and born_rowmax_err(p, ps, pd, rs, rd) <= 1e-5
    a, b = out
    assert (a[0] - b[0]).abs().max() <= 1e-6 * a[0].abs().max()


def test_config1_fp64_fields_and_born_matrix(hd):
    """The FP64 workload in full: 24x24x16, 8+8 optodes on the top face, 16 wavelengths."""
    p = workloads.config(1)
    rs, rd = osolve.fields_splu(p)
    with hd.Context.from_problem(p, precision="fp64", tol=1e-13, tol_cw=0.0) as ctx:
        ps, pd, st = ctx.solve_fields(0, p.n_lambda)
        assert rel_err(ps, rs) <= 1e-10 and rel_err(pd, rd) <= 1e-10
        J = ctx.born_assemble(ps, pd, 0, p.n_lambda)
        assert tuple(J.shape) == (1024, 36864)
        Jr = oborn.born_matrix(p, rs, rd)
        Jg = J.cpu().numpy()
        err = (np.abs(Jg - Jr).max(axis=1) / np.abs(Jr).max(axis=1)).max()
        assert err <= 1e-5


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_frequency_domain_cocg(hd, precision, tol):
    p = workloads.small(seed=8, nx=14, ny=12, nz=10, n_src=2, n_det=3, n_lambda=2, freq_mhz=100.0)
    rs, rd = osolve.fields_splu(p)
    with hd.Context.from_problem(p, precision=precision, tol=1e-13 if precision == "fp64" else 1e-10,
                                 tol_cw=0.0 if precision == "fp64" else 1e-8) as ctx:
        ps, pd, st = ctx.solve_fields(0, p.n_lambda)
    assert ps.dtype == (torch.complex128 if precision == "fp64" else torch.complex64)
    assert rel_err(ps, rs) <= tol and rel_err(pd, rd) <= tol


@pytest.mark.parametrize("grid,faces", [((38, 19, 21), (3.0,) * 6), ((34, 12, 10), (0.0, 3.0, 1.0, 3.0, 0.5, 2.0)),
                                         ((15, 12, 9), (3.0,) * 6)])
def test_frequency_domain_tma_and_generic_kernels_agree(hd, monkeypatch, grid, faces):
    """Complex64 COCG through the TMA rolling passes (nx even: 8-byte rows stay 16-byte aligned;
    ragged tiles in x, y and z, Dirichlet and Robin faces) and through the generic kernels (odd nx,
    or the TMA path switched off): both meet the oracle's complex128 fields to 1e-6."""
    nx, ny, nz = grid
    p = workloads.small(seed=41 + nx, nx=nx, ny=ny, nz=nz, n_src=2, n_det=3, n_lambda=2, freq_mhz=100.0,
                        robin_A=faces)
    rs, rd = osolve.fields_splu(p)
    out = []
    for flag in ("0", "1"):
        monkeypatch.setenv("HYDOT_NO_TMA", flag)
        with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8) as ctx:
            ps, pd, st = ctx.solve_fields(0, p.n_lambda)
        assert ps.dtype == torch.complex64 and st["n_not_converged"] == 0
        assert rel_err(ps, rs) <= 1e-6 and rel_err(pd, rd) <= 1e-6
        out.append((ps, pd))
    a, b = out
    assert (a[0] - b[0]).abs().max() <= 1e-6 * a[0].abs().max()


def test_frequency_domain_born_aware_floor(hd):
    """The Born-aware floor on complex fields (|A^-1| <= (Re A)^-1 entrywise for the constant
    imaginary shift): fields to 1e-6 and every Born product phi_s phi_d within 1e-5 of its row
    maximum against the oracle, in no more refinement cycles than the plain componentwise test."""
    p = workloads.make_problem(workloads.Grid(48, 40, 36, 2.0), 4, 4, 2, seed=24, geometry="transmission",
                               freq_mhz=100.0)
    rs, rd = osolve.fields_separable(p)
    cyc = {}
    for floor in (0.0, 100.0):
        with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=floor) as ctx:
            ps, pd, st = ctx.solve_fields(0, p.n_lambda)
        assert st["n_not_converged"] == 0
        assert rel_err(ps, rs) <= 1e-6 and rel_err(pd, rd) <= 1e-6
        assert born_rowmax_err(p, ps, pd, rs, rd) <= 1e-5
        cyc[floor] = st["cycles_max"]
    assert cyc[100.0] <= cyc[0.0]


def test_frequency_domain_roll_variants_and_graphs_bitwise(hd, monkeypatch):
    """The four complex slab shapes give the same bits, with and without CUDA-graph replay, and the
    autotuner reports the complex set."""
    p = workloads.make_problem(workloads.Grid(48, 40, 36, 2.0), 4, 4, 2, seed=22, geometry="transmission",
                               freq_mhz=100.0)
    out = []
    for v in range(4):
        monkeypatch.setenv("HYDOT_ROLL_VARIANT", str(v))
        for graphs in ("0", "1"):
            monkeypatch.setenv("HYDOT_NO_GRAPHS", graphs)
            with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8) as ctx:
                ps, pd, st = ctx.solve_fields(0, p.n_lambda)
                assert ctx.tuning()["variant"] == v and st["n_not_converged"] == 0
                tu = ctx.tuning()
            out.append((ps, pd))
    for ps, pd in out[1:]:
        assert torch.equal(ps, out[0][0]) and torch.equal(pd, out[0][1])
    # variant 3: the 2 x 4 slabs of variant 0 with four blocks per SM for pass 1; variant 2: pass 1
    # on 64 x 8 tiles of paired complex cells
    assert [(v["planes"], v["buffers"]) for v in tu["variants"]] == [(2, 4), (2, 6), (2, 3), (2, 4)]


def test_frequency_domain_variants_on_z_segments_bitwise(hd, monkeypatch):
    """Complex fields on blocks that own z-segments of 8 planes (a ragged last segment over nz = 21)
    and on a grid whose 64-wide paired-cell tiles are ragged (nx = 52): the four complex variants,
    the paired-cell one included, give the same bits, and every field converges."""
    monkeypatch.setenv("HYDOT_DIR_SEG", "8")
    p = workloads.make_problem(workloads.Grid(52, 19, 21, 2.0), 3, 2, 2, seed=26, geometry="transmission",
                               freq_mhz=100.0)
    out = []
    for v in range(4):
        monkeypatch.setenv("HYDOT_ROLL_VARIANT", str(v))
        with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8) as ctx:
            ps, pd, st = ctx.solve_fields(0, p.n_lambda)
            assert ctx.tuning()["variant"] == v and st["n_not_converged"] == 0
        out.append((ps, pd))
    for ps, pd in out[1:]:
        assert torch.equal(ps, out[0][0]) and torch.equal(pd, out[0][1])


def test_wavelength_slice_and_single_sets(hd, oracle_fields):
    p, (rs, rd) = oracle_fields["reflection-13x11x9"]
    with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, max_lambda_per_call=2) as ctx:
        ps, _, _ = ctx.solve_fields(1, 2, detectors=False)
        _, pd, _ = ctx.solve_fields(2, 1, sources=False)
        with pytest.raises(Exception):
            ctx.solve_fields(0, 3)  # larger than max_lambda_per_call
    assert rel_err(ps, rs[1:3]) <= 1e-6 and rel_err(pd, rd[2:3]) <= 1e-6


def test_degenerate_single_plane_grid(hd):
    """nz = 1: every cell has both z faces on the boundary; dense brute-force oracle."""
    p = workloads.small(seed=3, nx=9, ny=7, nz=1, n_src=2, n_det=2, n_lambda=2)
    rs, rd = osolve.fields_dense(p)
    with hd.Context.from_problem(p, precision="fp64", tol=1e-13, tol_cw=0.0) as ctx:
        ps, pd, _ = ctx.solve_fields(0, 2)
    assert rel_err(ps, rs) <= 1e-10 and rel_err(pd, rd) <= 1e-10


@pytest.mark.parametrize("freq", [0.0, 100.0])
@pytest.mark.parametrize("nz", [1, 2])
def test_thin_grids_mixed_precision(hd, nz, freq):
    """nz = 1 and 2 on the mixed path (continuous-wave and frequency domain): the double-float
    residual compiles its per-cell body per kind of plane, and on these grids every plane is a
    z-face plane (both faces at nz = 1, the lower and then the upper face at nz = 2); an odd nx
    keeps the launched generic passes. Dense brute-force oracle."""
    p = workloads.small(seed=30 + nz, nx=9, ny=7, nz=nz, n_src=2, n_det=2, n_lambda=2, freq_mhz=freq)
    rs, rd = osolve.fields_dense(p)
    with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8) as ctx:
        ps, pd, st = ctx.solve_fields(0, 2)
    assert st["n_not_converged"] == 0 and st["cw_max"] <= 1e-8
    assert rel_err(ps, rs) <= 1e-6 and rel_err(pd, rd) <= 1e-6


def test_single_cell_grid(hd):
    """1x1x1: the field is 1 / (mu_a h^3 + six face terms)."""
    p = workloads.make_problem(workloads.Grid(1, 1, 1, 2.0), 1, 0, 2, seed=4, geometry="reflection", margin=0)
    rs, _ = osolve.fields_dense(p)
    with hd.Context.from_problem(p, precision="fp64", tol=1e-13, tol_cw=0.0) as ctx:
        ps, pd, _ = ctx.solve_fields(0, 2)
    assert pd is None
    assert rel_err(ps, rs) <= 1e-13


def test_not_converged_status_and_best_iterate(hd):
    p = workloads.small(seed=5, nx=13, ny=11, nz=9, n_src=2, n_det=2, n_lambda=2)
    with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, max_iter=3) as ctx:
        with pytest.raises(hd.HydotError) as ei:
            ctx.solve_fields(0, 2)
        assert ei.value.code == -4
        ps, pd, st = ctx.solve_fields(0, 2, raise_not_converged=False)
    assert st["n_not_converged"] == st["n_fields"] == 8
    assert st["iters_max"] <= 3
    assert torch.isfinite(ps).all() and torch.isfinite(pd).all()


def test_bitwise_repeatable(hd):
    """Reductions use fixed-order per-tile partials: two runs give identical bits."""
    p = workloads.small(seed=5, nx=33, ny=17, nz=20, n_src=3, n_det=3, n_lambda=2)
    with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8) as ctx:
        a, b, _ = ctx.solve_fields(0, 2)
        c, d, _ = ctx.solve_fields(0, 2)
    assert torch.equal(a, c) and torch.equal(b, d)


@pytest.mark.parametrize("sweep", ["0", "1"])
def test_roll_variants_bitwise_identical_and_autotuner_settles(hd, oracle_fields, monkeypatch, sweep):
    """The slab shapes the autotuner chooses from give the same bits (two-pass and single-sweep
    forms); an untuned context times the variants on groups of inner iterations and then keeps one."""
    monkeypatch.setenv("HYDOT_SINGLE_SWEEP", sweep)
    monkeypatch.setenv("HYDOT_PERSISTENT", "0")
    p = workloads.make_problem(workloads.Grid(64, 40, 36, 2.0), 4, 4, 4, seed=21, geometry="transmission")
    out = []
    for v in range(4):
        monkeypatch.setenv("HYDOT_ROLL_VARIANT", str(v))
        with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=100.0) as ctx:
            ps, pd, st = ctx.solve_fields(0, p.n_lambda)
            assert ctx.tuning()["variant"] == v
        out.append((ps, pd))
    for ps, pd in out[1:]:
        assert torch.equal(ps, out[0][0]) and torch.equal(pd, out[0][1])
    monkeypatch.delenv("HYDOT_ROLL_VARIANT")
    with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=100.0) as ctx:
        assert ctx.tuning()["variant"] == -1
        for _ in range(3):
            ps, pd, st = ctx.solve_fields(0, p.n_lambda)
            assert torch.equal(ps, out[0][0]) and torch.equal(pd, out[0][1])
        tu = ctx.tuning()
    assert tu["variant"] in range(4)
    assert all(v["ns_per_cell"] > 0 for v in tu["variants"])
    # slab shapes {planes, buffers} of the two-pass and the single-sweep forms
    # (single-sweep variants 2 and 3 use 32 x 16 tiles, two cells per thread: the same bits)
    # (two-pass variants 1-3 run pass 1 on 64 x 8 pairs, 32 x 16 and 64 x 16 pairs)
    expect = [(4, 3), (3, 4), (3, 3), (4, 3)] if sweep == "1" else [(4, 4), (2, 6), (2, 6), (2, 4)]
    assert [(v["planes"], v["buffers"]) for v in tu["variants"]] == expect


@pytest.mark.parametrize("seg", [None, "8"])
def test_paired_cell_pass1_bitwise_on_ragged_tiles(hd, monkeypatch, seg):
    """Pass 1 on 64-wide tiles of x-adjacent cell pairs (two-pass variants 1 and 3) gives the bits of
    the 32-wide tiles (variants 0 and 2) where the 64-wide tiles are ragged: nx = 100 leaves a last
    tile with one full and one partial 32-cell half, ny = 19 a last 8-row group with three rows,
    nz = 21 a ragged last z-segment of 8 planes."""
    monkeypatch.setenv("HYDOT_SINGLE_SWEEP", "0")
    monkeypatch.setenv("HYDOT_PERSISTENT", "0")
    if seg:
        monkeypatch.setenv("HYDOT_DIR_SEG", seg)
    p = workloads.make_problem(workloads.Grid(100, 19, 21, 2.0), 3, 3, 3, seed=24, geometry="transmission")
    out = []
    for v in range(4):
        monkeypatch.setenv("HYDOT_ROLL_VARIANT", str(v))
        with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=100.0) as ctx:
            ps, pd, st = ctx.solve_fields(0, p.n_lambda)
            assert ctx.tuning()["variant"] == v and st["n_not_converged"] == 0
        out.append((ps, pd))
    for ps, pd in out[1:]:
        assert torch.equal(ps, out[0][0]) and torch.equal(pd, out[0][1])


@pytest.mark.parametrize("name", ["tma-ragged-36x19x21", "tma-faces-40x16x9"])
def test_single_sweep_and_two_pass_iterations_agree(hd, oracle_fields, monkeypatch, name):
    """The single-sweep inner iteration (Chronopoulos-Gear recurrences, s = A p recomputed on a
    two-cell ring) and the two-pass one are the same CG in exact arithmetic: both reach the oracle's
    fields and Born rows to the stated tolerances, with Krylov iteration counts within a few per cent."""
    p, (rs, rd) = oracle_fields[name]
    stats = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("HYDOT_SINGLE_SWEEP", flag)
        with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=100.0) as ctx:
            ps, pd, st = ctx.solve_fields(0, p.n_lambda)
        assert st["n_not_converged"] == 0
        assert rel_err(ps, rs) <= 1e-6 and rel_err(pd, rd) <= 1e-6
        assert born_rowmax_err(p, ps, pd, rs, rd) <= 1e-5
        stats[flag] = st
    assert abs(stats["0"]["iters_mean"] - stats["1"]["iters_mean"]) <= 0.05 * stats["1"]["iters_mean"] + 2


@pytest.mark.parametrize("sweep", ["0", "1"])
@pytest.mark.parametrize("seg", ["8", "16"])
def test_z_segmented_blocks(hd, oracle_fields, monkeypatch, seg, sweep):
    """Blocks that own a z-segment of a column instead of the whole column (segments of 8 or 16
    planes over nz = 21: a ragged last segment; each segment reads two planes beyond both its ends)
    reach the oracle's fields and Born rows to the same tolerances."""
    p, (rs, rd) = oracle_fields["tma-ragged-36x19x21"]
    monkeypatch.setenv("HYDOT_DIR_SEG", seg)
    monkeypatch.setenv("HYDOT_SINGLE_SWEEP", sweep)
    with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=100.0) as ctx:
        ps, pd, st = ctx.solve_fields(0, p.n_lambda)
    assert st["n_not_converged"] == 0
    assert rel_err(ps, rs) <= 1e-6 and rel_err(pd, rd) <= 1e-6
    assert born_rowmax_err(p, ps, pd, rs, rd) <= 1e-5


def test_graph_replay_matches_direct_launches(hd, monkeypatch):
    """Groups of inner iterations replayed from a CUDA graph give the bits of direct launches."""
    p = workloads.make_problem(workloads.Grid(24, 24, 16, 2.0), 8, 8, 4, seed=23, geometry="reflection")
    monkeypatch.setenv("HYDOT_ROLL_VARIANT", "0")
    res = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("HYDOT_NO_GRAPHS", flag)
        with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=100.0) as ctx:
            a = ctx.solve_fields(0, p.n_lambda)
            b_ = ctx.solve_fields(0, p.n_lambda)  # second call replays the cached graph
            c = ctx.solve_fields(1, 2)            # another batch: the graph is updated
        res[flag] = (a, b_, c)
    for q in range(3):
        assert torch.equal(res["0"][q][0], res["1"][q][0]) and torch.equal(res["0"][q][1], res["1"][q][1])
    assert torch.equal(res["0"][0][0], res["0"][1][0])


def test_bounded_wait_timeout_keeps_context_usable(hd):
    """Device waits that run out (an mbarrier nothing arrives at, through the kernels' bounded poll
    loop; the persistent solve's grid barrier with one of two co-resident blocks never arriving)
    come back as HYDOT_ERR_TIMEOUT; the context then solves as before."""
    p = workloads.small(seed=5, nx=16, ny=11, nz=9, n_src=2, n_det=2, n_lambda=2)
    with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8) as ctx:
        a, b, _ = ctx.solve_fields(0, 2)
        with pytest.raises(hd.HydotError) as ei:
            ctx.wait_selftest(2000)
        assert ei.value.code == -5
        c, d, st = ctx.solve_fields(0, 2)
        assert st["n_not_converged"] == 0
    assert torch.equal(a, c) and torch.equal(b, d)


@pytest.mark.parametrize("seg", [None, "8"])
@pytest.mark.parametrize("name", ["tma-ragged-36x19x21", "tma-faces-40x16x9"])
def test_persistent_inner_solve_matches_launched_sweeps(hd, oracle_fields, monkeypatch, name, seg):
    """The persistent form (one cooperative launch per refinement cycle: co-resident blocks iterate
    single sweeps over (field, column, z-segment) items with a grid barrier per iteration and stop
    on the device) does the same arithmetic as launched single sweeps with the same slabs: the same
    bits, and the oracle's fields and Born rows to the stated tolerances."""
    p, (rs, rd) = oracle_fields[name]
    monkeypatch.setenv("HYDOT_SINGLE_SWEEP", "1")
    monkeypatch.setenv("HYDOT_ROLL_VARIANT", "1")  # the persistent kernel's {3 planes, 4 buffers}
    if seg:
        monkeypatch.setenv("HYDOT_DIR_SEG", seg)
    out = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("HYDOT_PERSISTENT", flag)
        with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=100.0) as ctx:
            ps, pd, st = ctx.solve_fields(0, p.n_lambda)
            assert ctx.launch_mode()["mode"] == int(flag)
        assert st["n_not_converged"] == 0
        out[flag] = (ps, pd, st)
    assert torch.equal(out["0"][0], out["1"][0]) and torch.equal(out["0"][1], out["1"][1])
    assert out["0"][2]["iters_mean"] == out["1"][2]["iters_mean"]
    ps, pd, _ = out["1"]
    assert rel_err(ps, rs) <= 1e-6 and rel_err(pd, rd) <= 1e-6
    assert born_rowmax_err(p, ps, pd, rs, rd) <= 1e-5


def test_persistent_inner_solve_on_the_small_reflection_batch(hd):
    """The 24x24x16 reflection workload (8 + 8 optodes on the top face, 16 wavelengths: 256 fields,
    L2-resident) in the mixed form through one persistent launch per cycle, against the oracle's
    sparse-direct fields; then an untuned single-sweep context compares the two launch forms on
    whole cycles (same bits in both) and keeps one."""
    p = workloads.config(1)
    rs, rd = osolve.fields_splu(p)
    import os
    os.environ["HYDOT_PERSISTENT"] = "1"
    try:
        with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=100.0) as ctx:
            ps, pd, st = ctx.solve_fields(0, p.n_lambda)
            assert ctx.launch_mode()["mode"] == 1
    finally:
        os.environ.pop("HYDOT_PERSISTENT", None)
    assert st["n_not_converged"] == 0
    assert rel_err(ps, rs) <= 1e-6 and rel_err(pd, rd) <= 1e-6
    assert born_rowmax_err(p, ps, pd, rs, rd) <= 1e-5
    os.environ["HYDOT_SINGLE_SWEEP"] = "1"  # the launch-form tuner runs for single-sweep contexts
    try:
        with hd.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=100.0) as ctx:
            assert ctx.launch_mode()["mode"] == -1
            first, _, _ = ctx.solve_fields(0, p.n_lambda)
            for _ in range(5):
                qs, qd, st2 = ctx.solve_fields(0, p.n_lambda)
                assert st2["n_not_converged"] == 0
                assert torch.equal(qs, first)  # launched and persistent cycles give the same bits
            lm = ctx.launch_mode()
    finally:
        os.environ.pop("HYDOT_SINGLE_SWEEP", None)
    assert lm["mode"] in (0, 1) and lm["ns_per_cell_launched"] > 0 and lm["ns_per_cell_persistent"] > 0
    assert rel_err(qs, rs) <= 1e-6 and rel_err(qd, rd) <= 1e-6
