"""Shift-invariant initial guesses (Section 3, 3.2; base operator at the mean shift, Section 6.1):
the CUDA guesses against the oracle's Galerkin projections, solves started from them against the
oracle's fields, and the error paths.

The guesses are unique (they depend on the Krylov space, not on its basis), so they are compared
entry by entry; the CUDA bases are FP32, which moves a guess by ~1e-7 of its size times the
conditioning of the projected matrix, within the 2e-5 used here.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import shift as oshift
from oracle import solve as osolve

pytestmark = pytest.mark.gpu

CASES = {
    # nx % 4 == 0 (TMA inner kernels) and a ragged grid (generic kernels)
    "transmission-24x20x14": lambda: workloads.make_problem(workloads.Grid(24, 20, 14, 2.0), 3, 3, 4, seed=91,
                                                            geometry="transmission"),
    "reflection-ragged-17x13x11": lambda: workloads.small(seed=92, nx=17, ny=13, nz=11, n_src=2, n_det=3, n_lambda=3,
                                                          robin_A=(3.0, 3.0, 1.0, 3.0, 0.5, 3.0)),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("m", [8, 30])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_guesses_match_oracle(lib, name, m, precision):
    p = CASES[name]()
    gs_ref, gd_ref = oshift.shift_guess_fields(p, m)
    with lib.Context.from_problem(p, precision=precision, tol=1e-10, tol_cw=0.0) as ctx:
        ctx.set_shift_guess(m)
        gs, gd = ctx.shift_guess_fields(0, p.n_lambda)
    for got, ref in ((gs, gs_ref), (gd, gd_ref)):
        g = got.double().cpu().numpy()
        scale = np.abs(ref).max(axis=-1, keepdims=True)
        assert (np.abs(g - ref) / scale).max() <= 2e-5


def test_solves_from_the_guess_reach_the_oracle_fields_in_fewer_iterations(lib):
    p = workloads.make_problem(workloads.Grid(32, 28, 20, 2.0), 3, 3, 4, seed=93, geometry="transmission")
    rs, rd = osolve.fields_splu(p)
    iters = []
    for m in (0, 40):
        with lib.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=1e-8, cw_floor=100.0) as ctx:
            if m:
                ctx.set_shift_guess(m)
            ps, pd, st = ctx.solve_fields(0, p.n_lambda)
        for got, ref in ((ps, rs), (pd, rd)):
            g = got.double().cpu().numpy()
            assert (np.linalg.norm(g - ref, axis=-1) / np.linalg.norm(ref, axis=-1)).max() <= 1e-6
        assert st["n_not_converged"] == 0
        iters.append(st["iters_mean"])
    assert iters[1] < 0.95 * iters[0]


def test_fp64_solves_from_the_guess(lib):
    p = CASES["reflection-ragged-17x13x11"]()
    rs, rd = osolve.fields_splu(p)
    with lib.Context.from_problem(p, precision="fp64", tol=1e-13, tol_cw=0.0) as ctx:
        ctx.set_shift_guess(20)
        ps, pd, st = ctx.solve_fields(0, p.n_lambda)
        # removing the bases returns to the zero start
        ctx.set_shift_guess(0)
        ps0, pd0, st0 = ctx.solve_fields(0, p.n_lambda)
    for got in (ps, ps0):
        g = got.cpu().numpy()
        assert (np.linalg.norm(g - rs, axis=-1) / np.linalg.norm(rs, axis=-1)).max() <= 1e-10
    assert st["n_not_converged"] == 0 and st0["n_not_converged"] == 0
    assert st["iters_mean"] < st0["iters_mean"]


def test_error_paths(lib):
    p = CASES["reflection-ragged-17x13x11"]()
    with lib.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=0.0) as ctx:
        with pytest.raises(lib.HydotError):
            ctx.shift_guess_fields(0, 1)          # no bases yet
        with pytest.raises(lib.HydotError):
            ctx.set_shift_guess(65)               # basis too large
        ctx.set_shift_guess(4)
        with pytest.raises(lib.HydotError):
            ctx.shift_guess_fields(0, p.n_lambda + 1)
    with lib.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=0.0, deflation_k=4) as ctx:
        with pytest.raises(lib.HydotError):
            ctx.set_shift_guess(8)                # exclusive with the deflation basis
    pf = workloads.small(seed=94, nx=12, ny=10, nz=8, n_src=2, n_det=2, n_lambda=2, freq_mhz=100.0)
    with lib.Context.from_problem(pf, precision="mixed", tol=1e-8, tol_cw=0.0) as ctx:
        with pytest.raises(lib.HydotError):
            ctx.set_shift_guess(8)                # continuous-wave only
