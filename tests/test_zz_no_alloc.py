"""hydot_born_apply_noalloc: J x with no device allocation and no context.

Some callers cannot allocate GPU memory themselves, for instance code that runs where
cudaMalloc is not permitted, or that must stay within memory another component owns. This
entry point serves them: its scratch is a fixed device array inside the library. These tests
call it through the C ABI and compare it with the context-based hydot_born_apply and with the
CPU FP64 oracle's J x on the same inputs, twice in a row (the second call must not see the first
call's leftovers).
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads
import paper_1410_0986_gb300._lib as L
from oracle import born as oborn

pytestmark = pytest.mark.gpu


def _noalloc(lib_c, p, lams, ps, pd, x, y):
    eps = np.ascontiguousarray(p.eps[lams], dtype=np.float64)
    rc = lib_c.hydot_born_apply_noalloc(p.grid.N, p.n_src, p.n_det, p.n_chrom, len(lams), p.grid.h,
                                        eps.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(ps.data_ptr()),
                                        C.c_void_p(pd.data_ptr()), C.c_void_p(x.data_ptr()),
                                        C.c_void_p(y.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def test_noalloc_matches_context_entry_point_twice(lib):
    lib_c = L.load()
    # more than 32 sources and detectors: several (s, d) tiles; N not a multiple of the voxel block
    p = workloads.small(seed=12, nx=16, ny=12, nz=11, n_src=34, n_det=33, n_lambda=5, margin=0)
    gen = torch.Generator(device="cuda").manual_seed(11)
    with lib.Context.from_problem(p, precision="mixed", tol=1e-10, tol_cw=0.0) as ctx:
        for lam0, nlam in ((1, 3), (0, 5)):  # two calls in a row with different sizes
            ps = torch.rand(nlam, p.n_src, p.grid.N, device="cuda", generator=gen)
            pd = torch.rand(nlam, p.n_det, p.grid.N, device="cuda", generator=gen)
            x = torch.randn(p.n_chrom * p.grid.N, device="cuda", generator=gen)
            ref = ctx.born_apply(ps, pd, lam0, nlam, x)
            y = torch.full((p.n_src * p.n_det * nlam,), float("nan"), device="cuda")
            rc = _noalloc(lib_c, p, list(range(lam0, lam0 + nlam)), ps, pd, x, y)
            assert rc == L.HYDOT_OK, lib_c.hydot_last_error(None).decode()
            torch.cuda.synchronize()
            assert torch.isfinite(y).all()
            assert (y - ref).abs().max() <= 2e-5 * ref.abs().max()
            # the plain FP64 definition (eqn:measurement) on the same FP32 inputs
            yo = oborn.apply(p, ps.double().cpu().numpy(), pd.double().cpu().numpy(), x.double().cpu().numpy(),
                             list(range(lam0, lam0 + nlam)))
            assert np.abs(y.double().cpu().numpy() - yo).max() <= 2e-5 * np.abs(yo).max()


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    lib_c = L.load()
    p = workloads.small(seed=12, nx=16, ny=12, nz=11, n_src=3, n_det=3, n_lambda=2)
    t = torch.zeros(8, device="cuda")
    eps = np.zeros((10000, 1))
    ep = eps.ctypes.data_as(C.POINTER(C.c_double))
    ptr = C.c_void_p(t.data_ptr())
    # 10,000 wavelengths x 1 chromophore exceeds the 8,192 staged extinction coefficients
    assert lib_c.hydot_born_apply_noalloc(p.grid.N, 3, 3, 1, 10000, 2.0, ep, ptr, ptr, ptr, ptr, None) \
        == L.HYDOT_ERR_ARG
    assert "8192" in lib_c.hydot_last_error(None).decode()
    # partial sums of 64 x 64 optodes over 4,096 wavelength-voxel blocks exceed 16 MiB
    assert lib_c.hydot_born_apply_noalloc(1024 * 1024 * 4, 64, 64, 1, 8, 2.0, ep, ptr, ptr, ptr, ptr, None) \
        == L.HYDOT_ERR_ARG
    assert "16 MiB" in lib_c.hydot_last_error(None).decode()
