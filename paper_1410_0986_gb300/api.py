"""Python binding of libhydot: same calls as include/hydot.h, argument marshalling only.

PyTorch provides device memory and the stream; every step of the computation runs in
the library's CUDA kernels. There is no CPU fallback: constructing a Context without
the built library or without a CUDA device raises.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib

PRECISIONS = {"fp64": _lib.HYDOT_FP64, "mixed": _lib.HYDOT_MIXED}


class HydotError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Context:
    """One hydot_ctx: a grid, its spectra and optodes, and the solver workspace.

    Arrays passed to the methods are CUDA tensors laid out as include/hydot.h states;
    their dtype must be float64 ("fp64") or float32 ("mixed"), complex for omega != 0.
    """

    def __init__(self, nx: int, ny: int, nz: int, h: float, robin_A: Sequence[float], eps, c_bg, mus_prime,
                 src_ijk, det_ijk, *, omega: float = 0.0, c_medium: float = 299.792458 / 1.4,
                 precision: str = "mixed", tol: float = 1e-10, tol_cw: float = 1e-8, inner_tol: float = 0.0,
                 max_iter: int = 0, deflation_k: int = 0, max_lambda_per_call: int = 0, cw_floor: float = 0.0):
        if not torch.cuda.is_available():
            raise RuntimeError("libhydot needs a CUDA device; there is no CPU path")
        self.lib = _lib.load()
        self._eps = _f64(eps)
        self._cbg = _f64(c_bg)
        self._musp = _f64(mus_prime)
        self._src = np.ascontiguousarray(np.asarray(src_ijk, dtype=np.int32).reshape(-1, 3))
        self._det = np.ascontiguousarray(np.asarray(det_ijk, dtype=np.int32).reshape(-1, 3))
        p = _lib.Problem()
        p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
        p.h_mm = float(h)
        for f in range(6):
            p.robin_A[f] = float(robin_A[f])
        p.n_lambda, p.n_chrom = self._eps.shape
        p.eps = self._eps.ctypes.data_as(C.POINTER(C.c_double))
        p.c_bg = self._cbg.ctypes.data_as(C.POINTER(C.c_double))
        p.mus_prime = self._musp.ctypes.data_as(C.POINTER(C.c_double))
        p.omega = float(omega)
        p.c_medium = float(c_medium)
        p.n_src, p.n_det = len(self._src), len(self._det)
        p.src_ijk = self._src.ctypes.data_as(C.POINTER(C.c_int))
        p.det_ijk = self._det.ctypes.data_as(C.POINTER(C.c_int))
        p.precision = PRECISIONS[precision]
        p.tol, p.tol_cw, p.inner_tol = float(tol), float(tol_cw), float(inner_tol)
        p.max_iter, p.deflation_k, p.max_lambda_per_call = int(max_iter), int(deflation_k), int(max_lambda_per_call)
        p.cw_floor = float(cw_floor)
        self.problem = p
        self.nx, self.ny, self.nz, self.N = p.nx, p.ny, p.nz, p.nx * p.ny * p.nz
        self.n_lambda, self.n_chrom, self.n_src, self.n_det = p.n_lambda, p.n_chrom, p.n_src, p.n_det
        self.precision = precision
        self.complex = omega != 0.0
        real = torch.float64 if precision == "fp64" else torch.float32
        self.real_dtype = real
        self.dtype = (torch.complex128 if precision == "fp64" else torch.complex64) if self.complex else real
        torch.cuda.init()
        ptr = C.c_void_p()
        rc = self.lib.hydot_setup(C.byref(p), C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(ptr))
        if rc != 0:
            raise HydotError(rc, self.lib.hydot_last_error(None).decode())
        self._ctx = ptr

    @classmethod
    def from_problem(cls, prob, **kw) -> "Context":
        """Build from any object with the attributes of a synthetic problem description
        (grid.nx/ny/nz/h, robin_A, eps, c_bg, mus_prime, src_ijk, det_ijk, omega, c_medium)."""
        g = prob.grid
        return cls(g.nx, g.ny, g.nz, g.h, prob.robin_A, prob.eps, prob.c_bg, prob.mus_prime, prob.src_ijk,
                   prob.det_ijk, omega=prob.omega, c_medium=prob.c_medium, **kw)

    # ------------------------------------------------------------------ helpers
    def _check(self, rc: int, allow_not_converged: bool = False):
        if rc == 0 or (allow_not_converged and rc == _lib.HYDOT_ERR_NOT_CONVERGED):
            return rc
        raise HydotError(rc, self.lib.hydot_last_error(self._ctx).decode())

    def _stream(self):
        self.lib.hydot_set_stream(self._ctx, C.c_void_p(torch.cuda.current_stream().cuda_stream))

    def _ptr(self, t: Optional[torch.Tensor], shape, dtype=None) -> Optional[int]:
        if t is None:
            return None
        dtype = dtype or self.dtype
        if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() != int(np.prod(shape)):
            raise ValueError(f"expected a contiguous CUDA {dtype} tensor with {int(np.prod(shape))} elements, "
                             f"got {t.dtype} {tuple(t.shape)} on {t.device}")
        return t.data_ptr()

    def empty(self, *shape, dtype=None) -> torch.Tensor:
        return torch.empty(shape, dtype=dtype or self.dtype, device="cuda")

    # ------------------------------------------------------------------ calls
    def solve_fields(self, lam0: int, nlam: int, phi_src: Optional[torch.Tensor] = None,
                     phi_det: Optional[torch.Tensor] = None, *, sources: bool = True, detectors: bool = True,
                     raise_not_converged: bool = True):
        """hydot_solve_fields. Allocates the outputs when not given. Returns (phi_src, phi_det, stats)."""
        if phi_src is None and sources and self.n_src:
            phi_src = self.empty(nlam, self.n_src, self.N)
        if phi_det is None and detectors and self.n_det:
            phi_det = self.empty(nlam, self.n_det, self.N)
        st = _lib.Stats()
        self._stream()
        rc = self.lib.hydot_solve_fields(self._ctx, lam0, nlam, self._ptr(phi_src, (nlam, self.n_src, self.N)),
                                         self._ptr(phi_det, (nlam, self.n_det, self.N)), C.byref(st))
        self._check(rc, allow_not_converged=not raise_not_converged)
        return phi_src, phi_det, st.as_dict()

    def solve_adjoint(self, lam0: int, nlam: int, y: torch.Tensor, psi: Optional[torch.Tensor] = None,
                      raise_not_converged: bool = True):
        """hydot_solve_adjoint: psi[a][s] = A^-1 sum_d y[(s*n_det + d)*nlam + a] e_d. Returns (psi, stats)."""
        M = self.n_src * self.n_det * nlam
        if psi is None:
            psi = self.empty(nlam, self.n_src, self.N, dtype=self.real_dtype)
        st = _lib.Stats()
        self._stream()
        rc = self.lib.hydot_solve_adjoint(self._ctx, lam0, nlam, self._ptr(y, (M,), self.real_dtype),
                                          self._ptr(psi, (nlam, self.n_src, self.N), self.real_dtype), C.byref(st))
        self._check(rc, allow_not_converged=not raise_not_converged)
        return psi, st.as_dict()

    def born_apply_T_adjoint(self, phi_src, psi, lam0: int, nlam: int, g: Optional[torch.Tensor] = None):
        """hydot_born_apply_T_adjoint: g += J^T y from the source fields and the adjoint fields of y."""
        if g is None:
            g = torch.zeros(self.n_chrom * self.N, dtype=self.real_dtype, device="cuda")
        self._stream()
        rc = self.lib.hydot_born_apply_T_adjoint(self._ctx,
                                                 self._ptr(phi_src, (nlam, self.n_src, self.N), self.real_dtype),
                                                 self._ptr(psi, (nlam, self.n_src, self.N), self.real_dtype), lam0,
                                                 nlam, self._ptr(g, (self.n_chrom * self.N,), self.real_dtype))
        self._check(rc)
        return g

    def born_assemble(self, phi_src, phi_det, lam0: int, nlam: int, row0: int = 0, nrows: Optional[int] = None,
                      J: Optional[torch.Tensor] = None, ldJ: Optional[int] = None) -> torch.Tensor:
        M = self.n_src * self.n_det * nlam
        nrows = M - row0 if nrows is None else nrows
        cols = self.n_chrom * self.N
        ldJ = cols if ldJ is None else ldJ
        if J is None:
            J = self.empty(nrows, ldJ, dtype=self.real_dtype)
        self._stream()
        rc = self.lib.hydot_born_assemble(self._ctx, self._ptr(phi_src, (nlam, self.n_src, self.N), self.real_dtype),
                                          self._ptr(phi_det, (nlam, self.n_det, self.N), self.real_dtype), lam0, nlam,
                                          row0, nrows, self._ptr(J, (nrows, ldJ), self.real_dtype), ldJ)
        self._check(rc)
        return J

    def born_apply(self, phi_src, phi_det, lam0: int, nlam: int, x: torch.Tensor,
                   y: Optional[torch.Tensor] = None) -> torch.Tensor:
        M = self.n_src * self.n_det * nlam
        if y is None:
            y = self.empty(M, dtype=self.real_dtype)
        self._stream()
        rc = self.lib.hydot_born_apply(self._ctx, self._ptr(phi_src, (nlam, self.n_src, self.N), self.real_dtype),
                                       self._ptr(phi_det, (nlam, self.n_det, self.N), self.real_dtype), lam0, nlam,
                                       self._ptr(x, (self.n_chrom * self.N,), self.real_dtype),
                                       self._ptr(y, (M,), self.real_dtype))
        self._check(rc)
        return y

    def born_apply_T(self, phi_src, phi_det, lam0: int, nlam: int, y: torch.Tensor,
                     g: Optional[torch.Tensor] = None) -> torch.Tensor:
        M = self.n_src * self.n_det * nlam
        if g is None:
            g = torch.zeros(self.n_chrom * self.N, dtype=self.real_dtype, device="cuda")
        self._stream()
        rc = self.lib.hydot_born_apply_T(self._ctx, self._ptr(phi_src, (nlam, self.n_src, self.N), self.real_dtype),
                                         self._ptr(phi_det, (nlam, self.n_det, self.N), self.real_dtype), lam0, nlam,
                                         self._ptr(y, (M,), self.real_dtype),
                                         self._ptr(g, (self.n_chrom * self.N,), self.real_dtype))
        self._check(rc)
        return g

    # ------------------------------------------------------------------ randomised sketch
    def sketch_range(self, phi_src, phi_det, lam0: int, nlam: int, omega_t: torch.Tensor, ncols: int,
                     Y: Optional[torch.Tensor] = None, src0: int = 0, nsrc: Optional[int] = None) -> torch.Tensor:
        """hydot_sketch_range: Y = J Omega over the rows of sources src0 .. src0+nsrc-1 (Y has 224
        columns; omega_t is bfloat16 [n_chrom][ncols][N])."""
        nsrc = self.n_src - src0 if nsrc is None else nsrc
        M = nsrc * self.n_det * nlam
        if Y is None:
            Y = torch.empty(M, 224, dtype=torch.float32, device="cuda")
        if omega_t.dtype != torch.bfloat16 or not omega_t.is_contiguous() or omega_t.numel() != self.n_chrom * ncols * self.N:
            raise ValueError("omega_t must be a contiguous bfloat16 tensor [n_chrom][ncols][N]")
        self._stream()
        rc = self.lib.hydot_sketch_range(self._ctx, self._ptr(phi_src, (nlam, self.n_src, self.N), torch.float32),
                                         self._ptr(phi_det, (nlam, self.n_det, self.N), torch.float32), lam0, nlam,
                                         src0, nsrc, omega_t.data_ptr(), ncols,
                                         self._ptr(Y, (M, Y.shape[1]), torch.float32), Y.shape[1])
        self._check(rc)
        return Y

    def sketch_project(self, phi_src, phi_det, lam0: int, nlam: int, Q: torch.Tensor, ncols: int,
                       Bt: Optional[torch.Tensor] = None, src0: int = 0, nsrc: Optional[int] = None) -> torch.Tensor:
        """hydot_sketch_project: Bt += J^T Q over the slice and the rows of sources src0 .. src0+nsrc-1
        (Bt [n_chrom*N][224], accumulated)."""
        nsrc = self.n_src - src0 if nsrc is None else nsrc
        M = nsrc * self.n_det * nlam
        if Bt is None:
            Bt = torch.zeros(self.n_chrom * self.N, 224, dtype=torch.float32, device="cuda")
        self._stream()
        rc = self.lib.hydot_sketch_project(self._ctx, self._ptr(phi_src, (nlam, self.n_src, self.N), torch.float32),
                                           self._ptr(phi_det, (nlam, self.n_det, self.N), torch.float32), lam0, nlam,
                                           src0, nsrc, self._ptr(Q, (M, Q.shape[1]), torch.float32), ncols, Q.shape[1],
                                           self._ptr(Bt, (self.n_chrom * self.N, Bt.shape[1]), torch.float32),
                                           Bt.shape[1])
        self._check(rc)
        return Bt

    def sketch_orthonormalize(self, Y: torch.Tensor, ncols: int, return_smax: bool = False):
        """hydot_sketch_orthonormalize in place; returns the number of directions kept (and the largest
        singular value of the input when return_smax)."""
        k = C.c_int()
        smax = C.c_double()
        self._stream()
        self._check(self.lib.hydot_sketch_orthonormalize(self._ctx, self._ptr(Y, tuple(Y.shape), torch.float32),
                                                         Y.shape[0], ncols, Y.shape[1], C.byref(k), C.byref(smax)))
        return (k.value, smax.value) if return_smax else k.value

    def sketch_rank(self, Y: torch.Tensor, nq: int, col2: int, k: int, s1: float, tol: float):
        """hydot_sketch_rank with Q = Y[:, :nq] and the test sketch Y2 = Y[:, col2:col2+k] (both in one
        row-major buffer): (smallest adequate rank, its error estimate relative to s1)."""
        if col2 + k > Y.shape[1] or nq > col2:
            raise ValueError("Q and Y2 must be disjoint column ranges of Y")
        r = C.c_int()
        est = C.c_double()
        base = self._ptr(Y, tuple(Y.shape), torch.float32)
        self._stream()
        self._check(self.lib.hydot_sketch_rank(self._ctx, base, Y.shape[1], Y.shape[0], nq, base + 4 * col2,
                                               Y.shape[1], k, float(s1), float(tol), C.byref(r), C.byref(est)))
        return r.value, est.value

    def sketch_merge(self, f1, f2, tol: float, max_rank: int):
        """hydot_sketch_merge of two factorisations (U [m][r], S numpy [r], V [n][r]) of stacked row
        blocks; returns (U [m1+m2][rank], S [rank], V [n][rank])."""
        (U1, S1, V1), (U2, S2, V2) = f1, f2
        r1, r2 = U1.shape[1], U2.shape[1]
        n = V1.shape[0]
        cap = min(max_rank, r1 + r2)
        U = torch.empty(U1.shape[0] + U2.shape[0], cap, dtype=torch.float32, device="cuda")
        V = torch.empty(n, cap, dtype=torch.float32, device="cuda")
        S = np.zeros(r1 + r2)
        s1 = np.ascontiguousarray(S1, dtype=np.float64)
        s2 = np.ascontiguousarray(S2, dtype=np.float64)
        rank = C.c_int()
        dp = C.POINTER(C.c_double)
        self._stream()
        self._check(self.lib.hydot_sketch_merge(
            self._ctx, self._ptr(U1, tuple(U1.shape), torch.float32), r1, U1.shape[0], s1.ctypes.data_as(dp),
            self._ptr(V1, tuple(V1.shape), torch.float32), r1, r1,
            self._ptr(U2, tuple(U2.shape), torch.float32), r2, U2.shape[0], s2.ctypes.data_as(dp),
            self._ptr(V2, tuple(V2.shape), torch.float32), r2, r2, n, float(tol), cap,
            self._ptr(U, tuple(U.shape), torch.float32), cap, S.ctypes.data_as(dp),
            self._ptr(V, tuple(V.shape), torch.float32), cap, C.byref(rank)))
        r = rank.value
        return U[:, :r].contiguous(), S[:r].copy(), V[:, :r].contiguous()

    def sketch_factor(self, Q: torch.Tensor, Bt: torch.Tensor, ncols: int, rank: int):
        """hydot_sketch_factor: (U [rows][rank], S [rank] numpy, V [n_chrom*N][rank])."""
        U = torch.empty(Q.shape[0], rank, dtype=torch.float32, device="cuda")
        V = torch.empty(Bt.shape[0], rank, dtype=torch.float32, device="cuda")
        S = (C.c_double * rank)()
        self._stream()
        self._check(self.lib.hydot_sketch_factor(self._ctx, self._ptr(Q, tuple(Q.shape), torch.float32), Q.shape[0],
                                                 Q.shape[1], self._ptr(Bt, tuple(Bt.shape), torch.float32), Bt.shape[0],
                                                 Bt.shape[1], ncols, rank, U.data_ptr(), rank, S, V.data_ptr(), rank))
        return U, np.array(S[:]), V

    # ------------------------------------------------------------------ instrumentation
    def set_kernel_timing(self, on: bool = True):
        """Record CUDA events around the hot kernels from now on (resets the totals)."""
        self._check(self.lib.hydot_set_kernel_timing(self._ctx, 1 if on else 0))

    def launch_mode(self) -> dict:
        """Launch form of the inner solves: mode -1 while the tuner compares them, 0 launched
        iterations (graph replay), 1 one persistent launch per cycle; measured ns per cell-iteration."""
        m, a, b = C.c_int(0), C.c_double(0), C.c_double(0)
        self._check(self.lib.hydot_get_launch_mode(self._ctx, C.byref(m), C.byref(a), C.byref(b)))
        return {"mode": m.value, "ns_per_cell_launched": a.value, "ns_per_cell_persistent": b.value}

    def set_graphs(self, on: bool = True):
        """Replay groups of inner iterations from a CUDA graph (default) or launch every pass
        directly (each pass then gets its own events under set_kernel_timing)."""
        self._check(self.lib.hydot_set_graphs(self._ctx, 1 if on else 0))

    def kernel_stats(self) -> dict:
        """{kernel: {"ms", "launches", "bytes"}} since set_kernel_timing (synchronises)."""
        out = {}
        for name, kid in _lib.KERNELS.items():
            ms, n, by = C.c_double(), C.c_longlong(), C.c_double()
            self._check(self.lib.hydot_kernel_stats(self._ctx, kid, C.byref(ms), C.byref(n), C.byref(by)))
            out[name] = {"ms": ms.value, "launches": n.value, "bytes": by.value}
        return out

    def kernel_launches(self) -> int:
        return int(self.lib.hydot_kernel_launches(self._ctx))

    def set_absorption(self, dc: Optional[np.ndarray]) -> None:
        """hydot_set_absorption: dc [n_chrom * N] concentration changes (mM, chromophore-major), or
        None to return to the background medium."""
        if dc is None:
            self._check(self.lib.hydot_set_absorption(self._ctx, None))
            return
        a = np.ascontiguousarray(dc, dtype=np.float64).reshape(-1)
        if a.size != self.n_chrom * self.N:
            raise ValueError("dc must have n_chrom * N entries")
        self._stream()
        self._check(self.lib.hydot_set_absorption(self._ctx, a.ctypes.data_as(C.POINTER(C.c_double))))

    def set_shift_guess(self, m: int) -> None:
        """hydot_set_shift_guess: build the per-optode Krylov bases (m vectors each) of the
        mean-shift operator; later solves start from their Galerkin guesses. m = 0 removes them."""
        self._stream()
        self._check(self.lib.hydot_set_shift_guess(self._ctx, int(m)))

    def shift_guess_fields(self, lam0: int, nlam: int):
        """hydot_shift_guess_fields: the initial guesses (field units) of a wavelength slice,
        as (phi_src [nlam][n_src][N], phi_det [nlam][n_det][N])."""
        ps = torch.empty(nlam, self.n_src, self.N, dtype=self.real_dtype, device="cuda")
        pd = torch.empty(nlam, self.n_det, self.N, dtype=self.real_dtype, device="cuda")
        self._stream()
        self._check(self.lib.hydot_shift_guess_fields(self._ctx, int(lam0), int(nlam), C.c_void_p(ps.data_ptr()),
                                                      C.c_void_p(pd.data_ptr())))
        return ps, pd

    # ------------------------------------------------------------------ reconstruction (PaLS)
    @staticmethod
    def _host_f64(a, n=None):
        v = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        if n is not None and v.size != n:
            raise ValueError(f"expected {n} values, got {v.size}")
        return v

    def pals_shape(self, n_basis: int, p, tau=0.5, eps=0.1, nu=0.02) -> torch.Tensor:
        """hydot_pals_shape: mu [N] (FP32, device) of the parameters p [5 n_basis]."""
        pv = self._host_f64(p, 5 * n_basis)
        mu = torch.empty(self.N, dtype=torch.float32, device="cuda")
        self._stream()
        self._check(self.lib.hydot_pals_shape(self._ctx, int(n_basis), pv.ctypes.data_as(C.POINTER(C.c_double)),
                                              float(tau), float(eps), float(nu), C.c_void_p(mu.data_ptr())))
        return mu

    def pals_project(self, V: torch.Tensor, rank: int, n_basis: int, p, tau=0.5, eps=0.1, nu=0.02) -> np.ndarray:
        """hydot_pals_project: A [n_chrom][rank][1 + 5 n_basis] = V_c^T [mu, dmu/dp]."""
        if V.dtype != torch.float32 or not V.is_cuda or V.dim() != 2 or V.shape[0] != self.n_chrom * self.N:
            raise ValueError("V must be a CUDA float32 [n_chrom * N][>= rank] tensor")
        pv = self._host_f64(p, 5 * n_basis)
        A = np.empty((self.n_chrom, rank, 1 + 5 * n_basis))
        self._stream()
        self._check(self.lib.hydot_pals_project(self._ctx, C.c_void_p(V.data_ptr()), V.stride(0), int(rank), int(n_basis),
                                                pv.ctypes.data_as(C.POINTER(C.c_double)), float(tau), float(eps),
                                                float(nu), A.ctypes.data_as(C.POINTER(C.c_double))))
        return A

    def shape_compare(self, mu: torch.Tensor, mu_hat: torch.Tensor, level: float = 0.5):
        """hydot_shape_compare: (relative L2 error, Dice coefficient)."""
        for t in (mu, mu_hat):
            if t.dtype != torch.float32 or not t.is_cuda or t.numel() != self.N or not t.is_contiguous():
                raise ValueError("shapes must be contiguous CUDA float32 [N] tensors")
        l2, dc = C.c_double(), C.c_double()
        self._stream()
        self._check(self.lib.hydot_shape_compare(self._ctx, C.c_void_p(mu.data_ptr()), C.c_void_p(mu_hat.data_ptr()),
                                                 float(level), C.byref(l2), C.byref(dc)))
        return l2.value, dc.value

    def pals_reconstruct(self, U: torch.Tensor, S, V: torch.Tensor, y: torch.Tensor, n_basis: int, p0, c0, *,
                         tau=0.5, eps=0.1, nu=0.02, gamma=1.05, noise_norm=0.0, lm_nu0=1e-2, max_outer=10,
                         max_inner=20, fix_c=False):
        """hydot_pals_reconstruct (Algorithm alg:opt). U [rows][r], V [n_chrom N][r], y [rows]: CUDA float32;
        S [r], p0 [5 n_basis], c0 [n_chrom]: host. Returns (p, c, result dict)."""
        r = len(S)
        for t, rows in ((U, None), (V, self.n_chrom * self.N)):
            if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 2 or t.shape[1] < r or t.stride(1) != 1:
                raise ValueError("U and V must be CUDA float32 matrices with >= rank columns, unit column stride")
            if rows is not None and t.shape[0] != rows:
                raise ValueError("V must have n_chrom * N rows")
        if y.dtype != torch.float32 or not y.is_cuda or y.numel() != U.shape[0] or not y.is_contiguous():
            raise ValueError("y must be a contiguous CUDA float32 vector with one entry per row of U")
        Sv = self._host_f64(S, r)
        pv = self._host_f64(p0, 5 * n_basis).copy()
        cv = self._host_f64(c0, self.n_chrom).copy()
        opt = _lib.PalsOptions(float(tau), float(eps), float(nu), float(gamma), float(noise_norm), float(lm_nu0),
                               int(max_outer), int(max_inner), 1 if fix_c else 0)
        res = _lib.PalsResult()
        self._stream()
        dptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        self._check(self.lib.hydot_pals_reconstruct(self._ctx, C.c_void_p(U.data_ptr()), U.stride(0), U.shape[0],
                                                    dptr(Sv), C.c_void_p(V.data_ptr()), V.stride(0), r,
                                                    C.c_void_p(y.data_ptr()), int(n_basis), dptr(pv), dptr(cv),
                                                    C.byref(opt), C.byref(res)))
        return pv, cv, res.as_dict()

    def wait_selftest(self, polls: int = 1000) -> None:
        """hydot_wait_selftest: a bounded device wait that runs out; raises HydotError
        (HYDOT_ERR_TIMEOUT) as every pipelined kernel's timeout would."""
        self._check(self.lib.hydot_wait_selftest(self._ctx, int(polls)))

    def tuning(self) -> dict:
        """Autotuner state of the inner passes: chosen variant (-1 while tuning) and, per variant,
        slab planes, slab buffers and measured ns per cell-iteration (0 if not timed)."""
        n = _lib.ROLL_VARIANTS
        v = C.c_int(0)
        planes, bufs, ns = (C.c_int * n)(), (C.c_int * n)(), (C.c_double * n)()
        self._check(self.lib.hydot_get_tuning(self._ctx, C.byref(v), planes, bufs, ns))
        return {"variant": v.value, "variants": [{"planes": planes[i], "buffers": bufs[i], "ns_per_cell": ns[i]}
                                                 for i in range(n)]}

    def close(self):
        if getattr(self, "_ctx", None):
            self.lib.hydot_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def solve_batch(contexts: Sequence[Context], lam0, nlam, *, raise_not_converged: bool = True):
    """hydot_solve_batch: the fields of several contexts (one independent problem each, of any size)
    from one call, each context on a CUDA stream of its own so their solves overlap on the GPU.
    lam0 / nlam: one int for every context or one per context. Returns one (phi_src, phi_det, stats)
    per context, in order."""
    n = len(contexts)
    lam0 = [int(lam0)] * n if np.isscalar(lam0) else [int(v) for v in lam0]
    nlam = [int(nlam)] * n if np.isscalar(nlam) else [int(v) for v in nlam]
    if len(lam0) != n or len(nlam) != n:
        raise ValueError("lam0 and nlam need one entry per context")
    if n == 0:
        return []
    lib = contexts[0].lib
    cur = torch.cuda.current_stream()
    outs, srcs, dets = [], (C.c_void_p * n)(), (C.c_void_p * n)()
    for i, ctx in enumerate(contexts):
        ps = ctx.empty(nlam[i], ctx.n_src, ctx.N) if ctx.n_src else None
        pd = ctx.empty(nlam[i], ctx.n_det, ctx.N) if ctx.n_det else None
        outs.append((ps, pd))
        srcs[i], dets[i] = (None if ps is None else ps.data_ptr()), (None if pd is None else pd.data_ptr())
        # a side stream per context, ordered after the work that made the outputs' memory free
        s = getattr(ctx, "_batch_stream", None)
        if s is None:
            s = ctx._batch_stream = torch.cuda.Stream()
        s.wait_stream(cur)
        lib.hydot_set_stream(ctx._ctx, C.c_void_p(s.cuda_stream))
    st, status = (_lib.Stats * n)(), (C.c_int * n)()
    rc = lib.hydot_solve_batch((C.c_void_p * n)(*[c._ctx for c in contexts]), n, (C.c_int * n)(*lam0),
                               (C.c_int * n)(*nlam), srcs, dets, st, status)
    # every worker synchronised its stream before the call returned; later calls go back to torch's stream
    for ctx in contexts:
        ctx._stream()
    if rc != 0 and not (rc == _lib.HYDOT_ERR_NOT_CONVERGED and not raise_not_converged):
        whole = lib.hydot_last_error(None).decode()
        if whole:  # the lists themselves were rejected before any context ran
            raise HydotError(rc, whole)
        bad = next(i for i in range(n) if status[i] == rc)
        raise HydotError(rc, f"context {bad}: {lib.hydot_last_error(contexts[bad]._ctx).decode()}")
    return [(ps, pd, st[i].as_dict()) for i, (ps, pd) in enumerate(outs)]
