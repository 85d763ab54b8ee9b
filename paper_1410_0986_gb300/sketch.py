"""Randomised low-rank factorisation of the Born matrix, streamed over wavelength chunks.

Appendix A.1 (alg:randsvd) at a fixed target rank r with oversampling p, as the two passes the
paper's recursive scheme is built from (Section 4): the range pass Y = J Omega, an orthonormal
basis Q of range(Y), the projection pass B = Q^T J accumulated block by block over the row blocks
(the agglomeration of Section 4.2 as a sum), and the final recompression to rank r (Section 4.4).
Every step runs in libhydot (tensor-core passes, FP64 Gram orthonormalisation); this module only
sequences the calls. Fields are obtained per chunk from `fields(lam0, nlam)`, so they need not all
be resident: the projection pass asks for them again (for example by solving them again).
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

import torch

NCOLS_MAX = 224


def born_sketch(ctx, chunks: Sequence[Tuple[int, int]], omega_t: torch.Tensor, rank: int, oversample: int,
                fields: Callable[[int, int], Tuple[torch.Tensor, torch.Tensor]]):
    """Return (U, S, V, kept): J ~ U diag(S) V^T with U rows in chunk order.

    chunks: wavelength slices (lam0, nlam) covering the rows to factor; the rows of U are the slices'
    rows stacked in that order (inside a slice: (s, d, lambda - lam0), lambda fastest).
    omega_t: bfloat16 [n_chrom][rank + oversample][N] Gaussian test matrix (transposed per chromophore).
    """
    ncols = rank + oversample
    if ncols > NCOLS_MAX:
        raise ValueError(f"rank + oversample must be <= {NCOLS_MAX}")
    rows_of = [ctx.n_src * ctx.n_det * nlam for _, nlam in chunks]
    total = sum(rows_of)
    Y = torch.empty(total, NCOLS_MAX, dtype=torch.float32, device="cuda")
    r0 = 0
    for (lam0, nlam), nr in zip(chunks, rows_of):
        ps, pd = fields(lam0, nlam)
        ctx.sketch_range(ps, pd, lam0, nlam, omega_t, ncols, Y[r0:r0 + nr])
        r0 += nr
    kept = ctx.sketch_orthonormalize(Y, ncols)
    Bt = torch.zeros(ctx.n_chrom * ctx.N, NCOLS_MAX, dtype=torch.float32, device="cuda")
    r0 = 0
    for (lam0, nlam), nr in zip(chunks, rows_of):
        ps, pd = fields(lam0, nlam)
        ctx.sketch_project(ps, pd, lam0, nlam, Y[r0:r0 + nr], ncols, Bt)
        r0 += nr
    U, S, V = ctx.sketch_factor(Y, Bt, ncols, rank)
    return U, S, V, kept


def chunk_rows(ctx, chunks: Sequence[Tuple[int, int]]) -> List[int]:
    """Global row index (s*n_det + d)*n_lambda + lambda of every stacked row of born_sketch's U."""
    out = []
    for lam0, nlam in chunks:
        for s in range(ctx.n_src):
            for d in range(ctx.n_det):
                for a in range(nlam):
                    out.append((s * ctx.n_det + d) * ctx.n_lambda + lam0 + a)
    return out
