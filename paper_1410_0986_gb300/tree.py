"""Recursive low-rank compression of the Born matrix over a spatial bisection tree of the sources.

Section 4 of the paper: the rows of J split into one block per source (Section 4.1); the sources
are ordered by a geometric bisection tree (Algorithm alg:geom: split the bounding box across its
longest side at the midpoint until a cell holds at most two sources); each leaf block is factored by
the randomised SVD with the adaptive-rank error estimator (Appendix A.1, alg:randsvd), and sibling
factorisations are agglomerated up the tree (Section 4.3, Algorithm alg:recursive). Section 4.5
bounds the error of the result by 2^(L/2) (L+1) eps ||J||_F for leaf and merge tolerance eps and
depth L; `paper_tolerance` inverts that bound.

The sketch passes of libhydot take contiguous source ranges, so a problem's sources are first put
in tree order (`order_problem`); every node of the tree is then a range [lo, hi) of source indices.
This module holds the tree that libhydot's hydot_source_tree computes and sequences library calls
(range pass, orthonormalisation, rank estimate, projection, factorisation, merge); the arithmetic
runs in libhydot.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import _lib

NCOLS_MAX = 224


@dataclasses.dataclass
class Node:
    lo: int                      # first source (in tree order)
    hi: int                      # one past the last source
    children: Tuple["Node", ...] = ()

    @property
    def leaf(self) -> bool:
        return not self.children

    def depth(self) -> int:
        return 0 if self.leaf else 1 + max(c.depth() for c in self.children)

    def leaves(self) -> List["Node"]:
        return [self] if self.leaf else [x for c in self.children for x in c.leaves()]


def bisection_order(xy: np.ndarray, box_lo: Sequence[float], box_hi: Sequence[float], leaf_max: int = 2):
    """Algorithm alg:geom on 2-D source positions xy [n][2] inside the box [box_lo, box_hi], computed
    by hydot_source_tree.

    Returns (order, root): `order` lists the source indices leaf by leaf (depth first, the side
    at or below the split coordinate first), and `root` is the tree whose nodes are ranges of
    positions in `order`."""
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1, 2))
    n = len(xy)
    lib = _lib.load()
    order = (C.c_int * n)()
    nodes = (C.c_int * (8 * n))()
    n_nodes, root = C.c_int(), C.c_int()
    rc = lib.hydot_source_tree(xy.ctypes.data_as(C.POINTER(C.c_double)), n, float(box_lo[0]), float(box_lo[1]),
                               float(box_hi[0]), float(box_hi[1]), int(leaf_max), order, nodes, C.byref(n_nodes),
                               C.byref(root))
    if rc != 0:
        raise RuntimeError(lib.hydot_last_error(None).decode())

    def node(i: int) -> Node:
        lo, hi, c1, c2 = nodes[4 * i:4 * i + 4]
        return Node(lo, hi) if c1 < 0 else Node(lo, hi, (node(c1), node(c2)))

    return list(order), node(root.value)


def order_problem(problem):
    """The problem with its sources in bisection-tree order, the order, and the tree. Positions are
    the source cells' (i, j) on the source plane; the box is the face of the grid."""
    g = problem.grid
    xy = np.asarray(problem.src_ijk, dtype=np.float64)[:, :2] + 0.5
    order, root = bisection_order(xy, (0.0, 0.0), (float(g.nx), float(g.ny)))
    p = dataclasses.replace(problem, src_ijk=np.asarray(problem.src_ijk)[order])
    return p, order, root


def paper_tolerance(eps_d: float, depth: int, n_r: int) -> float:
    """Leaf and merge tolerance eps ~ eps_d / (2^(L/2) (L+1) sqrt(N_r)) for a target relative
    2-norm error eps_d (Section 4.5), N_r = min(M, N)."""
    return eps_d / (2.0 ** (depth / 2.0) * (depth + 1) * math.sqrt(n_r))


def leaf_factor(ctx, ps, pd, lam0: int, nlam: int, src0: int, nsrc: int, omega_t: torch.Tensor, n1: int, k: int,
                tol: float, max_rank: int):
    """alg:randsvd on the row block of sources src0 .. src0+nsrc-1: Y = J Omega with n1 sketch and k
    test columns, Q from the first n1, the smallest rank passing the error estimator (at most
    max_rank), B = Q^T J, and its SVD. Returns (U, S, V, estimate)."""
    rows = nsrc * ctx.n_det * nlam
    Y = ctx.sketch_range(ps, pd, lam0, nlam, omega_t, n1 + k, src0=src0, nsrc=nsrc)
    kept, s1 = ctx.sketch_orthonormalize(Y, n1, return_smax=True)
    r, est = ctx.sketch_rank(Y, kept, n1, k, s1, tol)
    r = max(1, min(r, max_rank, kept))
    Bt = torch.zeros(ctx.n_chrom * ctx.N, NCOLS_MAX, dtype=torch.float32, device="cuda")
    ctx.sketch_project(ps, pd, lam0, nlam, Y, r, Bt, src0=src0, nsrc=nsrc)
    U, S, V = ctx.sketch_factor(Y[:rows], Bt, r, r)
    return U, S, V, est


def compress(ctx, root: Node, ps, pd, lam0: int, nlam: int, omega_t: torch.Tensor, tol: float,
             oversample: int = 20, k_test: int = 10, leaf_rank: int = 190, merge_rank: int = 224,
             log: Optional[Callable[[str, Node, int], None]] = None):
    """Algorithm alg:recursive from `root` (sources in tree order). omega_t: bfloat16
    [n_chrom][n1 + k_test][N] with n1 = leaf_rank + oversample <= 224 - k_test. Returns (U, S, V)
    with U rows in tree order of the sources ((s, d, lambda - lam0) inside), and the per-node ranks
    through `log(kind, node, rank)`."""
    n1 = leaf_rank + oversample
    if n1 + k_test > NCOLS_MAX:
        raise ValueError(f"leaf_rank + oversample + k_test must be <= {NCOLS_MAX}")

    def rec(node: Node):
        if node.leaf:
            U, S, V, est = leaf_factor(ctx, ps, pd, lam0, nlam, node.lo, node.hi - node.lo, omega_t, n1, k_test, tol,
                                       leaf_rank)
            if log:
                log("leaf", node, U.shape[1])
            return U, S, V
        f = rec(node.children[0])
        for c in node.children[1:]:
            f = ctx.sketch_merge(f, rec(c), tol, merge_rank)
        if log:
            log("merge", node, f[0].shape[1])
        return f

    return rec(root)
