"""Randomized low-rank sketch of J at fixed rank (oracle).

Test infrastructure only (see the package docstring).

Appendix A.1 (alg:randsvd, after Halko, Martinsson & Tropp 2011) at a fixed
target rank r with oversampling p:
  1. Y = A Omega with Omega [n, r+p] i.i.d. N(0, 1);
  2. an orthonormal basis Q of range(Y) (the paper takes the leading left
     singular vectors of Y; here all r+p of them);
  3. B = Q^T A;
  4. SVD of B: B = U_B S V^T, and U = Q U_B;
  5. truncate to rank r (the final recompression of Section 4.4).
The merge across source-detector blocks (Section 4.2, agglomeration) is the
row-block sum B = sum_blocks Q_blk^T A_blk, which this unblocked restatement
computes in one product.

``truncated_svd`` is the optimum the sketch is compared with: the best rank-r
approximation error in the 2-norm is sigma_{r+1} (Section 4.2).
"""
from __future__ import annotations

import numpy as np


def randsvd_fixed(A: np.ndarray, Omega: np.ndarray, rank: int):
    """(U [m, rank], S [rank], V [n, rank]) with A ~ U diag(S) V^T."""
    Y = A @ Omega
    Qy, _, _ = np.linalg.svd(Y, full_matrices=False)
    B = Qy.T @ A
    Ub, S, Vt = np.linalg.svd(B, full_matrices=False)
    U = Qy @ Ub
    return U[:, :rank], S[:rank], Vt[:rank].T


def truncated_svd(A: np.ndarray, rank: int):
    U, S, Vt = np.linalg.svd(A, full_matrices=False)
    return U[:, :rank], S[:rank], Vt[:rank].T, S


def probe_error(A: np.ndarray, U: np.ndarray, S: np.ndarray, V: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Relative error ||A x - U S V^T x|| / ||A x|| for each probe column of X."""
    ax = A @ X
    lx = U @ (S[:, None] * (V.T @ X))
    return np.linalg.norm(ax - lx, axis=0) / np.linalg.norm(ax, axis=0)


# ----------------------------------------------------------------------------- recursive compression
# Section 4 (Algorithm alg:recursive, Algorithm alg:geom, Section 4.3 agglomeration, Section 4.5
# accuracy), restated with exact truncated SVDs at the leaves and at every agglomeration, so that
# the only approximation is the truncation the algorithm prescribes.

def geometric_bisection(points, lower, upper, max_leaf=2):
    """Algorithm alg:geom. points: [n][2] coordinates; the node box is [lower, upper]. A node with
    more than `max_leaf` points is cut across the box's widest side at its centre; points on the cut
    go to the lower side. Returns the tree as nested lists of point indices: a leaf is a list of
    ints, an inner node a list of two subtrees (lower side first)."""
    P = np.asarray(points, dtype=float)

    def build(members, lo, hi, level):
        if len(members) <= max_leaf or level > 64:
            return list(members)
        axis = int(np.argmax(np.asarray(hi) - np.asarray(lo)))
        cut = (lo[axis] + hi[axis]) / 2.0
        low = [m for m in members if P[m, axis] <= cut]
        high = [m for m in members if P[m, axis] > cut]
        lo_hi = list(hi)
        lo_hi[axis] = cut
        hi_lo = list(lo)
        hi_lo[axis] = cut
        parts = []
        if low:
            parts.append(build(low, list(lo), lo_hi, level + 1))
        if high:
            parts.append(build(high, hi_lo, list(hi), level + 1))
        return parts[0] if len(parts) == 1 else parts

    return build(list(range(len(P))), list(lower), list(upper), 0)


def tree_is_leaf(t) -> bool:
    return all(isinstance(v, (int, np.integer)) for v in t)


def tree_leaves(t):
    return [list(t)] if tree_is_leaf(t) else [leaf for sub in t for leaf in tree_leaves(sub)]


def tree_depth(t) -> int:
    return 0 if tree_is_leaf(t) else 1 + max(tree_depth(sub) for sub in t)


def _truncate(U, S, Vt, eps):
    """Keep the singular triplets with sigma > eps * sigma_1 (at least one)."""
    keep = max(1, int(np.sum(S > eps * S[0]))) if S.size and S[0] > 0 else 1
    return U[:, :keep], S[:keep], Vt[:keep].T


def recursive_lowrank(blocks, tree, eps):
    """Algorithm alg:recursive with exact SVDs. blocks: {source index: H_i (rows of that source)};
    tree: the output of geometric_bisection over the sources. Leaves: H_leaf (its sources' blocks
    stacked in leaf order) = truncated SVD at eps. Inner nodes: [U1 S1 V1^T; U2 S2 V2^T] =
    blockdiag(U1, U2) [S1 V1^T; S2 V2^T], the right factor's SVD truncated at eps (Section 4.3).
    Returns (U, S, V, ranks): U's rows are the sources' blocks in tree order; ranks lists
    (depth-first) the rank kept at every node."""
    ranks = []

    def rec(t):
        if tree_is_leaf(t):
            H = np.vstack([blocks[i] for i in t])
            U, S, Vt = np.linalg.svd(H, full_matrices=False)
            out = _truncate(U, S, Vt, eps)
            ranks.append(out[1].size)
            return out
        parts = [rec(sub) for sub in t]
        W = np.vstack([S[:, None] * V.T for (_, S, V) in parts])
        Uw, Sw, Vwt = np.linalg.svd(W, full_matrices=False)
        Uw, Sw, Vw = _truncate(Uw, Sw, Vwt, eps)
        rows = [U.shape[0] for (U, _, _) in parts]
        cols = [U.shape[1] for (U, _, _) in parts]
        Ublk = np.zeros((sum(rows), sum(cols)))
        r0 = c0 = 0
        for (U, _, _), m, k in zip(parts, rows, cols):
            Ublk[r0:r0 + m, c0:c0 + k] = U
            r0 += m
            c0 += k
        ranks.append(Sw.size)
        return Ublk @ Uw, Sw, Vw

    U, S, V = rec(tree)
    return U, S, V, ranks


def recursive_error_bound(eps, depth, frob_norm):
    """Section 4.5: ||H - H_hat||_F <~ 2^(L/2) (L+1) eps ||H||_F (first order in eps)."""
    return 2.0 ** (depth / 2.0) * (depth + 1) * eps * frob_norm
