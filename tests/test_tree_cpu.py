"""Host logic of the recursive compression (CPU): the source tree the package builds for its sketch
passes is the oracle's geometric bisection (Algorithm alg:geom), leaf by leaf and in the same order,
and the problem reordering keeps every other optode attribute."""
import numpy as np
import pytest

import workloads
from oracle import sketch as osk
from paper_1410_0986_gb300 import tree


@pytest.mark.parametrize("n,seed", [(7, 1), (37, 2), (64, 3), (2, 4)])
def test_bisection_order_matches_oracle(n, seed):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 12.0, size=(n, 2))
    order, root = tree.bisection_order(pts, (0.0, 0.0), (12.0, 12.0))
    ref = osk.geometric_bisection(pts, (0.0, 0.0), (12.0, 12.0))
    leaves = [order[l.lo:l.hi] for l in root.leaves()]
    assert leaves == osk.tree_leaves(ref)
    assert root.depth() == osk.tree_depth(ref)
    assert sorted(order) == list(range(n))


def test_order_problem_permutes_sources_only():
    p = workloads.config(5)
    q, order, root = tree.order_problem(p)
    assert np.array_equal(np.asarray(q.src_ijk), np.asarray(p.src_ijk)[order])
    assert np.array_equal(np.asarray(q.det_ijk), np.asarray(p.det_ijk))
    assert np.array_equal(q.eps, p.eps) and q.grid == p.grid
    assert root.lo == 0 and root.hi == p.n_src
    assert all(1 <= l.hi - l.lo <= 2 for l in root.leaves())
    assert root.depth() >= 5  # at least log2(64 / 2) levels (random positions: deeper in places)


def test_paper_tolerance_inverts_the_bound():
    eps = tree.paper_tolerance(0.1, 5, 10000)
    assert abs(osk.recursive_error_bound(eps, 5, 1.0) * np.sqrt(10000) - 0.1) < 1e-12
