"""Host logic of the recursive compression (CPU): the source tree the package builds for its sketch
passes is the oracle's geometric bisection (Algorithm alg:geom), leaf by leaf and in the same order,
and the problem reordering keeps every other optode attribute."""
import numpy as np
import pytest

import workloads
from oracle import sketch as osk
from paper_1410_0986_gb300 import tree


@pytest.mark.parametrize("n,seed,leaf", [(7, 1, 2), (37, 2, 2), (64, 3, 2), (2, 4, 2), (50, 5, 1), (50, 6, 5)])
def test_bisection_order_matches_oracle(n, seed, leaf):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 12.0, size=(n, 2))
    order, root = tree.bisection_order(pts, (0.0, 0.0), (12.0, 12.0), leaf_max=leaf)
    ref = osk.geometric_bisection(pts, (0.0, 0.0), (12.0, 12.0), max_leaf=leaf)
    leaves = [order[l.lo:l.hi] for l in root.leaves()]
    assert leaves == osk.tree_leaves(ref)
    assert root.depth() == osk.tree_depth(ref)
    assert sorted(order) == list(range(n))


def test_bisection_ties_duplicates_and_arguments():
    """Positions on the split lines go to the first side, a wider-than-tall box splits in x first,
    coincident positions end in one leaf once the depth limit is reached, and bad arguments are
    rejected with a message."""
    import ctypes as C
    import paper_1410_0986_gb300._lib as L
    grid = np.array([(x, y) for x in (0.0, 3.0, 6.0, 9.0, 12.0) for y in (0.0, 4.0, 8.0)])  # 5 x 3, on cuts
    dup = np.vstack([grid, np.full((5, 2), 6.0)])                                             # five at one point
    for pts, lo, hi in ((grid, (0.0, 0.0), (12.0, 8.0)), (dup, (0.0, 0.0), (12.0, 8.0))):
        order, root = tree.bisection_order(pts, lo, hi)
        ref = osk.geometric_bisection(pts, lo, hi)
        assert [order[l.lo:l.hi] for l in root.leaves()] == osk.tree_leaves(ref)
        assert root.depth() == osk.tree_depth(ref)
    lib = L.load()
    xy = np.zeros((1, 2))
    ip = (C.c_int * 8)()
    n, r = C.c_int(), C.c_int()
    assert lib.hydot_source_tree(xy.ctypes.data_as(C.POINTER(C.c_double)), 0, 0.0, 0.0, 1.0, 1.0, 2, ip, ip,
                                 C.byref(n), C.byref(r)) == L.HYDOT_ERR_ARG
    assert "leaf_max" in lib.hydot_last_error(None).decode()


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
