"""CPU FP64 oracle for the hyperspectral DOT Born hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or run
this package: only the tests, the smoke check and the benchmark's CPU-baseline
leg use it. It is a plain, slow, obviously-correct restatement of what the
method computes, written from Saibaba, Kilmer, Miller & Fantini, "Fast
algorithms for Hyperspectral Diffuse Optical Tomography" (arXiv:1410.0986),
and it shares no code with the CUDA library.

Modules
-------
model   Section 2.1-2.2: background coefficients (mu_a, D), the cell-centred
        finite-volume restatement of the diffusion operator with Robin /
        Dirichlet faces (eqn:diffusion, eqn:robin, eqn:discincident).
solve   Sparse-direct (SuperLU) fields, the definition of record; an
        independent separable fast-diagonalisation solver; dense brute force.
born    Eqn:lippschwin / eqn:measurement: explicit Born matrix J, J x, J^T y,
        and the adjoint-solve form of J^T y.
sketch  Appendix A.1: randomized range finder + SVD at fixed rank, and the
        exact truncated-SVD optimum it is compared with.

Parity status: every function is pinned by a ``-m "not gpu"`` test against
something other than itself (closed forms, conservation, finite differences
of the nonlinear forward model, brute force, a second solver, reciprocity).
"""
