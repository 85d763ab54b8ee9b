"""Write the stored expected values for the full-size parity tests and the benchmark's checks.

Calls only the oracle (sparse-direct FP64 fields, explicit Born products) and the seeded input
generator. Run: python tests/golden/make_golden.py [cfg2] [cfg1]   (config 2: about ten minutes on
an 8-core host; config 1: under a minute).

tests/golden/cw_mixed_64x64x48.npz -- the 64x64x48 / 32+32 optodes / 128-wavelength workload, for
two sampled wavelengths (each a one-wavelength slice of its own):
  lams        sampled wavelength indices
  vox         sampled voxel indices (seeded) followed by every optode voxel
  phis, phid  oracle fields at those voxels  [2][n][len(vox)]
  norms_s/d   2-norms of the full oracle fields [2][n]
  hmax        max_x |phi_s(x) phi_d(x)| for every (s, d)  [2][n_src][n_det]
  jx          y = J x over the whole slice (eqn:measurement), rows s*n_det + d  [2][n_src*n_det]
  jty         g = J^T y at the sampled voxels, every chromophore  [2][n_chrom][len(vox)]
  jty_max     max |g| over all voxels and chromophores  [2]
  with x = 0.05 |gaussian(X_SEED, n_chrom*N)| and y = |gaussian(Y_SEED, n_src*n_det)| (positive,
  as concentrations and measured intensities are, so the sums carry no cancellation).

tests/golden/cw_fp64_24x24x16.npz -- the 24x24x16 / 8+8 optodes / 16-wavelength workload, all
wavelengths as one slice (rows (s*n_det + d)*16 + lambda):
  rows, cols  seeded sample of J's entries  [8192]
  jval        J[rows, cols]
  rowmax      max_x |J[r, x]| for every row  [1024]
  jx          J x (x as above with N = 9,216)  [1024]
  jty         J^T y (y = |gaussian(Y_SEED, 1024)|)  [n_chrom*N]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads  # noqa: E402
from oracle import born, solve  # noqa: E402

LAMS = (3, 77)
X_SEED = 20141010
Y_SEED = 20141011


def born_inputs(p, nlam):
    """The positive probe vectors of the stored products (shared with the tests by this recipe)."""
    x = 0.05 * np.abs(workloads.gaussian(X_SEED, p.n_chrom * p.grid.N))
    y = np.abs(workloads.gaussian(Y_SEED, p.n_src * p.n_det * nlam))
    return x, y


def config2():
    p = workloads.config(2)
    rng = np.random.default_rng(20141009)
    vox = np.sort(rng.choice(p.grid.N, size=1024, replace=False))
    vox = np.concatenate([vox, p.src_voxels(), p.det_voxels()])
    phis, phid = solve.fields_splu_parallel(p, LAMS, workers=len(LAMS))
    hmax = np.empty((len(LAMS), p.n_src, p.n_det))
    for a in range(len(LAMS)):
        for s in range(p.n_src):
            hmax[a, s] = np.abs(phis[a, s][None, :] * phid[a]).max(axis=1)
    x, y = born_inputs(p, 1)
    N = p.grid.N
    jx = np.empty((len(LAMS), p.n_src * p.n_det))
    jty = np.empty((len(LAMS), p.n_chrom, vox.size))
    jty_max = np.empty(len(LAMS))
    for a, lam in enumerate(LAMS):
        jx[a] = born.apply(p, phis[a:a + 1], phid[a:a + 1], x, [lam])
        g = born.apply_T(p, phis[a:a + 1], phid[a:a + 1], y, [lam])
        jty[a] = g.reshape(p.n_chrom, N)[:, vox]
        jty_max[a] = np.abs(g).max()
    np.savez_compressed(os.path.join(HERE, "cw_mixed_64x64x48.npz"), lams=np.array(LAMS), vox=vox,
                        phis=phis[:, :, vox], phid=phid[:, :, vox], norms_s=np.linalg.norm(phis, axis=-1),
                        norms_d=np.linalg.norm(phid, axis=-1), hmax=hmax, jx=jx, jty=jty, jty_max=jty_max)


def config1():
    p = workloads.config(1)
    phis, phid = solve.fields_splu(p)
    J = born.born_matrix(p, phis, phid)
    rng = np.random.default_rng(20141012)
    rows = rng.integers(0, J.shape[0], size=8192)
    cols = rng.integers(0, J.shape[1], size=8192)
    x, y = born_inputs(p, p.n_lambda)
    np.savez_compressed(os.path.join(HERE, "cw_fp64_24x24x16.npz"), rows=rows, cols=cols, jval=J[rows, cols],
                        rowmax=np.abs(J).max(axis=1), jx=born.apply(p, phis, phid, x),
                        jty=born.apply_T(p, phis, phid, y))


if __name__ == "__main__":
    which = sys.argv[1:] or ["cfg2", "cfg1"]
    if "cfg1" in which:
        config1()
    if "cfg2" in which:
        config2()
