"""Write the stored expected values for the full-size parity tests.

Calls only the oracle (sparse-direct FP64 fields) and the seeded input generator.
Output: tests/golden/cw_mixed_64x64x48.npz with, for two sampled wavelengths of the
64x64x48 / 32+32 optodes / 128-wavelength workload:
  lams        sampled wavelength indices
  vox         sampled voxel indices (seeded) followed by every optode voxel
  phis, phid  oracle fields at those voxels  [2][n][len(vox)]
  norms_s/d   2-norms of the full oracle fields [2][n]
  hmax        max_x |phi_s(x) phi_d(x)| for every (s, d)  [2][n_src][n_det]
Run: python tests/golden/make_golden.py   (about ten minutes on an 8-core host)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads  # noqa: E402
from oracle import solve  # noqa: E402

LAMS = (3, 77)


def main():
    p = workloads.config(2)
    rng = np.random.default_rng(20141009)
    vox = np.sort(rng.choice(p.grid.N, size=1024, replace=False))
    vox = np.concatenate([vox, p.src_voxels(), p.det_voxels()])
    phis, phid = solve.fields_splu_parallel(p, LAMS, workers=len(LAMS))
    hmax = np.empty((len(LAMS), p.n_src, p.n_det))
    for a in range(len(LAMS)):
        for s in range(p.n_src):
            hmax[a, s] = np.abs(phis[a, s][None, :] * phid[a]).max(axis=1)
    np.savez_compressed(os.path.join(HERE, "cw_mixed_64x64x48.npz"), lams=np.array(LAMS), vox=vox,
                        phis=phis[:, :, vox], phid=phid[:, :, vox], norms_s=np.linalg.norm(phis, axis=-1),
                        norms_d=np.linalg.norm(phid, axis=-1), hmax=hmax)


if __name__ == "__main__":
    main()
