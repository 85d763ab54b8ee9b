"""The host-side symmetric eigensolver of libhydot (csrc/dense.h: Householder tridiagonalisation
and implicit-shift QR), compiled here with the host compiler and checked against numpy's eigh on
symmetric matrices of the sizes the sketch uses (Gram matrices up to 448 x 448), including
repeated and clustered eigenvalues and a rank-deficient case."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROG = r"""
#include <cstdio>
#include <vector>
#include "dense.h"
int main() {
  int n;
  while (std::scanf("%d", &n) == 1) {
    std::vector<double> A((size_t)n * n);
    for (auto& v : A) std::scanf("%lf", &v);
    std::vector<double> lam, V;
    if (!hydot::sym_eig(A, n, lam, V)) return 3;
    for (int i = 0; i < n; ++i) std::printf("%.17g\n", lam[i]);
    for (auto v : V) std::printf("%.17g\n", v);
  }
}
"""


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    d = tmp_path_factory.mktemp("eig")
    src, out = d / "eig.cpp", d / "eig"
    src.write_text(PROG)
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1410_0986_gb300", "csrc"), str(src),
                    "-o", str(out)], check=True)
    return str(out)


def _cases():
    rng = np.random.default_rng(5)
    out = []
    for n in (1, 2, 5, 64, 224, 448):
        X = rng.standard_normal((n, n))
        out.append(X @ X.T)
    Q, _ = np.linalg.qr(rng.standard_normal((50, 50)))
    lam = np.concatenate([np.full(10, 3.0), np.full(10, 3.0 + 1e-9), np.linspace(-1, 1, 30)])
    out.append((Q * lam) @ Q.T)                      # repeated and clustered eigenvalues
    X = rng.standard_normal((80, 20))
    out.append(X @ X.T)                               # rank 20 of 80
    out.append(np.diag(np.arange(6.0)))               # already diagonal
    return out


def test_sym_eig_matches_numpy(exe):
    cases = _cases()
    text = "".join(f"{A.shape[0]} " + " ".join(repr(float(v)) for v in A.ravel()) + "\n" for A in cases)
    vals = np.array(subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split(),
                    dtype=float)
    pos = 0
    for A in cases:
        n = A.shape[0]
        lam = vals[pos:pos + n]
        V = vals[pos + n:pos + n + n * n].reshape(n, n)
        pos += n + n * n
        scale = max(np.abs(A).max(), 1e-300)
        assert np.abs(np.sort(lam) - np.linalg.eigvalsh(A)).max() <= 1e-12 * scale * max(1, n / 32)
        assert np.abs(A @ V - V * lam).max() <= 1e-12 * scale * max(1, n / 32)
        assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12 * max(1, n / 32)


CAP_PROG = r"""
#include <cstdio>
#include <vector>
#include "dense.h"
int main() {
  // a symmetric 40 x 40 matrix with distinct eigenvalues: the QR iteration needs about 2 n bulge
  // chases; with a cap of 3 it must report that it did not converge, with the default it converges
  const int n = 40;
  std::vector<double> A((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = 1.0 / (1.0 + i + j) + (i == j ? i : 0.0);
  std::vector<double> lam, V;
  const bool capped = hydot::sym_eig(A, n, lam, V, 3);
  const bool full = hydot::sym_eig(A, n, lam, V);
  std::printf("%d %d\n", (int)capped, (int)full);
}
"""


def test_sym_eig_reports_non_convergence(tmp_path):
    """The eigensolver returns false when its sweep cap stops it before every coupling is deflated
    (its callers turn that into HYDOT_ERR_NOT_CONVERGED instead of using unconverged factors)."""
    src, out = tmp_path / "cap.cpp", tmp_path / "cap"
    src.write_text(CAP_PROG)
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1410_0986_gb300", "csrc"), str(src),
                    "-o", str(out)], check=True)
    r = subprocess.run([str(out)], capture_output=True, text=True, check=True)
    assert r.stdout.split() == ["0", "1"]
