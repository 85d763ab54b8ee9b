"""Seeded synthetic inputs for the hyperspectral DOT Born workloads.

This module only draws inputs: wavelengths, chromophore extinction spectra,
background concentrations, the reduced-scattering law of the synthetic medium,
source/detector cells, anomalies, noise and random probe matrices. It holds
none of the method's arithmetic (no diffusion coefficient, no operator, no
field, no Born entry), so that the CPU oracle and the CUDA path can both take
their inputs from here without sharing any computation.

Every draw comes from ``numpy.random.Generator(PCG64(seed))`` in a fixed order:
spectra -> background concentrations -> positions -> anomaly -> noise ->
probes / sketch matrix. The named workloads mirror the sizes of the paper's
problem ranges (Section 1, table of parameter ranges: 10-100 sources, 10-200
wavelengths, 32^3-100^3 unknowns) with four chromophores (Section 6, the
HbO2/HbR/water/lipid set) whose measured spectra are replaced by smooth
synthetic ones over the same 650-900 nm band.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

SEED_BASE = 14100986

# Faces in the order -x, +x, -y, +y, -z, +z.
FACES = ("-x", "+x", "-y", "+y", "-z", "+z")


@dataclasses.dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    h: float  # cell side, mm

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def voxel(self, i: int, j: int, k: int) -> int:
        """Linear voxel index, x fastest: (k*ny + j)*nx + i."""
        return (k * self.ny + j) * self.nx + i


@dataclasses.dataclass
class Problem:
    """One synthetic hyperspectral DOT problem (inputs only)."""

    name: str
    grid: Grid
    lambda_nm: np.ndarray  # [n_lambda]
    eps: np.ndarray  # [n_lambda, n_chrom] extinction, /mm/mM
    c_bg: np.ndarray  # [n_chrom] background concentration, mM
    mus_prime: np.ndarray  # [n_lambda] reduced scattering of the medium, /mm
    robin_A: np.ndarray  # [6] per-face Robin coefficient; 0 means Dirichlet
    src_ijk: np.ndarray  # [n_src, 3] int
    det_ijk: np.ndarray  # [n_det, 3] int
    omega: float = 0.0  # angular modulation frequency, rad/ns (0 => CW)
    c_medium: float = 299.792458 / 1.4  # speed of light in the medium, mm/ns
    seed: int = 0

    @property
    def n_lambda(self) -> int:
        return int(self.lambda_nm.shape[0])

    @property
    def n_chrom(self) -> int:
        return int(self.eps.shape[1])

    @property
    def n_src(self) -> int:
        return int(self.src_ijk.shape[0])

    @property
    def n_det(self) -> int:
        return int(self.det_ijk.shape[0])

    @property
    def M(self) -> int:
        return self.n_src * self.n_det * self.n_lambda

    def src_voxels(self) -> np.ndarray:
        g = self.grid
        return np.array([g.voxel(*p) for p in self.src_ijk], dtype=np.int64)

    def det_voxels(self) -> np.ndarray:
        g = self.grid
        return np.array([g.voxel(*p) for p in self.det_ijk], dtype=np.int64)


def _spectra(rng: np.random.Generator, lam: np.ndarray, n_chrom: int) -> np.ndarray:
    """Smooth synthetic extinction spectra: 0.01 plus two Gaussians, clipped to [0.01, 0.5]."""
    eps = np.empty((lam.shape[0], n_chrom))
    for c in range(n_chrom):
        a = rng.uniform(0.05, 0.24, size=2)
        m = rng.uniform(600.0, 950.0, size=2)
        w = rng.uniform(25.0, 100.0, size=2)
        v = 0.01 + sum(a[g] * np.exp(-0.5 * ((lam - m[g]) / w[g]) ** 2) for g in range(2))
        eps[:, c] = np.clip(v, 0.01, 0.5)
    return eps


def _face_cells(rng: np.random.Generator, grid: Grid, k: int, n: int,
                exclude: Optional[set] = None, margin: Optional[int] = None) -> np.ndarray:
    """Draw n distinct cells on the plane z-index k, at least max(2, n_axis/8) cells from the edges
    (or ``margin`` cells when given)."""
    mx = max(2, grid.nx // 8) if margin is None else margin
    my = max(2, grid.ny // 8) if margin is None else margin
    cand = [(i, j) for j in range(my, grid.ny - my) for i in range(mx, grid.nx - mx)]
    if exclude:
        cand = [c for c in cand if (c[0], c[1], k) not in exclude]
    if n > len(cand):
        raise ValueError("not enough face cells for the requested sources/detectors")
    pick = rng.choice(len(cand), size=n, replace=False)
    return np.array([(cand[p][0], cand[p][1], k) for p in pick], dtype=np.int64)


def make_problem(grid: Grid, n_src: int, n_det: int, n_lambda: int, *, seed: int,
                 n_chrom: int = 4, geometry: str = "transmission",
                 robin_A: Sequence[float] = (3.0,) * 6, freq_mhz: float = 0.0,
                 lambda_range=(650.0, 900.0), name: str = "custom",
                 margin: Optional[int] = None) -> Problem:
    """Draw a problem on ``grid``.

    geometry: "transmission" puts sources on the top plane (k = nz-1) and detectors
    on the bottom plane (k = 0), the paper's plate geometry (Section 4.3, Section 6);
    "reflection" puts both on the top plane in distinct cells.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = np.linspace(lambda_range[0], lambda_range[1], n_lambda)
    eps = _spectra(rng, lam, n_chrom)
    c_bg = rng.uniform(0.02, 0.1, size=n_chrom)
    top = grid.nz - 1
    if geometry == "reflection":
        cells = _face_cells(rng, grid, top, n_src + n_det, margin=margin)
        src, det = cells[:n_src], cells[n_src:]
    elif geometry == "transmission":
        src = _face_cells(rng, grid, top, n_src, margin=margin)
        det = _face_cells(rng, grid, 0, n_det, margin=margin)
    else:
        raise ValueError(geometry)
    mus_prime = (lam / 500.0) ** -1.2
    omega = 2.0 * math.pi * freq_mhz * 1e-3  # rad/ns
    return Problem(name=name, grid=grid, lambda_nm=lam, eps=eps, c_bg=c_bg,
                   mus_prime=mus_prime, robin_A=np.asarray(robin_A, dtype=np.float64),
                   src_ijk=src, det_ijk=det, omega=omega, seed=seed)


def ellipsoid_anomaly(grid: Grid, seed: int, n_blobs: int = 3, contrast: float = 0.05,
                      n_chrom: int = 4, rng: Optional[np.random.Generator] = None) -> np.ndarray:
    """Piecewise-constant co-located anomaly: n_blobs ellipsoids, centres in the middle half
    of the box, semi-axes U(3, 8) cells; every chromophore is +contrast mM inside.
    Returned chromophore-major, shape [n_chrom * N]."""
    if rng is None:
        rng = np.random.Generator(np.random.PCG64(seed))
    k, j, i = np.meshgrid(np.arange(grid.nz), np.arange(grid.ny), np.arange(grid.nx), indexing="ij")
    inside = np.zeros(grid.N, dtype=bool)
    for _ in range(n_blobs):
        cx = rng.uniform(0.25 * grid.nx, 0.75 * grid.nx)
        cy = rng.uniform(0.25 * grid.ny, 0.75 * grid.ny)
        cz = rng.uniform(0.25 * grid.nz, 0.75 * grid.nz)
        ax, ay, az = rng.uniform(3.0, 8.0, size=3)
        q = ((i + 0.5 - cx) / ax) ** 2 + ((j + 0.5 - cy) / ay) ** 2 + ((k + 0.5 - cz) / az) ** 2
        inside |= (q <= 1.0).reshape(-1)
    return np.tile(np.where(inside, contrast, 0.0), n_chrom)


def gaussian(seed: int, shape, dtype=np.float64) -> np.ndarray:
    """Standard normal draws (probe vectors, sketch test matrices, unit noise)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(size=shape).astype(dtype, copy=False)


# The five named workloads. Spacings other than the 24x24x16 workload's 2 mm are this
# project's choice (keeping the box near the paper's 12 cm phantom scale).
def config(cfg: int) -> Problem:
    s = SEED_BASE + cfg
    if cfg == 1:
        return make_problem(Grid(24, 24, 16, 2.0), 8, 8, 16, seed=s, geometry="reflection",
                            name="cw-fp64-24x24x16")
    if cfg == 2:
        return make_problem(Grid(64, 64, 48, 2.0), 32, 32, 128, seed=s, name="cw-mixed-64x64x48")
    if cfg == 3:
        return make_problem(Grid(96, 96, 64, 1.5), 24, 24, 256, seed=s, name="cw-grad-96x96x64")
    if cfg == 5:
        return make_problem(Grid(128, 128, 96, 1.0), 64, 64, 512, seed=s, name="cw-sketch-128x128x96")
    raise ValueError(f"config {cfg}: use config4_batch() for the frequency-domain batch")


CONFIG4_GRIDS = ((32, 32, 24), (48, 48, 32), (64, 48, 40), (80, 64, 48), (96, 80, 56), (112, 96, 64))


def config4_batch() -> list:
    """Six frequency-domain phantoms of uneven size, 16 sources + 16 detectors, 64 wavelengths,
    100 MHz modulation; one seed stream per phantom."""
    out = []
    for p, (nx, ny, nz) in enumerate(CONFIG4_GRIDS):
        out.append(make_problem(Grid(nx, ny, nz, 2.0), 16, 16, 64, seed=SEED_BASE + 4 + 1000 * p,
                                freq_mhz=100.0, name=f"fd-{nx}x{ny}x{nz}"))
    return out


def small(seed: int = 7, nx: int = 12, ny: int = 10, nz: int = 8, h: float = 2.0, n_src: int = 3,
          n_det: int = 3, n_lambda: int = 4, geometry: str = "reflection", freq_mhz: float = 0.0,
          robin_A=(3.0,) * 6, margin: int = 1) -> Problem:
    """A tiny problem for brute-force checks and ragged-size tests (sources one cell from the edges)."""
    return make_problem(Grid(nx, ny, nz, h), n_src, n_det, n_lambda, seed=seed, geometry=geometry,
                        freq_mhz=freq_mhz, robin_A=robin_A, name=f"small-{nx}x{ny}x{nz}", margin=margin)
