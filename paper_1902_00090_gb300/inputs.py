"""Seeded synthetic inputs for the FDFD solves (shared by the CUDA path and its tests).

This module only *draws* problem data: grid descriptions, permittivity maps and
random test vectors.  It holds none of the method's arithmetic (no operator, no
source vector, no PML, no solver step); the CUDA library and the CPU oracle each
compute those on their own from what is drawn here.

The paper's data set (wavelength-splitting gratings, 229x90 cells at 20 nm,
Fig. 1 and Methods) is not available, so the workloads are synthetic stand-ins
with the same structure: a high-index slab (eps = 12.25, silicon-like) in a
low-index background (eps = 2.1, oxide-like), with a design region whose
permittivity is either binary or a continuous density correlated along
optimisation-like trajectories (Methods: the data set mixes discrete and
continuous designs taken from every step of an optimisation).

Layout: every permittivity map is a float64 array of shape (ny, nx), row-major,
cell (i, j) at index j * nx + i, i along x (fastest).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

EPS_BG = 2.1          # oxide-like background permittivity
EPS_HI = 12.25        # silicon-like permittivity
EPS_SPAN = EPS_HI - EPS_BG


@dataclass(frozen=True)
class Grid:
    """One 2D TM (Ez) FDFD problem: Yee grid, wavelength, PML and source layout."""
    nx: int
    ny: int
    dx: float = 40e-9            # cell size [m]
    wavelength: float = 1550e-9  # vacuum wavelength [m]
    npml: int = 10               # PML thickness in cells, all four sides
    pml_order: float = 3.0       # polynomial grading order of the PML conductivity
    pml_R: float = 1e-8          # target normal-incidence reflection of the PML
    i_src: int = 20              # x index of the line-current source column
    sigma_src: float = 6.0       # Gaussian width of the source profile along y [cells]
    slab_cells: int = 8          # slab thickness [cells]
    design: tuple = field(default=None)  # (i0, i1, j0, j1) design box, half-open

    @property
    def D(self) -> int:
        return self.nx * self.ny

    @property
    def j_src(self) -> float:
        return self.ny / 2.0

    def design_box(self):
        if self.design is not None:
            return self.design
        if (self.nx, self.ny) == (128, 128):
            w, h = 64, 16
        else:
            w, h = self.nx // 2, self.ny // 8
        i0 = self.nx // 2 - w // 2
        j0 = self.ny // 2 - h // 2
        return (i0, i0 + w, j0, j0 + h)


def grid_128(**kw) -> Grid:
    """128x128 cells at 40 nm, 1550 nm, 10-cell PML, source at x = 20 cells."""
    return Grid(nx=128, ny=128, **kw)


def grid_for(nx: int, ny: int, **kw) -> Grid:
    """Same physical layout at another size (40 nm cells, 10-cell PML)."""
    return Grid(nx=nx, ny=ny, **kw)


def grid_1024(**kw) -> Grid:
    """1024x1024 at 20 nm: 20-cell PML, source at 40 cells, 12-cell source width,
    16-cell slab and a 512x256 design region (same physical sizes as at 40 nm)."""
    g = Grid(nx=1024, ny=1024, dx=20e-9, npml=20, i_src=40, sigma_src=12.0,
             slab_cells=16)
    return replace(g, design=(256, 768, 384, 640), **kw)


def background_eps(g: Grid) -> np.ndarray:
    """Slab of EPS_HI, slab_cells rows thick and centred in y, in EPS_BG."""
    eps = np.full((g.ny, g.nx), EPS_BG, dtype=np.float64)
    j0 = g.ny // 2 - g.slab_cells // 2
    eps[j0:j0 + g.slab_cells, :] = EPS_HI
    return eps


def rng_for(config: int, trajectory: int) -> np.random.Generator:
    """Seed convention: configuration c, trajectory t -> PCG64(1000 c + t)."""
    return np.random.Generator(np.random.PCG64(1000 * config + trajectory))


def bernoulli_eps(g: Grid, seed: int) -> np.ndarray:
    """Binary design: each design pixel is EPS_HI or EPS_BG with probability 1/2."""
    rng = rng_for(1, seed)
    eps = background_eps(g)
    i0, i1, j0, j1 = g.design_box()
    pix = rng.random((j1 - j0, i1 - i0)) < 0.5
    eps[j0:j1, i0:i1] = np.where(pix, EPS_HI, EPS_BG)
    return eps


def _gauss_taps(sigma: float, radius: int) -> np.ndarray:
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    return k / k.sum()


def blur(rho: np.ndarray, sigma: float = 1.5, radius: int = 6) -> np.ndarray:
    """Separable Gaussian blur, truncated at `radius`, mirror ('reflect') edges."""
    k = _gauss_taps(sigma, radius)
    out = rho
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (radius, radius)
        p = np.pad(out, pad, mode="symmetric")
        acc = np.zeros_like(out)
        n = out.shape[axis]
        for t, w in enumerate(k):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(t, t + n)
            acc += w * p[tuple(sl)]
        out = acc
    return out


def trajectory_eps(g: Grid, config: int, trajectory: int, steps: int = 16,
                   noise: float = 0.05) -> np.ndarray:
    """One design trajectory: `steps` correlated permittivity maps, shape (steps, ny, nx).

    Step 0: rho ~ U(0,1) on the design box, blurred.  Each later step adds
    N(0, noise^2), re-blurs and clips to [0, 1].  eps = 2.1 + 10.15 rho inside
    the design box; slab and background outside.
    """
    rng = rng_for(config, trajectory)
    i0, i1, j0, j1 = g.design_box()
    rho = blur(rng.random((j1 - j0, i1 - i0)))
    rho = np.clip(rho, 0.0, 1.0)
    base = background_eps(g)
    out = np.empty((steps, g.ny, g.nx), dtype=np.float64)
    for s in range(steps):
        if s > 0:
            rho = np.clip(blur(rho + noise * rng.standard_normal(rho.shape)), 0.0, 1.0)
        e = base.copy()
        e[j0:j1, i0:i1] = EPS_BG + EPS_SPAN * rho
        out[s] = e
    return out


def trajectory_set(g: Grid, config: int, n_traj: int, steps: int = 16) -> np.ndarray:
    """n_traj trajectories of `steps` maps each: shape (n_traj * steps, ny, nx),
    trajectory-major (the split into training and held-out sets is by trajectory)."""
    return np.concatenate([trajectory_eps(g, config, t, steps) for t in range(n_traj)])


def uniform_eps(g: Grid, value: float) -> np.ndarray:
    return np.full((g.ny, g.nx), float(value), dtype=np.float64)


def random_complex(n: int, seed: int, shape=None) -> np.ndarray:
    """Standard complex normal test vector(s), complex128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shp = (n,) if shape is None else shape
    return (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / np.sqrt(2.0)


def standard_normal(n: int, seed: int) -> np.ndarray:
    """n independent N(0, 1) draws (float64)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(n)
