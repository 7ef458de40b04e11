"""Seeded synthetic workloads for the direct-QPAT propagation path.

This module only *generates inputs*: grid sizes, time steps, acoustic media,
optical absorption maps, sensor positions and random direction vectors.  It
holds none of the method's arithmetic (no k-space operators, no PML, no
time stepping, no diffusion solve), so both the FP64 CPU oracle and the CUDA
path can draw their inputs from it without sharing any of the computation.

Units are SI throughout: metres, seconds, kg/m^3, optical coefficients in
1/m.  The paper quotes optical values in mm^-1 and attenuation in
dB MHz^-y cm^-1; the attenuation stays in those units (the conversion is part
of the method and lives on each side separately).

Geometry convention shared by every consumer: on the FFT grid of N_i nodes
along axis i (interior plus PML on both sides), node j sits at
x_j = (j - (N_i - 1)/2) * dx, so the grid is centred on the origin.  Arrays
are C-ordered with the *last* axis fastest, i.e. shape (ny, nx) in 2D and
(nz, ny, nx) in 3D; axis 0 of a position vector is x.

The workloads stand in for the paper's phantoms (Section 6, Tables 1 and 3),
whose images are not published as data: elliptic sound-speed/density
inclusions with tissue-like values, a background absorption map with disc
inclusions, and boundary or circular sensor arrays.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

MM = 1e-3


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic problem: sizes, medium recipe and sensor layout."""
    name: str
    dim: int
    n: int                 # interior nodes per axis
    pml: int               # PML nodes added on each side (outside the interior)
    dx: float              # grid spacing [m]
    nt: int                # number of recorded time samples
    cfl: float = 0.3
    c_bg: float = 1500.0
    rho_bg: float = 1000.0
    alpha_bg_db: float = 0.75      # dB MHz^-y cm^-1
    y: float = 1.3
    n_incl: int = 2
    incl_c: Tuple[float, float] = (1450.0, 1600.0)
    incl_rho_frac: float = 0.10
    incl_alpha_db: Optional[Tuple[float, float]] = None
    incl_fixed_c: bool = True       # True: inclusion k gets incl_c[k]; False: uniform in range
    mu_bg: float = 0.01 / MM        # background absorption [1/m]
    mu_discs: int = 3
    mu_disc_range: Tuple[float, float] = (0.02 / MM, 0.05 / MM)
    mu_smooth_sigma: float = 0.0    # >0: smooth random field instead of discs
    mus_prime: float = 1.0 / MM     # reduced scattering [1/m]
    sensors: str = "circle"         # "circle" | "perimeter" | "plane"
    n_sensors: int = 128
    sensor_radius: float = 5.5 * MM
    seed: int = 11685
    lossless: bool = False

    @property
    def grid(self) -> int:
        return self.n + 2 * self.pml

    @property
    def shape(self) -> Tuple[int, ...]:
        return (self.grid,) * self.dim

    @property
    def interior_shape(self) -> Tuple[int, ...]:
        return (self.n,) * self.dim


def c_max(w: Workload, c: np.ndarray) -> float:
    return float(np.max(c))


def time_step(w: Workload, c: np.ndarray) -> float:
    """dt = CFL * dx / c_max (the CFL number is part of each workload)."""
    return w.cfl * w.dx / float(np.max(c))


# --- the workloads -------------------------------------------------------

def small(n=24, pml=4, nt=40, dim=2, lossless=False, y=1.5, seed=7, sensors="circle",
          n_sensors=12, **kw) -> Workload:
    """A tiny heterogeneous lossy problem for oracle pins and quick parity."""
    dx = 0.1 * MM
    return Workload(name=f"small{dim}d-{n}", dim=dim, n=n, pml=pml, dx=dx, nt=nt,
                    y=y, lossless=lossless, seed=seed, sensors=sensors,
                    n_sensors=n_sensors, sensor_radius=0.35 * n * dx, **kw)


C1 = Workload(name="2d-128-fp64", dim=2, n=128, pml=20, dx=0.1 * MM, nt=600, y=1.3,
              n_incl=2, incl_c=(1450.0, 1600.0), sensors="circle", n_sensors=128,
              sensor_radius=5.5 * MM, seed=11685 + 0)

C2 = Workload(name="2d-512-fp32", dim=2, n=512, pml=32, dx=0.05 * MM, nt=2000, y=1.5,
              n_incl=6, incl_c=(1400.0, 1650.0), incl_fixed_c=False, incl_rho_frac=0.0,
              incl_alpha_db=(0.5, 1.0), sensors="perimeter", n_sensors=256,
              seed=11685 + 1)

C2_Y11 = dataclasses.replace(C2, name="2d-512-fp32-y1.1", y=1.1)

C3 = Workload(name="2d-1024-diff", dim=2, n=1024, pml=28, dx=0.05 * MM, nt=4000, y=1.5,
              n_incl=6, incl_c=(1400.0, 1650.0), incl_fixed_c=False, incl_rho_frac=0.0,
              incl_alpha_db=(0.5, 1.0), mu_bg=0.005 / MM, mu_discs=0,
              mu_smooth_sigma=8.0, mu_disc_range=(0.005 / MM, 0.05 / MM),
              sensors="perimeter", n_sensors=512, seed=11685 + 2)

C5 = Workload(name="3d-256-fp32", dim=3, n=256, pml=16, dx=0.1 * MM, nt=1500, y=1.3,
              n_incl=8, incl_c=(1400.0, 1650.0), incl_fixed_c=False,
              sensors="plane", n_sensors=128 * 128, mu_disc_range=(0.01 / MM, 0.04 / MM),
              seed=11685 + 4)


def c4_workloads():
    """The batched inexact-Newton inner-loop mix: 16 problems at each of three
    interior sizes; Nt is chosen so a wave at the background speed crosses
    the interior 1.5 times."""
    out = []
    for n, pml in ((256, 16), (384, 24), (512, 32)):
        w = Workload(name=f"2d-{n}-jvp", dim=2, n=n, pml=pml, dx=0.05 * MM, nt=1, y=1.5,
                     n_incl=6, incl_c=(1400.0, 1650.0), incl_fixed_c=False,
                     incl_rho_frac=0.0, incl_alpha_db=(0.5, 1.0), sensors="perimeter",
                     n_sensors=4 * (n // 8), seed=11685 + 3)
        out.append(w)
    return out


def c4_nt(w: Workload, c: np.ndarray) -> int:
    dt = time_step(w, c)
    return int(math.ceil(1.5 * w.n * w.dx / (w.c_bg * dt)))


# --- generators ----------------------------------------------------------

def node_coords(w: Workload):
    """1-D node coordinates of the FFT grid along one axis [m]."""
    g = w.grid
    return (np.arange(g) - (g - 1) / 2.0) * w.dx


def _mesh(w: Workload):
    x = node_coords(w)
    if w.dim == 2:
        Y, X = np.meshgrid(x, x, indexing="ij")
        return (X, Y)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return (X, Y, Z)


def acoustic_medium(w: Workload):
    """Sound speed c [m/s], density rho [kg/m^3] and attenuation alpha0
    [dB MHz^-y cm^-1] on the full FFT grid (PML included)."""
    rng = np.random.default_rng(w.seed)
    coords = _mesh(w)
    L = w.n * w.dx
    c = np.full(w.shape, w.c_bg)
    rho = np.full(w.shape, w.rho_bg)
    alpha = np.full(w.shape, 0.0 if w.lossless else w.alpha_bg_db)
    for k in range(w.n_incl):
        centre = rng.uniform(-1, 1, size=w.dim)
        centre *= 0.31 * L * rng.uniform(0, 1) ** (1.0 / w.dim) / max(np.linalg.norm(centre), 1e-12)
        semi = rng.uniform(0.04 * L, 0.16 * L, size=w.dim)
        if w.dim == 2:
            th = rng.uniform(0, np.pi)
            R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        else:
            A = rng.normal(size=(3, 3))
            R, _ = np.linalg.qr(A)
        rel = np.stack([coords[i] - centre[i] for i in range(w.dim)], axis=-1)
        loc = rel @ R          # coordinates in the ellipse frame
        mask = np.sum((loc / semi) ** 2, axis=-1) <= 1.0
        if w.incl_fixed_c and k < len(w.incl_c):
            cv = w.incl_c[k]
        else:
            cv = rng.uniform(*w.incl_c)
        sign = 1.0 if cv >= w.c_bg else -1.0
        if w.incl_rho_frac > 0:
            rv = w.rho_bg * (1.0 + sign * w.incl_rho_frac)
        else:
            rv = rng.uniform(900.0, 1100.0)
        c[mask] = cv
        rho[mask] = rv
        if w.incl_alpha_db is not None and not w.lossless:
            alpha[mask] = rng.uniform(*w.incl_alpha_db)
    return c, rho, alpha


def optical_absorption(w: Workload, seed_offset: int = 0):
    """mu_a [1/m] on the interior grid: background plus discs, or a smooth
    random field (Gaussian-filtered white noise) scaled into the range."""
    rng = np.random.default_rng(w.seed + 1000 + seed_offset)
    shape = w.interior_shape
    if w.mu_smooth_sigma > 0:
        from scipy.ndimage import gaussian_filter
        f = gaussian_filter(rng.normal(size=shape), w.mu_smooth_sigma, mode="wrap")
        f = (f - f.min()) / max(f.max() - f.min(), 1e-30)
        lo, hi = w.mu_disc_range
        return lo + (hi - lo) * f
    x = (np.arange(w.n) - (w.n - 1) / 2.0) * w.dx
    grids = np.meshgrid(*([x] * w.dim), indexing="ij")[::-1]   # (X, Y[, Z]) with x fastest
    mu = np.full(shape, w.mu_bg)
    L = w.n * w.dx
    for _ in range(w.mu_discs):
        centre = rng.uniform(-0.3 * L, 0.3 * L, size=w.dim)
        rad = rng.uniform(0.05 * L, 0.12 * L)
        r2 = sum((grids[i] - centre[i]) ** 2 for i in range(w.dim))
        mu[r2 <= rad * rad] = rng.uniform(*w.mu_disc_range)
    return mu


def optical_diffusion(w: Workload):
    """kappa = 1/(d (mu_a_bg + mu_s')) as a fixed field on the interior grid."""
    return np.full(w.interior_shape, 1.0 / (w.dim * (w.mu_bg + w.mus_prime)))


def sensor_positions(w: Workload):
    """(Ns, dim) sensor coordinates [m], x first."""
    half = (w.n - 1) / 2.0 * w.dx
    if w.sensors == "circle":
        th = 2 * np.pi * np.arange(w.n_sensors) / w.n_sensors
        pos = np.stack([w.sensor_radius * np.cos(th), w.sensor_radius * np.sin(th)], axis=1)
        if w.dim == 3:
            pos = np.concatenate([pos, np.zeros((w.n_sensors, 1))], axis=1)
        return pos
    if w.sensors == "perimeter":
        per = w.n_sensors // 4
        t = -half + 2 * half * np.arange(per) / per       # corners counted once
        s0 = np.stack([t, np.full(per, -half)], 1)         # bottom, left to right
        s1 = np.stack([np.full(per, half), t], 1)          # right, bottom to top
        s2 = np.stack([-t, np.full(per, half)], 1)         # top, right to left
        s3 = np.stack([np.full(per, -half), -t], 1)        # left, top to bottom
        return np.concatenate([s0, s1, s2, s3], 0)
    if w.sensors == "plane":
        m = int(round(math.sqrt(w.n_sensors)))
        t = -half + 2 * half * np.arange(m) / max(m - 1, 1)
        Y, X = np.meshgrid(t, t, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), np.full(m * m, -half)], 1)
    raise ValueError(w.sensors)


def random_field(shape, seed: int, dtype=np.float64):
    """Seeded standard-normal array."""
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


def smooth_p0(w: Workload, seed: int = 0):
    """A smooth seeded initial pressure on the interior grid (sum of Gaussians)."""
    rng = np.random.default_rng(w.seed + 500 + seed)
    x = (np.arange(w.n) - (w.n - 1) / 2.0) * w.dx
    grids = np.meshgrid(*([x] * w.dim), indexing="ij")[::-1]
    L = w.n * w.dx
    p0 = np.zeros(w.interior_shape)
    for _ in range(4):
        centre = rng.uniform(-0.3 * L, 0.3 * L, size=w.dim)
        sig = rng.uniform(0.03 * L, 0.08 * L)
        r2 = sum((grids[i] - centre[i]) ** 2 for i in range(w.dim))
        p0 += rng.uniform(0.5, 1.5) * np.exp(-r2 / (2 * sig * sig))
    return p0
