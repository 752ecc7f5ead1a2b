"""Seeded synthetic ocean grids for the free-surface elliptic system.

This module is the shared INPUT generator. It produces the fields that define
one problem instance (land/sea mask, face coefficients, diagonal shift, right
hand side) and nothing else: it holds none of the solver's arithmetic (no
operator assembly, no preconditioner, no iteration). Both the CPU oracle and
the CUDA library read its output.

Recipe (all fields are ``[ny][nx]`` row-major float64 / uint8; ``i`` runs
west->east and is periodic, ``j`` runs south->north and is closed):

* Mask: an N(0,1) field blurred with a Gaussian of sigma = max(nx, ny)/16
  cells (periodic in i, reflecting in j); exactly ``round(land * nx * ny)``
  lowest-valued cells are land.
* Depth: log H i.i.d. uniform on [ln 100, ln 5000], blurred with sigma = 3
  cells, affinely re-stretched to [ln 100, ln 5000] (a 50x depth contrast),
  then exponentiated.
* Scale factors e1 (east-west) and e2 (south-north): 1e5 m * (1 + 0.2 u) with
  u an independent blurred field (sigma = nx/8) stretched to [-1, 1].
  With ``pole_anisotropy > 0`` e1 is further multiplied by
  cos(phi_j), phi_j running from 0 at the southern row to
  ``pole_anisotropy * pi/2`` at the northern row, which reproduces the
  polar alpha >> beta regime of the paper's Section 2 (Eqs. 5-7).
* Face coefficients (Section 2, Eqs. 4-5 and Section 3, Eq. 8: the
  east-west coefficient carries e2/e1, the north-south one e1/e2):
  ``c_e[j,i]`` couples (i, j) with ((i+1) mod nx, j) and equals
  H_f * e2_f / e1_f; ``c_n[j,i]`` couples (i, j) with (i, j+1) and equals
  H_f * e1_f / e2_f. The face value of a field is the mean of its two cells.
  A face touching land, and every north face of the last row, is 0.
* Shift ``shift[j,i] = e1 * e2 / (g * dt^2)`` on wet cells (g = 9.81,
  dt = 5760 s), 0 on land: the mass term that the D^{n+1} part of the
  free-surface equation (Section 2, Eq. 2) adds to the diagonal.
* Right-hand side: N(0, 1) on wet cells, 0 on land.

Seeds: configuration c uses ``BASE_SEED + c``; ensemble member m of
configuration c uses ``BASE_SEED + 1000 * c + m``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 12101878
GRAVITY = 9.81
DT = 5760.0
H_MIN, H_MAX = 100.0, 5000.0


@dataclass
class Grid:
    nx: int
    ny: int
    wet: np.ndarray          # uint8 [ny][nx], 1 = ocean
    c_e: np.ndarray          # float64 [ny][nx]
    c_n: np.ndarray          # float64 [ny][nx]
    shift: np.ndarray        # float64 [ny][nx]
    b: np.ndarray            # float64 [ny][nx]
    H: np.ndarray = field(repr=False, default=None)
    e1: np.ndarray = field(repr=False, default=None)
    e2: np.ndarray = field(repr=False, default=None)
    seed: int = 0

    @property
    def n_wet(self) -> int:
        return int(self.wet.sum())


def _blur(field_: np.ndarray, sigma: float) -> np.ndarray:
    """Gaussian blur (transfer function exp(-2 pi^2 sigma^2 f^2)), periodic along
    i (axis 1) and half-sample reflecting along j (axis 0, done by mirroring the
    rows and blurring the doubled field periodically)."""
    if sigma <= 0:
        return field_
    ny, nx = field_.shape
    f = np.fft.rfftfreq(nx)
    out = np.fft.irfft(np.fft.rfft(field_, axis=1) * np.exp(-2.0 * math.pi ** 2 * sigma ** 2 * f ** 2)[None, :],
                       n=nx, axis=1)
    ext = np.concatenate([out, out[::-1]], axis=0)
    f = np.fft.rfftfreq(2 * ny)
    ext = np.fft.irfft(np.fft.rfft(ext, axis=0) * np.exp(-2.0 * math.pi ** 2 * sigma ** 2 * f ** 2)[:, None],
                       n=2 * ny, axis=0)
    return np.ascontiguousarray(ext[:ny])


def _stretch(u: np.ndarray, lo: float, hi: float) -> np.ndarray:
    umin, umax = float(u.min()), float(u.max())
    if umax - umin <= 0:
        return np.full_like(u, 0.5 * (lo + hi))
    return lo + (u - umin) * (hi - lo) / (umax - umin)


def make_grid(nx: int, ny: int, seed: int, land: float = 0.30,
              pole_anisotropy: float = 0.0, constant: bool = False) -> Grid:
    """Build one seeded grid. ``constant=True`` gives H = 1000 m, e1 = e2 = 1e5 m
    everywhere and an all-wet mask (used for closed-form spectrum checks)."""
    if nx < 1 or ny < 1:
        raise ValueError("grid must be at least 1x1")
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((ny, nx))
    logh = rng.uniform(math.log(H_MIN), math.log(H_MAX), size=(ny, nx))
    u1 = rng.standard_normal((ny, nx))
    u2 = rng.standard_normal((ny, nx))
    rhs = rng.standard_normal((ny, nx))

    if constant:
        wet = np.ones((ny, nx), dtype=np.uint8)
        H = np.full((ny, nx), 1000.0)
        e1 = np.full((ny, nx), 1e5)
        e2 = np.full((ny, nx), 1e5)
    else:
        m = _blur(noise, max(nx, ny) / 16.0)
        n_land = int(round(land * nx * ny))
        wet = np.ones(nx * ny, dtype=np.uint8)
        if n_land > 0:
            order = np.argsort(m.ravel(), kind="stable")
            wet[order[:n_land]] = 0
        wet = wet.reshape(ny, nx)
        H = np.exp(_stretch(_blur(logh, 3.0), math.log(H_MIN), math.log(H_MAX)))
        e1 = 1e5 * (1.0 + 0.2 * _stretch(_blur(u1, nx / 8.0), -1.0, 1.0))
        e2 = 1e5 * (1.0 + 0.2 * _stretch(_blur(u2, nx / 8.0), -1.0, 1.0))
    if pole_anisotropy > 0:
        phi = np.linspace(0.0, pole_anisotropy * math.pi / 2, ny, endpoint=False)
        e1 = e1 * np.cos(phi)[:, None]

    wetb = wet.astype(bool)
    # east faces: (i, j) -- ((i+1) mod nx, j)
    He = 0.5 * (H + np.roll(H, -1, axis=1))
    e1e = 0.5 * (e1 + np.roll(e1, -1, axis=1))
    e2e = 0.5 * (e2 + np.roll(e2, -1, axis=1))
    c_e = He * e2e / e1e
    c_e[~(wetb & np.roll(wetb, -1, axis=1))] = 0.0
    if nx == 1:
        c_e[:] = 0.0
    # north faces: (i, j) -- (i, j+1), none above the last row
    c_n = np.zeros((ny, nx))
    if ny > 1:
        Hn = 0.5 * (H[:-1] + H[1:])
        e1n = 0.5 * (e1[:-1] + e1[1:])
        e2n = 0.5 * (e2[:-1] + e2[1:])
        c_n[:-1] = Hn * e1n / e2n
        c_n[:-1][~(wetb[:-1] & wetb[1:])] = 0.0
    shift = np.where(wetb, e1 * e2 / (GRAVITY * DT * DT), 0.0)
    b = np.where(wetb, rhs, 0.0)
    return Grid(nx=nx, ny=ny, wet=np.ascontiguousarray(wet), c_e=np.ascontiguousarray(c_e),
                c_n=np.ascontiguousarray(c_n), shift=np.ascontiguousarray(shift),
                b=np.ascontiguousarray(b), H=H, e1=e1, e2=e2, seed=seed)


# The workloads, named by what they are.
TINY = dict(nx=32, ny=24, land=0.25)            # 32x24, ~25% land
COARSE = dict(nx=182, ny=149, land=0.30)        # ORCA2-like coarse global grid
ORCA1 = dict(nx=362, ny=292, land=0.30)
ORCA05 = dict(nx=722, ny=511, land=0.30)
ORCA025 = dict(nx=1442, ny=1021, land=0.30)     # eddy-permitting, ~1.47M points
ORCA12 = dict(nx=4322, ny=3059, land=0.30)      # eddy-resolving, ~13.2M points


def seed_for(config_index: int, member: int | None = None) -> int:
    if member is None:
        return BASE_SEED + config_index
    return BASE_SEED + 1000 * config_index + member


def next_rhs(b: np.ndarray, wet: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Serving workload: the next timestep's RHS is the previous one plus
    0.01 * N(0, 1) on wet cells."""
    step = rng.standard_normal(b.shape)
    return np.where(wet.astype(bool), b + 0.01 * step, 0.0)
