"""Seeded synthetic inputs for planar / line-detector photoacoustic imaging.

This module is shared by the oracle's tests, the GPU parity tests and the
benchmark.  It holds the *forward* physics (pressure recorded on the detector
line or plane for simple initial pressures) and nothing of the
reconstruction method itself: no node, weight, window or NUFFT arithmetic.

Model (the paper's Sec. 2): p solves the wave equation with sound speed c,
p(., 0) = f, dp/dt(., 0) = 0; the detectors sit on the plane (d = 3) or line
(d = 2) of depth 0 and record p at times t_n = n dt, n = 0..nt-1.  Objects lie
at positive depth.  Lateral detector positions are x_m = m dx (and y = m dy).

Forward models provided (each exact for its phantom class):

* ``balls_3d`` -- uniform balls: p(r, t) = A (r - c t) / (2 r) for
  |r - c t| < R (the N-shaped pressure of a uniform ball, r = distance from
  the detector to the centre, valid for r > R); smooth balls
  f = A (1 - s^2/R^2)^2: p = (r - c t) f(|r - c t|) / (2 r).  Both follow from
  the radial solution r p = [phi(r - ct) + phi(r + ct)]/2, phi(s) = s f(|s|).
* ``fcirc_2d`` -- the paper's circular object (Sec. 5.1), amplitude-scaled:
  f = A sqrt(1 - |x - x0|^2 / a^2).  It is the line integral (descent) of a
  uniform 3-D ball of radius a times A/(2a), so its 2-D data is the line
  integral of the N-wave:  p = A/(2a) * [ sqrt(r^2 - d^2) - ct ln(r + sqrt(r^2 - d^2)) ]
  evaluated between r_lo = max(d, ct - a) and r_hi = ct + a (d = detector to
  centre distance), a closed form at any grid size.
* ``spectral_2d`` -- any 2-D image, propagated exactly for its trigonometric
  interpolant in a zero-padded periodic box large enough that no periodic
  image reaches the detectors within the recorded time:
  p(x, 0, t) = Re sum_K fhat(K) cos(c |K| t) e^{i K x}.

All randomness comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class Geometry:
    """Detector / image grid of one reconstruction problem."""

    dim: int            # 2 (line detector) or 3 (planar detector)
    nx: int
    nt: int
    nz: int
    ny: int = 1
    dx: float = 1.0
    dy: float = 1.0
    dt: float = 1.0
    c: float = 1.0
    dz: float = 1.0

    @property
    def data_shape(self):
        return (self.nx, self.nt) if self.dim == 2 else (self.nx, self.ny, self.nt)

    @property
    def image_shape(self):
        return (self.nx, self.nz) if self.dim == 2 else (self.nx, self.ny, self.nz)

    @property
    def voxels(self) -> int:
        return self.nx * (self.ny if self.dim == 3 else 1) * self.nz


@dataclasses.dataclass
class Problem:
    geom: Geometry
    p: np.ndarray                 # data, float64, geom.data_shape
    f_true: Optional[np.ndarray]  # initial pressure on the image grid (None if not tabulated)
    objects: list                 # parameters of the phantom objects
    note: str = ""


# ---------------------------------------------------------------------------
# 3-D balls (closed-form N-waves)
# ---------------------------------------------------------------------------

def balls_3d(geom: Geometry, balls, smooth: bool = False, cell_average: bool = True):
    """Data p[x][y][n] for a sum of balls (centre (bx, by, bz), radius R, amplitude A).

    FP64, torch multithreaded CPU elementwise ops; only the time window in
    which a ball's wave passes a detector row is evaluated."""
    import torch
    assert geom.dim == 3
    x = torch.arange(geom.nx, dtype=torch.float64) * geom.dx
    y = torch.arange(geom.ny, dtype=torch.float64) * geom.dy
    ct = (geom.c * geom.dt) * torch.arange(geom.nt, dtype=torch.float64)
    p = torch.zeros(geom.data_shape, dtype=torch.float64)
    half = 0.5 * geom.c * geom.dt
    for (bx, by, bz, R, A) in balls:
        r = torch.sqrt((x[:, None] - bx) ** 2 + (y[None, :] - by) ** 2 + bz * bz)
        # samples n whose cell can meet |r - ct| < R for some detector
        n_lo = max(0, int(np.floor((float(r.min()) - R - 2 * half) / (geom.c * geom.dt))))
        n_hi = min(geom.nt, int(np.ceil((float(r.max()) + R + 2 * half) / (geom.c * geom.dt))) + 1)
        if n_hi <= n_lo:
            continue
        rr = r[:, :, None]
        c = ct[None, None, n_lo:n_hi]
        if smooth:
            s = torch.abs(rr - c)
            prof = torch.where(s < R, A * (1.0 - (s / R) ** 2) ** 2, torch.zeros((), dtype=torch.float64))
            p[:, :, n_lo:n_hi] += (rr - c) * prof / (2.0 * rr)
        elif not cell_average:
            p[:, :, n_lo:n_hi] += torch.where(torch.abs(rr - c) < R, A * (rr - c) / (2.0 * rr),
                                              torch.zeros((), dtype=torch.float64))
        else:
            lo = torch.maximum(c - half, rr - R)
            hi = torch.minimum(c + half, rr + R)
            val = ((rr * hi - 0.5 * hi * hi) - (rr * lo - 0.5 * lo * lo)) / (2.0 * rr) / (2 * half)
            p[:, :, n_lo:n_hi] += torch.where(hi > lo, A * val, torch.zeros((), dtype=torch.float64))
    return p.numpy()


def balls_3d_image(geom: Geometry, balls, smooth: bool = False):
    """The initial pressure of :func:`balls_3d` sampled on the image grid."""
    x = (np.arange(geom.nx) * geom.dx)[:, None, None]
    y = (np.arange(geom.ny) * geom.dy)[None, :, None]
    z = (np.arange(geom.nz) * geom.dz)[None, None, :]
    f = np.zeros(geom.image_shape)
    for (bx, by, bz, R, A) in balls:
        s = np.sqrt((x - bx) ** 2 + (y - by) ** 2 + (z - bz) ** 2)
        if smooth:
            f += np.where(s < R, A * (1 - (s / R) ** 2) ** 2, 0.0)
        else:
            f += np.where(s < R, A, 0.0)
    return f


# ---------------------------------------------------------------------------
# 2-D circular objects (closed form by descent from the 3-D ball)
# ---------------------------------------------------------------------------

def fcirc_2d(geom: Geometry, discs):
    """Data p[x][n] for a sum of f_circ objects (centre (x0, z0), radius a, amplitude A).

    Evaluated in FP64 with torch's multithreaded CPU elementwise ops (the same
    closed form as above, only faster than single-threaded numpy at 2048 x 4096)."""
    import torch
    assert geom.dim == 2
    x = torch.arange(geom.nx, dtype=torch.float64) * geom.dx
    tt = (geom.c * geom.dt) * torch.arange(geom.nt, dtype=torch.float64)[None, :]
    p = torch.zeros(geom.data_shape, dtype=torch.float64)
    for (x0, z0, a, A) in discs:
        d = torch.sqrt((x - x0) ** 2 + z0 * z0)[:, None]
        r_hi = tt + a
        r_lo = torch.maximum(d, tt - a)
        live = r_hi > r_lo
        d2 = d * d
        sh = torch.sqrt(torch.clamp(r_hi * r_hi - d2, min=0.0))
        sl = torch.sqrt(torch.clamp(r_lo * r_lo - d2, min=0.0))
        val = (sh - sl) - tt * torch.log((r_hi + sh) / (r_lo + sl))
        p += torch.where(live, (A / (2.0 * a)) * val, torch.zeros((), dtype=torch.float64))
    return p.numpy()


def fcirc_2d_image(geom: Geometry, discs):
    x = (np.arange(geom.nx) * geom.dx)[:, None]
    z = (np.arange(geom.nz) * geom.dz)[None, :]
    f = np.zeros(geom.image_shape)
    for (x0, z0, a, A) in discs:
        s2 = ((x - x0) ** 2 + (z - z0) ** 2) / (a * a)
        f += np.where(s2 < 1.0, A * np.sqrt(np.maximum(1.0 - s2, 0.0)), 0.0)
    return f


# ---------------------------------------------------------------------------
# 2-D spectral propagator (exact for the trigonometric interpolant)
# ---------------------------------------------------------------------------

def spectral_2d(geom: Geometry, image: np.ndarray, box: Optional[tuple] = None):
    """Data p[x][n] of a 2-D initial pressure given on the image grid.

    The image occupies box cells [0, nx) x [0, nz) (cell (m, q) at (m dx, q dz));
    everything else in the box is zero.  Requires dx == dz.
    """
    assert geom.dim == 2 and abs(geom.dx - geom.dz) < 1e-12 * geom.dx
    h = geom.dx
    T = geom.c * geom.nt * geom.dt
    need_x = geom.nx + int(np.ceil(T / h)) + 2
    need_z = geom.nz + int(np.ceil(T / h)) + 2
    if box is None:
        bx = 1 << int(np.ceil(np.log2(need_x)))
        bz = 1 << int(np.ceil(np.log2(need_z)))
    else:
        bx, bz = box
        assert bx >= need_x and bz >= need_z, "box too small: periodic images would reach the detectors"
    B = np.zeros((bx, bz))
    B[: geom.nx, : geom.nz] = image
    F = np.fft.fft2(B)
    Kx = 2 * np.pi * np.fft.fftfreq(bx, d=h)
    Kz = 2 * np.pi * np.fft.fftfreq(bz, d=h)
    Kabs = np.sqrt(Kx[:, None] ** 2 + Kz[None, :] ** 2)
    p = np.empty((geom.nx, geom.nt))
    for n in range(geom.nt):
        col = (F * np.cos(geom.c * Kabs * n * geom.dt)).sum(axis=1) / bz   # detector depth 0
        p[:, n] = np.fft.ifft(col).real[: geom.nx]
    return p


def disc_image_2d(geom: Geometry, discs):
    """Uniform discs (centre (x0, z0), radius a, amplitude A) sampled at cell centres."""
    x = (np.arange(geom.nx) * geom.dx)[:, None]
    z = (np.arange(geom.nz) * geom.dz)[None, :]
    f = np.zeros(geom.image_shape)
    for (x0, z0, a, A) in discs:
        f += np.where((x - x0) ** 2 + (z - z0) ** 2 < a * a, A, 0.0)
    return f


# ---------------------------------------------------------------------------
# Seeded random phantoms
# ---------------------------------------------------------------------------

def random_discs(rng, geom: Geometry, count: int, rmin: float, rmax: float, amin=0.5, amax=1.0):
    """Discs fully inside the image: x0 in [R, X - R], z0 in [R + 2, Z - R]."""
    X = geom.nx * geom.dx
    Z = geom.nz * geom.dz
    out = []
    for _ in range(count):
        R = rng.uniform(rmin, rmax)
        x0 = rng.uniform(R, X - R)
        z0 = rng.uniform(R + 2 * geom.dz, Z - R)
        A = rng.uniform(amin, amax)
        out.append((x0, z0, R, A))
    return out


def random_balls(rng, geom: Geometry, count: int, rmin: float, rmax: float, amin=1.0, amax=1.0):
    X, Y, Z = geom.nx * geom.dx, geom.ny * geom.dy, geom.nz * geom.dz
    out = []
    for _ in range(count):
        R = rng.uniform(rmin, rmax)
        out.append((rng.uniform(R, X - R), rng.uniform(R, Y - R), rng.uniform(R + 2 * geom.dz, Z - R), R,
                    rng.uniform(amin, amax)))
    return out


def plain_2d(seed: int = 0, nx: int = 128, nt: int = 256, nz: int = 128) -> Problem:
    """2-D line detector, 128 detectors x 256 samples -> 128 x 128 image; 1-8 uniform
    discs (radius U(2,12), amplitude U(0.5,1)) propagated by the spectral model."""
    rng = np.random.default_rng(seed)
    g = Geometry(dim=2, nx=nx, nt=nt, nz=nz)
    discs = random_discs(rng, g, int(rng.integers(1, 9)), 2.0, min(12.0, nz / 4))
    img = disc_image_2d(g, discs)
    return Problem(g, spectral_2d(g, img), img, discs, "uniform discs, spectral propagator")


def fcirc_problem_2d(seed: int, nx: int, nt: int, nz: int, count: int, rmin=2.0, rmax=12.0,
                     noise: float = 0.0) -> Problem:
    """2-D problem with f_circ discs (closed-form data) and optional white noise
    of standard deviation ``noise * max|p|``."""
    rng = np.random.default_rng(seed)
    g = Geometry(dim=2, nx=nx, nt=nt, nz=nz)
    discs = random_discs(rng, g, count, rmin, min(rmax, nz / 4))
    p = fcirc_2d(g, discs)
    if noise > 0:
        p = p + rng.standard_normal(p.shape) * (noise * np.abs(p).max())
    return Problem(g, p, fcirc_2d_image(g, discs), discs, "f_circ discs, closed form")


def large_2d(seed: int = 0) -> Problem:
    """2-D large: 2048 detectors x 4096 samples -> 2048 x 2048; 50 discs + 1 % noise."""
    return fcirc_problem_2d(seed, 2048, 4096, 2048, 50, noise=0.01)


def planar_3d(seed: int = 0, n: int = 128, nt: int = 256, nz: int = 128, rmin=3.0, rmax=15.0,
              max_balls: int = 20) -> Problem:
    """3-D planar: 128 x 128 detectors x 256 samples -> 128^3; 1-20 uniform balls."""
    rng = np.random.default_rng(seed)
    g = Geometry(dim=3, nx=n, ny=n, nt=nt, nz=nz)
    balls = random_balls(rng, g, int(rng.integers(1, max_balls + 1)), rmin, min(rmax, nz / 4))
    return Problem(g, balls_3d(g, balls), None, balls, "uniform balls, N-wave (time-cell averaged)")


def adjoint_3d(seed: int = 0) -> Problem:
    """Adjoint / autograd 3-D: 256 x 256 detectors x 512 samples -> 256^3."""
    return planar_3d(seed, n=256, nt=512, nz=256)


def batched_2d_geometries(seed: int = 0, count: int = 64) -> List[Geometry]:
    """Uneven batch: nx = 2*U{128..1024}, nt = 2*U{256..2048}, nz = nt/2 rounded down to even."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx = 2 * int(rng.integers(128, 1025))
        nt = 2 * int(rng.integers(256, 2049))
        nz = (nt // 2) & ~1
        out.append(Geometry(dim=2, nx=nx, nt=nt, nz=nz))
    return out


def batched_2d(seed: int = 0, count: int = 64) -> List[Problem]:
    geoms = batched_2d_geometries(seed, count)
    rng = np.random.default_rng(seed + 1000)
    probs = []
    for g in geoms:
        discs = random_discs(rng, g, int(rng.integers(1, 9)), 2.0, min(12.0 * g.nx / 128, g.nz / 4))
        probs.append(Problem(g, fcirc_2d(g, discs), None, discs, "f_circ discs, closed form"))
    return probs


def random_data(seed: int, geom: Geometry) -> np.ndarray:
    """White Gaussian data of the geometry's shape (for operator-level tests)."""
    return np.random.default_rng(seed).standard_normal(geom.data_shape)


def random_image(seed: int, geom: Geometry) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(geom.image_shape)
