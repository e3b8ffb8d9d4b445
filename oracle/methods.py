"""FP64 oracle of the other Fourier algorithms compared in Sec. 4.

TEST INFRASTRUCTURE ONLY, under the same rule as the rest of ``oracle/``:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may use it, and it never imports the CUDA library.

Each algorithm differs from the direct one only in how the temporal DFT of
Eq. (fft-2),  D(nu) = sum_{n<nt} e^{-2 pi i nu n / nt} g_n,  is evaluated at
the nodes nu of a lateral row.  Everything else -- the lateral DFT of
Eq. (fft-1a), the nodes and the weight (Eq. dft-2d, Eq. fft-0), the l = 0
rule and the inverse DFT of Eq. (fft-1) -- is the direct oracle's own
(``oracle.lateral_dft``, ``oracle.row_nodes``, ``oracle.image_from_spectrum``).

Methods (time-index units: the uniform grid of the oversampled DFT is
nu = j / c, j in Z, with c = M / nt for the padded length M):

* ``nearest`` / ``linear`` (Sec. 4, interpolation based algorithm): D is
  evaluated exactly on the grid by zero padding to M and one FFT, then
  interpolated at the node: the nearest grid value, or the straight line
  between the two grid neighbours.
* ``tsinc`` (Sec. 4, truncated sinc): Algorithm 1 with Psi the indicator of
  [-c pi, c pi]; then Psi = 1 on the samples and Psi_hat(w) = 2 sin(c pi w) / w.
* ``kb``: Algorithm 1 with the Kaiser-Bessel window of Sec. 3.2,
  alpha = pi (2c - 1)(1 - 1e-3) unless given.

Algorithm 1 is taken step by step: divide the samples by Psi(2 pi n/nt - pi),
scale by the constant, zero pad to c nt, one FFT (the vector G_hat_j of
Eq. nufft-b / nufft-c, wrapped modulo c nt), then the sum of Eq. (nufft-a)
over the terms with |j - c nu| <= c K, each with its factor
e^{-i pi (nu - j/c)} Psi_hat(nu - j/c).

Readings where Sec. 4 or Algorithm 1 leave a choice (also listed in the
design notes):
 * the step Delta in the definition of the interpolated spectrum is a common
   constant of every node value; it is carried by the weight, exactly as in
   the direct algorithm;
 * the grid wraps modulo M because D is nt-periodic in nu;
 * nearest neighbour rounds halves upward: j = floor(c nu + 1/2);
 * the constant in front of the oversampled DFT is 1/(2 pi c), the Fourier
   coefficient of a 2 pi c periodic function (printed as c/(2 pi));
 * the truncated sinc uses the same interpolation length as the
   Kaiser-Bessel window, K = 3, unless given.
"""
from __future__ import annotations

import math

import numpy as np

from . import _geom, image_from_spectrum, lateral_dft, row_nodes

METHODS = ("kb", "tsinc", "linear", "nearest")


def _padded_length(c: float, nt: int) -> int:
    M = int(round(c * nt))
    if abs(M - c * nt) > 1e-9 * max(1.0, c * nt) or M < nt:
        raise ValueError(f"c * nt must be an integer >= nt (c = {c}, nt = {nt})")
    return M


# ---------------------------------------------------------------------------
# windows of Algorithm 1: (Psi on [-pi, pi), Psi_hat on R)
# ---------------------------------------------------------------------------

def kb_window(alpha: float, K: float):
    """Kaiser-Bessel window Psi^{alpha,K}_KB and its Fourier transform (Sec. 3.2)."""
    i0aK = float(np.i0(alpha * K))

    def psi(theta):
        theta = np.asarray(theta, dtype=np.float64)
        inside = np.abs(theta) <= alpha
        r = np.sqrt(np.maximum(alpha * alpha - theta * theta, 0.0))
        return np.where(inside, np.i0(K * r) / i0aK, 0.0)

    def psi_hat(w):
        w = np.asarray(w, dtype=np.float64)
        d = K * K - w * w
        out = np.empty_like(w)
        pos = d > 0
        neg = d < 0
        zero = ~(pos | neg)
        s = np.sqrt(d[pos])
        out[pos] = 2.0 * np.sinh(alpha * s) / (i0aK * s)
        s = np.sqrt(-d[neg])
        out[neg] = 2.0 * np.sin(alpha * s) / (i0aK * s)
        out[zero] = 2.0 * alpha / i0aK
        return out

    return psi, psi_hat


def indicator_window(c: float):
    """Indicator of [-c pi, c pi] and its Fourier transform 2 sin(c pi w) / w."""

    def psi(theta):
        theta = np.asarray(theta, dtype=np.float64)
        return np.where(np.abs(theta) <= c * math.pi, 1.0, 0.0)

    def psi_hat(w):
        w = np.asarray(w, dtype=np.float64)
        out = np.empty_like(w)
        small = np.abs(w) < 1e-300
        out[small] = 2.0 * c * math.pi
        ws = w[~small]
        out[~small] = 2.0 * np.sin(c * math.pi * ws) / ws
        return out

    return psi, psi_hat


# ---------------------------------------------------------------------------
# evaluation of D(nu) at the nodes of one row
# ---------------------------------------------------------------------------

def grid_dft(gvec: np.ndarray, M: int) -> np.ndarray:
    """D_j = sum_{n<nt} e^{-2 pi i j n / M} g_n for j = 0..M-1 (last axis)."""
    return np.fft.fft(np.asarray(gvec, dtype=np.complex128), n=M, axis=-1)


def interpolate(D: np.ndarray, nu: np.ndarray, c: float, kind: str) -> np.ndarray:
    """Nearest / linear interpolation of the grid values D_j (at nu = j/c, j mod M)."""
    M = D.shape[-1]
    x = c * np.asarray(nu, dtype=np.float64)
    if kind == "nearest":
        j = np.floor(x + 0.5).astype(np.int64)
        return D[j % M]
    if kind != "linear":
        raise ValueError(kind)
    j0 = np.floor(x).astype(np.int64)
    f = x - j0
    return (1.0 - f) * D[j0 % M] + f * D[(j0 + 1) % M]


def nufft(gvec: np.ndarray, nu: np.ndarray, c: float, K: float, psi, psi_hat) -> np.ndarray:
    """Algorithm 1: the DFT of ``gvec`` at the nodes ``nu`` (time-index units)."""
    g = np.asarray(gvec, dtype=np.complex128)
    nt = g.shape[0]
    M = _padded_length(c, nt)
    theta = 2.0 * math.pi * np.arange(nt) / nt - math.pi
    G = np.fft.fft(g / psi(theta), n=M) / (2.0 * math.pi * c)
    nu = np.asarray(nu, dtype=np.float64)
    x = c * nu
    span = c * K
    lo = np.ceil(x - span - 1e-12).astype(np.int64)
    count = int(math.floor(2.0 * span)) + 2
    out = np.zeros(nu.shape, np.complex128)
    for t in range(count):
        j = lo + t
        keep = np.abs(j - x) <= span
        u = nu - j / c
        term = np.exp(-1j * math.pi * u) * psi_hat(u) * G[j % M]
        out += np.where(keep, term, 0.0)
    return out


def evaluate(gvec: np.ndarray, nu: np.ndarray, method: str, c: float = 2.0, K: float = 3.0,
             alpha: float | None = None) -> np.ndarray:
    """D(nu) of one row by ``method`` (see the module docstring)."""
    nt = np.asarray(gvec).shape[0]
    if method in ("nearest", "linear"):
        return interpolate(grid_dft(gvec, _padded_length(c, nt)), nu, c, method)
    if method == "tsinc":
        psi, psi_hat = indicator_window(c)
        return nufft(gvec, nu, c, K, psi, psi_hat)
    if method == "kb":
        a = alpha if alpha else math.pi * (2.0 * c - 1.0) * (1.0 - 1e-3)
        psi, psi_hat = kb_window(a, K)
        return nufft(gvec, nu, c, K, psi, psi_hat)
    raise ValueError(f"unknown method {method!r}")


# ---------------------------------------------------------------------------
# the whole reconstruction with a given evaluation method
# ---------------------------------------------------------------------------

def _signed(i: int, n: int) -> int:
    return i if i < n // 2 else i - n


def spectrum(g, p: np.ndarray, method: str, c: float = 2.0, K: float = 3.0, alpha: float | None = None,
             nthreads: int = 0) -> np.ndarray:
    """Weighted image spectrum fhat[kx][(ky)][l] (storage index l mod nz) with the
    temporal DFT evaluated at the nodes by ``method``."""
    gg = _geom(g)
    pt = lateral_dft(g, p, nthreads).reshape(gg.nx * gg.ny, gg.nt)
    out = np.empty((gg.nx * gg.ny, gg.nz), np.complex128)
    for row in range(gg.nx * gg.ny):
        kx = _signed(row // gg.ny, gg.nx)
        ky = _signed(row % gg.ny, gg.ny)
        nu, w = row_nodes(g, kx, ky)
        out[row] = w * evaluate(pt[row], nu, method, c, K, alpha)
    shape = (gg.nx, gg.nz) if gg.dim == 2 else (gg.nx, gg.ny, gg.nz)
    return out.reshape(shape)


def reconstruct(g, p: np.ndarray, method: str, c: float = 2.0, K: float = 3.0, alpha: float | None = None,
                nthreads: int = 0) -> np.ndarray:
    """Fourier reconstruction with the temporal DFT evaluated by ``method``."""
    return image_from_spectrum(g, spectrum(g, p, method, c, K, alpha, nthreads), nthreads)


def half_pixel_margin(g, c: float) -> float:
    """Smallest distance of c nu to a half integer over all nodes: the nearest-neighbour
    choice is decided identically in any precision finer than this margin."""
    gg = _geom(g)
    best = np.inf
    for row in range(gg.nx * gg.ny):
        nu, _ = row_nodes(g, _signed(row // gg.ny, gg.nx), _signed(row % gg.ny, gg.ny))
        x = c * nu
        best = min(best, float(np.min(np.abs(x - np.floor(x) - 0.5))))
    return best
