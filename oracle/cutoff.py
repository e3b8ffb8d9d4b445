"""FP64 oracle of the smooth data cutoff w_cut (Eq. data-part of Sec. 2, built as in Sec. 5).

TEST INFRASTRUCTURE ONLY, under the same rule as the rest of ``oracle/``:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may use it, and it never imports the CUDA library.

Partial (limited-view) data are modelled as g = w_cut * (Q f): the complete
data multiplied by a smooth nonnegative cutoff that is one well inside the
measured region and falls to zero at its edges.  Sec. 5 builds w_cut as the
convolution of a compactly supported mollifier phi_eps with the indicator of
the measurement box.

Readings (Sec. 5 prints phi_eps(x, t) = C exp(-1 / (eps - x^2 - t^2)^4) on
x^2 + t^2 < eps, with eps "a small multiple of the sampling step"):

* coordinates are measured in sampling steps along every data axis (the
  lateral axes in units of dx (dy), time in units of dt), so the box of the
  data grid [nx] ([ny]) [nt] is [0, n_a] on axis a: the samples sit at
  0 .. n_a - 1 inside (0, X) with X = n_a steps;
* the mollifier keeps the printed support |v|^2 < eps and exponent 4 but is
  written in the scale-free form phi_eps(v) = C exp(-1 / (1 - |v|^2/eps)^4).
  The printed form is not scale invariant: with the paper's X = 1 and
  eps ~ 4 / N it is a point mass (w_cut would be the hard indicator), and in
  sample units with eps >> 1 it is a flat disc with a knife edge.  The
  scale-free form is the same smooth bump at every eps; C makes its
  integral one;
* w_cut(u) = integral of phi_eps(v) chi_box(u - v) dv, evaluated at the
  sample positions u in R^d (d = 2: (x, t); d = 3: (x, y, t)).

The integral is a tensor Gauss-Legendre rule over the cube of v allowed by
the box, intersected with [-sqrt eps, sqrt eps]^d; phi_eps is smooth on R^d
(all derivatives vanish on the sphere), so the rule converges fast.  The
weight is that integral divided by the same rule over the full cube.
"""
from __future__ import annotations

import functools
import math

import numpy as np

QUAD_POINTS = 64


def bump(r2: np.ndarray, eps: float) -> np.ndarray:
    """exp(-1 / (1 - r^2/eps)^4) for r^2 < eps, zero elsewhere (unnormalised phi_eps)."""
    r2 = np.asarray(r2, dtype=np.float64)
    out = np.zeros_like(r2)
    m = r2 < eps
    out[m] = np.exp(-1.0 / (1.0 - r2[m] / eps) ** 4)
    return out


@functools.lru_cache(maxsize=None)
def _rule(n: int):
    return np.polynomial.legendre.leggauss(n)


def box_integral(lo, hi, eps: float, n: int = QUAD_POINTS) -> float:
    """Integral of the unnormalised bump over the box prod_a [lo_a, hi_a] (tensor Gauss-Legendre)."""
    x, w = _rule(n)
    r = math.sqrt(eps)
    axes, weights = [], []
    for a, b in zip(lo, hi):
        a, b = max(a, -r), min(b, r)
        if b <= a:
            return 0.0
        axes.append(0.5 * (b - a) * x + 0.5 * (b + a))
        weights.append(0.5 * (b - a) * w)
    grids = np.meshgrid(*axes, indexing="ij")
    r2 = sum(g * g for g in grids)
    f = bump(r2, eps)
    for wa in reversed(weights):
        f = f @ wa
    return float(f)


def normaliser(eps: float, dim: int, n: int = QUAD_POINTS) -> float:
    """1 / C_eps: the bump's integral over R^dim."""
    r = math.sqrt(eps)
    return box_integral([-r] * dim, [r] * dim, eps, n)


def weight_at(u, sizes, eps: float, n: int = QUAD_POINTS) -> float:
    """w_cut at the (real) position u for the box prod_a [0, sizes_a].

    chi_box(u - v) = 1  <=>  0 <= u_a - v_a <= n_a  <=>  u_a - n_a <= v_a <= u_a.
    """
    lo = [ua - na for ua, na in zip(u, sizes)]
    hi = list(u)
    return box_integral(lo, hi, eps, n) / normaliser(eps, len(sizes), n)


def weights(shape, eps: float, n: int = QUAD_POINTS) -> np.ndarray:
    """w_cut at every sample of a data grid ``shape`` = (nx, nt) or (nx, ny, nt).

    Integrals over the same clipped box are evaluated once (lru cache on the
    box bounds); every sample still gets the integral over its own box.
    """
    r = math.sqrt(eps)
    dim = len(shape)
    norm = normaliser(eps, dim, n)

    @functools.lru_cache(maxsize=None)
    def integral(bounds):
        return box_integral([b[0] for b in bounds], [b[1] for b in bounds], eps, n)

    def clip(ua, na):
        return (max(ua - na, -r), min(ua, r))

    out = np.empty(shape, np.float64)
    for idx in np.ndindex(*shape):
        out[idx] = integral(tuple(clip(float(i), float(s)) for i, s in zip(idx, shape))) / norm
    return out


def apply(p: np.ndarray, eps: float, n: int = QUAD_POINTS) -> np.ndarray:
    """g = w_cut * p for data p of shape (nx, nt) or (nx, ny, nt) (Eq. data-part)."""
    p = np.asarray(p, dtype=np.float64)
    return p * weights(p.shape, eps, n)
