"""Pins of the FP64 oracle of the compared Fourier algorithms (Sec. 4).

Each pin checks the oracle against something it does not compute itself:
the direct DFT (``oracle.nudft``, pinned in test_oracle_pins.py) at grid
nodes and between them, quadrature of the windows' Fourier integrals,
the 1/K decay of the sinc tail, and the error ordering of Table 1 against
the direct reconstruction.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.methods as om
import phantoms as ph


def _vec(nt=64, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(nt) + 1j * rng.standard_normal(nt)


def _err(v, ref, g):
    return float(np.max(np.abs(v - ref)) / np.sum(np.abs(g)))


@pytest.mark.parametrize("c", [1.0, 2.0])
@pytest.mark.parametrize("method", ["linear", "nearest", "tsinc"])
def test_exact_on_grid_nodes(method, c):
    """On the grid nu = j/c every method returns the DFT itself: the
    interpolation weights collapse to one grid value, and the sinc vanishes at
    every other integer.  Negative j and j beyond one period check the wrap
    modulo M, the phase e^{-i pi (nu - j/c)} and the constant 1/(2 pi c) (the
    printed c/(2 pi) would scale every value by c^2)."""
    if method == "tsinc" and c == 1.0:
        pytest.skip("Algorithm 1 needs c > 1")
    g = _vec()
    M = int(c * g.size)
    js = np.array([-3 * M - 1, -M, -5, -1, 0, 1, 7, M // 2, M - 1, M, 2 * M + 3])
    nu = js / c
    assert _err(om.evaluate(g, nu, method, c), oracle.nudft(g, nu), g) < 1e-13


@pytest.mark.parametrize("c", [1.0, 2.0])
def test_linear_between_grid_nodes(c):
    """Off the grid, linear interpolation is (1 - f) D(j/c) + f D((j+1)/c) of
    the direct DFT's values, including across the period boundary j = M - 1."""
    g = _vec(seed=1)
    M = int(c * g.size)
    for j in (-7, -1, 0, 5, M - 1, M + 2):
        for f in (0.25, 0.5, 0.9):
            nu = np.array([(j + f) / c])
            ref = (1 - f) * oracle.nudft(g, np.array([j / c])) + f * oracle.nudft(g, np.array([(j + 1) / c]))
            assert _err(om.evaluate(g, nu, "linear", c), ref, g) < 1e-13


@pytest.mark.parametrize("c", [1.0, 2.0])
def test_nearest_picks_the_closer_grid_node(c):
    g = _vec(seed=2)
    M = int(c * g.size)
    for j in (-9, -1, 0, 3, M - 1):
        for f, pick in ((0.2, j), (0.49, j), (0.5, j + 1), (0.51, j + 1), (0.8, j + 1)):
            v = om.evaluate(g, np.array([(j + f) / c]), "nearest", c)
            assert _err(v, oracle.nudft(g, np.array([pick / c])), g) < 1e-13


def test_kb_window_transform_is_its_fourier_integral():
    """Psi_hat_KB of Sec. 3.2 equals the integral of Psi_KB e^{-i w theta}
    (Psi is even and real, so the cosine integral), inside and outside
    [-K, K] and at |w| = K."""
    quad = pytest.importorskip("scipy.integrate").quad
    alpha, K = 3.0 * math.pi, 3.0
    psi, psi_hat = om.kb_window(alpha, K)
    for w in (0.0, 0.7, 2.5, 3.0, 3.4, 6.1):
        val, _ = quad(lambda t: float(psi(t)) * math.cos(w * t), -alpha, alpha, limit=400, epsabs=1e-13)
        assert abs(float(psi_hat(np.array([w]))[0]) - val) <= 1e-9 * abs(float(psi_hat(np.array([0.0]))[0]))


def test_indicator_window_transform_is_its_fourier_integral():
    quad = pytest.importorskip("scipy.integrate").quad
    c = 2.0
    psi, psi_hat = om.indicator_window(c)
    assert float(psi(np.array([math.pi]))[0]) == 1.0 and float(psi(np.array([-c * math.pi]))[0]) == 1.0
    for w in (0.0, 0.3, 1.0, 1.75, 4.2):
        val, _ = quad(lambda t: math.cos(w * t), -c * math.pi, c * math.pi, limit=200, epsabs=1e-13)
        assert abs(float(psi_hat(np.array([w]))[0]) - val) < 1e-10


def test_kb_algorithm1_reaches_the_direct_dft():
    """Algorithm 1 with the Kaiser-Bessel window (c = 2, K = 3) is the exact DFT
    up to the window's truncation error (Sec. 3.1 / 3.2: |Psi_hat(K)/Psi_hat(0)| ~ 3e-11
    for alpha = 3 pi)."""
    g = _vec(seed=3)
    nu = np.random.default_rng(4).uniform(-90, 90, 300)
    ref = oracle.nudft(g, nu)
    assert _err(om.evaluate(g, nu, "kb", 2.0, 3.0), ref, g) < 1e-10
    assert _err(om.evaluate(g, nu, "kb", 2.0, 3.0, alpha=3.0 * math.pi), ref, g) < 1e-9


def test_truncated_sinc_error_decays_like_one_over_K():
    """The sinc tail decays like 1/|w| (Remark on Shannon's formula): each
    fourfold K cuts the truncation error by roughly four, and at K = 3 it is far
    above the Kaiser-Bessel error."""
    g = _vec(seed=5)
    nu = np.random.default_rng(6).uniform(-80, 80, 300)
    ref = oracle.nudft(g, nu)
    errs = [_err(om.evaluate(g, nu, "tsinc", 2.0, K), ref, g) for K in (4.0, 16.0, 64.0)]
    assert errs[0] > 2.5 * errs[1] > 0 and errs[1] > 2.5 * errs[2] > 0
    assert errs[0] < 0.05
    assert _err(om.evaluate(g, nu, "tsinc", 2.0, 3.0), ref, g) > 1e4 * _err(om.evaluate(g, nu, "kb", 2.0, 3.0), ref, g)


def test_interpolation_error_shrinks_with_oversampling():
    """Interpolating the grid values of a smooth spectrum: linear error ~ (1/c)^2,
    nearest ~ 1/c.  A short pulse has a smooth DFT, so going from c = 1 to c = 4
    must cut both errors substantially."""
    nt = 64
    g = np.zeros(nt, np.complex128)
    g[:6] = np.hanning(8)[1:7]
    nu = np.random.default_rng(7).uniform(-30, 30, 400)
    ref = oracle.nudft(g, nu)
    e = {(m, c): _err(om.evaluate(g, nu, m, c), ref, g) for m in ("linear", "nearest") for c in (1.0, 4.0)}
    assert e[("linear", 4.0)] < e[("linear", 1.0)] / 8
    assert e[("nearest", 4.0)] < e[("nearest", 1.0)] / 2.5
    assert e[("linear", 1.0)] < e[("nearest", 1.0)]


def test_table1_error_ordering():
    """Table 1: against the direct reconstruction the errors order as
    Kaiser-Bessel < truncated sinc < linear (c=2) < nearest (c=2) < linear (c=1) <
    nearest (c=1).  f_circ discs (Sec. 5.1), closed-form data, N = 256."""
    N = 256
    pr = ph.fcirc_problem_2d(1, N, 2 * N, N, 3, rmin=N / 32, rmax=N / 8)
    ref = oracle.reconstruct(pr.geom, pr.p)
    order = [("kb", 2.0), ("tsinc", 2.0), ("linear", 2.0), ("nearest", 2.0), ("linear", 1.0), ("nearest", 1.0)]
    errs = []
    for m, c in order:
        f = om.reconstruct(pr.geom, pr.p, m, c)
        errs.append(float(np.linalg.norm(f - ref) / np.linalg.norm(ref)))
    assert errs[0] < 1e-8, errs
    assert all(a < b for a, b in zip(errs, errs[1:])), errs
    # the paper's magnitudes for the interpolation variants are tenths; the sinc hundredths
    assert 0.005 < errs[1] < 0.1 and errs[5] > 0.2, errs


def test_row_nodes_are_the_pinned_node_and_weight():
    g = ph.Geometry(dim=3, nx=8, ny=6, nt=16, nz=10, dx=0.9, dy=1.1, dt=0.7, c=1.3, dz=1.2)
    for kx, ky in ((0, 0), (3, -2), (-4, 1)):
        nu, w = oracle.row_nodes(g, kx, ky)
        for li in range(g.nz):
            l = li if li < g.nz // 2 else li - g.nz
            assert nu[li] == oracle.node(g, kx, ky, l) and w[li] == oracle.weight(g, kx, ky, l)
