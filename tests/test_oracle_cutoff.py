"""Pins of the FP64 oracle of the data cutoff w_cut (oracle/cutoff.py; Eq. data-part, Sec. 5).

Each pin checks the oracle's tensor Gauss-Legendre integrals against a route it
does not take: the bump's radial integral (scipy quad in polar / spherical
coordinates), the closed-form arc and spherical-cap fractions for one face, a
dense sampling of the angle inside a corner, and the values that the symmetry of
the bump fixes exactly (1/2 on a face, 1/4 and 1/8 in corners, F(s) + F(-s) = 1).
"""
import math

import numpy as np
import pytest

import oracle.cutoff as oc

quad = pytest.importorskip("scipy.integrate").quad


def _radial(eps, dim, extra=lambda r: 1.0):
    """Integral of bump(r^2) * surface(r) * extra(r) dr over [0, sqrt eps]."""
    surf = (lambda r: 2.0 * math.pi * r) if dim == 2 else (lambda r: 4.0 * math.pi * r * r)
    val, _ = quad(lambda r: float(oc.bump(np.array([r * r]), eps)[0]) * surf(r) * extra(r), 0.0, math.sqrt(eps),
                  epsabs=0.0, epsrel=1e-13, limit=400)
    return val


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("eps", [1.0, 16.0, 100.0])
def test_normaliser_is_the_radial_integral(eps, dim):
    assert abs(oc.normaliser(eps, dim) / _radial(eps, dim) - 1.0) < 1e-10


def test_bump_support_and_scale():
    """phi_eps vanishes for |v|^2 >= eps, peaks at exp(-1) at 0, and its shape
    depends on |v|^2/eps only."""
    assert oc.bump(np.array([0.0]), 9.0)[0] == pytest.approx(math.exp(-1.0), rel=1e-15)
    assert oc.bump(np.array([9.0, 9.5]), 9.0).tolist() == [0.0, 0.0]
    # the printed exponent 4: at |v|^2 = eps/2 the bump is exp(-2^4)
    assert oc.bump(np.array([4.5]), 9.0)[0] == pytest.approx(math.exp(-16.0), rel=1e-14)
    r2 = np.linspace(0, 0.99, 23)
    assert np.allclose(oc.bump(r2 * 4.0, 4.0), oc.bump(r2 * 49.0, 49.0), rtol=1e-14, atol=0)


def test_interior_is_one_and_faces_are_halves_2d():
    shape = (24, 40)
    w = oc.weights(shape, 16.0)
    assert abs(w[10, 20] - 1.0) < 1e-13
    assert abs(w[0, 20] - 0.5) < 1e-11 and abs(w[10, 0] - 0.5) < 1e-11
    assert abs(w[0, 0] - 0.25) < 1e-11
    # the box is [0, n]: the last sample is one step from the upper face, like sample 1 from the lower one
    assert abs(w[23, 20] - w[1, 20]) < 1e-13 and abs(w[10, 39] - w[10, 1]) < 1e-13
    assert abs(oc.weight_at((24.0, 20.0), shape, 16.0) - 0.5) < 1e-11
    assert np.all(w > 0) and np.all(w <= 1.0 + 1e-11)


def test_corners_and_edges_3d():
    shape = (10, 12, 20)
    eps = 9.0
    assert abs(oc.weight_at((0.0, 0.0, 0.0), shape, eps) - 0.125) < 1e-11
    assert abs(oc.weight_at((0.0, 6.0, 0.0), shape, eps) - 0.25) < 1e-11
    assert abs(oc.weight_at((5.0, 12.0, 10.0), shape, eps) - 0.5) < 1e-11
    assert abs(oc.weight_at((5.0, 6.0, 10.0), shape, eps) - 1.0) < 1e-13


@pytest.mark.parametrize("s", [0.3, 1.0, 2.5, 3.7])
def test_one_face_is_the_arc_fraction_2d(s):
    """Distance s to one face: polar form, the arc of radius r outside the
    half-plane v_1 > s has angle 2 arccos(s/r) for r > s."""
    eps = 16.0
    frac = lambda r: 1.0 - (math.acos(s / r) / math.pi if r > s else 0.0)
    ref = _radial(eps, 2, frac) / _radial(eps, 2)
    got = oc.weight_at((s, 30.0), (60, 60), eps)
    assert abs(got - ref) < 1e-9


@pytest.mark.parametrize("s", [0.4, 1.5, 2.9])
def test_one_face_is_the_cap_fraction_3d(s):
    """Spherical shells: the cap beyond the plane at distance s < r has area 2 pi r (r - s)."""
    eps = 9.0
    frac = lambda r: 1.0 - ((r - s) / (2.0 * r) if r > s else 0.0)
    ref = _radial(eps, 3, frac) / _radial(eps, 3)
    got = oc.weight_at((20.0, s, 20.0), (40, 40, 40), eps)
    assert abs(got - ref) < 1e-9


@pytest.mark.parametrize("s", [0.2, 1.3, 3.1])
def test_reflection_sums_to_one(s):
    """F(s) + F(-s) = 1: the bump is even, so the parts of it on either side of a face add up."""
    eps = 16.0
    a = oc.weight_at((s, 30.0), (60, 60), eps)
    b = oc.weight_at((-s, 30.0), (60, 60), eps)
    assert abs(a + b - 1.0) < 1e-11


def test_corner_against_sampled_angles_2d():
    """Near a corner (distances s1, s2 to two faces): polar form with the angle
    inside the quadrant {v_1 <= s1, v_2 <= s2} measured by dense sampling of the
    circle (midpoint rule, so only about 1e-5 accurate)."""
    eps, s1, s2 = 16.0, 1.2, 2.3
    th = (np.arange(200000) + 0.5) * (2.0 * math.pi / 200000)
    c, sn = np.cos(th), np.sin(th)
    frac = lambda r: float(np.mean((r * c <= s1) & (r * sn <= s2)))
    ref = _radial(eps, 2, frac) / _radial(eps, 2)
    got = oc.weight_at((s1, s2), (50, 50), eps)
    assert abs(got - ref) < 5e-5


def test_weight_grows_with_the_distance_to_the_face():
    w = oc.weights((30, 12), 25.0)[:, 6]
    assert np.all(np.diff(w[:15]) >= -1e-11) and w[5] == pytest.approx(1.0, abs=1e-13)
    assert w[0] == pytest.approx(0.5, abs=1e-11)


def test_apply_multiplies_the_data():
    rng = np.random.default_rng(3)
    p = rng.standard_normal((16, 20))
    assert np.array_equal(oc.apply(p, 4.0), p * oc.weights(p.shape, 4.0))
