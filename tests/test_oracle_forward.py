"""Pins of the FP64 oracle of the discrete forward model (the operator Q of
Sec. 2 on a zero-padded periodic box).

Pinned against: an independent implementation of the same spectral
propagator (phantoms.spectral_2d: library FFTs and per-time cosine sums), the
initial condition at t = 0 (the data equal the image's depth-0 layer), and the
closed-form N-shaped pressure of a smooth ball in 3-D (wave equation, radial
solution), which the discrete model must approach as the ball is resolved.
"""
import numpy as np
import pytest

import oracle
import phantoms as ph


def test_box_rule():
    g = ph.Geometry(dim=2, nx=32, nt=64, nz=24)
    assert oracle.forward_box(g) == (128, 1, 128)  # 32 + 64 + 2 -> 128; 24 + 64 + 2 -> 128
    g = ph.Geometry(dim=3, nx=20, ny=12, nt=16, nz=10, dx=2.0, dy=0.5, dt=1.0, c=1.0, dz=1.0)
    assert oracle.forward_box(g) == (32, 64, 32)   # 20+8+2, 12+32+2, 10+16+2


@pytest.mark.parametrize("shape", [(32, 64, 24), (40, 48, 40)])
def test_2d_equals_independent_spectral_propagator(shape):
    nx, nt, nz = shape
    g = ph.Geometry(dim=2, nx=nx, nt=nt, nz=nz)
    img = np.random.default_rng(3).standard_normal(g.image_shape)
    box = oracle.forward_box(g)
    got = oracle.forward_model(g, img, box)
    ref = ph.spectral_2d(g, img, box=(box[0], box[2]))
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("g", [ph.Geometry(dim=2, nx=24, nt=40, nz=16, dx=0.8, dt=0.5, c=1.3, dz=1.1),
                               ph.Geometry(dim=3, nx=12, ny=10, nt=20, nz=8, dx=0.9, dy=1.1, dt=0.7, c=1.3, dz=1.2)],
                         ids=["2d", "3d"])
def test_initial_condition(g):
    """At t = 0 the pressure is the initial pressure: the data's first sample is
    the image's depth-0 layer (the detectors sit at depth 0)."""
    img = np.random.default_rng(4).standard_normal(g.image_shape)
    p = oracle.forward_model(g, img)
    assert np.max(np.abs(p[..., 0] - img[..., 0])) <= 1e-12 * np.max(np.abs(img))


def test_3d_smooth_ball_approaches_the_closed_form():
    """Smooth balls (1 - s^2/R^2)^2: the model's data against the exact radial
    solution p = (r - ct) f(|r - ct|) / (2r).  The difference is the
    trigonometric interpolation error of the sampled ball: below 1 % and falling
    as the ball is resolved by more cells (R = 5, 7, 9: measured 0.93 %, 0.42 %,
    0.23 %)."""
    g = ph.Geometry(dim=3, nx=32, ny=32, nt=48, nz=32)
    errs = []
    for R in (5.0, 7.0, 9.0):
        balls = [(15.3, 16.1, 7.2 + R, R, 1.0)]
        img = ph.balls_3d_image(g, balls, smooth=True)
        ref = ph.balls_3d(g, balls, smooth=True, cell_average=False)
        got = oracle.forward_model(g, img)
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert errs[0] < 1.5e-2 and errs[2] < errs[1] < errs[0], errs
