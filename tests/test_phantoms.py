"""Checks of the seeded input generators (forward physics only)."""
import numpy as np

import phantoms as ph


def test_fcirc_closed_form_matches_spectral_propagator():
    """Two independent forward models of the paper's circular object agree:
    the closed form (descent from the 3-D ball) and exact spectral propagation
    of the sampled image; the gap shrinks with the radius (sampling of the
    sqrt edge)."""
    errs = []
    for a in (10.0, 20.0):
        g = ph.Geometry(dim=2, nx=128, nt=256, nz=128)
        discs = [(64.0, 50.0, a, 1.0)]
        p1 = ph.fcirc_2d(g, discs)
        p2 = ph.spectral_2d(g, ph.fcirc_2d_image(g, discs))
        errs.append(np.linalg.norm(p1 - p2) / np.linalg.norm(p1))
    assert errs[0] < 0.06 and errs[1] < errs[0] and errs[1] < 0.03


def test_uniform_ball_cell_average_matches_point_samples_on_average():
    g = ph.Geometry(dim=3, nx=8, ny=8, nt=400, nz=16, dt=0.25)
    balls = [(4.0, 4.0, 30.0, 5.0, 1.0)]
    pa = ph.balls_3d(g, balls, cell_average=True)
    pp = ph.balls_3d(g, balls, cell_average=False)
    # the N-wave integrates to zero over time; both samplings preserve that
    assert abs(pa.sum()) < 1e-9 * np.abs(pa).sum()
    assert np.linalg.norm(pa - pp) / np.linalg.norm(pp) < 0.15


def test_generators_are_seeded_and_shaped():
    a = ph.plain_2d(3)
    b = ph.plain_2d(3)
    assert a.p.shape == (128, 256) and np.array_equal(a.p, b.p)
    c = ph.planar_3d(1, n=32, nt=64, nz=32)
    assert c.p.shape == (32, 32, 64)
    geoms = ph.batched_2d_geometries(0)
    assert len(geoms) == 64
    for g in geoms:
        assert g.nx % 2 == 0 and g.nt % 2 == 0 and g.nz % 2 == 0
        assert 256 <= g.nx <= 2048 and 512 <= g.nt <= 4096
