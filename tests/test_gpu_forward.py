"""The discrete forward model on the GPU (pai_forward_plan / pai_forward_model)
against its FP64 oracle (oracle.forward_model): relative L2 <= 1e-5."""
import numpy as np
import pytest

import oracle
import phantoms as ph
from gpu_common import TOL, gdict, pai, rel, to_gpu, to_np  # noqa: F401

pytestmark = pytest.mark.gpu

CASES = [
    ph.Geometry(dim=2, nx=32, nt=64, nz=24),
    ph.Geometry(dim=2, nx=50, nt=90, nz=36, dx=0.8, dt=0.5, c=1.3, dz=1.1),
    ph.Geometry(dim=2, nx=128, nt=256, nz=128),
    ph.Geometry(dim=3, nx=12, ny=10, nt=20, nz=8, dx=0.9, dy=1.1, dt=0.7, c=1.3, dz=1.2),
    ph.Geometry(dim=3, nx=24, ny=16, nt=32, nz=20),
]


@pytest.mark.parametrize("g", CASES, ids=lambda g: f"{g.dim}d-{g.nx}x{g.ny}x{g.nt}-{g.nz}")
def test_forward_model_against_oracle(pai, g):
    model = pai.ForwardModel(gdict(g, K=3))
    assert model.box == oracle.forward_box(g)
    img = ph.random_image(90, g).astype(np.float32)
    got = to_np(model(to_gpu(img)))
    ref = oracle.forward_model(g, img.astype(np.float64))
    assert rel(got, ref) < TOL


def test_forward_model_ball_and_reconstruction(pai):
    """3-D smooth ball: the GPU model's data approach the closed-form pressure
    like the oracle's, and reconstructing them returns the ball's lateral
    position and depth (the limited-view reconstruction is blurred and loses
    each column's depth mean, so the check is the location of the maximum,
    within one cell)."""
    g = ph.Geometry(dim=3, nx=32, ny=32, nt=64, nz=32)
    balls = [(15.0, 16.0, 14.0, 7.0, 1.0)]
    img = ph.balls_3d_image(g, balls, smooth=True).astype(np.float32)
    model = pai.ForwardModel(gdict(g, K=3))
    data = to_np(model(to_gpu(img)))
    ref = ph.balls_3d(g, balls, smooth=True, cell_average=False)
    assert rel(data, ref) < 1.5e-2
    f = to_np(pai.Plan(gdict(g, K=3)).reconstruct(to_gpu(data)))
    peak = np.array(np.unravel_index(np.argmax(f), f.shape))
    assert np.all(np.abs(peak - np.array([15, 16, 14])) <= 1), peak


def test_forward_plan_rejects_other_calls(pai):
    import torch
    g = ph.Geometry(dim=2, nx=32, nt=64, nz=24)
    model = pai.ForwardModel(gdict(g))
    x = torch.zeros(32 * 64, device="cuda")
    y = torch.zeros(32 * 24, device="cuda")
    lib = pai.load_library()
    import ctypes
    assert lib.pai_reconstruct(model._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())) == 1
    assert lib.pai_adjoint(model._h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr())) == 1
    with pytest.raises(pai.PAIError):
        pai.ForwardModel(gdict(g, method="linear"))


@pytest.mark.parametrize("seed", range(6))
def test_forward_model_random_geometries(pai, seed):
    """Seeded random geometries (boxes kept at most 128 per axis) against the oracle."""
    rng = np.random.default_rng(700 + seed)
    dim = int(rng.integers(2, 4))
    even = lambda lo, hi: 2 * int(rng.integers(lo // 2, hi // 2 + 1))  # noqa: E731
    nx, ny = (even(2, 48), 1) if dim == 2 else (even(2, 16), even(2, 16))
    dx, dz, dt = (float(rng.uniform(0.8, 1.5)) for _ in range(3))
    c = float(rng.uniform(0.5, 1.0))
    g = ph.Geometry(dim=dim, nx=nx, ny=ny, nt=even(2, 48), nz=even(2, 40), dx=dx, dy=dx, dt=dt, c=c, dz=dz)
    model = pai.ForwardModel(gdict(g, K=3))
    assert max(model.box) <= 128, model.box
    img = ph.random_image(710 + seed, g).astype(np.float32)
    got = to_np(model(to_gpu(img)))
    assert rel(got, oracle.forward_model(g, img.astype(np.float64))) < TOL, g
