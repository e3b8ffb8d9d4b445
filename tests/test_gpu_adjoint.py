"""The GPU adjoint (pai_adjoint) and the autograd wrapper.

Checks: the dot-product identity <R p, h> = <p, R^T h> between the GPU
forward and the GPU adjoint (1e-6), the GPU adjoint against the oracle's exact
transpose (1e-5), gradients through PAIRecon against R^T(R p - f) and against
central finite differences."""
import numpy as np
import pytest

import oracle
import phantoms as ph
from gpu_common import DOT_TOL, TOL, gdict, pai, pipeline, rel, to_gpu, to_np  # noqa: F401

pytestmark = pytest.mark.gpu

CASES = [
    ph.Geometry(dim=2, nx=128, nt=256, nz=128),
    ph.Geometry(dim=2, nx=300, nt=700, nz=350, dx=1.0, dt=0.5, c=1.5, dz=0.8),
    ph.Geometry(dim=2, nx=6, nt=10, nz=4),
    ph.Geometry(dim=3, nx=20, ny=12, nt=48, nz=18, dx=0.9, dy=1.1, dt=0.7, c=1.3, dz=1.0),
    ph.Geometry(dim=3, nx=32, ny=32, nt=64, nz=32),
    ph.Geometry(dim=3, nx=64, ny=32, nt=128, nz=64, dy=1.2),
    ph.Geometry(dim=2, nx=256, nt=512, nz=256, dz=0.8),
    ph.Geometry(dim=2, nx=8, nt=8192, nz=64, dt=0.25),  # the largest padded length, M = 16384
]


@pytest.mark.parametrize("g", CASES, ids=lambda g: f"{g.dim}d-{g.nx}x{g.ny}x{g.nt}-{g.nz}")
def test_dot_product_identity(pai, g, pipeline):
    plan = pai.Plan(gdict(g, K=3))
    p = ph.random_data(50, g)
    h = ph.random_image(51, g)
    Rp = to_np(plan.reconstruct(to_gpu(p)))
    Rth = to_np(plan.adjoint(to_gpu(h)))
    p32 = p.astype(np.float32).astype(np.float64)
    h32 = h.astype(np.float32).astype(np.float64)
    lhs = float(np.vdot(Rp, h32))
    rhs = float(np.vdot(p32, Rth))
    scale = np.linalg.norm(Rp) * np.linalg.norm(h32)
    assert abs(lhs - rhs) < DOT_TOL * scale


@pytest.mark.parametrize("g", CASES, ids=lambda g: f"{g.dim}d-{g.nx}x{g.ny}x{g.nt}-{g.nz}")
def test_adjoint_against_oracle(pai, g, pipeline):
    plan = pai.Plan(gdict(g, K=3))
    h = ph.random_image(52, g).astype(np.float32)
    got = to_np(plan.adjoint(to_gpu(h)))
    ref = oracle.adjoint(g, h.astype(np.float64))
    assert rel(got, ref) < TOL


def test_adjoint_batched(pai, pipeline):
    geoms = [ph.Geometry(dim=2, nx=64, nt=130, nz=64), ph.Geometry(dim=2, nx=36, nt=512, nz=100),
             ph.Geometry(dim=3, nx=10, ny=8, nt=40, nz=16)]
    plan = pai.Plan([gdict(g, K=3) for g in geoms])
    hs = [ph.random_image(60 + i, g).astype(np.float32) for i, g in enumerate(geoms)]
    out = to_np(plan.adjoint(to_gpu(np.concatenate([h.ravel() for h in hs]))))
    off = 0
    for g, h in zip(geoms, hs):
        n = g.nx * g.ny * g.nt
        assert rel(out[off: off + n].reshape(g.data_shape), oracle.adjoint(g, h.astype(np.float64))) < TOL
        off += n


def test_autograd_gradient_is_adjoint_of_residual(pai):
    import torch
    g = ph.Geometry(dim=3, nx=24, ny=24, nt=48, nz=24)
    prob_p = ph.random_data(70, g)
    f_true = ph.random_image(71, g)
    plan = pai.Plan(gdict(g, K=3))
    p = to_gpu(prob_p).requires_grad_(True)
    ft = to_gpu(f_true)
    loss = 0.5 * ((pai.PAIRecon.apply(p, plan) - ft) ** 2).sum()
    loss.backward()
    with torch.no_grad():
        expect = plan.adjoint(plan.reconstruct(p.detach()) - ft)
    torch.cuda.synchronize()
    assert rel(to_np(p.grad), to_np(expect)) < 1e-6


@pytest.mark.parametrize("step,tol", [(1e-3, 5e-2), (1.0, 1e-4)])
def test_finite_differences(pai, step, tol):
    """Central differences at 32 random coordinates of p for the loss
    0.5 ||R p - f||^2, evaluated in FP64 from FP32 reconstructions as
    <a-b, (a+b)/2 - f>.  The loss is quadratic, so the central difference is
    exact at any step and only FP32 rounding separates it from the gradient:
    with step 1e-3 that rounding noise (~1e-7 of |R p| divided by the step)
    is a few percent, with step 1 it is ~1e-5."""
    g = ph.Geometry(dim=3, nx=24, ny=24, nt=48, nz=24)
    plan = pai.Plan(gdict(g, K=3))
    p0 = ph.random_data(72, g).astype(np.float32)
    f_true = ph.random_image(73, g)
    pt = to_gpu(p0).requires_grad_(True)
    loss = 0.5 * ((pai.PAIRecon.apply(pt, plan) - to_gpu(f_true)) ** 2).sum()
    loss.backward()
    grad = to_np(pt.grad).ravel()
    rng = np.random.default_rng(0)
    idx = rng.choice(p0.size, 32, replace=False)
    fd = []
    for i in idx:
        a = p0.ravel().copy()
        b = p0.ravel().copy()
        a[i] += step
        b[i] -= step
        ra = to_np(plan.reconstruct(to_gpu(a.reshape(g.data_shape)))).ravel()
        rb = to_np(plan.reconstruct(to_gpu(b.reshape(g.data_shape)))).ravel()
        d = ra - rb
        fd.append(np.dot(d, 0.5 * (ra + rb) - f_true.ravel()) / (2 * step))
    fd = np.array(fd)
    assert rel(fd, grad[idx]) < tol


def test_adjoint_3d_full_size(pai):
    """The 3-D adjoint workload at full size (256 x 256 detectors x 512 samples
    -> 256^3, c = 2, K = 3, the benchmark's gradient step): the gradient of
    0.5 ||R p - f||^2 through PAIRecon against the oracle's adjoint of the same
    residual on a 32 x 32 x 32 box of detector samples, the dot-product
    identity, and the directional derivative along 32 coordinates e_i.  R is
    linear, so the central difference (R(p + h e_i) - R(p - h e_i)) / 2h is R e_i
    for every step h; it is formed as R e_i directly, which keeps FP32 rounding
    of R p out of the difference."""
    import torch
    prob = ph.adjoint_3d(0)
    g = prob.geom
    plan = pai.Plan(gdict(g, oversampling=2, K=3))
    p0 = prob.p.astype(np.float32)
    f_true = ph.random_image(74, g).astype(np.float32)
    pt = to_gpu(p0).requires_grad_(True)
    ft = to_gpu(f_true)
    loss = 0.5 * ((pai.PAIRecon.apply(pt, plan) - ft) ** 2).sum()
    loss.backward()
    grad = to_np(pt.grad)
    with torch.no_grad():
        resid = to_np(plan.reconstruct(pt.detach()) - ft)
    box = ((112, 144), (112, 144), (240, 272))
    ref = oracle.adjoint_box(g, resid, *box)
    assert rel(grad[112:144, 112:144, 240:272], ref) < TOL
    # dot product identity at full size
    h = ph.random_image(75, g).astype(np.float32)
    Rp = to_np(plan.reconstruct(to_gpu(p0)))
    Rth = to_np(plan.adjoint(to_gpu(h)))
    lhs = float(np.vdot(Rp, h.astype(np.float64)))
    rhs = float(np.vdot(p0.astype(np.float64), Rth))
    assert abs(lhs - rhs) < DOT_TOL * np.linalg.norm(Rp) * np.linalg.norm(h)
    # directional derivatives along 32 coordinates (seed 0)
    idx = np.random.default_rng(0).choice(p0.size, 32, replace=False)
    e = torch.zeros(p0.size, device="cuda", dtype=torch.float32)
    dd = []
    for i in idx:
        e.zero_()
        e[int(i)] = 1.0
        Re = to_np(plan.reconstruct(e.view(g.data_shape))).ravel()
        dd.append(float(np.dot(Re, resid.ravel())))
    assert rel(np.array(dd), grad.ravel()[idx]) < 1e-5
