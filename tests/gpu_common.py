"""Helpers shared by the GPU parity tests (GPU path vs the FP64 oracle)."""
import numpy as np
import pytest

# Relative L2 bound for every GPU-vs-oracle comparison (FP32 arithmetic against
# the FP64 direct reconstruction).
TOL = 1e-5
# Dot-product (adjoint) bound: <R p, h> against <p, R^T h>, both from FP32 results.
DOT_TOL = 1e-6


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    b = np.asarray(b, dtype=np.complex128 if np.iscomplexobj(b) else np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def gdict(g, **over):
    d = dict(dim=g.dim, nx=g.nx, ny=g.ny, dx=g.dx, dy=g.dy, nt=g.nt, dt=g.dt, c=g.c, nz=g.nz, dz=g.dz)
    d.update(over)
    return d


@pytest.fixture(scope="session")
def pai():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0808_3510_gb300 import build
    build.build()
    import paper_0808_3510_gb300 as m
    return m


def to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def oracle_half_spectrum(g, F):
    """Map the oracle's full spectrum fhat[k][l] (all l) onto the library's half
    spectrum: scale 1/(n_lat nz) and the Nyquist entry as the mean of the l = -nz/2
    node of row k and the conjugate of row -k's (= the node at +nz/2)."""
    n_lat = g.nx * (g.ny if g.dim == 3 else 1)
    nzh = g.nz // 2
    E = F[..., : nzh + 1].copy() / (n_lat * g.nz)
    if g.dim == 2:
        neg = (-np.arange(g.nx)) % g.nx
        partner = np.conj(F[neg, nzh])
    else:
        nx_ = (-np.arange(g.nx)) % g.nx
        ny_ = (-np.arange(g.ny)) % g.ny
        partner = np.conj(F[nx_][:, ny_, nzh])
    E[..., nzh] = 0.5 * (F[..., nzh] + partner) / (n_lat * g.nz)
    return E


# Both pipelines a plan can run: every stage on the library's kernels (chosen
# when all sizes are powers of two and the tuner is off), or cuFFT for the
# inverse / adjoint image-side transforms.
PIPELINES = {
    "library_ffts": {"PAI_AUTOTUNE": "0", "PAI_FUSED_DEPTH": "1"},
    "cufft_inverse": {"PAI_FUSED_DEPTH": "0"},
}


@pytest.fixture(params=sorted(PIPELINES))
def pipeline(request, monkeypatch):
    for k, v in PIPELINES[request.param].items():
        monkeypatch.setenv(k, v)
    return request.param
