"""The allocation-free entry point pai_spectrum_rows_noalloc.

Some callers may not call cudaMalloc (device memory already reserved by
another allocator or pool, or a real-time loop where an allocation's implicit
synchronisation is not allowed); this entry point runs the fused row stage with
its scratch in a static device array.  Its output must match the planned entry point
pai_spectrum on the same data, within the tolerance the other GPU tests use,
on two calls in a row (the second call must not be disturbed by what the
first left in the shared array).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import phantoms as ph
from gpu_common import TOL, gdict, pai, rel, to_gpu  # noqa: F401

pytestmark = pytest.mark.gpu


def _lateral_rows(p, dim):
    import torch
    if dim == 2:
        return torch.fft.rfft(p, dim=0).contiguous()
    return torch.fft.rfft2(p, dim=(0, 1)).contiguous()


@pytest.mark.parametrize("g", [
    ph.Geometry(dim=2, nx=128, nt=256, nz=128),
    ph.Geometry(dim=2, nx=300, nt=700, nz=350, dx=1.0, dt=0.5, c=1.5, dz=0.8),
    ph.Geometry(dim=3, nx=20, ny=12, nt=48, nz=18, dx=0.9, dy=1.1, dt=0.7, c=1.3, dz=1.0),
], ids=["2d-128", "2d-ragged", "3d"])
def test_noalloc_matches_planned_spectrum_on_two_calls(pai, g):
    import torch
    d = gdict(g, K=3)
    plan = pai.Plan(d)
    lib = pai.load_library()
    gg = pai.geometry(d)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lz = g.nz // 2 + 1
    out = torch.empty(g.image_shape[:-1] + (lz,), device="cuda", dtype=torch.complex64)
    for call, seed in enumerate((80, 81)):
        p = to_gpu(ph.random_data(seed, g))
        expect = plan.spectrum(p).cpu().numpy()
        pt = _lateral_rows(p, g.dim)
        out.fill_(float("nan"))
        status = lib.pai_spectrum_rows_noalloc(ctypes.byref(gg), ctypes.c_void_p(pt.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()), stream)
        assert status == 0, lib.pai_status_string(status)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all(), f"call {call}: unwritten output"
        assert rel(got, expect) < TOL, f"call {call}"
