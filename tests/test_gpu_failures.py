"""Failure handling of plan construction and of the host-memory entry points,
provoked on the host only (no GPU fault): an allocation cap that makes a
device allocation fail like an exhausted device (PAI_FAULT_ALLOC_BYTES), and a
cuFFT plan creation that reports failure (PAI_FAULT_CUFFT_PLAN).  Every failed
call must return its status, leave the caller's out-pointer untouched, release
whatever the partly built plan held (device memory back to its level before
the call), and leave the context usable."""
import ctypes

import numpy as np
import pytest

import oracle
import phantoms as ph
from gpu_common import TOL, gdict, pai, rel, to_gpu, to_np  # noqa: F401

pytestmark = pytest.mark.gpu

SENTINEL = 0x5EED


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _try_plan(lib, gg, batched=0):
    h = ctypes.c_void_p(SENTINEL)
    if batched:
        arr = (type(gg) * batched)(*([gg] * batched))
        st = lib.pai_plan_batched(arr, batched, None, ctypes.byref(h))
    else:
        st = lib.pai_plan(ctypes.byref(gg), None, ctypes.byref(h))
    return st, h


G2 = ph.Geometry(dim=2, nx=256, nt=512, nz=256)
G3 = ph.Geometry(dim=3, nx=32, ny=24, nt=64, nz=32)


@pytest.mark.parametrize("g", [G2, G3], ids=["2d", "3d"])
@pytest.mark.parametrize("frac", [0.0, 0.001, 0.3, 0.7])
def test_allocation_cap_returns_oom_and_releases(pai, g, frac, monkeypatch):
    """Caps from nothing to 70 % of the single plan's workspace: the
    failure comes at every stage of the build (first buffer, tables, cuFFT work
    areas, work items)."""
    lib = pai.load_library()
    gg = pai.geometry(gdict(g, K=3))
    # warm up (cuFFT's modules, the library's kernels), then measure
    warm = pai.Plan(gdict(g, K=3))
    ws = warm.info["workspace_bytes"]
    warm.close()
    assert ws > 0
    budget = int(frac * ws)
    before = _free_bytes()
    monkeypatch.setenv("PAI_FAULT_ALLOC_BYTES", str(budget))
    for batched in (0, 3):
        st, h = _try_plan(lib, gg, batched)
        assert st == 3, lib.pai_status_string(st)  # PAI_ERR_OOM
        assert h.value == SENTINEL
    assert _free_bytes() == before
    monkeypatch.delenv("PAI_FAULT_ALLOC_BYTES")
    # the context still works
    p = ph.random_data(60, g)
    f = to_np(pai.Plan(gdict(g, K=3)).reconstruct(to_gpu(p)))
    assert rel(f, oracle.reconstruct(g, p.astype(np.float64))) < TOL


@pytest.mark.parametrize("which", [0, 1, 2, 3, 5])
def test_cufft_plan_failure_returns_cufft_and_releases(pai, which, monkeypatch):
    lib = pai.load_library()
    gg = pai.geometry(gdict(G2, K=3))
    st, h = _try_plan(lib, gg, 2)
    assert st == 0
    lib.pai_destroy(h)
    before = _free_bytes()
    monkeypatch.setenv("PAI_FAULT_CUFFT_PLAN", str(which))
    st, h = _try_plan(lib, gg, 2)  # two problems: eight plan creations
    assert st == 5, lib.pai_status_string(st)  # PAI_ERR_CUFFT
    assert h.value == SENTINEL
    assert _free_bytes() == before
    monkeypatch.delenv("PAI_FAULT_CUFFT_PLAN")
    st, h = _try_plan(lib, gg, 2)
    assert st == 0
    lib.pai_destroy(h)


def test_forward_plan_and_host_staging_failures(pai, monkeypatch):
    """The forward model's box buffers and the host entry point's staging
    buffers come from the same capped allocator: the forward plan fails with
    PAI_ERR_OOM, and a plan built with a cap just above its own workspace keeps
    working on the device while its host-memory call reports PAI_ERR_OOM."""
    import torch
    lib = pai.load_library()
    g = ph.Geometry(dim=2, nx=64, nt=128, nz=64)
    gg = pai.geometry(gdict(g, K=3))
    h = ctypes.c_void_p(SENTINEL)
    monkeypatch.setenv("PAI_FAULT_ALLOC_BYTES", "100000")
    assert lib.pai_forward_plan(ctypes.byref(gg), None, ctypes.byref(h)) == 3
    assert h.value == SENTINEL
    monkeypatch.delenv("PAI_FAULT_ALLOC_BYTES")
    ws = pai.Plan(gdict(g, K=3)).info["workspace_bytes"]
    monkeypatch.setenv("PAI_FAULT_ALLOC_BYTES", str(ws + 4096))  # staging needs 48 KiB more
    plan = pai.Plan(gdict(g, K=3))
    monkeypatch.delenv("PAI_FAULT_ALLOC_BYTES")
    p = ph.random_data(61, g).astype(np.float32)
    ok = to_np(plan.reconstruct(to_gpu(p)))
    assert rel(ok, oracle.reconstruct(g, p.astype(np.float64))) < TOL
    out = torch.empty(g.image_shape, dtype=torch.float32)
    with pytest.raises(pai.PAIError) as e:
        plan.reconstruct_host(torch.from_numpy(p.copy()), out)
    assert e.value.status == 3
    assert np.array_equal(to_np(plan.reconstruct(to_gpu(p))), ok)
