"""GB300 (sm_103a) NUFFT-based Fourier reconstruction for planar and line-detector
photoacoustic imaging (Haltmeier, Scherzer, Zangerl; Algorithm 2).

This module is the thin Python binding of ``libpai.so`` (C ABI in
``include/pai.h``): it marshals torch tensors into device pointers and the
current CUDA stream.  Every step of the reconstruction runs in the library's
CUDA kernels and cuFFT; there is no CPU or PyTorch fallback.  If the library
has not been built, every entry point raises.

Quick use::

    import torch, paper_0808_3510_gb300 as pai
    plan = pai.Plan(dict(dim=2, nx=128, nt=256, nz=128, dx=1, dt=1, c=1, dz=1))
    f = plan.reconstruct(p_cuda_float32)          # [nx][nz]
    f = pai.PAIRecon.apply(p, plan)                # differentiable in p
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Iterable, List, Optional, Sequence

import torch

__all__ = ["Plan", "ForwardModel", "PAIRecon", "PAIError", "Geometry", "PlanInfo", "ProblemInfo", "library_path", "load_library",
           "geometry", "window_probe", "cutoff_table", "cached_plan", "reconstruct", "adjoint"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libpai.so")
_lock = threading.Lock()
_lib = None

PAI_OK = 0
_STATUS = {
    0: "success", 1: "invalid argument", 2: "unsupported configuration", 3: "out of memory",
    4: "CUDA error", 5: "cuFFT error", 6: "device wait timed out",
}


class PAIError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {_STATUS.get(status, 'unknown status')} (pai_status {status})")
        self.status = status


class Geometry(ctypes.Structure):
    """Mirror of ``pai_geometry``."""

    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("nt", ctypes.c_int), ("dt", ctypes.c_double), ("c", ctypes.c_double),
        ("nz", ctypes.c_int), ("dz", ctypes.c_double),
        ("oversampling", ctypes.c_double), ("K", ctypes.c_double), ("alpha", ctypes.c_double),
        ("method", ctypes.c_int),
    ]


# How the temporal spectrum is evaluated at the nodes (the Fourier algorithms
# compared in Sec. 4): Algorithm 1 with the Kaiser-Bessel window (default) or
# with the indicator window (truncated sinc), or the exact oversampled DFT
# interpolated linearly / to the nearest grid node.
METHODS = {"kb": 0, "tsinc": 1, "linear": 2, "nearest": 3}


def method_code(m) -> int:
    if m is None:
        return 0
    if isinstance(m, str):
        if m not in METHODS:
            raise ValueError(f"unknown method {m!r}; expected one of {sorted(METHODS)}")
        return METHODS[m]
    return int(m)


class PlanInfo(ctypes.Structure):
    """Mirror of ``pai_plan_info``."""

    _fields_ = [
        ("count", ctypes.c_int), ("M", ctypes.c_int), ("taps", ctypes.c_int),
        ("oversampling", ctypes.c_double), ("K", ctypes.c_double), ("alpha", ctypes.c_double),
        ("predicted_error", ctypes.c_double), ("threads_per_cta", ctypes.c_int), ("ctas", ctypes.c_int),
        ("rows", ctypes.c_int), ("nodes", ctypes.c_longlong), ("workspace_bytes", ctypes.c_size_t),
        ("uses_graph", ctypes.c_int), ("library_ffts", ctypes.c_int),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class ProblemInfo(ctypes.Structure):
    """Mirror of ``pai_problem_info``."""

    _fields_ = [
        ("M", ctypes.c_int), ("taps", ctypes.c_int), ("oversampling", ctypes.c_double), ("K", ctypes.c_double),
        ("alpha", ctypes.c_double), ("predicted_error", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def library_path() -> str:
    return _LIB_PATH


def load_library() -> ctypes.CDLL:
    """Load libpai.so (built by ``paper_0808_3510_gb300.build``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                f"libpai.so not found at {_LIB_PATH}; build it with `python -m paper_0808_3510_gb300.build` "
                "(the reconstruction has no CPU fallback)")
        lib = ctypes.CDLL(_LIB_PATH)
        vp, fp = ctypes.c_void_p, ctypes.c_void_p
        st = ctypes.c_int
        G = ctypes.POINTER(Geometry)
        lib.pai_plan.argtypes = [G, vp, ctypes.POINTER(vp)]
        lib.pai_plan.restype = st
        lib.pai_plan_batched.argtypes = [G, ctypes.c_int, vp, ctypes.POINTER(vp)]
        lib.pai_plan_batched.restype = st
        for name in ("pai_reconstruct", "pai_adjoint", "pai_spectrum", "pai_reconstruct_host",
                     "pai_reconstruct_host_async"):
            getattr(lib, name).argtypes = [vp, fp, fp]
            getattr(lib, name).restype = st
        lib.pai_host_wait.argtypes = [vp]
        lib.pai_host_wait.restype = st
        lib.pai_forward_plan.argtypes = [G, vp, ctypes.POINTER(vp)]
        lib.pai_forward_plan.restype = st
        lib.pai_forward_model.argtypes = [vp, fp, fp]
        lib.pai_forward_model.restype = st
        ip = ctypes.POINTER(ctypes.c_int)
        lib.pai_forward_box.argtypes = [vp, ip, ip, ip]
        lib.pai_forward_box.restype = st
        lib.pai_profile_stages.argtypes = [vp, fp, fp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        lib.pai_profile_stages.restype = st
        lib.pai_set_deterministic.argtypes = [vp, ctypes.c_int]
        lib.pai_set_deterministic.restype = st
        lib.pai_set_stream.argtypes = [vp, vp]
        lib.pai_set_stream.restype = st
        lib.pai_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
        lib.pai_get_info.restype = st
        lib.pai_get_problem_info.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ProblemInfo)]
        lib.pai_get_problem_info.restype = st
        lib.pai_tuning_log.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
        lib.pai_tuning_log.restype = st
        lib.pai_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
        lib.pai_launch_count.restype = st
        lib.pai_destroy.argtypes = [vp]
        lib.pai_destroy.restype = st
        dp = ctypes.POINTER(ctypes.c_double)
        lib.pai_window_probe.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp, dp,
                                         dp]
        lib.pai_window_probe.restype = st
        lib.pai_spectrum_rows_noalloc.argtypes = [G, fp, fp, vp]
        lib.pai_spectrum_rows_noalloc.restype = st
        lib.pai_cutoff_table.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_int, ip]
        lib.pai_cutoff_table.restype = st
        lib.pai_set_cutoff.argtypes = [vp, ctypes.c_double]
        lib.pai_set_cutoff.restype = st
        lib.pai_cutoff.argtypes = [vp, fp, fp]
        lib.pai_cutoff.restype = st
        lib.pai_status_string.argtypes = [st]
        lib.pai_status_string.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != PAI_OK:
        raise PAIError(status, where)


def geometry(g) -> Geometry:
    """Build a ``pai_geometry`` from a dict or an object with the same field names
    (dim, nx, ny, dx, dy, nt, dt, c, nz, dz; optional oversampling, K, alpha and
    method, a name from ``METHODS`` or its code)."""
    get = (lambda k, d=None: g.get(k, d)) if isinstance(g, dict) else (lambda k, d=None: getattr(g, k, d))
    dim = int(get("dim"))
    return Geometry(
        dim, int(get("nx")), int(get("ny", 1) or 1) if dim == 3 else 1,
        float(get("dx", 1.0)), float(get("dy", 1.0) or 1.0) if dim == 3 else 1.0,
        int(get("nt")), float(get("dt", 1.0)), float(get("c", 1.0)),
        int(get("nz")), float(get("dz", 1.0)),
        float(get("oversampling", 0.0) or 0.0), float(get("K", 0.0) or 0.0), float(get("alpha", 0.0) or 0.0),
        method_code(get("method", 0)),
    )


def _numel(g: Geometry, last: int) -> int:
    return g.nx * (g.ny if g.dim == 3 else 1) * last


def _shape(g: Geometry, last: int):
    return (g.nx, last) if g.dim == 2 else (g.nx, g.ny, last)


def window_probe(H: int, beta: float, c: float, y=()):
    """Plan-time window math (host only): returns (phi(y)/phi(0) list, predicted
    truncation error, FP32 tap-polynomial fit error).  See ``pai_window_probe``."""
    lib = load_library()
    n = len(y)
    ya = (ctypes.c_double * max(n, 1))(*y)
    out = (ctypes.c_double * max(n, 1))()
    pe, fe = ctypes.c_double(), ctypes.c_double()
    _check(lib.pai_window_probe(H, beta, c, n, ya, out, ctypes.byref(pe), ctypes.byref(fe)), "pai_window_probe")
    return [out[i] for i in range(n)], pe.value, fe.value


def cutoff_table(dim: int, eps: float):
    """The weights of the data cutoff w_cut (``pai_cutoff_table``, host only) as a
    nested list of shape (R+1,)*dim indexed by the clipped distances to the
    faces (time last), and R."""
    lib = load_library()
    R = ctypes.c_int()
    _check(lib.pai_cutoff_table(int(dim), float(eps), None, 0, ctypes.byref(R)), "pai_cutoff_table")
    n = (R.value + 1) ** dim
    buf = (ctypes.c_double * n)()
    _check(lib.pai_cutoff_table(int(dim), float(eps), buf, n, ctypes.byref(R)), "pai_cutoff_table")
    flat = list(buf)
    r1 = R.value + 1
    if dim == 2:
        return [flat[i * r1:(i + 1) * r1] for i in range(r1)], R.value
    return [[flat[(i * r1 + j) * r1:(i * r1 + j + 1) * r1] for j in range(r1)] for i in range(r1)], R.value


def _apply_cutoff(obj, p: torch.Tensor, out: Optional[torch.Tensor]) -> torch.Tensor:
    g = obj.geom if isinstance(obj, ForwardModel) else obj.geoms[0]
    n = _numel(g, g.nt)
    for t, what in ((p, "p"), (out, "out")):
        if t is not None and (not isinstance(t, torch.Tensor) or t.device != obj.device or t.dtype != torch.float32
                              or not t.is_contiguous() or t.numel() != n):
            raise ValueError(f"{what} must be a contiguous float32 tensor on {obj.device} with {n} elements")
    if out is None:
        out = torch.empty(_shape(g, g.nt), device=obj.device, dtype=torch.float32)
    cur = torch.cuda.current_stream(obj.device).cuda_stream
    if cur != obj._stream:
        _check(obj._lib.pai_set_stream(obj._h, ctypes.c_void_p(cur)), "pai_set_stream")
        obj._stream = cur
    _check(obj._lib.pai_cutoff(obj._h, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(out.data_ptr())), "pai_cutoff")
    return out


def spectrum_rows_noalloc(g, pt: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
    """Fused row stage for callers that cannot allocate device memory
    (``pai_spectrum_rows_noalloc``).  ``pt``: complex64 lateral spectrum rows
    (an unnormalised real-to-complex FFT of the data over the lateral axes),
    ``out``: complex64 half image spectrum, both on the current device and
    contiguous; runs on torch's current stream and allocates nothing."""
    lib = load_library()
    gg = geometry(g)
    for t in (pt, out):
        if t.device.type != "cuda" or t.dtype != torch.complex64 or not t.is_contiguous():
            raise ValueError("pt and out must be contiguous complex64 CUDA tensors")
    rows = (gg.nx // 2 + 1) if gg.dim == 2 else gg.nx * (gg.ny // 2 + 1)
    if pt.numel() != rows * gg.nt or out.numel() != _numel(gg, gg.nz // 2 + 1):
        raise ValueError("pt / out have the wrong number of elements for this geometry")
    _check(lib.pai_spectrum_rows_noalloc(ctypes.byref(gg), ctypes.c_void_p(pt.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
           "pai_spectrum_rows_noalloc")
    return out


class Plan:
    """A reconstruction plan: one problem, or a batch of independent problems.

    ``Plan(g)`` wraps ``pai_plan``; ``Plan([g0, g1, ...])`` wraps
    ``pai_plan_batched`` (inputs and outputs are then flat concatenations).
    The plan lives on the current CUDA device; calls run on torch's current
    stream.
    """

    def __init__(self, geoms, stream: Optional[torch.cuda.Stream] = None, overrides: Optional[dict] = None):
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("paper_0808_3510_gb300 needs a CUDA device")
        single = not isinstance(geoms, (list, tuple))
        items = [geoms] if single else list(geoms)
        gs = []
        for g in items:
            gg = geometry(g)
            if overrides:
                for k, v in overrides.items():
                    setattr(gg, k, v)
            gs.append(gg)
        self.geoms: List[Geometry] = gs
        self.batched = not single
        self.device = torch.device("cuda", torch.cuda.current_device())
        s = stream if stream is not None else torch.cuda.current_stream()
        self._stream = s.cuda_stream
        arr = (Geometry * len(gs))(*gs)
        h = ctypes.c_void_p()
        if single:
            _check(lib.pai_plan(arr, ctypes.c_void_p(self._stream), ctypes.byref(h)), "pai_plan")
        else:
            _check(lib.pai_plan_batched(arr, len(gs), ctypes.c_void_p(self._stream), ctypes.byref(h)),
                   "pai_plan_batched")
        self._h = h
        self._lib = lib
        if torch.are_deterministic_algorithms_enabled():
            self.set_deterministic(True)
        self.data_numel = sum(_numel(g, g.nt) for g in gs)
        self.image_numel = sum(_numel(g, g.nz) for g in gs)
        self.spectrum_numel = sum(_numel(g, g.nz // 2 + 1) for g in gs)

    # -- helpers ---------------------------------------------------------
    def _sync_stream(self):
        cur = torch.cuda.current_stream(self.device).cuda_stream
        if cur != self._stream:
            _check(self._lib.pai_set_stream(self._h, ctypes.c_void_p(cur)), "pai_set_stream")
            self._stream = cur

    def _check_in(self, t: torch.Tensor, numel: int, what: str):
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != torch.float32:
            raise ValueError(f"{what} must be a float32 tensor on {self.device}")
        if not t.is_contiguous() or t.numel() != numel:
            raise ValueError(f"{what} must be contiguous with {numel} elements (got {tuple(t.shape)})")
        if t.data_ptr() % 8 != 0:
            raise ValueError(f"{what} must start on an 8-byte boundary (the library moves two floats at a time)")

    def _out_shape(self, last_attr: str):
        if self.batched:
            return (self.image_numel if last_attr == "nz" else self.data_numel,)
        g = self.geoms[0]
        return _shape(g, getattr(g, last_attr))

    # -- operators ---------------------------------------------------------
    def reconstruct(self, p: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """f = R p (Algorithm 2).  p: [nx][(ny)][nt] float32 on the plan's device."""
        self._check_in(p, self.data_numel, "p")
        if out is None:
            out = torch.empty(self._out_shape("nz"), device=self.device, dtype=torch.float32)
        self._check_in(out, self.image_numel, "out")
        self._sync_stream()
        _check(self._lib.pai_reconstruct(self._h, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(out.data_ptr())),
               "pai_reconstruct")
        return out

    def adjoint(self, h: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """p_bar = R^T h, the exact transpose of :meth:`reconstruct`."""
        self._check_in(h, self.image_numel, "h")
        if out is None:
            out = torch.empty(self._out_shape("nt"), device=self.device, dtype=torch.float32)
        self._check_in(out, self.data_numel, "out")
        self._sync_stream()
        _check(self._lib.pai_adjoint(self._h, ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(out.data_ptr())),
               "pai_adjoint")
        return out

    def spectrum(self, p: torch.Tensor) -> torch.Tensor:
        """Half image spectrum (steps 1-3), complex64 [nx][(ny)][nz/2+1] (flat when batched)."""
        self._check_in(p, self.data_numel, "p")
        out = torch.empty(self.spectrum_numel * 2, device=self.device, dtype=torch.float32)
        self._sync_stream()
        _check(self._lib.pai_spectrum(self._h, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(out.data_ptr())),
               "pai_spectrum")
        c = torch.view_as_complex(out.view(-1, 2))
        if not self.batched:
            g = self.geoms[0]
            c = c.view(_shape(g, g.nz // 2 + 1))
        return c

    def reconstruct_host(self, p_host: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """End to end from host memory (pai_reconstruct_host): copies in, reconstructs, copies out."""
        if p_host.device.type != "cpu" or p_host.dtype != torch.float32 or not p_host.is_contiguous():
            raise ValueError("p_host must be a contiguous float32 CPU tensor")
        if p_host.numel() != self.data_numel:
            raise ValueError("p_host has the wrong number of elements")
        if out is None:
            out = torch.empty(self._out_shape("nz"), dtype=torch.float32, pin_memory=p_host.is_pinned())
        self._sync_stream()
        _check(self._lib.pai_reconstruct_host(self._h, ctypes.c_void_p(p_host.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr())), "pai_reconstruct_host")
        return out

    def reconstruct_host_async(self, p_host: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
        """Pipelined end-to-end call (pai_reconstruct_host_async): enqueues the upload,
        the reconstruction and the download, and returns at once.  Neither tensor may be
        touched until :meth:`host_wait` returns; use page-locked tensors."""
        for t, n, what in ((p_host, self.data_numel, "p_host"), (out, self.image_numel, "out")):
            if t.device.type != "cpu" or t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != n:
                raise ValueError(f"{what} must be a contiguous float32 CPU tensor with {n} elements")
        self._sync_stream()
        _check(self._lib.pai_reconstruct_host_async(self._h, ctypes.c_void_p(p_host.data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr())), "pai_reconstruct_host_async")
        return out

    def host_wait(self):
        """Wait for every :meth:`reconstruct_host_async` call of this plan."""
        _check(self._lib.pai_host_wait(self._h), "pai_host_wait")

    def profile_stages(self, x: torch.Tensor, out: torch.Tensor, reps: int = 10, adjoint: bool = False):
        """Mean device milliseconds per pass of (first FFT stage, row kernel, last FFT stage)."""
        self._check_in(x, self.image_numel if adjoint else self.data_numel, "input")
        self._check_in(out, self.data_numel if adjoint else self.image_numel, "out")
        self._sync_stream()
        ms = (ctypes.c_double * 3)()
        _check(self._lib.pai_profile_stages(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                            int(reps), 1 if adjoint else 0, ms), "pai_profile_stages")
        return [ms[0], ms[1], ms[2]]

    def set_deterministic(self, on: bool = True):
        """Bit-identical adjoints on repeated calls (tap-phased or node-pair spread) instead
        of a faster spread that adds with shared-memory atomics (``pai_set_deterministic``).  Plans made
        while ``torch.use_deterministic_algorithms(True)`` is on start deterministic."""
        _check(self._lib.pai_set_deterministic(self._h, 1 if on else 0), "pai_set_deterministic")

    def set_cutoff(self, eps: float):
        """Attach the data cutoff w_cut with parameter eps (squared sampling steps; 0 removes it)."""
        _check(self._lib.pai_set_cutoff(self._h, float(eps)), "pai_set_cutoff")

    def cutoff(self, p: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """w_cut * p over the data grid (``pai_cutoff``); out may be p itself."""
        return _apply_cutoff(self, p, out)

    # -- introspection ------------------------------------------------------
    @property
    def info(self) -> dict:
        i = PlanInfo()
        _check(self._lib.pai_get_info(self._h, ctypes.byref(i)), "pai_get_info")
        return i.as_dict()

    @property
    def kernel_launches(self) -> int:
        n = ctypes.c_longlong()
        _check(self._lib.pai_launch_count(self._h, ctypes.byref(n)), "pai_launch_count")
        return int(n.value)

    def problem_info(self, index: int = 0) -> dict:
        """Padded length, taps, oversampling, K, alpha and predicted window error of
        problem ``index`` (``pai_get_problem_info``)."""
        i = ProblemInfo()
        _check(self._lib.pai_get_problem_info(self._h, int(index), ctypes.byref(i)), "pai_get_problem_info")
        return i.as_dict()

    @property
    def tuning_log(self) -> str:
        """What the tuner timed and kept when the plan was built (``pai_tuning_log``)."""
        return _tuning_log(self._lib, self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pai_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _tuning_log(lib, h) -> str:
    n = ctypes.c_size_t()
    _check(lib.pai_tuning_log(h, None, 0, ctypes.byref(n)), "pai_tuning_log")
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(lib.pai_tuning_log(h, buf, n.value + 1, None), "pai_tuning_log")
    return buf.value.decode()


class ForwardModel:
    """Discrete forward model (``pai_forward_plan`` / ``pai_forward_model``): detector
    data of an initial pressure on the image grid, the wave equation solved
    exactly for its trigonometric interpolant in a zero-padded periodic box.
    Calls run on torch's current stream."""

    def __init__(self, g, stream: Optional[torch.cuda.Stream] = None, cutoff: Optional[float] = None):
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("paper_0808_3510_gb300 needs a CUDA device")
        self.geom = geometry(g)
        self.device = torch.device("cuda", torch.cuda.current_device())
        s = stream if stream is not None else torch.cuda.current_stream()
        self._stream = s.cuda_stream
        h = ctypes.c_void_p()
        _check(lib.pai_forward_plan(ctypes.byref(self.geom), ctypes.c_void_p(self._stream), ctypes.byref(h)),
               "pai_forward_plan")
        self._h = h
        self._lib = lib
        b = [ctypes.c_int() for _ in range(3)]
        _check(lib.pai_forward_box(h, *[ctypes.byref(v) for v in b]), "pai_forward_box")
        self.box = tuple(v.value for v in b)
        if cutoff:
            self.set_cutoff(cutoff)
        if torch.are_deterministic_algorithms_enabled():
            self.set_deterministic(True)

    def set_deterministic(self, on: bool = True):
        """Bit-identical results on repeated calls (``pai_set_deterministic``)."""
        _check(self._lib.pai_set_deterministic(self._h, 1 if on else 0), "pai_set_deterministic")

    def set_cutoff(self, eps: float):
        """Return w_cut * (Q f) from now on (the data model of partial data); 0 removes the cutoff."""
        _check(self._lib.pai_set_cutoff(self._h, float(eps)), "pai_set_cutoff")

    def cutoff(self, p: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """w_cut * p over the detector data grid (``pai_cutoff``); out may be p itself."""
        return _apply_cutoff(self, p, out)

    def __call__(self, f: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        g = self.geom
        n_img, n_dat = _numel(g, g.nz), _numel(g, g.nt)
        if not isinstance(f, torch.Tensor) or f.device != self.device or f.dtype != torch.float32 \
                or not f.is_contiguous() or f.numel() != n_img:
            raise ValueError(f"f must be a contiguous float32 tensor on {self.device} with {n_img} elements")
        if out is None:
            out = torch.empty(_shape(g, g.nt), device=self.device, dtype=torch.float32)
        if out.device != self.device or out.dtype != torch.float32 or not out.is_contiguous() \
                or out.numel() != n_dat:
            raise ValueError(f"out must be a contiguous float32 tensor on {self.device} with {n_dat} elements")
        cur = torch.cuda.current_stream(self.device).cuda_stream
        if cur != self._stream:
            _check(self._lib.pai_set_stream(self._h, ctypes.c_void_p(cur)), "pai_set_stream")
            self._stream = cur
        _check(self._lib.pai_forward_model(self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr())),
               "pai_forward_model")
        return out

    @property
    def info(self) -> dict:
        i = PlanInfo()
        _check(self._lib.pai_get_info(self._h, ctypes.byref(i)), "pai_get_info")
        return i.as_dict()

    @property
    def kernel_launches(self) -> int:
        n = ctypes.c_longlong()
        _check(self._lib.pai_launch_count(self._h, ctypes.byref(n)), "pai_launch_count")
        return n.value

    @property
    def tuning_log(self) -> str:
        """What the box plan's tuner timed and kept (``pai_tuning_log``): the spread."""
        return _tuning_log(self._lib, self._h)

    def profile_stages(self, reps: int = 10):
        """Mean device ms of (image-side transforms, forward-model row kernel, lateral inverse) on the box."""
        bx, by, bz = self.box
        g = self.geom
        x = torch.zeros(bx * by * bz, device=self.device, dtype=torch.float32)
        y = torch.empty(bx * by * g.nt, device=self.device, dtype=torch.float32)
        ms = (ctypes.c_double * 3)()
        _check(self._lib.pai_profile_stages(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                            int(reps), 1, ms), "pai_profile_stages")
        return [ms[0], ms[1], ms[2]]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pai_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PAIRecon(torch.autograd.Function):
    """Differentiable reconstruction: forward = :meth:`Plan.reconstruct`,
    backward = :meth:`Plan.adjoint` (the operator is linear)."""

    @staticmethod
    def forward(ctx, p: torch.Tensor, plan: Plan):
        ctx.plan = plan
        return plan.reconstruct(p.contiguous())

    @staticmethod
    def backward(ctx, grad_f: torch.Tensor):
        return ctx.plan.adjoint(grad_f.contiguous()), None


# ---------------------------------------------------------------------------
# functional interface: cached plans per geometry and device
# ---------------------------------------------------------------------------

_PLAN_CACHE_SIZE = 8
_plan_cache: "dict" = {}
_plan_cache_lock = threading.Lock()


def _geometry_key(gg: Geometry):
    return tuple(getattr(gg, name) for name, _ in Geometry._fields_)


def cached_plan(g) -> Plan:
    """A single-problem :class:`Plan` for geometry ``g`` on the current device,
    created on first use and kept (least recently used first out, at most
    eight; a dropped plan is destroyed when its last user lets go of it)."""
    gg = geometry(g)
    key = (_geometry_key(gg), torch.cuda.current_device())
    with _plan_cache_lock:
        plan = _plan_cache.pop(key, None)
        if plan is None:
            plan = Plan(gg)
        _plan_cache[key] = plan
        while len(_plan_cache) > _PLAN_CACHE_SIZE:
            # dropped, not closed: an autograd graph may still hold it for its backward
            _plan_cache.pop(next(iter(_plan_cache)))
    return plan


def reconstruct(p: torch.Tensor, g) -> torch.Tensor:
    """Image [nx][ny][nz] from detector data ``p`` [nx][ny][nt] (Algorithm 2),
    differentiable in ``p`` (the backward pass is the exact adjoint).  ``g`` is
    a geometry dict or :class:`Geometry`; its plan is cached."""
    return PAIRecon.apply(p, cached_plan(g))


def adjoint(h: torch.Tensor, g) -> torch.Tensor:
    """The exact transpose of :func:`reconstruct`: data-shaped output from an
    image-shaped ``h``."""
    return cached_plan(g).adjoint(h.contiguous())
