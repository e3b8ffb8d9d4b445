"""FP64 CPU oracle for the planar photoacoustic Fourier reconstruction.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (the CUDA library and its Python binding)
never imports it, and this package never imports the product.

The arithmetic lives in ``pai_oracle.c`` (plain C99, FP64, pthreads over
lateral rows): the paper's *direct Fourier reconstruction* (Sec. 4, first
compared algorithm) -- Eq. (fft-1a) as a direct lateral DFT, Eq. (fft-2) by
direct summation at every node, the weight of Eq. (fft-0) and the inverse DFT
of Eq. (fft-1) -- plus its exact transpose.  This module only marshals numpy
arrays into that library.

Every function here is pinned by ``tests/test_oracle_pins.py`` against values
fixed by the paper or by mathematics (library FFTs at integer nodes, closed
forms, the wave equation's closed-form solutions, the adjoint identity).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pai_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libpai_oracle.so")
_lock = threading.Lock()
_lib = None


class _Geom(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("dx", ctypes.c_double),
        ("dy", ctypes.c_double),
        ("nt", ctypes.c_int),
        ("dt", ctypes.c_double),
        ("c", ctypes.c_double),
        ("nz", ctypes.c_int),
        ("dz", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile ``pai_oracle.c`` into ``oracle/_build/libpai_oracle.so``.

    Plain ``gcc -O2`` without fast-math, so every FP64 operation rounds as
    IEEE 754 prescribes.
    """
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        G = ctypes.POINTER(_Geom)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i = ctypes.c_int
        lib.oracle_node.argtypes = [G, i, i, i]
        lib.oracle_node.restype = ctypes.c_double
        lib.oracle_weight.argtypes = [G, i, i, i]
        lib.oracle_weight.restype = ctypes.c_double
        lib.oracle_row_nodes.argtypes = [G, i, i, dp, dp]
        lib.oracle_row_nodes.restype = None
        lib.oracle_nudft.argtypes = [i, dp, i, dp, dp]
        lib.oracle_nudft.restype = None
        lib.oracle_nudft_adjoint.argtypes = [i, dp, i, dp, dp]
        lib.oracle_nudft_adjoint.restype = None
        for name in ("oracle_lateral_dft", "oracle_spectrum"):
            getattr(lib, name).argtypes = [G, dp, dp, i]
            getattr(lib, name).restype = i
        lib.oracle_spectrum_rows.argtypes = [G, dp, i, ip, ip, dp, i]
        lib.oracle_spectrum_rows.restype = i
        lib.oracle_image_from_spectrum.argtypes = [G, dp, dp, i]
        lib.oracle_image_from_spectrum.restype = i
        lib.oracle_reconstruct.argtypes = [G, dp, dp, i]
        lib.oracle_reconstruct.restype = i
        lib.oracle_adjoint.argtypes = [G, dp, dp, i]
        lib.oracle_adjoint.restype = i
        lib.oracle_adjoint_box.argtypes = [G, dp, i, i, i, i, i, i, dp, i]
        lib.oracle_adjoint_box.restype = i
        lib.oracle_forward_model.argtypes = [G, dp, i, i, i, dp, i]
        lib.oracle_forward_model.restype = i
        lib.oracle_threads.argtypes = [i]
        lib.oracle_threads.restype = i
        _lib = lib
        return lib


def _geom(g) -> _Geom:
    """Accept any object (or dict) with the fields dim, nx, ny, dx, dy, nt, dt, c, nz, dz."""
    get = (lambda k: g[k]) if isinstance(g, dict) else (lambda k: getattr(g, k))
    dim = int(get("dim"))
    ny = int(get("ny")) if dim == 3 else 1
    dy = float(get("dy")) if dim == 3 else 1.0
    return _Geom(dim, int(get("nx")), ny, float(get("dx")), dy, int(get("nt")), float(get("dt")),
                 float(get("c")), int(get("nz")), float(get("dz")))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def threads(requested: int = 0) -> int:
    """Number of host threads the oracle uses for ``requested`` (0 = all online cores)."""
    return _load().oracle_threads(requested)


def node(g, kx: int, ky: int, l: int) -> float:
    """Node nu_{k,l} (time-index units) of Eq. (dft-2d) in the general grid."""
    gg = _geom(g)
    return _load().oracle_node(ctypes.byref(gg), kx, ky, l)


def weight(g, kx: int, ky: int, l: int) -> float:
    """Weight of Eq. (fft-0) in the general grid (0 on the l = 0 row)."""
    gg = _geom(g)
    return _load().oracle_weight(ctypes.byref(gg), kx, ky, l)


def row_nodes(g, kx: int, ky: int = 0):
    """Nodes and weights of one lateral row for every depth frequency, storage
    index l mod nz: the values of :func:`node` and :func:`weight`."""
    gg = _geom(g)
    nu = np.empty(gg.nz, np.float64)
    w = np.empty(gg.nz, np.float64)
    _load().oracle_row_nodes(ctypes.byref(gg), kx, ky, _dptr(nu), _dptr(w))
    return nu, w


def nudft(gvec: np.ndarray, nu: np.ndarray) -> np.ndarray:
    """Eq. (dft): sum_n e^{-i 2 pi nu n/N} g_n at arbitrary nodes, by direct summation."""
    gv = np.ascontiguousarray(gvec, dtype=np.complex128)
    nv = np.ascontiguousarray(nu, dtype=np.float64)
    out = np.empty(nv.shape[0], np.complex128)
    _load().oracle_nudft(gv.shape[0], _dptr(gv), nv.shape[0], _dptr(nv), _dptr(out))
    return out


def nudft_adjoint(h: np.ndarray, nu: np.ndarray, nt: int) -> np.ndarray:
    """Transpose-conjugate of :func:`nudft`: sum_i e^{+i 2 pi nu_i n/N} h_i."""
    hv = np.ascontiguousarray(h, dtype=np.complex128)
    nv = np.ascontiguousarray(nu, dtype=np.float64)
    out = np.empty(nt, np.complex128)
    _load().oracle_nudft_adjoint(nt, _dptr(hv), nv.shape[0], _dptr(nv), _dptr(out))
    return out


def _shape_data(g: _Geom):
    return (g.nx, g.ny, g.nt)


def _shape_img(g: _Geom):
    return (g.nx, g.ny, g.nz)


def _as_data(g: _Geom, p: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(p, dtype=np.float64)
    if a.size != g.nx * g.ny * g.nt:
        raise ValueError(f"data has {a.size} samples, geometry wants {g.nx}x{g.ny}x{g.nt}")
    return a.reshape(_shape_data(g))


def _out_shape(g: _Geom, last: int):
    return (g.nx, last) if g.dim == 2 else (g.nx, g.ny, last)


def lateral_dft(g, p: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """Eq. (fft-1a): direct lateral DFT of real data; returns complex [kx][(ky)][n]."""
    gg = _geom(g)
    a = _as_data(gg, p)
    out = np.empty(_shape_data(gg), np.complex128)
    if _load().oracle_lateral_dft(ctypes.byref(gg), _dptr(a), _dptr(out), nthreads):
        raise MemoryError("oracle_lateral_dft failed")
    return out.reshape(_out_shape(gg, gg.nt))


def spectrum(g, p: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """Weighted image spectrum fhat[kx][(ky)][l] (all l, storage index l mod nz):
    Eq. (fft-1a), Eq. (fft-2) by direct summation, Eq. (fft-0)."""
    gg = _geom(g)
    a = _as_data(gg, p)
    out = np.empty(_shape_img(gg), np.complex128)
    if _load().oracle_spectrum(ctypes.byref(gg), _dptr(a), _dptr(out), nthreads):
        raise MemoryError("oracle_spectrum failed")
    return out.reshape(_out_shape(gg, gg.nz))


def spectrum_rows(g, p: np.ndarray, kx, ky=None, nthreads: int = 0) -> np.ndarray:
    """Rows fhat[k, :] (all l) for selected signed lateral frequencies, each row
    computed directly from the data at cost O(nx ny nt + nz nt)."""
    gg = _geom(g)
    a = _as_data(gg, p)
    kxa = np.ascontiguousarray(np.atleast_1d(kx), dtype=np.int32)
    kya = np.zeros_like(kxa) if ky is None else np.ascontiguousarray(np.atleast_1d(ky), dtype=np.int32)
    if kxa.shape != kya.shape:
        raise ValueError("kx and ky must have the same length")
    out = np.empty((kxa.shape[0], gg.nz), np.complex128)
    ip = ctypes.POINTER(ctypes.c_int)
    rc = _load().oracle_spectrum_rows(ctypes.byref(gg), _dptr(a), kxa.shape[0], kxa.ctypes.data_as(ip),
                                      kya.ctypes.data_as(ip), _dptr(out), nthreads)
    if rc:
        raise MemoryError("oracle_spectrum_rows failed")
    return out


def image_from_spectrum(g, fhat: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """Eq. (fft-1): real part of the direct inverse DFT of the full spectrum."""
    gg = _geom(g)
    a = np.ascontiguousarray(fhat, dtype=np.complex128)
    if a.size != gg.nx * gg.ny * gg.nz:
        raise ValueError("spectrum size does not match the geometry")
    out = np.empty(_shape_img(gg), np.float64)
    if _load().oracle_image_from_spectrum(ctypes.byref(gg), _dptr(a), _dptr(out), nthreads):
        raise MemoryError("oracle_image_from_spectrum failed")
    return out.reshape(_out_shape(gg, gg.nz))


def reconstruct(g, p: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """Direct Fourier reconstruction (the exact quantity Algorithm 2 approximates)."""
    gg = _geom(g)
    a = _as_data(gg, p)
    out = np.empty(_shape_img(gg), np.float64)
    if _load().oracle_reconstruct(ctypes.byref(gg), _dptr(a), _dptr(out), nthreads):
        raise MemoryError("oracle_reconstruct failed")
    return out.reshape(_out_shape(gg, gg.nz))


def adjoint(g, h: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """Exact transpose of :func:`reconstruct` under real inner products."""
    gg = _geom(g)
    a = np.ascontiguousarray(h, dtype=np.float64)
    if a.size != gg.nx * gg.ny * gg.nz:
        raise ValueError("image size does not match the geometry")
    out = np.empty(_shape_data(gg), np.float64)
    if _load().oracle_adjoint(ctypes.byref(gg), _dptr(a), _dptr(out), nthreads):
        raise MemoryError("oracle_adjoint failed")
    return out.reshape(_out_shape(gg, gg.nt))


def adjoint_box(g, h: np.ndarray, x, y, n, nthreads: int = 0) -> np.ndarray:
    """:func:`adjoint` evaluated only on the box of output samples x = range(*x),
    y = range(*y) (ignored in 2-D), n = range(*n), each a (start, stop) pair;
    for grids whose full adjoint is too costly to form directly."""
    gg = _geom(g)
    a = np.ascontiguousarray(h, dtype=np.float64)
    if a.size != gg.nx * gg.ny * gg.nz:
        raise ValueError("image size does not match the geometry")
    y = (0, 1) if gg.dim == 2 else y
    cx, cy, cn = x[1] - x[0], y[1] - y[0], n[1] - n[0]
    out = np.empty((cx, cy, cn), np.float64)
    rc = _load().oracle_adjoint_box(ctypes.byref(gg), _dptr(a), x[0], cx, y[0], cy, n[0], cn, _dptr(out), nthreads)
    if rc == -2:
        raise ValueError("box outside the data grid")
    if rc:
        raise MemoryError("oracle_adjoint_box failed")
    return out.reshape((cx, cn)) if gg.dim == 2 else out


def forward_box(g) -> tuple:
    """Box extents of the discrete forward model: per axis the next power of two
    (at least 32) >= the image extent + ceil(c nt dt / spacing) + 2."""
    import math
    gg = _geom(g)

    def ext(n, d):
        need = n + math.ceil(gg.c * gg.nt * gg.dt / d - 1e-9) + 2
        b = 32
        while b < need:
            b *= 2
        return b
    return (ext(gg.nx, gg.dx), ext(gg.ny, gg.dy) if gg.dim == 3 else 1, ext(gg.nz, gg.dz))


def forward_model(g, f: np.ndarray, box=None, nthreads: int = 0) -> np.ndarray:
    """Discrete forward model (Sec. 2, the operator Q): detector data of the
    initial pressure f on the image grid, the exact wave-equation solution for
    the trigonometric interpolant of f zero-padded to the periodic box ``box``
    (default :func:`forward_box`), by direct sums; returns [nx][(ny)][nt]."""
    gg = _geom(g)
    a = np.ascontiguousarray(f, dtype=np.float64)
    if a.size != gg.nx * gg.ny * gg.nz:
        raise ValueError("image size does not match the geometry")
    bx, by, bz = box if box is not None else forward_box(g)
    out = np.empty(_shape_data(gg), np.float64)
    rc = _load().oracle_forward_model(ctypes.byref(gg), _dptr(a), bx, by, bz, _dptr(out), nthreads)
    if rc == -2:
        raise ValueError("box smaller than the image")
    if rc:
        raise MemoryError("oracle_forward_model failed")
    return out.reshape(_out_shape(gg, gg.nt))
