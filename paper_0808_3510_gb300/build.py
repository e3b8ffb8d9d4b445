"""Build libpai.so (the CUDA library behind include/pai.h) for sm_103a.

Translation units are compiled in parallel with nvcc and linked into
``paper_0808_3510_gb300/_build/libpai.so`` (in-tree, git-ignored).  Run as
``python -m paper_0808_3510_gb300.build`` or through ``__graft_entry__.build()``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpai.so")
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# (source, extra defines, object name)
UNITS = [
    ("pai_api.cu", [], "pai_api.o"),
    ("pai_launch.cu", [], "pai_launch.o"),
    ("pai_window.cpp", [], "pai_window.o"),
    ("pai_plan_math.cpp", [], "pai_plan_math.o"),
    ("pai_noalloc.cu", [], "pai_noalloc.o"),
    ("pai_lateral.cu", [], "pai_lateral.o"),
    ("pai_cutoff.cu", [], "pai_cutoff.o"),
    ("pai_row_inst.cu", ["-DPAI_HLO=2", "-DPAI_HHI=4"], "pai_row_h2.o"),
    ("pai_row_inst.cu", ["-DPAI_HLO=5", "-DPAI_HHI=6"], "pai_row_h5.o"),
    ("pai_row_inst.cu", ["-DPAI_HLO=7", "-DPAI_HHI=8"], "pai_row_h7.o"),
    ("pai_row_inst.cu", ["-DPAI_HLO=9", "-DPAI_HHI=12"], "pai_row_h9.o"),
]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpai")


def _cuda_lib_dir(nvcc: str) -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        d = os.path.join(root, sub)
        if os.path.exists(os.path.join(d, "libcufft.so")):
            return d
    return os.path.join(root, "lib64")


def _sources_newer(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "pai.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every unit for sm_103a and link libpai.so; returns its path."""
    if not force and not _sources_newer(LIB):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    libdir = _cuda_lib_dir(nvcc)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]

    def compile_unit(u):
        src, defs, obj = u
        cmd = [nvcc] + common + defs + ["-c", os.path.join(CSRC, src), "-o", os.path.join(BUILD, obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + [os.path.join(BUILD, o) for o in objs] + [
        "-L", libdir, "-lcufft", "-Xlinker", f"-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
