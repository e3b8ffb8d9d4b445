#!/usr/bin/env python
"""Benchmark of the GB300 NUFFT Fourier reconstruction (libpai).

Metric: reconstructed voxels per second (whole job, all ranks), inputs already
resident in HBM, one step = one pai_reconstruct of one problem (or of the whole
batch for --config batched2d).  L2 is flushed (512 MiB write) before every
timed step; each step is timed with CUDA events on the launching stream.

Also reported on the same JSON line:
  roofline      the row kernel (the dominant hand-written kernel): algorithmic
                bytes per launch / its event-timed duration vs the measured HBM
                copy bandwidth, plus the ncu DRAM traffic recorded for it;
  e2e           the same metric through pai_reconstruct_host_async (pinned host
                buffers, H2D and D2H copies inside the timed region);
  cpu_baseline  the FP64 oracle (direct Fourier reconstruction) timed on this
                host's cores on a bounded sample of the same workload;
  clocks        nvidia-smi SM clock and throttle reasons sampled while timing.

``--impl reference`` times the oracle alone (the reference arm) on the same
workload, metric and unit.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reconstructed voxels/s and NUFFT-kernel HBM GB/s at rel L2<=1e-5, batched vs plain"
# workloads of several problems in one batched plan
MULTI_CONFIGS = ("batched2d", "frames2d")
# the GPU tests that hold each workload to the oracle
PARITY_TESTS = {
    "large2d": "tests/test_gpu_parity.py::test_large_2d_sampled_rows",
    "plain2d": "tests/test_gpu_parity.py::test_plain_2d_128x256",
    "planar3d": "tests/test_gpu_parity.py::test_3d_planar_128",
    "adjoint3d": "tests/test_gpu_adjoint.py",
    "batched2d": "tests/test_gpu_parity.py::test_batched_64_full_size_sampled_rows",
    "frames2d": "tests/test_gpu_parity.py::test_large_2d_sampled_rows (per frame), test_batched_*",
}
UNIT = "voxels/s"
L2_FLUSH_BYTES = 512 << 20


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def workload(name: str, seed: int = 0):
    """Returns (description, list of geometry dicts, list of float32 data arrays)."""
    import phantoms as ph

    def gd(g, **kw):
        d = dict(dim=g.dim, nx=g.nx, ny=g.ny, dx=g.dx, dy=g.dy, nt=g.nt, dt=g.dt, c=g.c, nz=g.nz, dz=g.dz)
        d.update(kw)
        return d

    if name == "large2d":
        pr = ph.large_2d(seed)
        return ("2-D line detector: 2048 detectors x 4096 samples -> 2048 x 2048 image, 50 f_circ discs "
                "(closed-form data) + white noise at 1% of peak; oversampling 2, K = 4 (16 taps)",
                [gd(pr.geom, oversampling=2.0, K=4.0)], [pr.p.astype(np.float32)])
    if name == "plain2d":
        pr = ph.plain_2d(seed)
        return ("2-D line detector: 128 detectors x 256 samples -> 128 x 128, 1-8 uniform discs (spectral "
                "propagation); oversampling 2, K = 3 (12 taps)",
                [gd(pr.geom, oversampling=2.0, K=3.0)], [pr.p.astype(np.float32)])
    if name == "planar3d":
        pr = ph.planar_3d(seed)
        return ("3-D planar detector: 128 x 128 detectors x 256 samples -> 128^3, 1-20 uniform balls (N-waves); "
                "oversampling 2, K = 3", [gd(pr.geom, oversampling=2.0, K=3.0)], [pr.p.astype(np.float32)])
    if name == "adjoint3d":
        pr = ph.adjoint_3d(seed)
        return ("3-D planar detector: 256 x 256 detectors x 512 samples -> 256^3, uniform balls; oversampling 2, K = 3",
                [gd(pr.geom, oversampling=2.0, K=3.0)], [pr.p.astype(np.float32)])
    if name == "frames2d":
        probs = [ph.large_2d(seed * 8 + i) for i in range(8)]
        return ("8 frames of the 2-D large workload (2048 x 4096 -> 2048 x 2048, independent seeds) in one batched "
                "plan; oversampling 2, K = 4", [gd(p.geom, oversampling=2.0, K=4.0) for p in probs],
                [p.p.astype(np.float32) for p in probs])
    if name == "batched2d":
        probs = ph.batched_2d(seed)
        return ("64 uneven 2-D problems (nx = 2 U{128..1024}, nt = 2 U{256..2048}, nz = nt/2) in one plan; "
                "f_circ disc phantoms; window left open: chosen by the plan's window tuner (truncation error <= 1e-7)",
                [gd(p.geom) for p in probs], [p.p.astype(np.float32) for p in probs])
    raise SystemExit(f"unknown config {name}")


def voxels_of(geoms) -> int:
    return sum(g["nx"] * (g["ny"] if g["dim"] == 3 else 1) * g["nz"] for g in geoms)


# ---------------------------------------------------------------------------
# oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

# wall-clock budget of a whole `--impl reference` run (the oracle on the host cores)
REF_BUDGET_S = 150.0


def oracle_rate(geoms, datas, target_s: float = 10.0, per_row_hint: float = 0.0):
    """Voxels/s of the FP64 oracle, estimated from a bounded sample: direct
    lateral DFT rows plus direct NUDFT rows (steps 1-3 of the direct Fourier
    reconstruction) for a subset of lateral frequencies of the first problem,
    extrapolated to all rows of every problem.  The final inverse DFT is not
    timed, so the rate is an upper bound on the oracle's speed.  per_row_hint:
    wall seconds per row measured earlier (skips the calibration run); at
    least one row per thread is timed."""
    import oracle
    import phantoms as ph

    g0 = geoms[0]
    G = ph.Geometry(**{k: g0[k] for k in ("dim", "nx", "ny", "dx", "dy", "nt", "dt", "c", "nz", "dz")})
    p = datas[0].astype(np.float64).reshape(G.data_shape)
    rng = np.random.default_rng(1)
    nrows_total = G.nx * (G.ny if G.dim == 3 else 1)

    def run(nrows):
        kx = rng.integers(-G.nx // 2, G.nx // 2, nrows)
        ky = rng.integers(-G.ny // 2, G.ny // 2, nrows) if G.dim == 3 else np.zeros(nrows, int)
        t = time.perf_counter()
        oracle.spectrum_rows(G, p, kx, ky)
        return time.perf_counter() - t

    n = max(1, oracle.threads())
    per_row = per_row_hint if per_row_hint > 0 else run(n) / n
    rows = int(min(nrows_total, max(n, target_s / max(per_row, 1e-9))))
    t = run(rows)
    per_row = t / rows
    # every problem costs rows x (nx ny nt + nz nt) in this model; scale by op count
    def cost(g):
        nl = g["nx"] * (g["ny"] if g["dim"] == 3 else 1)
        return nl * (nl * g["nt"] + g["nz"] * g["nt"])
    est = per_row / (G.nx * (G.ny if G.dim == 3 else 1) * G.nt + G.nz * G.nt) * sum(cost(g) for g in geoms)
    sample = (f"{rows} of {nrows_total} lateral-frequency rows of problem 0 (direct lateral DFT row + direct "
              f"NUDFT at {G.nz} nodes, FP64), {t:.1f} s wall on {n} threads, extrapolated by operation count "
              f"to the whole workload; inverse DFT not timed (rate is an upper bound)")
    return voxels_of(geoms) / est, n, sample, per_row


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

NVML_LOOP = r"""
import ctypes, sys, time
lib = ctypes.CDLL("libnvidia-ml.so.1")
assert lib.nvmlInit_v2() == 0
h = ctypes.c_void_p()
assert lib.nvmlDeviceGetHandleByUUID(sys.argv[1].encode(), ctypes.byref(h)) == 0
reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or lib.nvmlDeviceGetCurrentClocksThrottleReasons
clk, mx, mw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
out = open(sys.argv[2], "w", buffering=1)
while True:
    t = time.time()
    if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0
            and reasons(h, ctypes.byref(rs)) == 0):
        pw = mw.value / 1000.0 if lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(mw)) == 0 else -1.0
        out.write("%.6f %d %d %.3f %d\n" % (t, clk.value, mx.value, pw, rs.value))
    time.sleep(0.010)
"""


class NvmlClocks:
    """SM clock, power and clock-event-reason samples every 10 ms through NVML
    (read-only queries of the driver library) in a separate process, so that a
    timed region of a few milliseconds still holds samples and this process's
    launches do not wait on the sampler.  (Sampling every 2 ms measurably
    slowed 20-us steps; every 10 ms did not.)"""
    # NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, uuid):
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="pai_nvml_", suffix=".txt")
        os.close(fd)
        self.proc = subprocess.Popen([sys.executable, "-c", NVML_LOOP, uuid, self.path],
                                     stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        self.samples = []

    def start(self):
        # wait (at most 2 s) for the first sample so the timed region is covered
        t_end = time.time() + 2.0
        while time.time() < t_end and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            for line in open(self.path):
                f = line.split()
                if len(f) == 5:
                    pw = float(f[3])
                    self.samples.append((float(f[0]), float(f[1]), float(f[2]), pw if pw >= 0 else None, int(f[4])))
        except Exception:
            pass
        try:
            os.unlink(self.path)
        except OSError:
            pass


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.samples = []
        self.proc = None
        self.thread = None
        self.dev = device_index
        self.nvml = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        uuid = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
        except Exception:
            pass
        if uuid:
            uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            cmd += ["-i", uuid]
            try:
                self.nvml = NvmlClocks(uuid)
                self.nvml.start()
            except Exception:
                self.nvml = None
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.nvml:
            self.nvml.stop()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self, t0: float, t1: float):
        if self.nvml:
            inside = [r for r in self.nvml.samples if t0 <= r[0] <= t1]
            window = "timed region"
            if not inside:
                # a region shorter than the 10 ms period: the samples next to it
                inside = [r for r in self.nvml.samples if t0 - 0.015 <= r[0] <= t1 + 0.015]
                window = "timed region +- 15 ms"
            if inside:
                pw = [r[3] for r in inside if r[3] is not None]
                reasons = sorted({name for r in inside for bit, name in NvmlClocks.REASONS.items() if r[4] & bit})
                return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                        "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(inside),
                        "window": window, "source": "NVML, every 10 ms, separate process"}
        rows = []
        for ts, line in self.samples:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            rows.append((ts, parts))
        inside = [r for r in rows if t0 <= r[0] <= t1]
        window = "timed region"
        if not inside:
            inside = rows
            window = "whole run (no sample fell inside the timed region)"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(p[0]) for _, p in inside if num(p[0]) is not None]
        mx = [num(p[1]) for _, p in inside if num(p[1]) is not None]
        pw = [num(p[2]) for _, p in inside if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, p in inside for i in range(4) if p[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(inside),
                "window": window}


# ---------------------------------------------------------------------------
# measured peaks and committed ncu traffic
# ---------------------------------------------------------------------------

def hbm_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s)"


def kernel_source_hash() -> str:
    """Hash of the row kernels' source with // comments and blank lines removed
    (a comment edit leaves the recorded traffic valid; any code edit voids it)."""
    import re
    h = hashlib.sha256()
    for f in ("pai_row_kernels.cuh",):
        text = open(os.path.join(ROOT, "paper_0808_3510_gb300", "csrc", f), encoding="utf-8").read()
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()[:16]


def recorded_traffic(config: str):
    """DRAM bytes per launch of the forward row kernel from the committed ncu
    summary, or None when absent or recorded for different kernel source."""
    path = os.path.join(ROOT, "profiles", "row_forward_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get(config)
    if not e or e.get("kernel_source_sha") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# multi-rank aggregation (replicas: one independent problem per rank)
# ---------------------------------------------------------------------------

def aggregate_over_ranks(ms_local: float, voxels_local: int, device=None):
    """Whole-job numbers for independent replicas: the step time is the max over
    ranks, the throughput is the voxels all ranks reconstructed per step divided
    by that time.  Works with any torch.distributed backend (gloo / nccl); with
    no process group it is the single-rank case."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms_local, voxels_local / (ms_local * 1e-3)
    t = torch.tensor([ms_local, float(voxels_local)], dtype=torch.float64, device=device)
    m = t[:1].clone()
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    s = t[1:].clone()
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    ms_max = float(m.item())
    return ms_max, float(s.item()) / (ms_max * 1e-3)



def nvtx_range(push: bool, name: str = "timed_steps"):
    """Open (push) or close the NVTX range around the timed steps (no effect
    unless a profiler listens)."""
    try:
        import torch
        if push:
            torch.cuda.nvtx.range_push(name)
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def timed_steps(fn, reps, flush, stream):
    """Mean CUDA-event milliseconds of fn() over reps steps, L2 flushed before each."""
    import torch
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    for i in range(reps):
        flush.fill_(float(i & 7))
        e0[i].record(stream)
        fn()
        e1[i].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / reps


def window_summary(plan, count):
    """The window the plan's tuner kept for a batch (taps, padded lengths,
    oversampling, worst predicted error) and its tuning log."""
    infos = [plan.problem_info(i) for i in range(count)]
    return {"taps": sorted({i["taps"] for i in infos}),
            "M_range": [min(i["M"] for i in infos), max(i["M"] for i in infos)],
            "oversampling_range": [min(i["oversampling"] for i in infos), max(i["oversampling"] for i in infos)],
            "max_predicted_error": max(i["predicted_error"] for i in infos),
            "tuning_log": plan.tuning_log.strip().splitlines()}


def compare_batched_plain(pai, geoms, p, out, batched_ms, flush, stream, reps=20):
    """The problems of a batched plan as separate single-problem plans run one
    after another on the same stream: graph-replayed plans (each plan replays
    its own captured CUDA graph, as a user's single plan does) and eager plans
    (no graph).  Returns the batched-vs-plain record of the bench line."""
    import torch
    ins, outs, off_i, off_o = [], [], 0, 0
    sizes = []
    for g in geoms:
        gg = pai.geometry(g)
        ni = gg.nx * (gg.ny if gg.dim == 3 else 1) * gg.nt
        no = gg.nx * (gg.ny if gg.dim == 3 else 1) * gg.nz
        sizes.append((ni, no))
    res = {"batched_ms_per_step": batched_ms, "problems": len(geoms)}
    for mode in ("graph", "eager"):
        if mode == "eager":
            os.environ["PAI_USE_GRAPH"] = "0"
        try:
            plans = [pai.Plan(g) for g in geoms]
        finally:
            os.environ.pop("PAI_USE_GRAPH", None)
        ins, outs, off_i, off_o = [], [], 0, 0
        for pl, (ni, no) in zip(plans, sizes):
            ins.append(p.view(-1)[off_i: off_i + ni].view(pl._out_shape("nt")))
            outs.append(out.view(-1)[off_o: off_o + no].view(pl._out_shape("nz")))
            off_i += ni
            off_o += no

        def run_all():
            for pl, a, o in zip(plans, ins, outs):
                pl.reconstruct(a, o)
        for _ in range(3):
            run_all()
        torch.cuda.synchronize()
        res[f"plain_{mode}_ms_per_step"] = timed_steps(run_all, reps, flush, stream)
        for pl in plans:
            pl.close()
    res["plain_ms_per_step"] = res["plain_graph_ms_per_step"]
    res["speedup"] = res["plain_graph_ms_per_step"] / batched_ms
    res["speedup_vs_plain_eager"] = res["plain_eager_ms_per_step"] / batched_ms
    res["plain"] = (f"{len(geoms)} separate single-problem plans on the same stream, one after another; "
                    "'speedup' against graph-replayed plans, 'speedup_vs_plain_eager' against eager plans")
    return res


def fp32_fma_peak(dev, clocks):
    """FP32 FMA peak in TFLOP/s: SMs (queried) x 128 FP32 lanes per SM (sm_100
    family) x 2 flops x the maximum SM clock (nvidia-smi, sampled during the
    timed region; else the measured-peaks file)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz, src = None, None
    if clocks and clocks.get("sm_max_mhz"):
        mhz, src = float(clocks["sm_max_mhz"]), "nvidia-smi clocks.max.sm"
    else:
        try:
            mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
            src = "MEASURED_PEAKS.json sm_max_mhz"
        except Exception:
            mhz, src = 2070.0, "nominal 2070 MHz"
    peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    return peak, f"FP32 FMA: {sms} SMs x 128 lanes x 2 flops x {mhz:g} MHz ({src})"

# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

# ---------------------------------------------------------------------------
# the discrete forward model (pai_forward_model): image -> detector data
# ---------------------------------------------------------------------------

FORWARD_CONFIGS = {
    "forward3d": "3-D: 128^3 initial pressure (1-20 uniform balls) -> 128 x 128 detectors x 256 samples",
    "forward2d": "2-D: 2048 x 2048 initial pressure (50 f_circ discs) -> 2048 detectors x 4096 samples",
    "datamodel2d": "2-D partial data g = w_cut Q f (Eq. data-part): forward2d with the cutoff eps = 16 fused into "
                   "the copy of the detector rows",
}


def run_forward_model(args, rank, world, local_rank):
    """One step = one pai_forward_model call (image resident in HBM, data written
    to HBM); value = image voxels per second over all ranks."""
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the FP64 oracle of the forward model evaluates "
                              "every (box frequency, time) cosine directly; a bounded sample of this workload is "
                              "not representative"}))
        return
    import torch
    import phantoms as ph
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    else:
        torch.cuda.set_device(0)
    from paper_0808_3510_gb300 import build as pai_build
    if rank == 0 or world == 1:
        pai_build.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_0808_3510_gb300 as pai
    rng = np.random.default_rng(rank)
    if args.config == "forward3d":
        g = ph.Geometry(dim=3, nx=128, ny=128, nt=256, nz=128)
        img = ph.balls_3d_image(g, ph.random_balls(rng, g, int(rng.integers(1, 21)), 3.0, 15.0))
        K = 3.0
    else:
        g = ph.Geometry(dim=2, nx=2048, nt=4096, nz=2048)
        img = ph.fcirc_2d_image(g, ph.random_discs(rng, g, 50, 2.0, 12.0))
        K = 4.0
    gdict_ = dict(dim=g.dim, nx=g.nx, ny=g.ny, dx=g.dx, dy=g.dy, nt=g.nt, dt=g.dt, c=g.c, nz=g.nz, dz=g.dz,
                  oversampling=2.0, K=K)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    model = pai.ForwardModel(gdict_, cutoff=16.0 if args.config == "datamodel2d" else None)
    f = torch.from_numpy(img.astype(np.float32)).to(dev)
    out = torch.empty(g.data_shape, device=dev, dtype=torch.float32)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev, dtype=torch.float32)
    for _ in range(args.warmup):
        model(f, out)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    l0 = model.kernel_launches
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    for i in range(args.steps):
        flush.fill_(float(i & 7))
        starts[i].record(stream)
        model(f, out)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t1 = time.time()
    launches = model.kernel_launches - l0
    ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / args.steps
    time.sleep(0.2)
    sampler.stop()
    clocks = sampler.summary(t0, t1)
    ms_max, value = aggregate_over_ranks(ms, g.voxels, dev)
    st = model.profile_stages(reps=20)
    bx, by, bz = model.box
    rows = bx * (by // 2 + 1) if g.dim == 3 else bx // 2 + 1
    nbytes_alg = rows * (bz + g.nt) * 8  # depth spectrum rows in, temporal rows out
    peak, peak_src = hbm_peak()
    achieved = nbytes_alg / (st[1] * 1e-3) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.config}: {FORWARD_CONFIGS[args.config]}; padded box {bx} x {by} x {bz}, "
                       f"oversampling 2, K = {K:g}", "voxels_per_step": g.voxels, "box": [bx, by, bz],
                       "l2": "flushed before every timed step (512 MiB write)", "parallelism": f"replicas x{world}"},
            "step": "forward model (image -> detector data)",
            "parity": {"checked_by": "tests/test_gpu_cutoff.py::test_data_model_against_oracle"
                       if args.config == "datamodel2d" else "tests/test_gpu_forward.py", "bar_rel_l2": 1e-5},
            "roofline": {"bound": "hbm", "kernel": "row_adjoint in forward-model mode (node pairs, spread, inverse "
                         "FFT, crop)", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": peak_src, "algorithmic_bytes_per_launch": nbytes_alg,
                         "kernel_ms": st[1], "stage_ms": {"image_fft": st[0], "row_kernel": st[1],
                                                           "lateral_inverse_fft": st[2]}},
            "cpu_baseline": None, "e2e": {"value": None, "unit": UNIT, "note": "no host-memory entry point"},
            "gpu_launches": launches, "clocks": clocks, "wall_s_timed_region": t1 - t0,
            "tuning_log": model.tuning_log.strip().splitlines(),
        }))
    model.close()


# ---------------------------------------------------------------------------
# the data cutoff w_cut (pai_cutoff): partial data g = w_cut * p
# ---------------------------------------------------------------------------

CUTOFF_DESC = ("2-D: w_cut (Eq. data-part) applied to 2048 detectors x 4096 samples of random data, eps = 16 "
               "squared sampling steps (support radius 4 steps), out of place")


def run_cutoff(args, rank, world, local_rank):
    """One step = one out-of-place pai_cutoff over the 2-D large data grid
    (33.6 MB read, 33.6 MB written); value = data samples per second over all
    ranks.  The in-place call (only the samples within reach of a face are
    rewritten) is timed beside it."""
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle of w_cut integrates the mollifier "
                              "over each sample's own box; it is a checker, not a timed program"}))
        return
    import torch
    import phantoms as ph
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    else:
        torch.cuda.set_device(0)
    from paper_0808_3510_gb300 import build as pai_build
    if rank == 0 or world == 1:
        pai_build.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_0808_3510_gb300 as pai
    g = ph.Geometry(dim=2, nx=2048, nt=4096, nz=2048)
    eps = 16.0
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    plan = pai.Plan(dict(dim=2, nx=g.nx, nt=g.nt, nz=g.nz, K=4.0))
    plan.set_cutoff(eps)
    rng = np.random.default_rng(rank)
    p = torch.from_numpy(rng.standard_normal((g.nx, g.nt)).astype(np.float32)).to(dev)
    out = torch.empty_like(p)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev, dtype=torch.float32)
    samples = g.nx * g.nt

    def timed(fn, steps):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i & 7))
            starts[i].record(stream)
            fn()
            ends[i].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / steps

    for _ in range(args.warmup):
        plan.cutoff(p, out)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    l0 = plan.kernel_launches
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    ms = timed(lambda: plan.cutoff(p, out), args.steps)
    if world > 1:
        torch.distributed.barrier()
    t1 = time.time()
    launches = plan.kernel_launches - l0
    time.sleep(0.2)
    sampler.stop()
    clocks = sampler.summary(t0, t1)
    ms_in_place = timed(lambda: plan.cutoff(p, p), min(args.steps, 200))
    ms_max, value = aggregate_over_ranks(ms, samples, dev)
    nbytes_alg = samples * 8
    peak, peak_src = hbm_peak()
    achieved = nbytes_alg / (ms * 1e-3) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": "data samples/s through w_cut", "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"cutoff2d: {CUTOFF_DESC}", "samples_per_step": samples, "eps": eps,
                       "l2": "flushed before every timed step (512 MiB write)", "parallelism": f"replicas x{world}"},
            "step": "data cutoff (pai_cutoff, out of place)",
            "parity": {"checked_by": "tests/test_gpu_cutoff.py::test_cutoff_full_size_sampled",
                       "bar": "2.5e-7 relative per sample"},
            "roofline": {"bound": "hbm", "kernel": "cutoff_kernel (one streaming pass)", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                         "peak_source": peak_src, "algorithmic_bytes_per_launch": nbytes_alg, "kernel_ms": ms},
            "in_place_ms": ms_in_place,
            "cpu_baseline": None, "e2e": {"value": None, "unit": "samples/s", "note": "no host-memory entry point"},
            "gpu_launches": launches, "clocks": clocks, "wall_s_timed_region": t1 - t0,
        }))
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 2000; 20 for --impl reference)")
    ap.add_argument("--warmup", type=int, default=None, help="warm-up steps (default 20; 3 for --impl reference)")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--config", default="large2d", choices=["large2d", "plain2d", "planar3d", "adjoint3d",
                                                            "batched2d", "frames2d", "forward3d", "forward2d",
                                                            "datamodel2d", "cutoff2d"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 64-problem batched-vs-plain measurement of the default run")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 20 if args.impl == "reference" else 2000
    if args.warmup is None:
        args.warmup = 3 if args.impl == "reference" else 20
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.config in FORWARD_CONFIGS:
        return run_forward_model(args, rank, world, local_rank)
    if args.config == "cutoff2d":
        return run_cutoff(args, rank, world, local_rank)

    if args.impl == "reference":
        if rank != 0:
            return
        desc, geoms, datas = workload(args.config)
        vals = []
        cores, sample = 0, ""
        # each step a bounded sample: about REF_BUDGET_S seconds for the whole
        # run, at most 2 s and at least one row per thread per step
        target = min(2.0, REF_BUDGET_S / (args.warmup + args.steps))
        per_row = 0.0
        for i in range(args.warmup + args.steps):
            v, cores, sample, per_row = oracle_rate(geoms, datas, target_s=target, per_row_hint=per_row)
            if i >= args.warmup:
                vals.append(v)
        value = float(statistics.median(vals))
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.config}: {desc}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    import torch

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    else:
        torch.cuda.set_device(0)

    from paper_0808_3510_gb300 import build as pai_build
    if rank == 0 or world == 1:
        pai_build.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_0808_3510_gb300 as pai

    desc, geoms, datas = workload(args.config, seed=rank)
    flat = np.concatenate([d.ravel() for d in datas]).astype(np.float32)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    multi = args.config in MULTI_CONFIGS
    plan = pai.Plan(geoms if multi else geoms[0])
    p_host = torch.from_numpy(flat).pin_memory()
    p = p_host.to(dev)
    out = torch.empty(plan.image_numel, device=dev, dtype=torch.float32)
    if not multi:
        out = out.view(plan._out_shape("nz"))
        p = p.view(plan._out_shape("nt"))
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev, dtype=torch.float32)
    vox = voxels_of(geoms)

    # Parity with the FP64 oracle is established by the GPU tests, at this
    # workload's size and launch configuration as well (sampled spectrum rows);
    # this script runs the oracle only in its CPU-baseline and reference legs.
    parity = {"checked_by": PARITY_TESTS.get(args.config, "tests/test_gpu_parity.py"), "bar_rel_l2": 1e-5}

    grad_mode = args.config == "adjoint3d"
    if grad_mode:
        # one step = the gradient of 0.5 ||R p - f_true||^2 with respect to p
        import phantoms as ph
        g0 = geoms[0]
        G = ph.Geometry(**{k: g0[k] for k in ("dim", "nx", "ny", "dx", "dy", "nt", "dt", "c", "nz", "dz")})
        prob = ph.adjoint_3d(rank)
        f_true = torch.from_numpy(ph.balls_3d_image(G, prob.objects).astype(np.float32)).to(dev)
        grad = torch.empty_like(p)

    def step():
        if grad_mode:
            plan.reconstruct(p, out)
            out.sub_(f_true)
            plan.adjoint(out, grad)
        else:
            plan.reconstruct(p, out)

    # warm-up (also captures the CUDA graphs)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = plan.kernel_launches
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    nvtx_range(True)  # marks the timed steps for a profiler's launch filter
    for i in range(args.steps):
        flush.fill_(float(i & 7))
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    nvtx_range(False)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t1 = time.time()
    launches = plan.kernel_launches - launches0
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps
    time.sleep(0.2)
    sampler.stop()
    clocks = sampler.summary(t0, t1)
    ms_max, value = aggregate_over_ranks(ms, vox, dev)

    # roofline of the row kernel
    st = plan.profile_stages(p, out, reps=50)
    st_adj = plan.profile_stages(out, grad, reps=20, adjoint=True) if grad_mode else None
    info = plan.info
    # algorithmic bytes of the row kernel: the scope table's per-node figure for
    # the gather with the weight (each oversampled-spectrum element inside some
    # node's tap window read once, 8 B written per node: about 20 B per node in
    # the half-lateral layout) times the nodes one launch evaluates; and, beside
    # it, the fused kernel's own input and output (lateral spectrum rows in,
    # half image spectrum out), which is all it moves through HBM
    nbytes_alg = 0
    nbytes_io = 0
    for g in geoms:
        nl = g["nx"] * (g["ny"] if g["dim"] == 3 else 1)
        half = (g["ny"] if g["dim"] == 3 else g["nx"]) // 2 + 1
        rows = (g["nx"] if g["dim"] == 3 else 1) * half
        nbytes_alg += 20 * nl * g["nz"]
        nbytes_io += rows * g["nt"] * 8 + nl * (g["nz"] // 2 + 1) * 8
    peak, peak_src = hbm_peak()
    achieved = nbytes_alg / (st[1] * 1e-3) / 1e9
    achieved_io = nbytes_io / (st[1] * 1e-3) / 1e9
    # ALU view of the same launch: 5 M log2 M flops per row FFT; per +-nu pair task
    # 16 H (tap accumulation: two nodes x 2H taps x 2 FMA) + 16 H (per tap pair two
    # 4-term polynomials in z^2 and the two weights) + 40 (node position, phase,
    # weight) flops
    flops = 0
    for i, g in enumerate(geoms):
        pinfo = plan.problem_info(i)
        H = max(pinfo["taps"] // 2, 1)
        M = pinfo["M"]
        half = (g["ny"] if g["dim"] == 3 else g["nx"]) // 2 + 1
        rows = (g["nx"] if g["dim"] == 3 else 1) * half
        flops += rows * (5 * M * math.log2(M) + (g["nz"] // 2 + 1) * (32 * H + 40))
    fp32_peak, fp32_src = fp32_fma_peak(dev, clocks)
    roofline = {"bound": "hbm", "kernel": "row_forward (prescale + oversampled FFT + KB gather + weight)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(args.config), "peak_source": peak_src,
                "algorithmic_bytes_per_launch": nbytes_alg,
                "algorithmic_bytes": "20 B per node (gather + weight, half-lateral layout) x nodes per launch",
                "fused_io": {"bytes_per_launch": nbytes_io, "achieved": achieved_io, "frac": achieved_io / peak,
                             "what": "lateral spectrum rows in + half image spectrum out"},
                "kernel_ms": st[1],
                "stage_ms": {"lateral_fft": st[0], "row_kernel": st[1], "inverse_fft": st[2]},
                "alu_view": {"flops_per_launch": flops, "achieved_tflops": flops / (st[1] * 1e-3) / 1e12,
                             "peak_tflops": fp32_peak, "frac": flops / (st[1] * 1e-3) / 1e12 / fp32_peak,
                             "peak_source": fp32_src}}
    if st_adj is not None:
        roofline["adjoint_stage_ms"] = {"image_fft": st_adj[0], "row_adjoint_kernel": st_adj[1],
                                        "lateral_inverse_fft": st_adj[2]}

    # batched vs plain: the same problems as separate single-problem plans, one
    # after another (graph-replayed, the fair comparison, and eager)
    batched = None
    if multi:
        batched = compare_batched_plain(pai, geoms, p, out, ms, flush, stream)
        batched["window"] = window_summary(plan, len(geoms))
    elif args.config == "large2d" and not args.no_batched and rank == 0:
        # the default run also measures the batched half of the metric on the
        # 64-problem uneven batch (the headline value stays the single problem)
        bdesc, bgeoms, bdatas = workload("batched2d", seed=0)
        bflat = torch.from_numpy(np.concatenate([d.ravel() for d in bdatas]).astype(np.float32)).to(dev)
        del bdatas
        bplan = pai.Plan(bgeoms)
        bout = torch.empty(bplan.image_numel, device=dev, dtype=torch.float32)
        for _ in range(3):
            bplan.reconstruct(bflat, bout)
        torch.cuda.synchronize()
        bms = timed_steps(lambda: bplan.reconstruct(bflat, bout), 20, flush, stream)
        batched = compare_batched_plain(pai, bgeoms, bflat, bout, bms, flush, stream)
        batched["workload"] = f"batched2d: {bdesc}"
        batched["voxels_per_step"] = voxels_of(bgeoms)
        batched["batched_voxels_per_s"] = voxels_of(bgeoms) / (bms * 1e-3)
        batched["window"] = window_summary(bplan, len(bgeoms))
        bplan.close()
        del bflat, bout
        torch.cuda.empty_cache()

    # end to end through host memory: a stream of steps through the pipelined
    # host call (upload, transforms and download of consecutive steps overlap);
    # every step's upload and download lie inside the timed region
    e2e = None
    if not args.no_e2e and grad_mode:
        e2e = {"value": None, "unit": UNIT,
               "note": "the gradient step has no host-memory entry point; the forward's end-to-end "
                       "number is reported by --config planar3d / large2d"}
    elif not args.no_e2e:
        src = p_host if multi else p_host.view(plan._out_shape("nt"))
        ins = [src, src.clone().pin_memory()]
        outs = [torch.empty(plan._out_shape("nz"), dtype=torch.float32).pin_memory() for _ in range(2)]
        for i in range(4):
            plan.reconstruct_host_async(ins[i % 2], outs[i % 2])
        plan.host_wait()
        reps = 200  # a stream long enough that filling and draining the pipeline is a small part
        torch.cuda.synchronize()
        t = time.perf_counter()
        for i in range(reps):
            plan.reconstruct_host_async(ins[i % 2], outs[i % 2])
        plan.host_wait()
        el = (time.perf_counter() - t) / reps
        # one synchronous call (upload, transforms, download back to back) for its latency
        for _ in range(3):
            plan.reconstruct_host(ins[0], outs[0])
        t = time.perf_counter()
        for _ in range(10):
            plan.reconstruct_host(ins[0], outs[0])
        lat = (time.perf_counter() - t) / 10
        e2e = {"value": vox * world / el, "unit": UNIT, "h2d_bytes_per_step": int(flat.nbytes),
               "d2h_bytes_per_step": int(plan.image_numel * 4), "ms_per_step": el * 1e3,
               "api": "pai_reconstruct_host_async over page-locked buffers, steps pipelined",
               "sync_call_ms": lat * 1e3}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, cores, sample, _ = oracle_rate(geoms, datas, target_s=10.0)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.config}: {desc}", "problems": len(geoms), "voxels_per_step": vox,
                       "M": info["M"], "taps": info["taps"], "oversampling": info["oversampling"],
                       "K": info["K"], "predicted_window_error": info["predicted_error"],
                       "threads_per_cta": info["threads_per_cta"], "ctas": info["ctas"],
                       "cuda_graph": bool(info["uses_graph"]),
                       "l2": "flushed before every timed step (512 MiB write)",
                       "parallelism": f"replicas x{world}"},
            "parity": parity,
            "roofline": roofline,
            "batched_vs_plain": batched,
            "tuning_log": plan.tuning_log.strip().splitlines(),
            "step": "gradient of 0.5||R p - f||^2 (reconstruct + residual + adjoint)" if grad_mode else "reconstruct",
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "wall_s_timed_region": t1 - t0,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
