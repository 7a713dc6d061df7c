#!/usr/bin/env python
"""Benchmark: cell-updates per second per Runge-Kutta stage on the bulk
workload (256 x 256 x 64 cells of 2 nm, 64 Voronoi grains, FP32 fields), the
plain FP64 path beside it, and the CPU oracle as baseline.

One step = one classic RK4 step = four full stages of the hot path (demag by
the five FFT passes, local terms + LLG + RK combination, renormalisation).
value = cells x 4 x steps / device time, summed over ranks (replicas: every
rank solves its own copy; no data-path collective).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.
"""
import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK stage at 256x256x64 (FP32 fields)"
UNIT = "cell-updates/s"
WORKLOAD = "bulk 256x256x64 cells of 2 nm, Ms 1e6 A/m, A 1.5e-11 J/m, Ku1 4e5 J/m^3 on 64 Voronoi grains, alpha 0.1, RK4 dt 5e-14 s"
STAGES_PER_STEP = 4
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (non-tensor) nominal rate: used only if the probe cannot run


# ----------------------------------------------------------------- models --
def padded(n):
    """The library's padded FFT extents (mm_fft_extent)."""
    from paper_2302_08843_gb300.binding import padded_extents
    return list(padded_extents(n))


def kernel_bytes(n, s, grains=True, ms_cell=False):
    """Algorithmic HBM bytes per launch of each kernel (data the kernel must
    read or write once), for real size s (4 FP32, 8 FP64)."""
    nx, ny, nz = n
    N = nx * ny * nz
    LX, LY, LZ = padded(n)
    KX = LX // 2 + 1
    cs = 2 * s
    S1 = 3 * nz * ny * KX * cs
    S2 = 3 * nz * LY * KX * cs
    tens = 6 * (LZ // 2 + 1) * (LY // 2 + 1) * KX * s
    v3 = 3 * N * s
    g = N if grains else 0
    mc = N * s if ms_cell else 0
    # stage kernel of RK4, averaged over the four stages:
    # reads m_s, h_demag, m_n (all stages), acc (stages 2-4), grain ids; writes acc (1-3), next (all)
    stage = (4 * (3 * v3 + g + mc) + 3 * v3 + 3 * v3 + 4 * v3) / 4.0
    # fused x-inverse + stage + x-forward: reads S1, m_s, m_n, grain ids, acc (3 of 4 stages);
    # writes acc (3 of 4), next and S1
    k5 = S1 + (4 * (3 * v3 + g) + 3 * v3 + 3 * v3 + 4 * v3) / 4.0 + S1
    return {
        "k5_fused": k5,
        "p1_x_forward": v3 + mc + S1,
        "p2_y_forward": S1 + S2,
        "p3_z_conv": 2 * S2 + tens,
        "p4_y_inverse": S2 + S1,
        "p5_x_inverse": S1 + v3,
        "stage_llg": stage,
    }


def model_stage_bytes(n, s):
    """The per-stage traffic model of the design notes (one HBM read+write per
    FFT axis pass, tensor once, 73 B/cell of local/RK traffic at FP32; scaled
    with the real size)."""
    nx, ny, nz = n
    LX, LY, LZ = padded(n)
    KX = LX // 2 + 1
    cs = 2 * s
    fft = 4 * 3 * cs * KX * ny * nz + 4 * 3 * cs * KX * LY * nz
    tens = 6 * s * KX * (ny + 1) * (nz + 1)
    local = (73.0 / 4.0) * s * nx * ny * nz
    return fft + tens + local


def floor_stage_bytes(n, s):
    """Compulsory traffic of one stage with no intermediates: m_s read once,
    the tensor spectrum once, and the RK state (m_n, acc read/write, grain id,
    m_{s+1} write)."""
    nx, ny, nz = n
    LX, LY, LZ = padded(n)
    KX = LX // 2 + 1
    N = nx * ny * nz
    tens = 6 * s * KX * (ny + 1) * (nz + 1)
    return tens + N * (3 * s + 1 + 3 * s + 2 * (3 * s) * 0.75 + 3 * s)


def stage_flops(n):
    """Floating-point operations of one stage (5 L log2 L per complex line
    transform, half for a real line, 30 per k-point for the 3x3 multiply,
    about 150 per cell for local terms, LLG and the RK combination)."""
    nx, ny, nz = n
    LX, LY, LZ = padded(n)
    KX = LX // 2 + 1
    lg = lambda L: math.log2(L) if L > 1 else 0.0
    f = 2 * 3 * ny * nz * 2.5 * LX * lg(LX)                 # P1 + P5
    f += 2 * 3 * nz * KX * 5 * LY * lg(LY)                  # P2 + P4
    f += KX * LY * 3 * 2 * 5 * LZ * lg(LZ) + KX * LY * LZ * 30   # P3
    f += 150 * nx * ny * nz
    return f


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self, gpu_indices):
        if self.p is None:
            return None
        time.sleep(0.3)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    idx = int(parts[0])
                except ValueError:
                    continue
                if idx in gpu_indices:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows)}


class UtilSampler:
    """nvidia-smi utilization.gpu (the share of each sample period in which a
    kernel was running) sampled every 200 ms while the served stream runs."""

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=index,utilization.gpu",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self, gpu_indices):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        vals = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) == 2 and parts[0].isdigit() and parts[1].isdigit() and int(parts[0]) in gpu_indices:
                    vals.append(float(parts[1]))
        os.unlink(self.f.name)
        if not vals:
            return None
        return {"mean": round(statistics.mean(vals) / 100.0, 4), "median": round(statistics.median(vals) / 100.0, 4),
                "samples": len(vals)}


# ---------------------------------------------------------- FP64 peak --
def fp64_peak_measure(torch, gpu_indices):
    """FP64 FMA rate of this GPU: the library's probe kernel (8 CTAs of 256
    threads per SM, every thread 8 independent chains of dependent FMAs),
    timed with CUDA events on the launching stream after warm-up launches,
    with the SM clock sampled meanwhile.  Changes no GPU setting."""
    from paper_2302_08843_gb300.binding import probe_fp64_fma
    stream = torch.cuda.current_stream()
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, iters = 8 * nsm, 4096
    for _ in range(3):
        probe_fp64_fma(stream.cuda_stream, sink.data_ptr(), blocks, iters)
    torch.cuda.synchronize()
    sampler = ClockSampler()
    sampler.start()
    time.sleep(0.3)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    fl = 0.0
    a.record(stream)
    for _ in range(40):
        fl += probe_fp64_fma(stream.cuda_stream, sink.data_ptr(), blocks, iters)
    b.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop(gpu_indices)
    ms = a.elapsed_time(b)
    return {"tflops": round(fl / (ms / 1e3) / 1e12, 4), "launches": 40, "ms": round(ms, 3),
            "kernel": "fp64_fma_probe_kernel (%d CTAs x 256 threads, 8 chains x %d FMAs per thread)" % (blocks, iters),
            "clocks": clocks}


# ---------------------------------------------------------- CPU baseline --
def _oracle_sample(result_path, n_stages, crop):
    """Time RK stages of the unmodified oracle on the bulk workload (or a crop
    of the same construction), then three stages of each small configuration
    (plain 32x32x4, thin film 512x128x1, multilayer crop 64x64x8).  Runs in a
    spawned process."""
    sys.path.insert(0, ROOT)
    from oracle.llg import Problem
    from paper_2302_08843_gb300 import workloads as W

    def stages(w, n, **kw):
        prob = Problem(w.n, w.dx, Ms=w.Ms, A=w.A, alpha=w.alpha, Ku1=w.Ku1, ku_axis=w.ku_axis_cells(),
                       h_ext=w.h_ext(0.0) if callable(w.h_ext) else w.h_ext, **kw)
        m = w.m0
        t0 = time.perf_counter()
        for s in range(n):
            k = prob.rhs(m, s * w.dt)
            m = m + 0.5 * w.dt * k
        return time.perf_counter() - t0

    w = W.bulk(crop=crop)
    el = stages(w, n_stages)
    small = {}
    for name, ws, kw in (("plain_fp64_32x32x4", W.plain_fp64(), {}), ("thin_film_512x128x1", W.thin_film(), {}),
                         ("multilayer_64x64x8", W.multilayer(n=(64, 64, 8)), None)):
        if kw is None:
            kw = {"layers": ws.extra["layers"]}
        sec = stages(ws, 3, **kw)
        small[name] = {"cell_updates_per_s": ws.ncells * 3 / sec, "stages": 3, "seconds": round(sec, 3)}
    from oracle.demag import FFT_BACKEND, FFT_WORKERS
    json.dump({"seconds": el, "stages": n_stages, "cells": w.ncells, "n": list(w.n), "small": small,
               "cpu_count": os.cpu_count(), "fft": FFT_BACKEND, "fft_workers": FFT_WORKERS},
              open(result_path, "w"))


def start_cpu_baseline(n_stages=1, crop=None):
    ctx = mp.get_context("spawn")
    path = tempfile.NamedTemporaryFile(suffix=".json", delete=False).name
    p = ctx.Process(target=_oracle_sample, args=(path, n_stages, crop))
    p.start()
    return p, path


def finish_cpu_baseline(p, path, sample_desc):
    p.join()
    try:
        r = json.load(open(path))
    except Exception:
        return None
    finally:
        try:
            os.unlink(path)
        except OSError:
            pass
    return {"value": r["cells"] * r["stages"] / r["seconds"], "unit": UNIT, "cores": r["fft_workers"],
            "kind": "oracle", "sample": sample_desc % r, "host_cpu_count": r["cpu_count"],
            "threads": "FFTs: %s; the element-wise NumPy terms: 1 thread" % r["fft"],
            "small_configs": r.get("small")}


# ------------------------------------------------------------------ ours --
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(torch, dist, v, device):
    """The largest of every rank's v (all ranks get it); v itself without a
    process group."""
    if dist is None:
        return v
    tt = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def serve_replicas(torch, dist, rank, ws, requests, server):
    """Replicas only: rank r serves requests r, r+ws, ... of the stream with
    its own server (no collective on the data path); rank 0 gathers every
    result and the max elapsed time.  Returns (results in stream order,
    elapsed) on rank 0 and (None, elapsed) elsewhere."""
    from paper_2302_08843_gb300.serving import shard, unshard
    mine = shard(requests, rank, ws)
    res = server.run(mine, realtime=True)
    elapsed = max_over_ranks(torch, dist, server.elapsed, "cpu" if dist is None or
                             dist.get_backend() == "gloo" else "cuda")
    if dist is None:
        return res, elapsed
    parts = [None] * ws if rank == 0 else None
    dist.gather_object(res, parts, dst=0)
    return (unshard(parts, len(requests)) if rank == 0 else None), elapsed


def traffic_for(kernel, precision):
    """ncu DRAM bytes per launch from the committed profile summary, or None
    when the kernel sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("source_hash") != source_hash():
        return None
    e = d.get("kernels", {}).get(precision, {}).get(kernel)
    return None if e is None else e.get("dram_bytes_per_launch")


# the files that define the timed FP32 stage kernels (device code and the
# launch configuration); a change to any of them invalidates stored counters
KERNEL_SOURCES = ("demag_passes.cu", "demag_rt.cu", "fft_engine.cuh", "fft_pair.cuh", "common.cuh", "tma.cuh",
                  "demag.h")


def source_hash():
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2302_08843_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(f.encode())
        h.update(open(os.path.join(src, f), "rb").read())
    return h.hexdigest()[:16]


def time_precision(torch, w, precision, steps, warmup, peaks):
    from paper_2302_08843_gb300.binding import setup_workload
    stream = torch.cuda.current_stream()
    s = setup_workload(w, precision, stream=stream)
    t = 0.0
    for _ in range(warmup):
        t, _ = s.step(w.dt, t, "rk4")
    torch.cuda.synchronize()
    # the timed steps run without per-kernel events (an event between two
    # launches would also cancel their programmatic overlap); the per-kernel
    # split comes from a second, profiled run of the same steps
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        t, _ = s.step(w.dt, t, "rk4")
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    s.profile_enable(True)
    for _ in range(steps):
        t, _ = s.step(w.dt, t, "rk4")
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile_enable(False)
    return s, ms, prof


def e2e_measure(torch, s, w, steps, warmup):
    """Same metric through the C ABI with host buffers: every step copies m in
    from pinned host memory (mm_set_m), runs one RK4 step (mm_llg_step) and
    reads m back to pinned host memory (mm_get_m, which waits for the copy).
    Two states on two CUDA streams take the steps in turn, so that step k's
    copy in and compute overlap step k-1's copy out; the timed region holds
    every step's copies."""
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import to_soa
    dt = "float32" if s.dtype == torch.float32 else "float64"
    s2 = setup_workload(w, "fp32" if s.dtype == torch.float32 else "fp64", stream=torch.cuda.Stream())
    states = [s, s2]
    mh = [torch.from_numpy(to_soa(w.m0).astype(dt)).pin_memory() for _ in range(2)]
    out = [torch.empty_like(mh[0]).pin_memory() for _ in range(2)]
    t = [0.0, 0.0]

    def run(n):
        for k in range(n):
            q = k & 1
            states[q].set_m(mh[q])
            t[q], _ = states[q].step(w.dt, t[q], "rk4")
            if k >= 1:
                states[q ^ 1].get_m_host(out[q ^ 1])
        states[(n - 1) & 1].get_m_host(out[(n - 1) & 1])

    run(warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run(steps)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    s2.close()
    nbytes = mh[0].numel() * mh[0].element_size()
    return el, nbytes


def b1_cufft_measure(torch, w, steps, warmup, s32):
    """Comparison baseline B1: the same RK4 stage written as library FFTs and
    separate elementwise PyTorch kernels -- torch.fft (cuFFT) rfftn/irfftn over
    the full zero-padded grid, the 3x3 multiply with the unfolded real tensor
    spectrum, the exchange stencil by slicing, anisotropy, LLG and the RK4
    combination as tensor expressions.  FP32, inputs resident, timed with CUDA
    events like the main path.  Also returns its field's relative max-norm
    difference from mm_heff's FP32 field on the same m."""
    from paper_2302_08843_gb300.binding import demag_spectrum_host, padded_extents
    from paper_2302_08843_gb300.workloads import to_soa
    mu0, gamma = 4e-7 * math.pi, 2.21e5
    dev = "cuda"
    nx, ny, nz = w.n
    Px, Py, Pz = padded_extents(w.n)
    oct_ = torch.from_numpy(demag_spectrum_host(w.n, w.dx)).float().to(dev)     # [6][Pz/2+1][Py/2+1][Kx]
    kz = torch.arange(Pz, device=dev)
    ky = torch.arange(Py, device=dev)
    kzf = torch.minimum(kz, Pz - kz) if Pz > 1 else kz
    kyf = torch.minimum(ky, Py - ky) if Py > 1 else ky
    sz = torch.where(2 * kz <= Pz, 1.0, -1.0).to(dev)[:, None, None]
    sy = torch.where(2 * ky <= Py, 1.0, -1.0).to(dev)[None, :, None]
    full = oct_[:, kzf][:, :, kyf]                                                # [6][Pz][Py][Kx]
    Nxx, Nxy, Nxz, Nyy, Nyz, Nzz = full[0], full[1] * sy, full[2] * sz, full[3], full[4] * sy * sz, full[5]
    del oct_, full
    Ms, A, Ku, al = float(w.Ms), float(w.A), float(w.Ku1), float(w.alpha)
    axes = torch.from_numpy(to_soa(w.ku_axis_cells().astype(np.float32))).to(dev)   # [3][nz][ny][nx]
    cex = 2.0 * A / (mu0 * Ms)
    cani = 2.0 * Ku / (mu0 * Ms)
    gp = -gamma / (1.0 + al * al)
    idx2 = [1.0 / (d * d) for d in w.dx]

    def heff(m):
        Mp = torch.zeros((3, Pz, Py, Px), device=dev, dtype=torch.float32)
        Mp[:, :nz, :ny, :nx] = Ms * m
        Mh = torch.fft.rfftn(Mp, dim=(1, 2, 3))
        hx = Nxx * Mh[0] + Nxy * Mh[1] + Nxz * Mh[2]
        hy = Nxy * Mh[0] + Nyy * Mh[1] + Nyz * Mh[2]
        hz = Nxz * Mh[0] + Nyz * Mh[1] + Nzz * Mh[2]
        h = torch.fft.irfftn(torch.stack((hx, hy, hz)), s=(Pz, Py, Px), dim=(1, 2, 3), norm="forward")
        h = h[:, :nz, :ny, :nx].contiguous()
        mp = torch.nn.functional.pad(m[None], (1, 1, 1, 1, 1, 1), mode="replicate")[0]
        lap = (idx2[0] * (mp[:, 1:-1, 1:-1, 2:] + mp[:, 1:-1, 1:-1, :-2] - 2 * m)
               + idx2[1] * (mp[:, 1:-1, 2:, 1:-1] + mp[:, 1:-1, :-2, 1:-1] - 2 * m)
               + idx2[2] * (mp[:, 2:, 1:-1, 1:-1] + mp[:, :-2, 1:-1, 1:-1] - 2 * m))
        h = h + cex * lap + cani * (axes * m).sum(0, keepdim=True) * axes
        return h

    def rhs(m):
        h = heff(m)
        c = torch.cross(m, h, dim=0)
        return gp * (c + al * torch.cross(m, c, dim=0))

    def rk4(m, dt):
        k1 = rhs(m)
        k2 = rhs(m + 0.5 * dt * k1)
        k3 = rhs(m + 0.5 * dt * k2)
        k4 = rhs(m + dt * k3)
        y = m + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        return y / torch.linalg.vector_norm(y, dim=0, keepdim=True)

    m = torch.from_numpy(to_soa(w.m0.astype(np.float32))).to(dev)
    h_ours = s32.heff(m).double()
    h_b1 = heff(m).double()
    diff = float((h_b1 - h_ours).abs().max() / h_ours.abs().max())
    for _ in range(warmup):
        m = rk4(m, w.dt)
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        m = rk4(m, w.dt)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    return {"value": w.ncells * STAGES_PER_STEP * steps / (ms / 1e3), "unit": UNIT,
            "ms_per_stage": round(ms / steps / STAGES_PER_STEP, 4), "steps": steps,
            "field_rel_diff_vs_libmm_fp32": diff,
            "what": "torch.fft rfftn/irfftn (cuFFT) over the full padded grid + separate elementwise "
                    "PyTorch kernels, FP32"}


def layers_bytes(n, s):
    """Algorithmic HBM bytes of one p3_layers launch for real size s: the 3 nz
    complex planes of the y-spectrum read and written once, and the tensor's
    stored pairs i <= j read once (the mirrored ky reads the same row)."""
    nx, ny, nz = n
    LX, LY, _ = padded(n)
    KX = LX // 2 + 1
    spectrum = 2 * 3 * nz * KX * LY * 2 * s
    tensor = 6 * (nz * (nz + 1) // 2) * (LY // 2 + 1) * KX * s
    return spectrum + tensor


def layers_measure(torch, hbm_peak, steps=20, warmup=3):
    """The non-equidistant stack (Sec. 4.4): 256x256x8 cells in 8 layers of
    unequal thickness, per-layer materials, RK4 in FP32 and FP64 fields;
    cell-updates/s per RK stage (device-timed, no per-kernel events), then a
    profiled run of the same steps for the per-kernel split and the coupling
    pass against the HBM roofline."""
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import to_soa
    w = W.multilayer()
    out = {"layers_nm": [round(v * 1e9, 3) for v in w.extra["layers"]]}
    stream = torch.cuda.current_stream()
    for prec, rs in (("fp32", 4), ("fp64", 8)):
        s = State(w.n, w.dx, prec, stream)
        s.set_material(Ms=0.0, A=0.0, alpha=w.alpha, Ku1=0.0, ku_axis=w.ku_axis,
                       Ms_cell=to_soa(w.Ms), A_cell=to_soa(w.A), Ku1_cell=to_soa(w.Ku1))
        s.set_zeeman(h=w.h_ext)
        s.set_layers(w.extra["layers"])
        s.demag_setup(20)
        s.set_m(to_soa(w.m0))
        t = 0.0
        for _ in range(warmup):
            t, _ = s.step(w.dt, t, "rk4")
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            t, _ = s.step(w.dt, t, "rk4")
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        s.profile_enable(True)
        for _ in range(steps):
            t, _ = s.step(w.dt, t, "rk4")
        torch.cuda.synchronize()
        prof = s.profile_read()
        s.profile_enable(False)
        s.close()
        tot = sum(v[1] for v in prof.values())
        split = {k: {"launches": v[0], "us_per_launch": round(1e3 * v[1] / max(v[0], 1), 2),
                     "share": round(v[1] / tot, 4)} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
        ent = {"ms_per_step": round(ms / steps, 4),
               "cell_updates_per_s": w.ncells * 4 * steps / (ms / 1e3),
               "kernels": split}
        if "p3_layers" in prof:
            n_l, t_l = prof["p3_layers"]
            us = 1e3 * t_l / n_l
            byt = layers_bytes(w.n, rs)
            ent["p3_layers_roofline"] = {"algorithmic_bytes": byt, "us": round(us, 2),
                                         "achieved_gbs": round(byt / (us * 1e-6) / 1e9, 1),
                                         "frac_of_measured_hbm": round(byt / (us * 1e-6) / 1e9 / hbm_peak, 4)}
        out[prec] = ent
    torch.cuda.empty_cache()
    return out


def mixed_measure(torch, hbm_peak, n=(192, 192, 48), steps=20, warmup=3):
    """The bulk construction on a grid whose padded axes are mixed-radix
    lengths (192x192x48 -> 384x384x96; powers of two would need 512x512x128,
    2.4x the points): RK4 in FP32 and FP64 through the classic passes,
    cell-updates/s per stage (device-timed), and each pass's algorithmic bytes
    against the HBM roofline from a profiled run of the same steps."""
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    w = W.bulk(n=n)
    stream = torch.cuda.current_stream()
    out = {"n": list(n), "padded": padded(n)}
    for prec, rs in (("fp32", 4), ("fp64", 8)):
        st = steps if prec == "fp32" else max(2, steps // 10)
        s = setup_workload(w, prec, stream=stream)
        t = 0.0
        for _ in range(warmup):
            t, _ = s.step(w.dt, t, "rk4")
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(st):
            t, _ = s.step(w.dt, t, "rk4")
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        s.profile_enable(True)
        for _ in range(st):
            t, _ = s.step(w.dt, t, "rk4")
        torch.cuda.synchronize()
        prof = s.profile_read()
        s.profile_enable(False)
        s.close()
        kb = kernel_bytes(n, rs, grains=True)
        tot = sum(v[1] for v in prof.values())
        kern = {}
        for name, (cnt, tms) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
            us = 1e3 * tms / max(cnt, 1)
            e = {"launches": cnt, "us_per_launch": round(us, 2), "share": round(tms / tot, 4)}
            if name in kb:
                e["algorithmic_bytes"] = int(kb[name])
                e["frac_of_measured_hbm"] = round(kb[name] / (us * 1e-6) / 1e9 / hbm_peak, 4)
            kern[name] = e
        out[prec] = {"ms_per_step": round(ms / st, 4), "cell_updates_per_s": w.ncells * 4 * st / (ms / 1e3),
                     "kernels": kern}
    torch.cuda.empty_cache()
    return out


def workloads_measure(torch, hbm_peak=6800.0):
    """Time to solution of the paper-shaped configurations beside the bulk one
    (wall time with the device synchronised): plain FP64 (32x32x4, 200 RK4
    steps), the thin film (512x128x1, DP45 with rtol 1e-5 to 1 ns, FP64 and
    FP32 fields), the inverse design (128x128x1, 2000 FP32 RK4 steps and the
    gradient of the time-averaged output m_y by the checkpointed adjoint), the
    non-equidistant multilayer (256x256x8, RK4, layers_measure) and the
    mixed-radix grid (192x192x48, RK4, mixed_measure)."""
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.autodiff import rk4_observable
    from paper_2302_08843_gb300.binding import State, setup_workload
    from paper_2302_08843_gb300.workloads import to_soa
    out = {}
    w = W.plain_fp64()
    s = setup_workload(w, "fp64")
    s.step(w.dt, 0.0, "rk4")
    s.set_m(to_soa(w.m0))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t = 0.0
    for _ in range(w.steps):
        t, _ = s.step(w.dt, t, "rk4")
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    out["plain_fp64_32x32x4_rk4_200"] = {"seconds": round(el, 4), "steps": w.steps}
    s.close()
    w = W.thin_film()
    for prec in ("fp64", "fp32"):
        s = setup_workload(w, prec)
        # untimed warm-up (first launches of the DP45 kernels), then from m0 again
        t, dt = 0.0, 1e-13
        for _ in range(3):
            t, dt = s.step(dt, t, "dp45", w.extra["rtol"])
        s.set_m(to_soa(w.m0))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t, dt, steps = 0.0, 1e-13, 0
        while t < 1e-9:
            t, dt = s.step(min(dt, 1e-9 - t), t, "dp45", w.extra["rtol"])
            steps += 1
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        out["thin_film_512x128x1_dp45_1ns_" + prec] = {"seconds": round(el, 3), "accepted_steps": steps,
                                                        "cell_steps_per_s": w.ncells * steps / el}
        s.close()
    w = W.inverse_design()
    s = State(w.n, w.dx, "fp32")
    s.set_zeeman(fn=w.h_ext, weight=to_soa(w.h_ext_weight))
    s.demag_setup(20)
    m0 = torch.from_numpy(to_soa(w.m0)).float().cuda()
    weight = np.zeros(w.n + (3,))
    (x0, x1), (y0, y1) = w.extra["out_box"]
    weight[x0:x1, y0:y1, :, 1] = 1.0 / ((x1 - x0) * (y1 - y0))
    weight = torch.from_numpy(to_soa(weight)).float().cuda()
    wt = torch.tensor(to_soa(w.extra["w"]), dtype=torch.float64, device="cuda", requires_grad=True)
    # untimed warm-up: a 200-step rollout and its gradient (first launches of
    # the adjoint kernels and of autograd take seconds in a fresh process)
    rk4_observable(torch.sigmoid(wt) * w.extra["Ms0"], s, m0, weight, w.dt, 200, 100,
                   dict(A=w.A, alpha=w.alpha)).mean().backward()
    wt.grad = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    obs = rk4_observable(torch.sigmoid(wt) * w.extra["Ms0"], s, m0, weight, w.dt, w.steps, 100,
                         dict(A=w.A, alpha=w.alpha))
    loss = obs.mean()
    torch.cuda.synchronize()
    fwd = time.perf_counter() - t0
    loss.backward()
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    out["inverse_design_128x128x1_fp32_2000_steps"] = {"forward_seconds": round(fwd, 3),
                                                       "forward_and_gradient_seconds": round(total, 3),
                                                       "checkpoint_every": 100}
    s.close()
    torch.cuda.empty_cache()
    out["multilayer_256x256x8_rk4"] = layers_measure(torch, hbm_peak)
    out["mixed_radix_192x192x48_rk4"] = mixed_measure(torch, hbm_peak)
    return out


def serve_measure(torch, n_requests, dist=None, rank=0, ws=1):
    """The served stream (Poisson arrivals, mean 2 ms; five grid shapes; FP32
    batched relax under a 40 GB footprint cap): p50/p99 latency and
    throughput of its first n_requests requests, next to the plain per-solve
    path (one mm_relax per request, FP64 and FP32) timed over a bounded number
    of DP45 steps on one request of every shape, compared in accepted
    cell-steps/s.  The FP32 field error is measured against the FP64 path on
    each shape."""
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.serving import Server, latency_summary
    stream = W.serving_stream()
    reqs = stream[:n_requests]
    srv = Server(precision="fp32", hbm_cap=40e9)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    idx = [int(x) for x in vis.split(",")] if vis and all(x.strip().isdigit() for x in vis.split(",")) \
        else list(range(ws))
    util = UtilSampler()
    util.start()
    res, elapsed = serve_replicas(torch, dist, rank, ws, reqs, srv)
    busy = util.stop(set(idx[rank:rank + 1]) if ws > 1 else set(idx[:1]))
    launches, peak = srv.launches, srv.peak_used
    srv.close()
    torch.cuda.empty_cache()
    if rank != 0:
        return None
    summ = latency_summary(res, elapsed)
    cell_steps = sum(w.ncells * r["steps"] for (_, w), r in zip(reqs, res))
    by_shape = {}
    for (_, w), r in zip(reqs, res):
        e = by_shape.setdefault("%dx%dx%d" % tuple(w.n), {"requests": 0, "steps": 0, "hit_max_steps": 0,
                                                          "latency_s": []})
        e["requests"] += 1
        e["steps"] += r["steps"]
        e["hit_max_steps"] += int(r["status"] == 3)
        e["latency_s"].append(r["latency"])
    for e in by_shape.values():
        lat = e.pop("latency_s")
        e["mean_steps"] = round(e.pop("steps") / e["requests"], 1)
        e["p50_s"] = round(float(np.percentile(lat, 50)), 3)
    summ["by_shape"] = by_shape
    summ["device_busy"] = busy
    summ.update({"elapsed_s": round(elapsed, 3), "graph_launches_rank0": launches,
                 "cell_steps_per_s": cell_steps / elapsed, "peak_footprint_bytes_rank0": int(peak),
                 "replicas": ws,
                 "sample": "first %d of the 512-request stream (arrivals as drawn)%s" %
                           (len(reqs), "" if ws == 1 else ", request i served by rank i mod %d" % ws)})
    per = {}
    ferr = {}
    shapes = []
    for _, w in stream:
        if tuple(w.n) not in shapes:
            shapes.append(tuple(w.n))
            per_w = w
            for prec in ("fp64", "fp32"):
                st = setup_workload(per_w, prec)
                nsteps = 100
                st.relax(tol=1e-30, max_steps=5, allow_unconverged=True)          # warm-up
                st.set_m(W.to_soa(per_w.m0))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                k, _, _, _ = st.relax(tol=1e-30, max_steps=nsteps, allow_unconverged=True)
                torch.cuda.synchronize()
                el = time.perf_counter() - t0
                a = per.setdefault(prec, [0.0, 0.0])
                a[0] += per_w.ncells * k
                a[1] += el
                st.close()
            s64 = setup_workload(per_w, "fp64")
            s32 = setup_workload(per_w, "fp32")
            h64 = s64.heff().double()
            h32 = s32.heff().double()
            ferr["%dx%dx%d" % tuple(per_w.n)] = float((h32 - h64).abs().max() / h64.abs().max())
            s64.close()
            s32.close()
        if len(shapes) == len(W.SERVING_GRIDS):
            break
    summ["per_solve"] = {prec: {"cell_steps_per_s": v[0] / v[1],
                                "sample": "100 DP45 steps of mm_relax on one request of each shape"}
                         for prec, v in per.items()}
    # batched rate per shape with every slot running (no admission, no host
    # loop): what the device sustains for each bucket, against the served rate
    from paper_2302_08843_gb300.binding import Batch
    from paper_2302_08843_gb300.serving import auto_capacity
    batch_rate = {}
    for shp in W.SERVING_GRIDS:
        rq = [w for _, w in stream if tuple(w.n) == tuple(shp)]
        cap = auto_capacity(shp)
        b = Batch(shp, rq[0].dx, "fp32", capacity=cap)
        for sl in range(cap):
            w = rq[sl % len(rq)]
            b.set_slot(sl, w.Ms, w.A, w.alpha, W.to_soa(w.m0).astype(np.float32))
        b.begin(16, 1e-5, 1e-30, 10 ** 9)
        b.end()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            b.begin(16, 1e-5, 1e-30, 10 ** 9)
            b.end()
        el = time.perf_counter() - t0
        cells = cap * int(np.prod(shp))
        batch_rate["%dx%dx%d" % tuple(shp)] = {"slots": cap, "ms_per_attempt": round(el / 48 * 1e3, 4),
                                               "cell_attempts_per_s": cells * 48 / el}
        b.close()
    summ["batched_rate_by_shape"] = batch_rate
    summ["served_vs_fp64_per_solve"] = summ["cell_steps_per_s"] / summ["per_solve"]["fp64"]["cell_steps_per_s"]
    summ["fp32_field_rel_err_vs_fp64"] = ferr
    return summ


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    from paper_2302_08843_gb300 import workloads as W
    # --nz crops the bulk construction to its first nz planes: a small case for
    # profiler captures, never a bench line
    w = W.bulk() if not args.nz else W.bulk(crop=((0, 256), (0, 256), (0, args.nz)))
    w.steps = args.steps
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = start_cpu_baseline(n_stages=3)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def allmax(v):
        return max_over_ranks(torch, dist, v, "cuda")

    results = {}
    clocks = None
    for precision in (("fp32",) if args.nz else ("fp32", "fp64")):
        steps = args.steps if precision == "fp32" else max(2, args.steps // 10)
        barrier()
        sampler = ClockSampler() if (rank == 0 and precision == "fp32") else None
        if sampler:
            sampler.start()
            time.sleep(0.5)
        s, ms, prof = time_precision(torch, w, precision, steps, args.warmup, peaks)
        barrier()
        if sampler:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES")
            idx = [int(x) for x in vis.split(",")] if vis and all(x.strip().isdigit() for x in vis.split(",")) \
                else list(range(ws))
            clocks = sampler.stop(set(idx[:ws]))
        ms_max = allmax(ms)
        el_e2e = nbytes = None
        b1 = None
        if precision == "fp32":
            el_e2e, nbytes = e2e_measure(torch, s, w, max(8, steps // 2), 2)
            el_e2e = allmax(el_e2e)
            if not args.nz and not args.no_b1:
                b1 = b1_cufft_measure(torch, w, max(3, steps // 5), 2, s)
                torch.cuda.empty_cache()
        results[precision] = dict(ms=ms_max, steps=steps, prof=prof, e2e=(el_e2e, nbytes, max(8, steps // 2)), b1=b1)
        s.close()
        del s
        torch.cuda.empty_cache()

    fp64_peak = None
    if not args.nz:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        idx = [int(x) for x in vis.split(",")] if vis and all(x.strip().isdigit() for x in vis.split(",")) \
            else list(range(ws))
        fp64_peak = fp64_peak_measure(torch, set(idx[local:local + 1]) if ws > 1 else set(idx[:1]))
    # the oracle process has overlapped the device-timed sections; the served
    # stream and the other configurations are partly host-bound (launch loops,
    # field callbacks), so they run after it has finished
    cpu_res = None
    if cpu is not None:
        cpu_res = finish_cpu_baseline(*cpu, sample_desc="%(stages)d RK stages of the FP64 oracle on the "
                                      "full 256x256x64 bulk workload (%(seconds).1f s; %(fft)s)")
    serving = None
    if args.serve_requests > 0 and not args.nz:
        serving = serve_measure(torch, args.serve_requests, dist, rank, ws)
    other = workloads_measure(torch, hbm_peak) if (rank == 0 and not args.nz and not args.no_workloads) else None
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    N = w.ncells
    r32 = results["fp32"]
    value = ws * N * STAGES_PER_STEP * r32["steps"] / (r32["ms"] / 1e3)
    ms_step = r32["ms"] / r32["steps"]

    def roofline_info(prof, s_bytes, precision, steps):
        # kernel_bytes gives each pass's algorithmic bytes per stage; a pass
        # run as several launches per stage (kx chunks of the y/z/y passes)
        # has that figure split evenly over its launches
        kb = kernel_bytes(w.n, s_bytes, grains=True)
        nstages = steps * STAGES_PER_STEP
        total = sum(v[1] for v in prof.values())
        kernels = {}
        for name, (cnt, tms) in prof.items():
            avg = tms / max(cnt, 1)
            ent = {"launches": cnt, "total_ms": round(tms, 4), "share": round(tms / total, 4),
                   "avg_us": round(avg * 1e3, 2)}
            if name in kb:
                per_launch = kb[name] * nstages / cnt if cnt > nstages else kb[name]
                ach = per_launch / (avg / 1e3) / 1e9
                ent.update({"algorithmic_bytes": int(per_launch), "achieved_gbs": round(ach, 1),
                            "frac_of_measured_hbm": round(ach / hbm_peak, 4)})
                if cnt > nstages:
                    ent["launches_per_stage"] = round(cnt / nstages, 3)
            kernels[name] = ent
        dom = max(kernels, key=lambda k: kernels[k]["total_ms"])
        return kernels, dom

    kernels32, dom = roofline_info(r32["prof"], 4, "fp32", r32["steps"])
    kd = kernels32[dom]
    roof = {"bound": "hbm", "kernel": dom, "achieved": kd.get("achieved_gbs"), "peak": hbm_peak, "unit": "GB/s",
            "frac": kd.get("frac_of_measured_hbm"), "traffic": traffic_for(dom, "fp32"),
            "peak_source": peak_src + " hbm_gbs (copy)"}
    launches = sum(v[0] for v in r32["prof"].values())
    stage_ms = ms_step / STAGES_PER_STEP
    model_b = model_stage_bytes(w.n, 4)
    ach_stage = model_b / (stage_ms / 1e3) / 1e9
    kern_sum = sum(kernel_bytes(w.n, 4).values()) * 1.0
    floor_b = floor_stage_bytes(w.n, 4)
    stage_roof = {"model_bytes_per_stage": int(model_b), "ms_per_stage": round(stage_ms, 4),
                  "achieved_gbs": round(ach_stage, 1), "frac": round(ach_stage / hbm_peak, 4),
                  "kernel_bytes_per_stage": int(kern_sum),
                  "floor_bytes_per_stage": int(floor_b),
                  "frac_of_floor": round(floor_b / (stage_ms / 1e3) / 1e9 / hbm_peak, 4)}
    if args.nz:
        print(json.dumps({"profiling_case": "bulk cropped to %dx%dx%d" % tuple(w.n), "value": value,
                          "kernels": kernels32}))
        return
    r64 = results["fp64"]
    v64 = ws * N * STAGES_PER_STEP * r64["steps"] / (r64["ms"] / 1e3)
    fl = stage_flops(w.n)
    st64 = r64["ms"] / r64["steps"] / STAGES_PER_STEP
    kernels64, dom64 = roofline_info(r64["prof"], 8, "fp64", r64["steps"])
    if fp64_peak is not None:
        p64, p64_src = fp64_peak["tflops"], "measured: FP64 FMA probe on this GPU (fp64.peak_probe)"
    else:
        p64, p64_src = FP64_NOMINAL_TFLOPS, "nominal GB300 FP64 rate (probe not run)"
    fp64 = {"value": v64, "unit": UNIT, "ms_per_step": round(r64["ms"] / r64["steps"], 4), "steps": r64["steps"],
            "roofline": {"bound": "alu", "achieved": round(fl / (st64 / 1e3) / 1e12, 4),
                         "peak": p64, "unit": "TFLOP/s",
                         "frac": round(fl / (st64 / 1e3) / 1e12 / p64, 4),
                         "peak_source": p64_src, "flops_per_stage": int(fl)},
            "kernels": kernels64, "dominant": dom64, "peak_probe": fp64_peak}
    el, nbytes, e2e_steps = r32["e2e"]
    e2e = {"value": ws * N * STAGES_PER_STEP * e2e_steps / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
           "how": "mm_set_m from pinned host memory, mm_llg_step, mm_get_m to pinned host memory every step; "
                  "two states on two streams in turn (a step's copy in and compute overlap the previous "
                  "step's copy out)"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": r32["steps"],
           "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "cells": N, "padded_fft": padded(w.n),
                      "stages_per_step": STAGES_PER_STEP, "parallelism": "replicas x%d" % ws,
                      "l2": "per-stage working set ~0.7 GB > 129 MB L2, no flush"},
           "roofline": roof, "stage_roofline": stage_roof, "kernels": kernels32,
           "gpu_launches": launches, "e2e": e2e, "fp64": fp64, "clocks": clocks}
    if r32.get("b1"):
        out["b1_cufft"] = dict(r32["b1"], ours_over_b1=round(value / r32["b1"]["value"], 3))
    if serving is not None:
        out["serving"] = serving
    if other is not None:
        out["workloads"] = other
    if cpu is not None:
        out["cpu_baseline"] = cpu_res
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------- reference --
def run_reference(args):
    """The oracle (the method written plainly in FP64 NumPy) as the reference
    arm, on the host cores.  Each step is one RK stage of the bulk workload's
    construction on a crop sized so that the whole run stays within a few
    minutes."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    total = args.steps + args.warmup
    # oracle stage cost per cell is roughly flat; pick the largest crop with
    # (steps + warmup) stages <= ~120 s on one core (about 6 us per cell-stage)
    crops = [((0, 256), (0, 256), (0, 64)), ((0, 128), (0, 128), (0, 32)), ((0, 64), (0, 64), (0, 16)),
             ((0, 32), (0, 32), (0, 8))]
    crop = crops[-1]
    for c in crops:
        cells = (c[0][1] - c[0][0]) * (c[1][1] - c[1][0]) * (c[2][1] - c[2][0])
        if cells * total * 6e-6 <= 120.0:
            crop = c
            break
    sys.path.insert(0, ROOT)
    from oracle.llg import Problem
    from paper_2302_08843_gb300 import workloads as W
    w = W.bulk(crop=None if crop == crops[0] else crop)
    prob = Problem(w.n, w.dx, Ms=w.Ms, A=w.A, alpha=w.alpha, Ku1=w.Ku1, ku_axis=w.ku_axis_cells(), h_ext=w.h_ext)
    m = w.m0
    for s in range(args.warmup):
        m = m + 0.5 * w.dt * prob.rhs(m, 0.0)
    t0 = time.perf_counter()
    for s in range(args.steps):
        m = m + 0.5 * w.dt * prob.rhs(m, 0.0)
    el = time.perf_counter() - t0
    value = w.ncells * args.steps / el
    from oracle.demag import FFT_BACKEND, FFT_WORKERS
    sample = ("one RK stage per step of the FP64 oracle on the %dx%dx%d crop of the bulk workload (%s; "
              "element-wise NumPy terms on 1 thread)" % (tuple(w.n) + (FFT_BACKEND,)))
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": WORKLOAD, "sample_grid": list(w.n)},
                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": FFT_WORKERS, "kind": "oracle",
                                       "sample": sample, "host_cpu_count": os.cpu_count()},
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_layers_only(args):
    import torch
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    res = layers_measure(torch, peaks.get("hbm_gbs", 6800.0), steps=args.steps, warmup=args.warmup)
    print(json.dumps({"case": "multilayer 256x256x8 (profiling case)", "layers": res}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-b1", action="store_true", help="skip the cuFFT + elementwise comparison baseline")
    ap.add_argument("--no-workloads", action="store_true", help="skip the other configurations' timings")
    ap.add_argument("--nz", type=int, default=0,
                    help="profiling case: the bulk workload cropped to nz planes (the printed line is not a bench "
                         "result)")
    ap.add_argument("--serve-requests", type=int, default=512,
                    help="requests of the served stream to run (512 = all; 0 = skip)")
    ap.add_argument("--mixed-only", action="store_true",
                    help="profiling case: only the 192x192x48 mixed-radix grid (the printed line is not a bench "
                         "result)")
    ap.add_argument("--layers-only", action="store_true",
                    help="profiling case: only the 256x256x8 non-equidistant stack (the printed line is not a "
                         "bench result)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.layers_only:
        run_layers_only(args)
    elif args.mixed_only:
        import torch
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        res = mixed_measure(torch, peaks.get("hbm_gbs", 6800.0), steps=args.steps, warmup=args.warmup)
        print(json.dumps({"case": "mixed-radix 192x192x48 (profiling case)", "mixed": res}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
