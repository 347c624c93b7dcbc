#!/usr/bin/env python
"""Throughput of the STARRED loss-and-gradient hot path on GB300.

Default workload: the uneven batch of 256 SN + host fields (stamp sizes
32..128, 10..500 epochs each, f = 2, 64x64 narrow PSFs, 1 point source,
4-6 starlet scales) together with the 16-star PSF reconstruction (64x64
stamps, f = 2, 5 scales).  One step = one loss-and-gradient evaluation of
every field of the batch and of the PSF fit, plus the fused AdaBelief update
of all their parameters.  The metric is epoch-pixels per second: data pixels
of all epochs (and star stamps) evaluated per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank evaluates its own
batch (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2402_08725_gb300 import synthetic as syn  # noqa: E402

WORKLOADS = {
    "config4": "uneven batch of 256 SN+host fields (N 32-128, E 10-500, f=2, K=64, M=1, J 4-6) "
               "+ 16-star PSF fit (64x64, f=2, J=5)",
    "config3": "lensed quasar: 300 epochs of 64x64, f=2, K=64, M=4, J=4",
    "config1": "joint deconvolution: 4 epochs of 32x32, f=2, K=64, M=2, J=4",
    "config5": "JWST-like: 6 frames of 512x512, f=3, K=255, M=40, J=6",
    "config2": "PSF fit: 16 stars of 64x64, f=2, J=5",
}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="config4")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave out the per-configuration measurements (configs 1, 2, 3, 5 each on its own)")
    ap.add_argument("--no-noise", action="store_true",
                    help="skip the Monte Carlo prior weights, point-source prior and extraction measurements")
    ap.add_argument("--conv-mode", choices=["auto", "direct", "fft"], default="auto",
                    help="convolution form of every field (auto: timed per shape on first use)")
    ap.add_argument("--fields", type=int, default=0,
                    help="config4 only: evaluate the first FIELDS fields (a smaller case for profiling)")
    ap.add_argument("--schedule", default="",
                    help="EPOCHS,PAIRS: the transform form's schedule instead of tuning it (profiling runs, "
                         "whose timings under a profiler would mislead the tuner)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# --- workloads ---------------------------------------------------------------------------

def make_workload(name, rank, n_fields=0):
    """(deconv fields, psf problem or None); rank shifts the seeds (weak scaling)."""
    seed_shift = 7919 * rank
    if name == "config4":
        sel = range(n_fields) if n_fields else None
        fields = syn.config4(seed=syn.BASE_SEED + 4 + seed_shift, fields=sel)
        return fields, syn.config2(seed=syn.BASE_SEED + 2 + seed_shift)
    if name == "config3":
        return [syn.config3(seed=syn.BASE_SEED + 3 + seed_shift)], None
    if name == "config1":
        return [syn.config1(seed=syn.BASE_SEED + 1 + seed_shift)], None
    if name == "config5":
        return [syn.config5(seed=syn.BASE_SEED + 5 + seed_shift)], None
    if name == "config2":
        return [], syn.config2(seed=syn.BASE_SEED + 2 + seed_shift)
    raise ValueError(name)


def units_of(fields, pb):
    u = sum(fd.epoch_pixels for fd in fields)
    if pb is not None:
        u += pb.epoch_pixels
    return u


def folded_taps_1d(N, f, K):
    """sum over data pixels p of #{fine u in [0, F): f p - u in the folded-kernel support}."""
    o = K // 2
    t_lo, t_hi = -o - f + 1, K - 1 - o
    F = f * N
    p = np.arange(N)
    lo = np.maximum(f * p - t_hi, 0)
    hi = np.minimum(f * p - t_lo, F - 1)
    return int(np.maximum(hi - lo + 1, 0).sum())


def fwd_flops(fields):
    """Algorithmic FLOPs of one forward (= one adjoint) tile-kernel launch: 2 per
    in-bounds tap of the D-folded convolution, over all epochs of all fields."""
    return sum(2.0 * fd.E * folded_taps_1d(fd.N, fd.f, fd.K) ** 2 for fd in fields)


def fwd_bytes(fields):
    """Algorithmic DRAM bytes of one forward launch: data, weights, folded kernels, e out, h in."""
    b = 0
    for fd in fields:
        Tk = -(-(fd.K + fd.f - 1) // fd.f) + 1
        b += fd.E * fd.N * fd.N * 4 * 3 + fd.E * fd.f * fd.f * Tk * Tk * 4 + fd.F * fd.F * 4
    return b


FFT_SIZES = (24, 32, 40, 48, 56, 64, 72, 80, 96, 112, 128, 144)   # in shared memory
BIG_SIZES = (192, 240, 288, 384, 576, 768)                          # through global memory


def fft_size(N, K, f):
    """Transform size of the frequency-domain form (the library's rule): the smallest listed
    L >= N + max(tau_hi, -tau_lo) that also holds the folded kernel (L >= Tk); the in-shared-memory
    sizes first, then the global-memory ones."""
    o = K // 2
    t_lo, t_hi = -o - f + 1, K - 1 - o
    tau_lo = -((-t_lo) // f)
    tau_hi = (t_hi + f - 1) // f
    need = max(N + max(tau_hi, -tau_lo), tau_hi - tau_lo + 1)
    return next(L for L in FFT_SIZES + BIG_SIZES if L >= need)


FFT_CHUNK = 16  # epochs per work item of the frequency-domain form (the library's value)


def fft_bytes(fields):
    """Algorithmic DRAM bytes of one evaluation's transform kernels.  In shared memory: each epoch
    reads its f^2 folded-kernel spectra (L x (L/2+1) complex) and its data and weights; each chunk of
    epochs writes its f^2 accumulated adjoint spectra, read back once by the per-field reduction;
    each field's h spectra are written and read once.  Through global memory: each frame's kernel
    spectra are read once and its image spectra written and read once, its data and weights read
    and its residual written; the f^2 adjoint spectra are written and read once per pair of
    frames; h is read and its gradient written."""
    b = 0
    for fd in fields:
        L = fft_size(fd.N, fd.K, fd.f)
        LH = L * (L // 2 + 1)
        nph = fd.f * fd.f
        if L in BIG_SIZES:
            pairs = -(-fd.E // 2)
            b += fd.E * (3 * nph * LH * 8 + 12 * fd.N * fd.N) + pairs * nph * LH * 8 * 2 + 8 * fd.F ** 2
            continue
        chunks = -(-fd.E // FFT_CHUNK)
        b += fd.E * (nph * LH * 8 + 8 * fd.N * fd.N) + chunks * nph * LH * 8 * 2 + 2 * nph * LH * 8 + 8 * fd.F ** 2
    return b


def fft_flops(fields):
    """Nominal FLOPs of the transform kernels: 5 n log2 n per complex transform of n points
    (a real L x L transform counted as L^2/2 complex points), 2 per epoch, plus the complex
    products of the spectra (model, adjoint, and the 3 Parseval products per source)."""
    import math
    fl = 0.0
    for fd in fields:
        L = fft_size(fd.N, fd.K, fd.f)
        LH = L * (L // 2 + 1)
        nph = fd.f * fd.f
        n = L * L / 2
        per = 2 * 5 * n * math.log2(n) + nph * LH * (8 + 8 + fd.M * (8 + 3 * 6 + 6))
        fl += fd.E * per + 2 * nph * 5 * n * math.log2(n)
    return fl


CHUNK_SRCS = [os.path.join(ROOT, "paper_2402_08725_gb300", "csrc", n)
              for n in ("fft_pair.cu", "fft_pair.cuh", "common.cuh", "cplx.cuh", "ffsum.cuh")]
CHUNK_PROFILE = os.path.join(ROOT, "profiles", "fft_chunk_pair_kernel_config4.md")


def chunk_source_hash():
    """First 16 hex digits of the sha256 of the transform chunk kernel's source files, in order."""
    import hashlib
    h = hashlib.sha256()
    for path in CHUNK_SRCS:
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes (read + write) of one config-4 launch of the transform chunk kernel, from the
    committed ncu summary (a 24-field capture scaled by the epoch-pixels to the full batch), or
    None if that summary was taken on another version of the kernel's source (its recorded hash
    differs)."""
    import re
    try:
        txt = open(CHUNK_PROFILE).read()
        want = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", txt).group(1)
        if want != chunk_source_hash():
            return None
        return float(re.search(r"dram_bytes_per_launch_full:\s*(\d+)", txt).group(1))
    except (OSError, AttributeError, ValueError):
        return None


def lr_groups(fd):
    amp = float(np.mean(np.abs(fd.params[fd.F ** 2:fd.F ** 2 + fd.E * fd.M]))) if fd.M else 1.0
    return (1e-2 * max(float(np.max(np.abs(fd.params[:fd.F ** 2]))), 1.0) / 100.0, 1e-2 * amp, 1e-3, 1e-3, 1e-2)


# --- clocks --------------------------------------------------------------------------------

class _NvmlClocks:
    """Read-only NVML queries through ctypes (libnvidia-ml ships with the driver): the SM clock,
    its maximum and the active clock-event reasons of one GPU, sampled by a host thread."""
    # nvmlClocksEventReasons bits (nvml.h)
    BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        ok = False
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(cuda_index).uuid)
            for u in (uuid, "GPU-" + uuid):
                if self.lib.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(self.h)) == 0:
                    ok = True
                    break
        except Exception:
            ok = False
        if not ok:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            ids = [x for x in vis.split(",") if x.strip()]
            idx = int(ids[cuda_index]) if ids and all(x.strip().isdigit() for x in ids) else cuda_index
            if self.lib.nvmlDeviceGetHandleByIndex_v2(idx, ctypes.byref(self.h)) != 0:
                raise OSError("no NVML handle")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        c, m, r = self.ct.c_uint(), self.ct.c_uint(), self.ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, self.ct.byref(c)) != 0:
            return None
        if self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, self.ct.byref(m)) != 0:
            return None
        if self.reasons_fn(self.h, self.ct.byref(r)) != 0:
            return None
        return float(c.value), float(m.value), {n for bit, n in self.BITS.items() if r.value & bit}

    def close(self):
        self.lib.nvmlShutdown()


class ClockSampler:
    """Clocks and throttle reasons during the timed region: NVML every 10 ms from a host thread
    (the main thread waits in a stream synchronisation meanwhile), else nvidia-smi every 200 ms."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.nvml = None
        self.thread = None
        self.samples = []

    def start(self):
        try:
            self.nvml = _NvmlClocks(self.gpu)
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            import threading
            self.stop_ev = threading.Event()
            first = self.nvml.sample()
            if first is not None:
                self.samples.append(first)

            def run():
                while not self.stop_ev.wait(0.010):
                    v = self.nvml.sample()
                    if v is not None:
                        self.samples.append(v)
            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.nvml is not None:
            self.stop_ev.set()
            self.thread.join(timeout=5)
            last = self.nvml.sample()
            if last is not None:
                self.samples.append(last)
            self.nvml.close()
            if not self.samples:
                return None
            reasons = set()
            for _, _, r in self.samples:
                reasons |= r
            return {"sm_mhz": statistics.median(v[0] for v in self.samples),
                    "sm_max_mhz": max(v[1] for v in self.samples), "reasons": sorted(reasons),
                    "samples": len(self.samples), "source": "NVML, every 10 ms during the timed steps"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi, every 200 ms during the timed steps"}


def load_peaks():
    try:
        with open(PEAKS_FILE) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# --- CPU baseline (the FP64 oracle as it stands) --------------------------------------------

def oracle_sample(fields, pb, budget_macs=2.0e11, seed=0):
    """Pick fields (seeded order) until the literal oracle's estimated work reaches the budget."""
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(fields)) if fields else []
    cost = [2.0 * fd.E * (fd.F ** 2) * (fd.K ** 2) for fd in fields]
    picked, macs = [], 0.0
    for i in order:
        if macs + cost[i] > budget_macs:
            continue
        picked.append(int(i))
        macs += cost[i]
        if macs >= 0.5 * budget_macs:
            break
    if not picked and fields:  # no field fits the budget alone: the cheapest one
        picked = [int(np.argmin(cost))]
    return picked


def time_oracle(fields, picked, pb):
    import oracle
    t0 = time.perf_counter()
    units = 0
    for i in picked:
        fd = fields[i]
        oracle.deconv_loss_grad(fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s, fd.W, fd.params)
        units += fd.epoch_pixels
    if pb is not None:
        oracle.psf_loss_grad(pb.S, pb.N, pb.f, pb.J, pb.lam, pb.t, pb.sigma, pb.W, pb.params)
        units += pb.epoch_pixels
    dt = time.perf_counter() - t0
    return units, dt, oracle.max_threads()


def cpu_baseline(fields, pb, budget_macs=6.0e11):
    """The oracle on all host cores, and on one core with a smaller sample."""
    import oracle
    picked = oracle_sample(fields, pb, budget_macs)
    units, dt, cores = time_oracle(fields, picked, pb)
    desc = f"{len(picked)} of {len(fields)} fields (" + ", ".join(
        f"N={fields[i].N} E={fields[i].E}" for i in picked) + ")" + (" + the PSF fit" if pb is not None else "") + \
        ", one loss+gradient evaluation each, literal FP64 oracle (OpenMP)"
    one = None
    try:
        oracle.set_threads(1)
        picked1 = oracle_sample(fields, None, budget_macs / 40, seed=1)
        units1, dt1, _ = time_oracle(fields, picked1, None)
        one = {"value": units1 / dt1, "unit": "epoch-px/s", "cores": 1, "seconds": dt1,
               "sample": f"{len(picked1)} of {len(fields)} fields (" + ", ".join(
                   f"N={fields[i].N} E={fields[i].E}" for i in picked1) + "), one loss+gradient evaluation each"}
    finally:
        oracle.set_threads(cores)
    return {"value": units / dt, "unit": "epoch-px/s", "cores": cores, "kind": "oracle", "sample": desc,
            "seconds": dt, "one_core": one}


# --- our implementation --------------------------------------------------------------------

NOISE_REALISATIONS = 5000  # App. B


def measure_noise(stream, fp32_peak, with_cpu, reps=3, cpu_sample=256):
    """Monte Carlo prior weights (sec. 2.3) on a config-3 field: 64 x 64 stamps, f = 2
    (F = 128), co-added noise of its 300 epochs, the first epoch's 64 x 64 PSF, 4 starlet planes,
    5000 realisations.  The dominant kernel is the S_1^T correlation, FP32 FMA issue bound; its
    algorithmic work is 2 FLOP per in-bounds tap of the "same" correlation with zero fill,
    2 (sum_u n(u))^2 per realisation with n(u) = #{t < K : 0 <= u + t - K//2 < F}; the kernel also
    multiplies the zero taps outside the grid (2 F^2 K^2 per realisation, reported beside it)."""
    import torch
    from paper_2402_08725_gb300 import synthetic as syn
    from paper_2402_08725_gb300.binding import noise_weights
    fd = syn.config3()
    N, f, K, J, n = fd.N, fd.f, fd.K, fd.J, NOISE_REALISATIONS
    F = f * N
    with torch.cuda.stream(stream):
        sg = torch.from_numpy(np.ascontiguousarray(fd.sigma, dtype=np.float32)).cuda()
        sk = torch.from_numpy(np.ascontiguousarray(fd.s[0], dtype=np.float32)).cuda()
        stream.synchronize()
        for _ in range(2):
            noise_weights(N, f, K, J, sg, sk, n, 1, want_map=False, stream=stream)
        times = []
        for r in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            W, _, _ = noise_weights(N, f, K, J, sg, sk, n, 1 + r, want_map=False, stream=stream)
            e1.record(stream)
            stream.synchronize()
            times.append(e0.elapsed_time(e1))
        _, _, tm = noise_weights(N, f, K, J, sg, sk, n, 1, want_map=False, timing=True, stream=stream)
    ms = float(np.median(times))
    o = K // 2
    taps_1d = sum(max(0, min(K, o - u + F) - max(0, o - u)) for u in range(F))
    flops_real = 2.0 * taps_1d * taps_1d      # in-bounds taps per realisation
    flops_dense = 2.0 * F * F * K * K         # every tap, zero fill included
    flops = flops_real * n
    ach = flops / (tm["corr_ms"] / 1e3) / 1e12
    out = {"workload": f"config-3 field: {N}x{N} stamps, f={f} (F={F}), co-added noise of {fd.E} epochs, "
                       f"epoch-1 PSF {K}x{K}, J={J}, {n} realisations",
           "ms": round(ms, 3), "value": round(n / (ms / 1e3), 1), "unit": "realisations/s",
           "W": [float(w) for w in W],
           "phases_ms": {k: round(tm[k], 3) for k in ("draw_ms", "corr_ms", "starlet_ms", "final_ms")},
           "launches": tm["launches"], "batch": tm["batch"],
           "roofline": {"bound": "alu", "achieved": round(ach, 2), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                        "frac": round(ach / fp32_peak, 4), "traffic": None, "kernel": "noise_corr_kernel",
                        "flops_per_launch": flops_real * tm["batch"],
                        "dense_flops_per_launch": flops_dense * tm["batch"],
                        "dense_tflops": round(flops_dense * n / (tm["corr_ms"] / 1e3) / 1e12, 2),
                        "in_bounds_fraction": round(flops_real / flops_dense, 4),
                        "peak_source": "measured FFMA microbenchmark (sr_measure_fp32_peak)"},
           "timing": "CUDA events around the whole call on its stream (workspace allocation included), "
                     "median of 3 after 2 warm-up calls; phases from the call's own events",
           "l2": "batch buffers sized to stay in L2 by design (no flush)"}
    if with_cpu:
        import oracle
        m = cpu_sample
        t0 = time.perf_counter()
        oracle.noise_weights(N, f, K, J, fd.sigma.astype(np.float64), fd.s[0].astype(np.float64), m, 1)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": round(m / dt, 2), "unit": "realisations/s", "cores": oracle.max_threads(),
                               "kind": "oracle",
                               "sample": f"the first {m} realisations of the same workload (FP64 C, OpenMP over "
                                         f"realisations), {dt:.1f} s"}
    return out


def measure_pts(stream, evals=10, warm=3):
    """Point-source prior (Eq. 11, third term) on the config-3 lensed quasar (E = 300, N = 64,
    f = 2, M = 4, J = 4), where blending makes the term necessary: one loss-and-gradient
    evaluation without and with the term (lambda_pts = 0.5 lambda, the starting value of App. C),
    and the App. C estimate."""
    import torch
    from paper_2402_08725_gb300 import synthetic as syn
    from paper_2402_08725_gb300.binding import Problem
    fd = syn.config3()
    with torch.cuda.stream(stream):
        prob = Problem.from_field(fd, stream=stream)
        P = torch.from_numpy(np.ascontiguousarray(fd.params, dtype=np.float32)).cuda()
        g = torch.empty_like(P)
        stream.synchronize()

        def timed():
            for _ in range(warm):
                prob.loss_and_grad(P, g, sync=False)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(evals):
                prob.loss_and_grad(P, g, sync=False)
            e1.record(stream)
            stream.synchronize()
            return e0.elapsed_time(e1) / evals

        ms0, n0 = timed(), prob.launches_per_eval()
        prob.set_lambda_pts(0.5 * fd.lam)
        ms1, n1 = timed(), prob.launches_per_eval()
        t0 = time.perf_counter()
        est = prob.estimate_lambda_pts(P)
        est_ms = (time.perf_counter() - t0) * 1e3
        prob.close()
    return {"workload": f"config-3 field: E={fd.E}, N={fd.N}, f={fd.f}, K={fd.K}, M={fd.M}, J={fd.J}, "
                        f"lambda={fd.lam}",
            "eval_ms_without": round(ms0, 4), "eval_ms_with": round(ms1, 4),
            "overhead_ms": round(ms1 - ms0, 4), "launches_without": n0, "launches_with": n1,
            "lambda_pts": 0.5 * fd.lam, "estimate_app_c": round(est, 6), "estimate_call_ms": round(est_ms, 3),
            "timing": f"CUDA events over {evals} evaluations after {warm} warm-up ones (per evaluation); "
                      "the estimate call by the host clock (it allocates, runs and synchronises)"}


def measure_extraction(stream, n_steps=200):
    """End-to-end light-curve extraction (sec. 3) on the scale of the paper's runtime statement
    (about 1000 epochs of 32 x 32 cutouts, 64 x 64 deconvolved, in about 10 s on one GPU including
    2-3 s of compilation; 200 AdaBelief iterations as in its runtime figure): a supernova light
    curve on the sky background, 1000 epochs, N = 32, f = 2, K = 64; four point sources (a
    lensed-quasar configuration) over 300 epochs of 64 x 64; and the two host workloads, a config-3
    field and a config-4 field whose host is drawn through each epoch's own seeing (so that one h
    fits every epoch); AdaBelief (200 steps) and L-BFGS-B (100 iterations) from the same start.  Host-clock time of the whole call
    (problem creation, uploads, starting point, graph capture, the steps, read-back), device time of
    the steps, and the metrics of sec. 3 against the generator's truth."""
    import torch
    from paper_2402_08725_gb300 import metrics as mt
    from paper_2402_08725_gb300 import synthetic as syn
    from paper_2402_08725_gb300.extract import extract
    out = []
    cases = [("supernova, 1000 epochs of 32x32, 1 point source",
              syn.point_source_field(2402, 1000, 32, 1, light_curve=syn.supernova_light_curve(1000, 400),
                                     positions=[[1.5, -2.0]])),
             ("lensed quasar, 300 epochs of 64x64, 4 point sources",
              syn.point_source_field(2403, 300, 64, 4, positions=[[6, 0], [0, 6], [-6, 0], [0, -6]])),
             ("config 3: lensed quasar (4 images) with ring arc and lens galaxy, 300 epochs of 64x64, "
              "the host seen through each epoch's seeing", syn.config3(host_blur="epoch")),
             ("config-4 field: supernova on a bulge + disc host, 250 epochs of 64x64, "
              "the host seen through each epoch's seeing", syn.config4_field(7, 64, 250, 4, host_blur="epoch"))]
    extract(cases[0][1], np.zeros((1, 2)), n_steps=2, lambda_pts=0.0, stream=stream)  # library loaded, warm
    for name, fd in cases:
        _, a_t, c_t, _, _ = syn.unpack_deconv(fd.params.astype(np.float64), fd.E, fd.N, fd.f, fd.M)
        c0 = c_t + np.random.default_rng(1).normal(0.0, 0.2, c_t.shape)
        bright = a_t >= 0.1 * a_t.max(axis=0, keepdims=True)
        row = {"workload": name, "epochs": fd.E, "N": fd.N}
        for opt, steps in (("adabelief", n_steps), ("lbfgsb", n_steps // 2)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            # fields with a host take the point-source prior at the App. C estimate, which keeps h
            # from absorbing the point sources (sec. 2.2); point sources alone need none
            lp = "app_c" if "host" in name else 0.0
            r = extract(fd, c0, n_steps=steps, lambda_pts=lp, stream=stream, optimizer=opt)
            wall = time.perf_counter() - t0
            row[opt] = {"steps": steps, "lambda_pts": lp, "loss_evaluations": r["evaluations"], "wall_s": round(wall, 3),
                        "device_ms": round(r["ms"], 2),
                        "chi2_over_half_npix": round(float(r["losses"][-1]) / (0.5 * fd.E * fd.N * fd.N), 4),
                        "A_photo": round(mt.a_photo(a_t, r["a"], bright), 5),
                        "P_photo": round(mt.p_photo(a_t, r["a"], bright), 5),
                        "P_astro_px": round(mt.p_astro(c_t, r["c"]), 5),
                        "max_position_error_px": round(float(np.max(np.abs(r["c"] - c_t))), 4)}
        out.append(row)
    return {"cases": out, "paper_context": "about 10 s for about 1000 epochs of 32x32 (2-3 s of it compilation), "
                                           "one consumer GPU (RTX 3060 in its runtime figure)",
            "photometry_epochs": "epochs whose true flux is at least 10 % of the source's peak"}


def measure_psf_fit(stream, steps=300):
    """PSF reconstruction quality (sec. 3, MAE_PSF) on config 2 (16 stars of 64 x 64, f = 2): the
    fit from b = 0, alpha x 1.3, beta = 3.5, amplitudes from the background-subtracted stamp sums
    and centres 0.1 px off, by AdaBelief (300 steps) and by L-BFGS-B (100 iterations) with the
    prior weights of the noise propagation of sec. 2.3 (sr_noise_weights, 1000 realisations, the
    2-px Gaussian as the operator on b, the noise in units of the normalised stars), and by
    AdaBelief with the workload's synthetic weights (in data units, not scaled to the stars' fluxes:
    the prior then weighs about a star amplitude too little and b fits the noise).  The stars
    of config 2 are drawn on the data grid from the Moffat profile of the effective width times a
    faint copy of a random texture, not through the model, so no narrow PSF reproduces them exactly;
    the reference PSF is the Moffat that drew them, both PSFs normalised to unit sum.  Beside each
    MAE_PSF the fitted PSF's negative mass (the sum of its negative pixels at unit sum) is given: for
    two non-negative unit-sum PSFs the L1 difference cannot exceed 2, so an MAE above 2 is carried by
    negative lobes of the pixel grid b."""
    import torch
    from paper_2402_08725_gb300 import metrics as mt
    from paper_2402_08725_gb300 import synthetic as syn
    from paper_2402_08725_gb300.binding import Problem, optim_cfg
    pb = syn.config2()
    S, N, f = pb.S, pb.N, pb.f
    F = f * N
    truth = pb.params.astype(np.float64)
    ref_p = truth.copy()
    ref_p[:F * F] = 0.0
    start = truth.copy()
    start[:F * F] = 0.0
    start[F * F] *= 1.3
    start[F * F + 1] = 3.5
    sums = np.array([float(np.sum(pb.t[k] - np.median(pb.t[k]))) for k in range(S)])
    start[F * F + 2:F * F + 2 + S] = np.maximum(sums, 1.0)
    start[F * F + 2 + S:] += np.random.default_rng(3).normal(0.0, 0.1, 2 * S)
    out = {"workload": f"config 2: {S} stars of {N}x{N}, f={f}"}
    with torch.cuda.stream(stream):
        prob = Problem.from_psf(pb, stream=stream)
        unit = lambda t: (t / t.sum()).cpu().numpy().astype(np.float64)
        s_ref = unit(prob.psf_model(torch.from_numpy(ref_p.astype(np.float32)).cuda()))
        P0 = torch.from_numpy(start.astype(np.float32)).cuda()
        out["mae_psf_start"] = round(mt.mae_psf(s_ref, unit(prob.psf_model(P0))), 5)
        # prior weights by the noise propagation of sec. 2.3: for a PSF fit the pixel grid b is
        # convolved with the 2-px-FWHM Gaussian r (Eq. 3), the stars' noise co-added in units of
        # the normalised stars (sigma_k / a_k, a_k from the starting amplitudes)
        from paper_2402_08725_gb300.binding import noise_weights
        K = 9
        yy, xx = np.mgrid[0:K, 0:K] - K // 2
        r = np.exp(-(xx * xx + yy * yy) * np.log(2.0))
        sig_n = (pb.sigma / start[F * F + 2:F * F + 2 + S, None, None]).astype(np.float32)
        W_mc, _, _ = noise_weights(N, f, K, pb.J, torch.from_numpy(sig_n).cuda(),
                                   torch.from_numpy((r / r.sum()).astype(np.float32)).cuda(), 1000, 7,
                                   want_map=False, stream=stream)
        out["noise_weights"] = [float(w) for w in W_mc]
        out["workload_weights"] = [float(w) for w in pb.W]
        for opt in ("adabelief", "lbfgsb", "adabelief_workload_weights"):
            P = P0.clone()
            prob.reset_optimizer()
            prob.set_weights(pb.W if opt == "adabelief_workload_weights" else W_mc)
            stream.synchronize()
            t0 = time.perf_counter()
            if opt.startswith("adabelief"):
                amp = float(np.mean(start[F * F + 2:F * F + 2 + S]))
                last = prob.step(P, steps, optim_cfg("adabelief", lr=(2e-5, 1e-2, 1e-2 * amp, 1e-3)))
                info = {"steps": steps, "loss": last}
            else:
                r = prob.lbfgsb(P, max_iter=steps // 3, pgtol=0.0, factr=0.0)
                info = {"steps": r["iterations"], "loss_evaluations": r["evaluations"], "loss": r["f"],
                        "status": r["status"]}
            stream.synchronize()
            info["wall_s"] = round(time.perf_counter() - t0, 3)
            fit = P.cpu().numpy().astype(np.float64)
            s_fit = unit(prob.psf_model(P))
            info["mae_psf"] = round(mt.mae_psf(s_ref, s_fit), 5)
            info["negative_mass"] = round(float(-np.sum(np.minimum(s_fit, 0.0))), 5)
            info["alpha"], info["beta"] = round(fit[F * F], 4), round(fit[F * F + 1], 4)
            info["P_astro_px"] = round(mt.p_astro(truth[F * F + 2 + S:].reshape(S, 2),
                                                  fit[F * F + 2 + S:].reshape(S, 2)), 5)
            info["A_photo"] = round(mt.a_photo(truth[F * F + 2:F * F + 2 + S], fit[F * F + 2:F * F + 2 + S]), 5)
            info["P_photo"] = round(mt.p_photo(truth[F * F + 2:F * F + 2 + S], fit[F * F + 2:F * F + 2 + S]), 5)
            out[opt] = info
        prob.close()
    out["truth"] = {"alpha": round(truth[F * F], 4), "beta": round(truth[F * F + 1], 4)}
    out["reference"] = "the Moffat(alpha, beta) that drew the stars, unit sum; MAE = L1 of the difference"
    return out


def run_ours(args):
    import torch
    rank, world, local_rank = dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2402_08725_gb300.binding import Batch, Problem, optim_cfg

    t_gen = time.perf_counter()
    fields, pb = make_workload(args.workload, rank, args.fields)
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.Stream()
    units = units_of(fields, pb)
    with torch.cuda.stream(stream):
        # each field's uploads and set-up run on one of a few side streams (they overlap on the
        # GPU); the batch evaluates on `stream` after waiting for them
        side = [torch.cuda.Stream() for _ in range(SIDE_STREAMS)]
        probs = [Problem.from_field(fd, conv_mode=args.conv_mode, stream=side[i % SIDE_STREAMS])
                 for i, fd in enumerate(fields)]
        torch.cuda.synchronize()
        batch = Batch(probs, stream=stream) if probs else None
        # the transform form's schedule (epochs per work item, pair cap), timed on the batch
        schedule = None
        if batch is not None and args.schedule:
            ce, cg = (int(x) for x in args.schedule.split(","))
            batch.set_schedule(ce, cg)
            schedule = {"epochs_per_item": ce, "pairs_per_group": cg, "ms_per_eval": None, "fixed": True}
        elif batch is not None:
            schedule = batch.tune_schedule()
        # the PSF fit is independent of the batch: it runs on its own stream, forked from and
        # joined to `stream` in every step, so that its small launches overlap the batch's
        psf_stream = torch.cuda.Stream()
        psf = Problem.from_psf(pb, stream=psf_stream) if pb is not None else None
        fork, join = torch.cuda.Event(), torch.cuda.Event()
        P = torch.from_numpy(batch.pack([fd.params for fd in fields])).cuda() if batch else None
        P0 = P.clone() if P is not None else None
        Q = torch.from_numpy(pb.params).cuda() if psf else None
        Q0 = Q.clone() if Q is not None else None
        cfg = optim_cfg("adabelief", lr=lr_groups(fields[0])) if fields else None
        cfg_psf = optim_cfg("adabelief", lr=(1e-5, 1e-3, 10.0, 1e-3))  # b, (alpha, beta), a, c
        stream.synchronize()

        def one_step():
            # queued without host synchronisation; the step ends when `stream` has joined the
            # PSF fit's stream
            if psf is not None:
                fork.record(stream)
                psf_stream.wait_event(fork)
                psf.step(Q, 1, cfg_psf, sync=False)
                join.record(psf_stream)
            if batch is not None:
                batch.step(P, 1, cfg, sync=False)
            if psf is not None:
                stream.wait_event(join)

        for _ in range(args.warmup):
            one_step()
        if batch is not None:
            batch.profile(True)
        stream.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local_rank)
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            one_step()
        e1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        clk = clocks.stop()
        n_ev, fwd_ms, adj_ms, fft_ms = batch.profile_read() if batch is not None else (0, 0.0, 0.0, 0.0)
        if batch is not None:
            batch.profile(False)
        # per problem and step: the evaluation's launches, the loss record, and the optimiser's
        # prologue and update
        launches = 0
        if batch is not None:
            launches += (batch.launches_per_eval() + 3) * args.steps
        if psf is not None:
            launches += (psf.launches_per_eval() + 3) * args.steps
        # the same steps replayed from the captured CUDA graph (no kernel events)
        graph_ms = None
        if batch is not None:
            stream.synchronize()
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            for _ in range(args.steps):
                one_step()
            g1.record(stream)
            stream.synchronize()
            graph_ms = g0.elapsed_time(g1) / args.steps

    ms_max = ms
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    value = units * args.steps * world / (ms_max / 1e3)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e and batch is not None:
        e2e = measure_e2e(fields, probs, batch, psf, pb, max(2, min(args.steps, 10)), stream, side)

    peaks, peak_src = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local_rank).multi_processor_count
    fp32_nominal = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    from paper_2402_08725_gb300.binding import measure_fp32_peak
    fp32_peak = measure_fp32_peak()  # register-resident FFMA kernel, after the timed steps
    roof = None
    kernels = None
    if batch is not None and n_ev > 0:
        forms = batch.field_forms()
        direct_fields = [fd for fd, m in zip(fields, forms) if m == "direct"]
        fft_fields = [fd for fd, m in zip(fields, forms) if m == "fft"]
        avg_f, avg_a, avg_t = fwd_ms / n_ev, adj_ms / n_ev, fft_ms / n_ev
        kernels = {"fwd_ms": round(avg_f, 4), "adj_ms": round(avg_a, 4), "fft_ms": round(avg_t, 4),
                   "evals_profiled": n_ev, "fields_direct": len(direct_fields), "fields_fft": len(fft_fields)}
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        kernels.update({"fp32_peak_tflops_measured": round(fp32_peak, 2),
                        "fp32_peak_tflops_nominal": round(fp32_nominal, 2)})
        if direct_fields:
            fl = fwd_flops(direct_fields)
            kernels.update({"fwd_tflops": round(fl / avg_f / 1e9, 3) if avg_f > 0 else None,
                            "adj_tflops": round(fl / avg_a / 1e9, 3) if avg_a > 0 else None,
                            "direct_flops_per_launch": fl})
        if fft_fields:
            tb = fft_bytes(fft_fields)
            tf = fft_flops(fft_fields)
            kernels.update({"fft_bytes_per_launch": tb, "fft_flops_per_launch": tf,
                            "fft_gbs": round(tb / (avg_t / 1e3) / 1e9, 1), "fft_tflops": round(tf / (avg_t / 1e3) / 1e12, 3)})
        if avg_t >= max(avg_f, avg_a):
            ach = fft_bytes(fft_fields) / (avg_t / 1e3) / 1e9
            full = args.workload == "config4" and not args.fields and not direct_fields
            roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(ach / hbm, 4), "traffic": profiled_traffic() if full else None,
                    "kernel": "fft_hhat_pair_kernel + fft_chunk_pair_kernel",
                    "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"}
            if roof["traffic"] is not None:
                roof["traffic_source"] = ("fft_chunk_pair_kernel DRAM bytes per launch: ncu on the first 24 fields, "
                                          "scaled by the epoch-pixels (profiles/fft_chunk_pair_kernel_config4.md)")
        else:
            fl = fwd_flops(direct_fields)
            dom_ms, dom = (avg_f, "fwd") if avg_f >= avg_a else (avg_a, "adj")
            achieved = fl / (dom_ms / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                    "frac": round(achieved / fp32_peak, 4), "traffic": None, "kernel": f"{dom}_kernel<16>",
                    "peak_source": f"measured FFMA microbenchmark (sr_measure_fp32_peak); nominal {n_sm} SMs x "
                                   f"{FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz = {fp32_nominal:.1f}"}

    # L-BFGS-B on the same batch (sec. 2.4's second optimiser): cost per evaluation next to the
    # captured AdaBelief step, and the loss decrease over 20 iterations from the bench's start
    lbfgsb_batch = None
    if batch is not None and not args.no_noise and rank == 0:
        with torch.cuda.stream(stream):
            Pl = P0.clone()
            stream.synchronize()
            t0 = time.perf_counter()
            r = batch.lbfgsb(Pl, max_iter=20, pgtol=0.0, factr=0.0)
            wall = time.perf_counter() - t0
        lbfgsb_batch = {"iterations": r["iterations"], "evaluations": r["evaluations"], "status": r["status"],
                        "wall_s": round(wall, 3), "ms_per_evaluation": round(1e3 * wall / max(r["evaluations"], 1), 3),
                        "adabelief_ms_per_step": round(ms_max / args.steps, 3),
                        "loss_start": float(r["history"][0]), "loss_end": float(r["f"]),
                        "timing": "host clock around the call (each iteration synchronises with the host)"}
        # one L-BFGS-B per field (independent runs advanced together, one batched evaluation per
        # line-search round)
        with torch.cuda.stream(stream):
            Pl = P0.clone()
            stream.synchronize()
            t0 = time.perf_counter()
            rf, rounds = batch.lbfgsb_fields(Pl, max_iter=20, pgtol=0.0, factr=0.0)
            wall = time.perf_counter() - t0
        st_count = {}
        for q in rf:
            st_count[q["status"]] = st_count.get(q["status"], 0) + 1
        lbfgsb_batch["per_field"] = {
            "fields": len(rf), "batched_evaluations": rounds + 1, "wall_s": round(wall, 3),
            "ms_per_batched_evaluation": round(1e3 * wall / (rounds + 1), 3),
            "iterations_min_max": [min(q["iterations"] for q in rf), max(q["iterations"] for q in rf)],
            "status": st_count, "loss_start": float(sum(q["history"][0] for q in rf)),
            "loss_end": float(sum(q["f"] for q in rf)),
            "timing": "host clock around the call (per iteration: the per-field host algebra on host threads; "
                      "per line-search round one batched evaluation)"}

    plain = None
    if not args.no_plain and fields and rank == 0:
        plain = measure_plain(fields, value / world, stream)

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_baseline(fields, pb)

    noise = None
    if not args.no_noise and rank == 0:
        noise = measure_noise(stream, fp32_peak, with_cpu=not args.no_cpu and world == 1)
    pts = measure_pts(stream) if not args.no_noise and rank == 0 else None
    extraction = measure_extraction(stream) if not args.no_noise and rank == 0 else None
    psf_fit = measure_psf_fit(stream) if not args.no_noise and rank == 0 else None
    configs = None
    if not args.no_configs and rank == 0 and args.workload == "config4" and not args.fields:
        configs = measure_configs(stream, fp32_peak, float(peaks.get("hbm_gbs", 6800.0)),
                                  with_cpu=not args.no_cpu and world == 1)

    if rank == 0:
        line = {
            "metric": "loss+grad evals/sec (epoch-pixels/s), batched adjoint vs plain, % HBM roofline",
            "value": value, "unit": "epoch-px/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload + (f" (first {args.fields} fields)" if args.fields else ""),
                       "description": WORKLOADS[args.workload],
                       "epoch_pixels_per_step": units, "fields": len(fields), "psf_stars": pb.S if pb else 0,
                       "conv_mode": args.conv_mode,
                       "l2": "inputs larger than L2" if units * 12 > 129e6 else "inputs smaller than L2 (no flush)",
                       "generation_s": round(t_gen, 1)},
            "graph_ms_per_step": graph_ms,
            "schedule": schedule,
            "gpu_launches": launches,
            "clocks": clk,
            "roofline": roof,
            "kernels": kernels,
            "e2e": e2e,
            "plain": plain,
            "cpu_baseline": cpu,
            "noise_weights": noise,
            "pts_prior": pts,
            "lc_extraction": extraction,
            "psf_fit": psf_fit,
            "lbfgsb_batch": lbfgsb_batch,
            "configs": configs,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


SIDE_STREAMS = 8


# --- each configuration on its own ------------------------------------------------------------

L2_FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2: written between timed steps


def timed_steps(step, steps, warm, stream, flush):
    """Mean ms of `step` over `steps` calls, each bracketed by CUDA events on `stream`, with the
    L2 flushed (a 256 MB write) before each call, outside the events."""
    import torch
    for _ in range(warm):
        step()
    total = 0.0
    evs = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    stream.synchronize()
    for e0, e1 in evs:
        total += e0.elapsed_time(e1)
    return total / steps


def first_epochs(fd, k):
    """The field restricted to its first k epochs (data, noise, PSFs and per-epoch parameters)."""
    h, a, c, dl, gm = syn.unpack_deconv(fd.params, fd.E, fd.N, fd.f, fd.M)
    return syn.DeconvField(k, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d[:k], fd.sigma[:k], fd.s[:k], fd.W,
                           syn.pack_deconv(h, a[:k], c, dl[:k], gm[:k]))


def oracle_rate(fields, pb):
    """epoch-px/s of one literal FP64 oracle evaluation of each field (and the PSF fit)."""
    import oracle
    t0 = time.perf_counter()
    units = 0
    for fd in fields:
        oracle.deconv_loss_grad(fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s, fd.W, fd.params)
        units += fd.epoch_pixels
    if pb is not None:
        oracle.psf_loss_grad(pb.S, pb.N, pb.f, pb.J, pb.lam, pb.t, pb.sigma, pb.W, pb.params)
        units += pb.epoch_pixels
    dt = time.perf_counter() - t0
    return units / dt, dt, oracle.max_threads()


def measure_config(name, stream, fp32_peak, hbm, with_cpu, steps=10, warm=3):
    """One configuration alone: loss + gradient + AdaBelief step per step, L2 flushed between steps;
    the dominant kernel against its roof; the plain per-epoch form; the oracle on the host cores."""
    import torch
    from paper_2402_08725_gb300.binding import Batch, Problem, optim_cfg
    fields, pb = make_workload(name, 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {"description": WORKLOADS[name], "unit": "epoch-px/s", "steps": steps, "warmup": warm,
           "l2": "flushed between steps (256 MB write)"}
    with torch.cuda.stream(stream):
        if fields:
            probs = [Problem.from_field(fd, stream=stream) for fd in fields]
            batch = Batch(probs, stream=stream)
            out["schedule"] = batch.tune_schedule()
            P = torch.from_numpy(batch.pack([fd.params for fd in fields])).cuda()
            cfg = optim_cfg("adabelief", lr=lr_groups(fields[0]))
            ms = timed_steps(lambda: batch.step(P, 1, cfg, sync=False), steps, warm, stream, flush)
            batch.profile(True)
            for _ in range(3):
                batch.loss_and_grad(P)
            stream.synchronize()
            n_ev, fwd_ms, adj_ms, fft_ms = batch.profile_read()
            batch.profile(False)
            forms = batch.field_forms()
            f_ms, a_ms, t_ms = fwd_ms / n_ev, adj_ms / n_ev, fft_ms / n_ev
            if t_ms >= max(f_ms, a_ms):
                tb = fft_bytes(fields)
                ach = tb / (t_ms / 1e3) / 1e9
                L = fft_size(fields[0].N, fields[0].K, fields[0].f)
                kern = ("fft_load_rows/cols/rows + big_window_adj (global-memory transforms, L = %d)" % L
                        if L in BIG_SIZES else "fft_hhat_pair_kernel + fft_chunk_pair_kernel (L = %d)" % L)
                out["roofline"] = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                                   "frac": round(ach / hbm, 4), "traffic": None, "kernel": kern,
                                   "kernel_ms": round(t_ms, 4), "bytes_per_launch": tb,
                                   "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
            else:
                fl = fwd_flops(fields)
                dom_ms, dom = (f_ms, "fwd") if f_ms >= a_ms else (a_ms, "adj")
                ach = fl / (dom_ms / 1e3) / 1e12
                out["roofline"] = {"bound": "alu", "achieved": round(ach, 3), "peak": round(fp32_peak, 2),
                                   "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4), "traffic": None,
                                   "kernel": f"{dom}_kernel<16>", "kernel_ms": round(dom_ms, 4),
                                   "peak_source": "measured FFMA microbenchmark"}
            out["forms"] = sorted(set(forms))
            units = units_of(fields, None)
            # the plain per-epoch form on the same fields
            if name == "config5":
                # the plain form's kernels hold the whole PSF in shared memory (K = 255 does not fit):
                # the direct D-folded form on the same frames instead
                dp = [Problem.from_field(fd, conv_mode="direct", stream=stream) for fd in fields]
                db = Batch(dp, stream=stream)
                dms = timed_steps(lambda: db.step(P, 1, cfg, sync=False), 2, 1, stream, flush)
                out["plain"] = None
                out["direct"] = {"value": units / (dms / 1e3), "unit": "epoch-px/s", "ms_per_step": round(dms, 3),
                                 "speedup_transform_over_direct": dms / ms}
                db.close()
                for pr in dp:
                    pr.close()
            else:
                pp = [Problem.from_field(fd, conv_mode="plain", stream=stream) for fd in fields]
                Pp = [torch.from_numpy(fd.params).cuda() for fd in fields]
                Gp = [torch.empty_like(x) for x in Pp]

                def plain_eval():
                    for pr, x, g in zip(pp, Pp, Gp):
                        pr.loss_and_grad(x, g, sync=False)
                pms = timed_steps(plain_eval, 2, 1, stream, flush)
                plain_v = units / (pms / 1e3)
                out["plain"] = {"value": plain_v, "unit": "epoch-px/s", "ms_per_eval": round(pms, 3),
                                "speedup_batched_over_plain": (units / (ms / 1e3)) / plain_v}
                for pr in pp:
                    pr.close()
            batch.close()
            for pr in probs:
                pr.close()
        else:
            psf = Problem.from_psf(pb, stream=stream)
            Q = torch.from_numpy(pb.params).cuda()
            cfg_psf = optim_cfg("adabelief", lr=(1e-5, 1e-3, 10.0, 1e-3))
            ms = timed_steps(lambda: psf.step(Q, 1, cfg_psf, sync=False), steps, warm, stream, flush)
            units = units_of([], pb)
            # algorithmic bytes of a PSF-fit step: stars and weights read, b read and its gradient
            # written, the optimiser's 28 B per parameter
            byts = pb.S * pb.N * pb.N * 8 + pb.F * pb.F * 8 + 28 * pb.n_params
            ach = byts / (ms / 1e3) / 1e9
            out["roofline"] = {"bound": "hbm", "achieved": round(ach, 2), "peak": hbm, "unit": "GB/s",
                               "frac": round(ach / hbm, 5), "traffic": None,
                               "kernel": "the whole PSF-fit step (9 launches; latency-bound at this size)",
                               "bytes_per_step": byts, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
            out["plain"] = None
            psf.close()
    out["value"] = units / (ms / 1e3)
    out["ms_per_step"] = round(ms, 4)
    out["epoch_pixels_per_step"] = units
    if with_cpu:
        cf = fields if name != "config5" else [syn.config5(E=1, N=128)]
        cs = "all of it" if name != "config5" else "one 128x128 frame of the config-5 kind (f = 3, K = 255, 40 sources)"
        if name == "config3":   # a tenth of the epochs
            cf = [first_epochs(fields[0], 30)]
            cs = "the first 30 of the 300 epochs"
        v, dt, cores = oracle_rate(cf, pb if not fields else None)
        out["cpu_baseline"] = {"value": v, "unit": "epoch-px/s", "cores": cores, "kind": "oracle", "sample": cs,
                               "seconds": round(dt, 2)}
    return out


def measure_configs(stream, fp32_peak, hbm, with_cpu):
    return {name: measure_config(name, stream, fp32_peak, hbm, with_cpu, steps=5 if name == "config5" else 10)
            for name in ("config1", "config2", "config3", "config5")}


def measure_e2e(fields, probs, batch, psf, pb, steps, stream, side):
    """Host arrays in page-locked memory; each step copies data, noise, PSFs and parameters to
    the device through the C ABI, evaluates, and reads back the gradient and the loss.  The
    batch's inputs go in packed, one call per kind for all fields (sr_batch_set_psfs first, so that
    the PSFs' folding and kernel spectra run under the data and noise copies, which the library
    issues on its copy stream), then the evaluation from host buffers.  Two ways: pipelined (the
    evaluations queued with sr_batch_loss_and_grad_host_async and, for the PSF fit,
    sr_loss_and_grad_host_async, so that the next step's input copies run under this step's
    evaluation; one synchronisation at the end, every step's gradient and loss read back into
    page-locked memory), the reported value; and synchronous (each step waits for its results
    before the next step's copies), for comparison.  The first timed step fills the pipeline."""
    import torch

    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()

    dcat = pinned(np.concatenate([fd.d.ravel() for fd in fields]))
    scat = pinned(np.concatenate([fd.sigma.ravel() for fd in fields]))
    pcat = pinned(np.concatenate([fd.s.ravel() for fd in fields]))
    params = pinned(np.concatenate([fd.params for fd in fields])).numpy()
    grads = [torch.empty(batch.n_params, dtype=torch.float32).pin_memory().numpy() for _ in range(2)]
    totals = [torch.empty(1, dtype=torch.float64).pin_memory().numpy() for _ in range(2)]
    h2d = (dcat.numel() + scat.numel() + pcat.numel()) * 4 + params.nbytes
    d2h = grads[0].nbytes + 8
    if psf is not None:
        qd, qs = pinned(pb.t), pinned(pb.sigma)
        qp = pinned(pb.params).numpy()
        qg = torch.empty(psf.n_params, dtype=torch.float32).pin_memory().numpy()
        ql = torch.empty(1, dtype=torch.float64).pin_memory().numpy()
        h2d += (qd.numel() + qs.numel()) * 4 + qp.nbytes
        d2h += qg.nbytes + 8
    units = units_of(fields, pb)

    def one(k, pipelined):
        if psf is not None:
            psf.set_data(qd)
            psf.set_noise(qs)
            if pipelined:
                psf.loss_and_grad_host_async(qp, qg, ql)
            else:
                ql[0] = psf.loss_and_grad_host(qp, qg)[0]
        batch.set_psfs(pcat)
        batch.set_data(dcat)
        batch.set_noise(scat)
        if pipelined:
            batch.loss_and_grad_host_async(params, grads[k & 1], totals[k & 1])
        else:
            totals[0][0] = batch.loss_and_grad_host(params, grads[0])[0]

    out = {}
    for pipelined in (False, True):
        def sync():
            batch.sync()
            if psf is not None:
                psf.sync()
            stream.synchronize()
        one(0, pipelined)
        sync()
        t0 = time.perf_counter()
        for k in range(steps):
            one(k, pipelined)
        sync()
        dt = time.perf_counter() - t0
        if not all(np.isfinite(t[0]) for t in totals) or (psf is not None and not np.isfinite(ql[0])):
            raise RuntimeError("non-finite total in the end-to-end steps")
        out[pipelined] = units * steps / dt
    return {"value": out[True], "unit": "epoch-px/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps,
            "mode": "pipelined: each step's input copies run under the previous step's evaluation",
            "synchronous": {"value": out[False], "unit": "epoch-px/s",
                            "mode": "each step waits for its evaluation before the next step's copies"}}


def measure_plain(fields, batched_value, stream, max_fields=6, evals=2):
    """The plain per-epoch form (fine-grid convolution, D, residual, D^T,
    correlation as separate launches per epoch) on a sample of the fields,
    against the batched fused form's per-GPU throughput."""
    import torch
    from paper_2402_08725_gb300.binding import Problem
    rng = np.random.default_rng(1)
    idx = sorted(rng.permutation(len(fields))[:max_fields].tolist())
    with torch.cuda.stream(stream):
        probs = [Problem.from_field(fields[i], conv_mode="plain", stream=stream) for i in idx]
        ps = [torch.from_numpy(fields[i].params).cuda() for i in idx]
        gs = [torch.empty_like(p) for p in ps]
        for pr, p, g in zip(probs, ps, gs):
            pr.loss_and_grad(p, g, sync=False)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(evals):
            for pr, p, g in zip(probs, ps, gs):
                pr.loss_and_grad(p, g, sync=False)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        for pr in probs:
            pr.close()
    units = sum(fields[i].epoch_pixels for i in idx) * evals
    val = units / (ms / 1e3)
    return {"value": val, "unit": "epoch-px/s", "fields": idx, "speedup_batched_over_plain": batched_value / val}


# --- reference arm: the oracle as it stands ----------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    fields, pb = make_workload(args.workload, 0)
    # each step a bounded sample of the workload (a few seconds of CPU work)
    picked = oracle_sample(fields, pb, budget_macs=1.5e10, seed=2)
    for _ in range(args.warmup):
        time_oracle(fields, picked[:1], None)
    tot_units, tot_dt, cores = 0, 0.0, 1
    for _ in range(args.steps):
        u, dt, cores = time_oracle(fields, picked, pb)
        tot_units += u
        tot_dt += dt
    value = tot_units / tot_dt
    desc = f"{len(picked)} of {len(fields)} fields per step (" + ", ".join(
        f"N={fields[i].N} E={fields[i].E}" for i in picked) + ")" + (" + the PSF fit" if pb is not None else "")
    line = {
        "metric": "loss+grad evals/sec (epoch-pixels/s), batched adjoint vs plain, % HBM roofline",
        "value": value, "unit": "epoch-px/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_dt / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload]},
        "cpu_baseline": {"value": value, "unit": "epoch-px/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "epoch-px/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
