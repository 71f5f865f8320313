#!/usr/bin/env python
"""Throughput of the projected t-SVD hot path (*Q-SVDII, Alg. 4.2) on GB300.

One step = one tsvdqII call through the C ABI on the video-shaped workload
(A 120 x 160 x 300 FP32, Q = leading p = 50 left singular vectors of the mode-3
unfolding, gamma = 0.99): projection, facewise Jacobi SVDs, global energy
selection, truncated factors, low-rank rebuild, back-projection and the error
terms.  Metric: tensor entries compressed per second (l*m*n / step time).

Our arm:       python bench.py [--gpus N --steps K --warmup W]
Reference arm: python bench.py --impl reference ...   (the FP64 CPU oracle)

Timing: inputs resident in HBM; L2 flushed (256 MiB write) before every step,
outside the per-step CUDA events; K steps bracketed by barrier + synchronize;
max over ranks.  The same line carries the p = n (*M) run at equal
reconstruction error, the roofline of the dominant kernel (the Jacobi SVD,
timed live with stage events on the launching stream), the end-to-end number
through host buffers, the oracle CPU baseline and the SM clocks sampled during
the timed region.
"""
from __future__ import annotations

import argparse
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L, M, N, P, GAMMA = 120, 160, 300, 50, 0.99
WORKLOAD = "video-shaped tSVDQII 120x160x300 (l x m x frames), Q = U3 leading p=50, gamma=0.99"
METRIC = "tensor entries compressed/sec (tSVDQ)"
UNIT = "entries/s"
FP32_LANES_PER_SM = 128


def nominal_svd_flops(l, m, p):
    """Textbook Golub-Kahan-Reinsch count for sigma and V of an a x b slice
    (a >= b): 4ab^2 + 8b^3, times p slices."""
    a, b = max(l, m), min(l, m)
    return p * (4.0 * a * b * b + 8.0 * b ** 3)


def pipeline_roofline(l, m, n, p, kappa, hbm_gbs, fp32_tflops, stage_ms):
    """T_roof = sum of the stage bounds of the hot path (algorithmic work per
    tensor): projection 4(lmn + np + plm) bytes at HBM bandwidth; facewise SVD
    the nominal 4ab^2 + 8b^3 flops per slice at the FP32 FMA peak; select 8 p b
    bytes; rebuild + back-projection 4 lmn + 4 kappa (l + m) + 4 np bytes.
    frac = T_roof / T_step (the measured stage sum)."""
    b = min(l, m)
    t = {"projection": 4.0 * (l * m * n + n * p + p * l * m) / (hbm_gbs * 1e9),
         "svd": nominal_svd_flops(l, m, p) / (fp32_tflops * 1e12),
         "select": 8.0 * p * b / (hbm_gbs * 1e9),
         "rebuild_backproj": 4.0 * (l * m * n + kappa * (l + m) + n * p) / (hbm_gbs * 1e9)}
    t_roof = sum(t.values())
    t_step = sum(stage_ms) / 1e3
    return {"t_roof_ms": 1e3 * t_roof, "t_step_ms": 1e3 * t_step, "frac": t_roof / t_step,
            "stage_bound_ms": {k: 1e3 * v for k, v in t.items()}}


def measure_peaks(torch, binding, stream):
    """FP32 FMA and tcgen05 tf32 throughput from the library's probe kernels
    (CUDA events on the launching stream, best of 3 after a warm-up), at the
    clocks the GPU runs at."""
    out = {}
    for kind, name, reps in ((0, "fp32_fma_tflops", 16384), (1, "tf32_tensor_tflops", 20000)):
        best = None
        with torch.cuda.stream(stream):
            binding.peak_probe(kind, reps, stream)
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fl = binding.peak_probe(kind, reps, stream)
                e1.record(stream)
                e1.synchronize()
                v = fl / (e0.elapsed_time(e1) / 1e3) / 1e12
                best = v if best is None else max(best, v)
        out[name] = best
    return out


def stage_traffic(kernels):
    """DRAM bytes per launch of the SVD stage's kernels from the committed ncu
    captures (summed), or None when any kernel's source has changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        with open(path) as f:
            recs = json.load(f)
        total = 0
        for k in kernels:
            rec = recs[k]
            with open(os.path.join(ROOT, rec["source"]), "rb") as f:
                sha = hashlib.sha256(f.read()).hexdigest()
            if not sha.startswith(rec["sha256_prefix"]):
                return None
            total += rec["dram_bytes_per_launch"]
        return total
    except (OSError, KeyError, ValueError):
        return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs():
    from paper_2409_19402_gb300 import inputs
    A = inputs.video(l=L, m=M, n=N)
    Qp = inputs.u3_q(A, P)
    Qn = inputs.u3_q(A, N)
    return A, Qp, Qn


# ------------------------------------------------------------------ reference arm
REF_BUDGET_S = 150.0

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    A, Qp, _ = make_inputs()
    # Each step is a bounded sample: the whole tensor when (steps + warmup) full
    # oracle steps fit REF_BUDGET_S, else the leading rows of every frame (a
    # smaller tSVDQII problem of the same kind, same Q and gamma).
    t0 = time.perf_counter()
    oracle.tsvdqII(A, Qp, GAMMA)                      # first warm-up step, full size
    t_full = time.perf_counter() - t0
    per_step = REF_BUDGET_S / max(1, args.steps + args.warmup)
    rows = L if t_full <= per_step else max(8, int(L * per_step / t_full))
    As = np.ascontiguousarray(A[:, :rows, :])
    for _ in range(max(0, args.warmup - 1)):
        oracle.tsvdqII(As, Qp, GAMMA)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.tsvdqII(As, Qp, GAMMA)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = rows * M * N * args.steps / total
    sample = ("each step: one full oracle tsvdqII of the workload" if rows == L else
              f"each step: oracle tsvdqII of the leading {rows} of {L} rows of every frame "
              f"({rows}x{M}x{N}, same Q and gamma)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l": L, "m": M, "n": N, "p": P, "gamma": GAMMA},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm
class Runner:
    """Preallocated buffers and a direct C-ABI call for one tsvdqII configuration."""

    def __init__(self, A_dev, Q_dev, gamma, torch, binding, precond=True):
        import ctypes
        self.t, self.b, self.ct = torch, binding, ctypes
        self.A, self.Q, self.gamma = A_dev, Q_dev, gamma
        n, l, m = A_dev.shape
        p = Q_dev.shape[1]
        r = min(l, m)
        self.dims = (l, m, n, p)
        d = A_dev.device
        self.rho = torch.empty(p, dtype=torch.int32, device=d)
        self.offs = torch.empty(p + 1, dtype=torch.int64, device=d)
        self.Uh = torch.empty(p * r * l, dtype=torch.float32, device=d)
        self.s = torch.empty(p * r, dtype=torch.float32, device=d)
        self.Vh = torch.empty(p * r * m, dtype=torch.float32, device=d)
        self.Ak = torch.empty((n, l, m), dtype=torch.float32, device=d)
        self.rep = torch.zeros(binding.REPORT_BYTES, dtype=torch.uint8, device=d)
        nb = binding.workspace_bytes(binding.PP_OP_TSVDQII, l=l, m=m, n=n, p=p)
        self.ws = torch.empty(nb, dtype=torch.uint8, device=d)
        self.opts = binding.pp_opts()
        self.opts.precond = 0 if precond else -1

    def __call__(self, stream):
        P_ = lambda x: self.ct.c_void_p(x.data_ptr())
        l, m, n, p = self.dims
        st = self.b.lib().tsvdqII(P_(self.A), P_(self.Q), l, m, n, p, float(self.gamma),
                                  P_(self.rho), P_(self.offs), P_(self.Uh), P_(self.s),
                                  P_(self.Vh), P_(self.Ak), P_(self.rep),
                                  self.ct.byref(self.opts), P_(self.ws), self.ws.numel(),
                                  self.ct.c_void_p(stream.cuda_stream))
        if st != 0:
            raise RuntimeError(self.b.status_str(st))

    def report(self):
        return self.b.read_report(self.rep)


class TruncRunner:
    """Preallocated buffers and a direct C-ABI call for one tsvdq_trunc (Alg. 4.1)
    configuration."""

    def __init__(self, A_dev, Q_dev, k, torch, binding):
        import ctypes
        self.t, self.b, self.ct = torch, binding, ctypes
        self.A, self.Q, self.k = A_dev, Q_dev, k
        n, l, m = A_dev.shape
        p = Q_dev.shape[1]
        self.dims = (l, m, n, p)
        d = A_dev.device
        self.Uh = torch.empty(p * l * k, dtype=torch.float32, device=d)
        self.s = torch.empty(p * k, dtype=torch.float32, device=d)
        self.Vh = torch.empty(p * m * k, dtype=torch.float32, device=d)
        self.Ak = torch.empty((n, l, m), dtype=torch.float32, device=d)
        self.rep = torch.zeros(binding.REPORT_BYTES, dtype=torch.uint8, device=d)
        nb = binding.workspace_bytes(binding.PP_OP_TSVDQ, l=l, m=m, n=n, p=p, k=k)
        self.ws = torch.empty(nb, dtype=torch.uint8, device=d)
        self.opts = binding.pp_opts()

    def __call__(self, stream):
        P_ = lambda x: self.ct.c_void_p(x.data_ptr())
        l, m, n, p = self.dims
        st = self.b.lib().tsvdq_trunc(P_(self.A), P_(self.Q), l, m, n, p, int(self.k), P_(self.Uh),
                                      P_(self.s), P_(self.Vh), P_(self.Ak), P_(self.rep),
                                      self.ct.byref(self.opts), P_(self.ws), self.ws.numel(),
                                      self.ct.c_void_p(stream.cuda_stream))
        if st != 0:
            raise RuntimeError(self.b.status_str(st))

    def report(self):
        return self.b.read_report(self.rep)


def equal_error_gamma(binding, A_d, Qn_d, err_target):
    """gamma' for the p = n (*M) path whose *Q-SVDII error is at most err_target:
    the smallest K whose discarded energy plus projection error fits."""
    n, l, m = A_d.shape
    full = binding.tsvdq_trunc(A_d, Qn_d, min(l, m), want_ak=False)
    import torch
    torch.cuda.synchronize()
    sig = full.s.double().cpu().numpy()
    keys = np.sort((sig ** 2).ravel())[::-1]
    c = np.cumsum(keys)
    total = c[-1]
    frep = full.report()
    proj = max(frep.normA2 - frep.normAh2, 0.0)
    need = total - (err_target - proj)
    Kp = int(np.searchsorted(c, need, side="left")) + 1
    Kp = min(max(Kp, 1), len(c))
    return min(1.0, c[Kp - 1] / total)


def sigma_error(sig_gpu, sig_ref, rel_floor=1e-3):
    """Normwise |s~ - s|_2 / |s|_2 over all slices and the largest elementwise
    relative error among the singular values >= rel_floor * max."""
    sg, sr = np.asarray(sig_gpu, np.float64), np.asarray(sig_ref, np.float64)
    nw = float(np.linalg.norm(sg - sr) / np.linalg.norm(sr))
    big = sr >= rel_floor * sr.max()
    ew = float(np.max(np.abs(sg[big] - sr[big]) / sr[big])) if big.any() else 0.0
    return {"normwise": nw, "max_rel_retained": ew}


def run_hyperspectral(args, torch, binding, stream, dev, hbm, fp32_peak):
    """The hyperspectral-shaped workload (512 x 512 x 224, Q = U3 with p in {10,
    25, 50, 100}; tSVDQII at gamma 0.99 and 0.9, fixed rank k in {5, 20, 50}),
    each timed with stage events (best of 2 after a warm-up; A is 235 MB, larger
    than L2), its pipeline roofline fraction, and the p = n = 224 (*M) path at
    equal reconstruction error for p = 10 and p = 100.  Singular values of
    slice 0 at p = 10 are compared with the oracle's."""
    from paper_2409_19402_gb300 import inputs
    A = inputs.hyperspectral()
    n, l, m = A.shape
    A_d = torch.from_numpy(A).to(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    for e in ev:
        e.record(stream)
    stream.synchronize()

    def time_run(run):
        binding.set_stage_events(ev)
        best = None
        with torch.cuda.stream(stream):
            run(stream)
            for _ in range(2):
                run(stream)
                stream.synchronize()
                st = [ev[j].elapsed_time(ev[j + 1]) for j in range(5)]
                if best is None or sum(st) < sum(best):
                    best = st
        binding.set_stage_events(None)
        return best

    out = {"workload": "hyperspectral-shaped 512x512x224, Q = U3 leading p", "configs": []}
    for p in (10, 25, 50, 100):
        Qn = inputs.u3_q(A, p)
        Q_d = torch.from_numpy(Qn).to(dev)
        for kind, par in (("tsvdqII", 0.99), ("tsvdqII", 0.9), ("tsvdq_trunc", 5),
                          ("tsvdq_trunc", 20), ("tsvdq_trunc", 50)):
            run = (Runner(A_d, Q_d, par, torch, binding) if kind == "tsvdqII"
                   else TruncRunner(A_d, Q_d, par, torch, binding))
            st = time_run(run)
            rep = run.report()
            kappa = int(rep.kappa)
            ms = sum(st)
            pipe = pipeline_roofline(l, m, n, p, kappa, hbm, fp32_peak, st)
            svd_tf = nominal_svd_flops(l, m, p) / (st[1] / 1e3) / 1e12
            cfg = {"p": p, kind == "tsvdqII" and "gamma" or "k": par, "op": kind,
                   "ms_per_step": ms, "value": l * m * n / (ms / 1e3), "unit": UNIT,
                   "stages_ms": dict(zip(("projection", "svd", "select", "factors_rebuild",
                                          "backproj_errors"), st)),
                   "svd_frac_fp32": svd_tf / fp32_peak, "pipeline_frac": pipe["frac"],
                   "kappa": kappa, "sweeps": int(rep.sweeps), "status": int(rep.status),
                   "RE": math.sqrt(rep.err2 / rep.normA2)}
            if kind == "tsvdqII" and par == 0.99 and p in (10, 100):
                # the full invertible *M form at equal reconstruction error
                Qfull = torch.from_numpy(inputs.u3_q(A, n)).to(dev)
                g2 = equal_error_gamma(binding, A_d, Qfull, rep.err2)
                runn = Runner(A_d, Qfull, g2, torch, binding)
                stn = time_run(runn)
                repn = runn.report()
                cfg["pn_compare"] = {"p": n, "gamma": g2, "ms_per_step": sum(stn),
                                     "err2": repn.err2, "err2_target": rep.err2,
                                     "kappa": int(repn.kappa),
                                     "speedup_p_lt_n": sum(stn) / ms}
                del runn, Qfull
            out["configs"].append(cfg)
            del run
        if p == 10:   # every singular value of slice 0, for the oracle comparison
            full = binding.tsvdq_trunc(A_d, Q_d, min(l, m), want_ak=False)
            torch.cuda.synchronize()
            out["_sig0_p10"] = full.s[0].double().cpu().numpy()
            out["_inputs_p10"] = (A, Qn)
            del full
    return out


def cpu_baseline_leg(args, A, Qp, sig_gpu_video, hs):
    """The oracle on the host cores: the video workload's full tSVDQII, single
    thread (the reported baseline) and OpenMP over slices (all cores), and one
    hyperspectral slice's SVD (p = 10, slice 0).  The same oracle outputs give
    the singular-value error of the GPU results (normwise over every slice of
    the video workload; slice 0 of the hyperspectral one)."""
    import oracle
    t0 = time.perf_counter()
    ref = oracle.tsvdqII(A, Qp, GAMMA)
    dt = time.perf_counter() - t0
    cpu = {"value": L * M * N / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "one full oracle tsvdqII step of the workload (FP64, single thread)",
           "seconds": dt}
    sig_err = {"video": sigma_error(sig_gpu_video, ref.sig_all)}
    cpu_omp = None
    if oracle.has_openmp():
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        oracle.tsvdqII(A, Qp, GAMMA, omp=True)
        dt2 = time.perf_counter() - t0
        cpu_omp = {"value": L * M * N / dt2, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "one full oracle tsvdqII step, OpenMP over slices and mode-3 "
                             "output slices (same arithmetic per slice), all host cores",
                   "seconds": dt2}
    if hs is not None and "_sig0_p10" in hs:
        Ah_A, Qn = hs.pop("_inputs_p10")
        t0 = time.perf_counter()
        Ah0 = oracle.mode3(Ah_A, np.asarray(Qn, np.float64)[:, :1].T)[0]
        s0 = oracle.svd(Ah0)[1]
        dt3 = time.perf_counter() - t0
        sig_err["hyperspectral_p10_slice0"] = sigma_error(hs.pop("_sig0_p10"), s0)
        hs["cpu_baseline_sample"] = {"seconds": dt3, "cores": 1, "kind": "oracle",
                                     "sample": "projection and SVD of slice 0 (512 x 512), p = 10"}
    return cpu, cpu_omp, sig_err


def timed_steps(run, steps, warmup, torch, flush, stream, stage_events=None):
    """Per-step CUDA-event times (ms) with an L2 flush before every step."""
    for _ in range(warmup):
        flush.zero_()
        run(stream)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    stage_ms = []
    times = []
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            evs[i][0].record(stream)
            run(stream)
            evs[i][1].record(stream)
        if stage_events is not None:
            stream.synchronize()
            stage_ms.append([stage_events[j].elapsed_time(stage_events[j + 1])
                             for j in range(len(stage_events) - 1)])
    torch.cuda.synchronize()
    times = [a.elapsed_time(b) for a, b in evs]
    return times, stage_ms


def max_over_ranks(x, dist, device):
    """The largest x over the ranks: the job takes as long as its slowest rank
    (x itself with one process)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, total_ms):
    """Whole-job entries/s: every rank processes its own tensor of the workload
    each step (weak scaling), in the slowest rank's time."""
    return world * L * M * N * steps / (total_ms / 1e3)


def run_ours(args):
    import torch

    import __graft_entry__
    from paper_2409_19402_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    binding.lib()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)

    A, Qp, Qn = make_inputs()
    A_d = torch.from_numpy(A).to(dev)
    Qp_d = torch.from_numpy(Qp).to(dev)
    Qn_d = torch.from_numpy(Qn).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # launch-shape autotuning of the Jacobi SVD on this problem (setup, untimed)
    from paper_2409_19402_gb300 import autotune
    if args.jacobi_shape:                          # fixed shape (profiling runs)
        C, GW, pc = (int(x) for x in args.jacobi_shape.split(","))
        binding.set_jacobi_shape(L, M, P, C, GW)
        tuned = (C, GW, None, bool(pc))
    else:
        tuned = autotune.tune_jacobi(A_d, Qp_d, gamma=GAMMA, use_cache=False)
    tuned_n = autotune.tune_jacobi(A_d, Qn_d, gamma=GAMMA, use_cache=False) if not args.no_pn else None
    run = Runner(A_d, Qp_d, GAMMA, torch, binding, precond=tuned[3])

    # stage events: created by recording once, then registered with the library
    stage_events = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    for e in stage_events:
        e.record(stream)
    stream.synchronize()
    binding.set_stage_events(stage_events)

    # ---------------- timed region (p < n)
    launches0 = binding.kernel_launches()
    clocks = ClockSampler(local)       # samples warm-up + timed steps (20 ms period)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    times, stage_ms = timed_steps(run, args.steps, args.warmup, torch, flush, stream,
                                  stage_events)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    if dist is not None:
        dist.barrier()
    launches = binding.kernel_launches() - launches0
    per_step_launches = launches / (args.steps + args.warmup)
    binding.set_stage_events(None)
    rep = run.report()
    if rep.status != 0:
        raise RuntimeError(f"device status {binding.status_str(rep.status)}")

    total_ms = max_over_ranks(sum(times), dist, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(world, args.steps, total_ms)

    # ---------------- dominant kernel roofline (Jacobi SVD, stage 1 -> 2)
    peaks, peak_kind = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    probes = measure_peaks(torch, binding, stream)
    fp32_peak = probes["fp32_fma_tflops"]
    fp32_nominal = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12     # TFLOP/s
    stage_mean = [statistics.mean(s[j] for s in stage_ms) for j in range(5)]
    jac_ms = stage_mean[1]
    flops = nominal_svd_flops(L, M, P)
    achieved = flops / (jac_ms / 1e3) / 1e12
    # the QR kernel that runs for this slice shape: register-resident up to 128
    # vectors of up to 176 entries, else the shared-memory one
    qr_kernel = "qrcp_reg_kernel" if min(L, M) <= 128 and max(L, M) <= 176 else "qrcp_kernel"
    stage_kernels = ([qr_kernel] if tuned[3] else []) + ["jacobi_cluster_kernel"]
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    pipe = pipeline_roofline(L, M, N, P, int(rep.kappa), hbm, fp32_peak, stage_mean)
    roofline = {"kernel": " + ".join(stage_kernels) + " (facewise SVD stage)", "bound": "alu",
                "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": stage_traffic(stage_kernels),
                "peak_kind": "measured: FP32 FMA probe kernel (pp_peak_probe kind 0) on this "
                             f"GPU; nominal {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                             f"{sm_max:.0f} MHz = {fp32_nominal:.1f}",
                "work": "nominal 4ab^2+8b^3 per slice (Golub-Kahan-Reinsch), p=50",
                "pipeline_frac": pipe["frac"], "pipeline": pipe,
                "hbm_peak_gbs": hbm, "hbm_peak_kind": f"{peak_kind} (MEASURED_PEAKS.json copy)",
                "probes": probes}
    proj_bytes = 4.0 * (L * M * N + N * P + P * L * M)
    back_bytes = 4.0 * (L * M * N * 2 + P * L * M + N * P)  # read A_k-hat and A, write A_k
    stages = {"projection_ms": stage_mean[0], "jacobi_ms": stage_mean[1],
              "select_ms": stage_mean[2], "factors_rebuild_ms": stage_mean[3],
              "backproj_errors_ms": stage_mean[4],
              "projection_hbm_frac": proj_bytes / (stage_mean[0] / 1e3) / 1e9 / hbm,
              "backproj_hbm_frac": back_bytes / (stage_mean[4] / 1e3) / 1e9 / hbm}

    # ---------------- p = n (*M) at equal reconstruction error
    pn = None
    if not args.no_pn:
        err_target = rep.err2
        full = binding.tsvdq_trunc(A_d, Qn_d, min(L, M), want_ak=False)
        torch.cuda.synchronize()
        sig = full.s.double().cpu().numpy()
        keys = np.sort((sig ** 2).ravel())[::-1]
        c = np.cumsum(keys)
        total = c[-1]
        frep = full.report()
        proj = max(frep.normA2 - frep.normAh2, 0.0)
        need = total - (err_target - proj)          # kept energy needed
        Kp = int(np.searchsorted(c, need, side="left")) + 1
        Kp = min(max(Kp, 1), len(c))
        gamma_pn = min(1.0, c[Kp - 1] / total)
        run_pn = Runner(A_d, Qn_d, gamma_pn, torch, binding, precond=tuned_n[3])
        t_pn, _ = timed_steps(run_pn, args.steps, args.warmup, torch, flush, stream)
        rpn = run_pn.report()
        ms_pn = sum(t_pn) / args.steps
        pn = {"p": N, "gamma": gamma_pn, "ms_per_step": ms_pn,
              "jacobi_shape": {"C": tuned_n[0], "GW": tuned_n[1], "qr_precond": tuned_n[3]},
              "value": L * M * N / (ms_pn / 1e3), "err2": rpn.err2, "err2_target": err_target,
              "kappa": int(rpn.kappa), "speedup_p_lt_n": ms_pn / ms_per_step}

    # ---------------- batched uneven workload (64 tensors): eager fork/join vs CUDA graph
    batched = None
    if world == 1 and not args.no_batched:
        batched = run_batched(args, torch, binding, stream, dev)

    # ---------------- differentiable projected product (config: W 256x256x512, X 256x64x512)
    diff = None
    if world == 1 and not args.no_diff:
        diff = run_diff(args, torch, stream, dev)

    # ---------------- complex transformation: DFT rows, p = 50 (tsvdqII_c)
    cplx = None
    if world == 1 and not args.no_complex:
        cplx = run_complex(args, torch, binding, A_d, stream, dev)

    # ---------------- end to end through host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, torch, binding, run, A, Qp, stream, dist, dev, world)

    # ---------------- hyperspectral-shaped workload (N = 1)
    hs = None
    if world == 1 and not args.no_hyperspectral:
        hs = run_hyperspectral(args, torch, binding, stream, dev, hbm, fp32_peak)

    # ---------------- oracle CPU baseline (rank 0, N = 1 only)
    cpu = cpu_omp = sig_err = None
    if world == 1 and not args.no_cpu:
        full = binding.tsvdq_trunc(A_d, Qp_d, min(L, M), want_ak=False)
        torch.cuda.synchronize()
        cpu, cpu_omp, sig_err = cpu_baseline_leg(args, A, Qp, full.s.double().cpu().numpy(), hs)
    if hs is not None:
        hs.pop("_sig0_p10", None)
        hs.pop("_inputs_p10", None)
    return finish(args, rank, world, rep, value, ms_per_step, roofline, stages, pn, e2e, cpu,
                  per_step_launches, clk, t_wall, dist, tuned, batched, diff, cplx,
                  hs=hs, cpu_omp=cpu_omp, sig_err=sig_err)


def run_complex(args, torch, binding, A_d, stream, dev):
    """The video workload with a complex Q: the first p = 50 DFT rows
    (Q = F(1:p,:)^H), *Q-SVDII with gamma = 0.99 through tsvdqII_c."""
    from paper_2409_19402_gb300 import inputs
    Qc = torch.from_numpy(inputs.dft_qc(N, P)).to(dev)
    ws = binding.workspace(binding.workspace_bytes(binding.PP_OP_TSVDQII_C, l=L, m=M, n=N, p=P),
                           dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            out = binding.tsvdqII_c(A_d, Qc, GAMMA, ws=ws, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            out = binding.tsvdqII_c(A_d, Qc, GAMMA, ws=ws, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    r = out.report()
    return {"q": "DFT rows F(1:50,:)^H (complex)", "gamma": GAMMA, "ms_per_step": ms,
            "value": L * M * N / (ms / 1e3), "unit": UNIT, "kappa": int(r.kappa),
            "sweeps": int(r.sweeps), "RE": math.sqrt(r.err2 / r.normA2),
            "status_ok": r.status == 0}


def run_diff(args, torch, stream, dev):
    """One training step of the projected-product layer Y = W *Q X (forward, loss
    1/2 |Y - T|^2, hand-written backward with the Stiefel-projected Q gradient)
    at W 256x256x512, X 256x64x512 (BF16 values, computed in FP32), Q 512x64."""
    from paper_2409_19402_gb300 import autograd as ag
    g = torch.Generator(device="cpu").manual_seed(4)
    W = (torch.randn((512, 256, 256), generator=g) / 16).to(torch.bfloat16).float().to(dev)
    X = (torch.randn((512, 256, 64), generator=g) / 16).to(torch.bfloat16).float().to(dev)
    Q = torch.linalg.qr(torch.randn((512, 64), generator=g, dtype=torch.float64))[0].float().to(dev)
    Ws = (torch.randn((512, 256, 256), generator=g) / 16).to(dev)
    Qs = torch.linalg.qr(torch.randn((512, 64), generator=g, dtype=torch.float64))[0].float().to(dev)
    with torch.no_grad():
        T = ag.qprod(Ws, X, Qs)
    W.requires_grad_(); X.requires_grad_(); Q.requires_grad_()

    def step():
        W.grad = X.grad = Q.grad = None
        loss = 0.5 * ((ag.qprod(W, X, Q) - T) ** 2).sum()
        loss.backward()
        return loss

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            loss = step()
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    eager_loss = float(loss.detach())
    # the same step captured once as a CUDA graph (forward, loss and backward)
    # and replayed: the GPU time without the host's per-launch cost
    gph = torch.cuda.CUDAGraph()
    W.grad = X.grad = Q.grad = None
    with torch.cuda.graph(gph, stream=stream):
        static_loss = 0.5 * ((ag.qprod(W, X, Q) - T) ** 2).sum()
        static_loss.backward()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            gph.replay()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            gph.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1) / args.steps
    n, n1, m, n2, p = 512, 256, 256, 64, 64
    flops = 2.0 * (n * p * (n1 * m + m * n2) + p * n1 * m * n2 + n * p * n1 * n2)  # forward
    return {"shapes": "W 256x256x512, X 256x64x512, Q 512x64", "ms_fwd_bwd": ms,
            "ms_fwd_bwd_graph": ms_graph, "loss": eager_loss,
            "loss_graph": float(static_loss.detach()), "forward_flops": flops,
            "note": "includes the torch loss/residual ops; all products in the library; "
                    "_graph: the step replayed as one CUDA graph"}


def run_batched(args, torch, binding, stream, dev):
    """64 uneven Tucker-rank-10 tensors (tSVDQII, gamma = 0.95, Q = U3 per tensor):
    one tsvdqII_batched call per step, timed eagerly and as a replayed CUDA graph.
    The inputs (1.3 GB) exceed L2, so no flush is needed between steps."""
    from paper_2409_19402_gb300 import inputs
    items = inputs.batched()
    pairs = [(torch.from_numpy(A).to(dev), torch.from_numpy(inputs.u3_q(A, p)).to(dev))
             for A, p in items]
    entries = sum(int(A.numel()) for A, _ in pairs)
    B = binding.Batch(pairs, 0.95)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    launches0 = binding.kernel_launches()
    ms_eager = timed(lambda: B(stream))
    per_call = (binding.kernel_launches() - launches0) / (args.steps + args.warmup)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        B(stream)
    ms_graph = timed(lambda: g.replay())
    reps = [o.report() for o in B.outs]
    return {"tensors": len(pairs), "entries": entries, "gamma": 0.95,
            "ms_eager": ms_eager, "ms_graph": ms_graph,
            "value_eager": entries / (ms_eager / 1e3), "value_graph": entries / (ms_graph / 1e3),
            "unit": UNIT, "kernels_per_call": per_call,
            "status_ok": all(r.status == 0 for r in reps),
            "max_sweeps": max(r.sweeps for r in reps)}


def run_e2e(args, torch, binding, run, A, Qp, stream, dist, dev, world):
    """Same metric through host buffers: every step copies its inputs (A, Q) in
    from pinned host memory and its compressed representation (report, rho,
    offs, the packed factors) out to pinned host memory.  Two buffer sets and
    a copy stream pipeline the steps, as a streaming user would: step i's
    inputs go in while step i-1 computes and step i-2's result comes out.
    The serial variant (each step copies in, computes and copies out before
    the next begins) is reported beside it."""
    A_h = torch.from_numpy(A).pin_memory()
    Q_h = torch.from_numpy(Qp).pin_memory()
    n_steps = args.warmup + args.steps

    def d2h_bytes(kappa):
        return (binding.REPORT_BYTES + run.rho.numel() * 4 + run.offs.numel() * 8 +
                4 * kappa * (L + M + 1))

    # ---- serial
    serial = []
    for i in range(n_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            run.A.copy_(A_h, non_blocking=True)
            run.Q.copy_(Q_h, non_blocking=True)
            run(stream)
            hdr = torch.empty(binding.REPORT_BYTES, dtype=torch.uint8).pin_memory()
            hdr.copy_(run.rep, non_blocking=True)
            offs_h = run.offs.to("cpu", non_blocking=True)
        stream.synchronize()
        kappa = int(offs_h[-1])
        with torch.cuda.stream(stream):
            run.Uh[:kappa * L].to("cpu", non_blocking=True)
            run.s[:kappa].to("cpu", non_blocking=True)
            run.Vh[:kappa * M].to("cpu", non_blocking=True)
        stream.synchronize()
        if i >= args.warmup:
            serial.append(time.perf_counter() - t0)
    serial_s = sum(serial)

    # ---- pipelined: two buffer sets, copies on their own stream
    runs = [run, Runner(torch.empty_like(run.A), torch.empty_like(run.Q), run.gamma, torch,
                        binding, precond=run.opts.precond >= 0)]
    cps = torch.cuda.Stream(device=dev)
    h2d_done = [torch.cuda.Event(), torch.cuda.Event()]
    comp_done = [torch.cuda.Event(), torch.cuda.Event()]
    out_done = [torch.cuda.Event(), torch.cuda.Event()]
    small = [(torch.empty(binding.REPORT_BYTES, dtype=torch.uint8).pin_memory(),
              torch.empty(run.offs.numel(), dtype=torch.int64).pin_memory(),
              torch.empty(run.rho.numel(), dtype=torch.int32).pin_memory()) for _ in range(2)]
    cap = run.s.numel()
    big = [(torch.empty(cap * L, dtype=torch.float32).pin_memory(),
            torch.empty(cap, dtype=torch.float32).pin_memory(),
            torch.empty(cap * M, dtype=torch.float32).pin_memory()) for _ in range(2)]
    moved = []
    torch.cuda.synchronize()

    def finish(j):                      # step j's result out (after its compute)
        bj = j % 2
        comp_done[bj].synchronize()
        kappa = int(small[bj][1][-1])
        r = runs[bj]
        with torch.cuda.stream(cps):
            big[bj][0][:kappa * L].copy_(r.Uh[:kappa * L], non_blocking=True)
            big[bj][1][:kappa].copy_(r.s[:kappa], non_blocking=True)
            big[bj][2][:kappa * M].copy_(r.Vh[:kappa * M], non_blocking=True)
            out_done[bj].record(cps)
        moved.append(d2h_bytes(kappa))

    t0 = None
    for i in range(n_steps):
        if i == args.warmup:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            moved.clear()
        bi = i % 2
        r = runs[bi]
        with torch.cuda.stream(cps):                # inputs in (buffer free once step i-2 left)
            if i >= 2:
                cps.wait_event(out_done[bi])
            r.A.copy_(A_h, non_blocking=True)
            r.Q.copy_(Q_h, non_blocking=True)
            h2d_done[bi].record(cps)
        with torch.cuda.stream(stream):
            stream.wait_event(h2d_done[bi])
            r(stream)
            small[bi][0].copy_(r.rep, non_blocking=True)
            small[bi][1].copy_(r.offs, non_blocking=True)
            small[bi][2].copy_(r.rho, non_blocking=True)
            comp_done[bi].record(stream)
        if i >= 1:
            finish(i - 1)
    finish(n_steps - 1)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    serial_s = max_over_ranks(serial_s, dist, dev)
    return {"value": job_throughput(world, args.steps, 1e3 * e2e_s), "unit": UNIT,
            "h2d_bytes_per_step": int(A.nbytes + Qp.nbytes),
            "d2h_bytes_per_step": int(statistics.mean(moved[:args.steps])),
            "ms_per_step": 1e3 * e2e_s / args.steps,
            "pipelined": "two buffer sets; inputs in on a copy stream while the previous step computes",
            "serial": {"value": job_throughput(world, args.steps, 1e3 * serial_s),
                       "ms_per_step": 1e3 * serial_s / args.steps}}


def finish(args, rank, world, rep, value, ms_per_step, roofline, stages, pn, e2e, cpu,
           per_step_launches, clk, t_wall, dist, tuned=None, batched=None, diff=None, cplx=None,
           hs=None, cpu_omp=None, sig_err=None):
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "l": L, "m": M, "n": N, "p": P, "gamma": GAMMA,
                       "parallelism": f"replicas x{world}" if world > 1 else "single",
                       "l2": "flushed before every step (256 MiB write), outside the events",
                       "K": int(rep.K), "kappa": int(rep.kappa), "sweeps": int(rep.sweeps),
                       "jacobi_shape": {"C": tuned[0], "GW": tuned[1], "qr_precond": tuned[3]},
                       "RE": math.sqrt(rep.err2 / rep.normA2)},
            "roofline": roofline,
            "stages": stages,
            "pn_compare": pn,
            "batched_64": batched,
            "diff_step": diff,
            "complex_dft": cplx,
            "hyperspectral": hs,
            "sigma_error_vs_oracle": sig_err,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "cpu_baseline_openmp": cpu_omp,
            "gpu_launches": int(round(per_step_launches * args.steps)),
            "clocks": clk,
            "wall_s_timed_region": t_wall,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-complex", action="store_true")
    ap.add_argument("--jacobi-shape", default="",
                    help="C,GW,precond: fixed Jacobi launch shape instead of autotuning")
    ap.add_argument("--no-pn", action="store_true", help="skip the p = n comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer run")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-tensor batched run")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiation step run")
    ap.add_argument("--no-hyperspectral", action="store_true",
                    help="skip the hyperspectral-shaped runs")
    ap.add_argument("--diff-only", action="store_true",
                    help="run only the differentiation step and print its timing (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.diff_only:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        dev = torch.device("cuda:0")
        print(json.dumps(run_diff(args, torch, torch.cuda.Stream(), dev)))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
