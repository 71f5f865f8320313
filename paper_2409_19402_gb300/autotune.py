"""Autotuner for the facewise Jacobi SVD.

For a problem of p slices of l x m it times tsvdqII with every launchable
shape -- one CTA per slice, or a cluster of C = 2..8 CTAs per slice with 8,
16 or 32 lanes per rotated pair -- each with and without the QR
preconditioner (pp_opts.precond), on the caller's data (or a seeded Gaussian
stand-in), registers the fastest shape with pp_set_jacobi_shape, and caches
the choice in a JSON file keyed by device name and (l, m, p).  The caller
passes the returned precond choice in its options.  The timing uses CUDA
events on the current stream after one warm-up call per configuration.
"""
from __future__ import annotations

import json
import os

import torch

from . import binding

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json")


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _key(l, m, p):
    return f"{torch.cuda.get_device_name()}|{l}x{m}|p{p}"


def candidates(l: int, m: int):
    b = min(l, m)
    out = [(1, 16)]
    for C in range(2, 9):
        if b >= 4 * C:
            for GW in (16, 32, 8):
                out.append((C, GW))
    return out


def tune_jacobi(A: torch.Tensor = None, Q: torch.Tensor = None, shape=None, gamma: float = 0.99,
                reps: int = 5, use_cache: bool = True, verbose: bool = False):
    """Pick and register the fastest Jacobi shape.  Give (A, Q) device tensors, or
    shape = (l, m, n, p) for a Gaussian stand-in.  Returns (C, GW, ms_per_call,
    precond) with precond the preconditioner setting of the fastest call."""
    if A is None:
        l, m, n, p = shape
        g = torch.Generator(device="cuda").manual_seed(0)
        A = torch.randn((n, l, m), device="cuda", generator=g)
        Q, _ = torch.linalg.qr(torch.randn((n, p), device="cuda", generator=g, dtype=torch.float64))
        Q = Q.float().contiguous()
    n, l, m = A.shape
    p = Q.shape[1]
    cache = _load() if use_cache else {}
    key = _key(l, m, p)
    if key in cache and len(cache[key]) == 4:
        C, GW, ms, pc = cache[key]
        binding.set_jacobi_shape(l, m, p, C, GW)
        return C, GW, ms, bool(pc)
    ws = binding.workspace(binding.workspace_bytes(binding.PP_OP_TSVDQII, l=l, m=m, n=n, p=p),
                           A.device)
    best = None
    for C, GW in candidates(l, m):
        binding.set_jacobi_shape(l, m, p, C, GW)
        for pc in (True, False):
            try:
                binding.tsvdqII(A, Q, gamma, want_ak=False, ws=ws, precond=pc)     # warm-up
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    binding.tsvdqII(A, Q, gamma, want_ak=False, ws=ws, precond=pc)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
            except binding.PPError:
                continue
            if verbose:
                print(f"  jacobi shape C={C} GW={GW} precond={pc}: {ms:.3f} ms")
            if best is None or ms < best[2]:
                best = (C, GW, ms, pc)
    C, GW, ms, pc = best
    binding.set_jacobi_shape(l, m, p, C, GW)
    if use_cache:
        cache = _load()
        cache[key] = [C, GW, ms, pc]
        tmp = CACHE + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, CACHE)
    return C, GW, ms, pc
