"""Autotuner for the solve's launch configuration.

It times the library's real entry points with CUDA events (after warm-up, on
the launching stream) over the knobs the kernels expose:

* rollout block size (threads per tile): 32, 64, 96, 128 -- the rollout
  kernel is built for 96 registers, five 128-thread blocks per SM;
* for batch plans, the CUDA-graph form: one concurrent branch per
  (objective, noise type, block) group, or one serial chain;
* where the normals are drawn: a separate Philox pass, inside the rollout
  (stored), or inside the rollout and again in the update (never stored:
  no noise memory); the same draws in every form;
* samples per thread (a block covers block x spt samples, fewer blocks per
  solve), searched for every block size with the best graph form and noise
  generation;
* optionally the noise storage (float32 or bfloat16; bfloat16 changes the
  numerics, so it is only searched when the caller allows it).

Results are cached in a JSON file keyed by GPU name, objective, K bucket (next
power of two) and N bucket (next multiple of 16).
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

from . import mppi as M
from . import workloads as W

BLOCKS = (32, 64, 96, 128)
DEFAULT_CACHE = os.environ.get("MPPI_AUTOTUNE_CACHE",
                               os.path.join(os.path.expanduser("~"), ".cache", "mppi_autotune.json"))


def _torch():
    import torch
    return torch


def gpu_name() -> str:
    torch = _torch()
    return torch.cuda.get_device_name(torch.cuda.current_device()).replace(" ", "_")


def bucket_key(objective: int, K: int, N: int) -> str:
    kb = 1 << max(0, math.ceil(math.log2(max(1, K))))
    nb = 16 * math.ceil(max(1, N) / 16)
    return f"{gpu_name()}|obj{objective}|K{kb}|N{nb}"


class Cache:
    def __init__(self, path: str = DEFAULT_CACHE):
        self.path = path
        self.data: Dict[str, dict] = {}
        if path and os.path.exists(path):
            try:
                with open(path) as f:
                    self.data = json.load(f)
            except (OSError, ValueError):
                self.data = {}

    def get(self, key: str) -> Optional[dict]:
        return self.data.get(key)

    def put(self, key: str, value: dict) -> None:
        self.data[key] = value
        if self.path:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def time_single(mc, sc, track, block: int, noise_dtype: int = M.NOISE_F32, reps: int = 20, warmup: int = 5,
                x0=None, t0: float = 0.0, noise_gen: int = M.NOISEGEN_KERNEL) -> float:
    """Mean device time (ms) of one mppi_solve_async with this block size."""
    torch = _torch()
    ctl = M.Controller(mc, sc, track, noise_dtype=noise_dtype, block=block, noise_gen=noise_gen)
    x = x0 if x0 is not None else W.hover_state_before_gate(track.gates, 0, 1.0)
    s = torch.cuda.Stream()
    dx = torch.tensor(np.float32(x), device="cuda")
    du = torch.zeros(5, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        for _ in range(warmup):
            M.mppi_solve_async(ctl.h, dx.data_ptr(), t0, s, du.data_ptr())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            M.mppi_solve_async(ctl.h, dx.data_ptr(), t0, s, du.data_ptr())
        e1.record(s)
    s.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ctl.close()
    return ms


def tune_single(mc, sc, track, blocks: Sequence[int] = BLOCKS, allow_bf16: bool = False,
                cache: Optional[Cache] = None, x0=None, t0: float = 0.0,
                noise_gens: Sequence[int] = (M.NOISEGEN_KERNEL, M.NOISEGEN_FUSED, M.NOISEGEN_REGEN)) -> dict:
    """Best block, noise generation (and noise storage, if allowed) for one
    solve shape."""
    key = bucket_key(sc.objective, sc.K, sc.N)
    if cache is not None and cache.get(key):
        return cache.get(key)
    dtypes = (M.NOISE_F32, M.NOISE_BF16) if allow_bf16 else (M.NOISE_F32,)
    table = []
    for dt in dtypes:
        for g in noise_gens:
            if g == M.NOISEGEN_REGEN and dt != M.NOISE_F32:
                continue  # regenerated noise is never stored, so it has no bfloat16 form
            for b in blocks:
                table.append({"block": b, "noise_dtype": dt, "noise_gen": g,
                              "ms": time_single(mc, sc, track, b, dt, x0=x0, t0=t0, noise_gen=g)})
    best = min(table, key=lambda r: r["ms"])
    out = {"block": best["block"], "noise_dtype": best["noise_dtype"], "noise_gen": best["noise_gen"],
           "ms": best["ms"], "table": table}
    if cache is not None:
        cache.put(key, out)
    return out


def time_batch(make_handles: Callable[..., List], x0s: np.ndarray, t0: float, mode: int, block: int,
               reps: int = 10, warmup: int = 3, noise_gen: Optional[int] = None, spt: int = 1) -> float:
    """Mean device time (ms) of one batched solve (mppi_batch_solve_async)."""
    torch = _torch()
    kw = {}
    if noise_gen is not None:
        kw["noise_gen"] = noise_gen
    if spt != 1:
        kw["spt"] = spt
    ctls = make_handles(block, **kw)
    plan = M.mppi_batch_create([c.h for c in ctls], use_graph=mode)
    n = len(ctls)
    s = torch.cuda.Stream()
    dx = torch.tensor(np.float32(x0s), device="cuda")
    dt = torch.full((n,), float(t0), dtype=torch.float64, device="cuda")
    du = torch.zeros((n, 5), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        for _ in range(warmup):
            M.mppi_batch_solve_async(plan, dx.data_ptr(), dt.data_ptr(), s, du.data_ptr())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            M.mppi_batch_solve_async(plan, dx.data_ptr(), dt.data_ptr(), s, du.data_ptr())
        e1.record(s)
    s.synchronize()
    ms = e0.elapsed_time(e1) / reps
    M.mppi_batch_destroy(plan)
    for c in ctls:
        c.close()
    return ms


def tune_batch(make_handles: Callable[..., List], x0s: np.ndarray, t0: float,
               blocks: Sequence[int] = BLOCKS, modes: Sequence[int] = (1, 2), cache: Optional[Cache] = None,
               key: Optional[str] = None, noise_gens: Optional[Sequence[int]] = None,
               spts: Sequence[int] = (1,)) -> dict:
    """Best (block, graph form[, noise generation][, samples per thread])
    for a batch; make_handles(block) builds the batch's Controllers with that
    block size (make_handles(block, noise_gen=g) when noise_gens is given,
    make_handles(block, ..., spt=s) for the samples-per-thread stage).  The
    samples per thread are searched for every block size, with the best graph
    form and noise generation of the first stage."""
    full_key = f"{gpu_name()}|batch|{key}" if key else None
    if cache is not None and full_key and cache.get(full_key):
        return cache.get(full_key)
    gens = list(noise_gens) if noise_gens else [None]
    table = []
    for g in gens:
        for b in blocks:
            for m in modes:
                table.append({"block": b, "graph_mode": m, "noise_gen": M.NOISEGEN_DEFAULT if g is None else g,
                              "spt": 1, "ms": time_batch(make_handles, x0s, t0, m, b, noise_gen=g)})
    best = min(table, key=lambda r: r["ms"])
    # samples per thread: each block size, with the best graph form and noise generation
    for s in spts:
        if s == 1:
            continue
        g = None if noise_gens is None else best["noise_gen"]
        for b in blocks:
            table.append({"block": b, "graph_mode": best["graph_mode"], "noise_gen": best["noise_gen"],
                          "spt": s, "ms": time_batch(make_handles, x0s, t0, best["graph_mode"], b,
                                                     noise_gen=g, spt=s)})
    best = min(table, key=lambda r: r["ms"])
    out = {"block": best["block"], "graph_mode": best["graph_mode"], "noise_gen": best["noise_gen"],
           "spt": best["spt"], "ms": best["ms"], "table": table}
    if cache is not None and full_key:
        cache.put(full_key, out)
    return out
