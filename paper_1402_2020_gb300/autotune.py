"""Autotuner for the library's launch shapes.

The cost kernel's row band (rows per CTA), its popcount form (carry-save tree or plain POPC) and the
batched cost kernel's task height change only speed, never results. This module times candidate
shapes with CUDA events on synthetic descriptor planes of the workload's size, keeps the fastest per
(GPU, descriptor length, aggregation window, dmax bucket, size bucket) in a JSON cache, and applies
it to a context with bsm_set_tuning.

Cache file: $BSM_AUTOTUNE_CACHE, else ~/.cache/bsm_gb300/autotune.json.
"""
from __future__ import annotations

import json
import os

from . import bsm

COST_ROWS = (16, 32, 64, 128, 256)
POPC_FORMS = (0, 1, 2)
VARIANTS = (1, 2, 3)  # one or two columns per lane, tensor cores
BATCH_ROWS = (32, 64, 128)


def cache_path() -> str:
    return os.environ.get("BSM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "bsm_gb300", "autotune.json"))


def bucket(v: int) -> int:
    """Round up to a power of two (buckets of image sizes and disparity ranges)."""
    b = 1
    while b < v:
        b *= 2
    return b


def key(gpu: str, n_bits: int, win: int, w: int, h: int, dmax: int) -> str:
    return f"{gpu}|n{n_bits}|win{win}|d{bucket(dmax)}|px{bucket(w * h)}|v4"


def load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(cache: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def choose(candidates, measure):
    """Fastest candidate by `measure(candidate) -> milliseconds` (ties keep the earlier candidate)."""
    best, best_t = None, float("inf")
    timings = {}
    for c in candidates:
        t = measure(c)
        timings[str(c)] = t
        if t < best_t:
            best, best_t = c, t
    return best, timings


def _time_cost(ctx, planes, w, h, dmax, rows, popc, variant, dv, reps, torch):
    dL = torch.empty((h, w), dtype=torch.int32, device="cuda")
    dR = torch.empty_like(dL)
    bsm.bsm_set_tuning(ctx, rows, popc, 0, variant, *dv)
    s = torch.cuda.current_stream()
    for _ in range(2):
        bsm.bsm_cost_aggregate_wta(ctx, *planes, w, h, dmax, dL, dR)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        bsm.bsm_cost_aggregate_wta(ctx, *planes, w, h, dmax, dL, dR)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_cost(ctx, n_bits: int, win: int, w: int, h: int, dmax: int, reps: int = 3, use_cache: bool = True) -> dict:
    """Best (cost_rows, cost_popc_plain, cost_variant) for this workload shape; applied to ctx and cached.
    The context's describe variant and tile copies are kept."""
    import torch

    cur0 = bsm.bsm_get_tuning(ctx)
    dv = (cur0["describe_variant"], cur0["describe_copies"])
    gpu = torch.cuda.get_device_name()
    k = key(gpu, n_bits, win, w, h, dmax)
    cache = load() if use_cache else {}
    if k not in cache:
        nw = n_bits // 32
        gen = torch.Generator(device="cuda").manual_seed(1234)
        planes = [torch.randint(-2 ** 31, 2 ** 31 - 1, (h, w, nw), dtype=torch.int32, device="cuda", generator=gen)
                  for _ in range(4)]
        forms = POPC_FORMS if nw == 8 else (0,)
        variants = VARIANTS if nw == 8 else ((1, 2) if nw == 4 else (1,))
        if 3 in variants:  # the tensor-core kernel is refused for the both-masks ablation
            try:
                bsm.bsm_set_tuning(ctx, 0, 0, 0, 3, *dv)
            except bsm.BsmError:
                variants = tuple(v for v in variants if v != 3)
        cands = [(r, p, v) for v in variants if v != 3 for r in COST_ROWS if r <= max(16, 2 * h) for p in forms
                 if not (v == 1 and p == 2)]
        if 3 in variants:  # the tensor-core kernel: its own band heights, popcount form unused
            cands += [(r, 0, 3) for r in (0, 16, 32, 64, 128) if r <= max(16, 2 * h)]
        best, timings = choose(cands, lambda c: _time_cost(ctx, planes, w, h, dmax, c[0], c[1], c[2], dv, reps, torch))
        cache[k] = {"cost_rows": best[0], "cost_popc_plain": best[1], "cost_variant": best[2], "timings_ms": timings}
        if use_cache:
            merged = load()
            merged[k] = cache[k]
            store(merged)
    t = cache[k]
    cur = bsm.bsm_get_tuning(ctx)
    bsm.bsm_set_tuning(ctx, t["cost_rows"], t["cost_popc_plain"], cur["batch_rows"], t.get("cost_variant", 0), *dv)
    return t


def tune_batch(ctx, descs, n_bits: int, win: int, reps: int = 2, use_cache: bool = True) -> dict:
    """Best batch task height for a batch (keyed by its total size); applied to ctx and cached."""
    import torch

    gpu = torch.cuda.get_device_name()
    px = sum(d.w * d.h for d in descs)
    k = f"{gpu}|n{n_bits}|win{win}|batch|px{bucket(px)}"
    cache = load() if use_cache else {}
    if k not in cache:
        cur = bsm.bsm_get_tuning(ctx)

        def measure(rows):
            bsm.bsm_set_tuning(ctx, cur["cost_rows"], cur["cost_popc_plain"], rows, cur["cost_variant"],
                               cur["describe_variant"], cur["describe_copies"])
            s = torch.cuda.current_stream()
            bsm.bsm_batch_run(ctx, descs)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                bsm.bsm_batch_run(ctx, descs)
            e1.record(s)
            e1.synchronize()
            return e0.elapsed_time(e1) / reps

        best, timings = choose(BATCH_ROWS, measure)
        cache[k] = {"batch_rows": best, "timings_ms": timings}
        if use_cache:
            merged = load()
            merged[k] = cache[k]
            store(merged)
    t = cache[k]
    cur = bsm.bsm_get_tuning(ctx)
    bsm.bsm_set_tuning(ctx, cur["cost_rows"], cur["cost_popc_plain"], t["batch_rows"], cur["cost_variant"],
                       cur["describe_variant"], cur["describe_copies"])
    return t
