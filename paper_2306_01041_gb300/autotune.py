"""Autotuner for the batched persistent Voronoi sweep (rt_batch_create's launch knobs).

The knobs are the wavelength chunk carried by each work item (grid, direction, chunk) and the
block size (warps per level).  Chunks are derived from one scale factor: a grid of n sites gets
chunk = round(scale * total_sites * nlam * ndir / (items_target * n)), which balances the work of
the items across grids of uneven size.  Every candidate is timed with CUDA events on the caller's
inputs (after one warm-up) and the fastest is cached in a JSON file keyed by device name, grid
sizes, level counts and wavelength count, so later runs reuse it without timing.
"""
from __future__ import annotations

import json
import os

import torch

from .api import Batch

CACHE = os.environ.get("RT_AUTOTUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "rt_gb300_autotune.json"))


def _key(grids, nlam):
    dev = torch.cuda.get_device_name()
    return f"{dev}|nlam={nlam}|" + ",".join(f"{g.npt}:{g.max_levels}" for g in grids)


def _load():
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(table):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def chunks_for(grids, nlam, scale, items_target):
    total = sum(g.npt for g in grids)
    out = []
    for g in grids:
        c = int(round(scale * total * nlam * g.ndir / (items_target * g.npt)))
        out.append(max(1, min(nlam, c)))
    return out


def tune_batch(grids, alphas, Ss, nlam, candidates=None, reps=2, use_cache=True):
    """Returns (Batch, choice dict); ``choice`` = {"lam_chunk": [...], "threads": T, "ms": t}."""
    key = _key(grids, nlam)
    table = _load() if use_cache else {}
    if key in table:
        c = table[key]
        return Batch(grids, nlam, lam_chunk=c["lam_chunk"], threads=c["threads"]), c
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    if candidates is None:
        candidates = [(s, t) for t in (256, 512) for s in (0.0625, 0.125, 0.25, 0.5, 1.0)]
    best = None
    for scale, threads in candidates:
        lc = chunks_for(grids, nlam, scale, 4 * nsm)
        b = Batch(grids, nlam, lam_chunk=lc, threads=threads)
        Js = [torch.empty_like(a) for a in alphas]
        b.formal_solution(alphas, Ss, Js=Js)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.formal_solution(alphas, Ss, Js=Js)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        if best is None or ms < best[0]:
            best = (ms, lc, threads, b)
    ms, lc, threads, b = best
    choice = {"lam_chunk": lc, "threads": threads, "ms": round(ms, 3)}
    if use_cache:
        table[key] = choice
        _store(table)
    return b, choice
