"""Autotuner for the launch knobs of the persistent trace.

Knobs: rays a warp takes from the queue at a time (``chunk``), threads per block
(``block_threads``) and the level-buffer capacity (``queue_capacity``, which sets how many
rays one phase of the persistent schedule holds). Each candidate is timed with CUDA events on
a sample of the grid's sources (the cost of a trace is a sum over sources, so a sample ranks
the candidates like the whole set). A small sample separates the candidates that differ by
several percent but not the close ones, whose order can change with the number of sources in
flight, so the fastest few are timed again on a larger sample when the workload has more
sources than the first one. The winner is cached in a JSON file keyed by the grid shape, the
number of sources and the base level, so later runs of the same workload shape skip the
search.
"""
from __future__ import annotations

import dataclasses
import itertools
import json
import os

import numpy as np
import torch

from . import art as A

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")

DEFAULT_SPACE = {
    "chunk": [32, 64, 96, 128],
    "block_threads": [128, 256, 512],
    "queue_capacity": [16 << 20, 64 << 20, 256 << 20],  # rays per deep-level buffer (16 B each)
}


def _key(shape, nsrc, params: A.Params) -> str:
    return f"{shape[0]}x{shape[1]}x{shape[2]}|src{nsrc}|l0{params.level0}|m{params.m_ray}"


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _time_knobs(g, params: A.Params, knobs: dict, repeats: int, stream) -> float:
    """Best of ``repeats`` timed traces with these knobs (after one untimed trace, which also
    allocates); inf if the trace reports an error."""
    p = dataclasses.replace(params, schedule="persistent", **knobs)
    g.trace(p, force=False)
    best = float("inf")
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.trace(p, force=False, stats=False)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best if g.stats()["status"] == 0 else float("inf")


def tune(nH0: torch.Tensor, dx: float, pos, L, params: A.Params, sample: int = 16,
         space: dict | None = None, repeats: int = 2, cache_path: str | None = CACHE,
         nH: torch.Tensor | None = None, lo=(0.0, 0.0, 0.0), verbose: bool = False,
         refine_sample: int = 128, finalists: int = 3) -> A.Params:
    """Returns ``params`` with the fastest knobs for this workload shape: every candidate
    timed on ``sample`` sources, then the ``finalists`` fastest on ``refine_sample`` sources
    (when the workload has more sources than the first sample)."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    L = np.asarray(L, dtype=np.float64).reshape(-1)
    key = _key(tuple(nH0.shape), len(L), params)
    cache = _load_cache(cache_path) if cache_path else {}
    if key in cache:
        return dataclasses.replace(params, **cache[key]["knobs"])
    space = space or DEFAULT_SPACE
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(len(L), size=min(sample, len(L)), replace=False))
    stream = torch.cuda.current_stream(nH0.device)
    g = A.Grid(nH0, dx, lo=lo, nH=nH, stream=stream)
    g.add_sources(pos[idx], L[idx])
    results = []
    names = list(space)
    for combo in itertools.product(*(space[n] for n in names)):
        knobs = dict(zip(names, combo))
        best = _time_knobs(g, params, knobs, repeats, stream)
        if best == float("inf"):
            continue
        results.append((best, knobs))
        if verbose:
            print(f"  {knobs}: {best:.3f} ms")
    g.close()
    if not results:
        raise RuntimeError("autotune: every candidate failed")
    results.sort(key=lambda r: r[0])
    nsample = len(idx)
    if finalists > 1 and len(L) > len(idx) and len(results) > 1:
        idx2 = np.sort(rng.choice(len(L), size=min(refine_sample, len(L)), replace=False))
        g = A.Grid(nH0, dx, lo=lo, nH=nH, stream=stream)
        g.add_sources(pos[idx2], L[idx2])
        refined = []
        for _, knobs in results[:finalists]:
            best = _time_knobs(g, params, knobs, repeats, stream)
            if best < float("inf"):
                refined.append((best, knobs))
            if verbose:
                print(f"  refined {knobs}: {best:.3f} ms")
        g.close()
        if refined:
            results = sorted(refined, key=lambda r: r[0])
            nsample = len(idx2)
    ms, knobs = results[0]
    if cache_path:
        cache = _load_cache(cache_path)
        cache[key] = {"knobs": knobs, "ms_sample": ms, "sample_sources": int(nsample),
                      "candidates": int(np.prod([len(v) for v in space.values()]))}
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return dataclasses.replace(params, **knobs)
