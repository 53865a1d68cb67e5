"""Empirical launch-shape tuner for the UST sampler.

Walkers per tree and the kernel's register variant trade walker count against
conflicts between walkers of one tree; the best point depends on the graph
(short BA walks vs. long grid walks at large alpha).  The tuner times a few
candidate shapes on one wave of trees of the caller's graph, keeps the fastest
and caches the choice per (size bucket, mean-degree bucket, weighted, trees)
in a JSON file next to the built library.  Shapes never change results.
"""
from __future__ import annotations

import json
import math
import os
import time

import torch

from . import build as _build

CANDIDATES = [(0, 40), (0, 64), (128, 64), (256, 64), (512, 64), (256, 40)]
_CACHE = os.path.join(_build.BUILD, "sampler_shapes.json")


def _key(G, tau: int) -> str:
    nb = int(math.log2(max(G.n, 1)))
    db = int(math.log2(max(1.0, G.nnz / max(G.n, 1))))
    tb = int(math.log2(max(1, tau * G.n_alpha)))
    return f"n{nb}_d{db}_w{int(G.weighted)}_a{G.n_alpha}_t{tb}"


def _load():
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def autotune(G, tau: int, probe_trees: int | None = None, seed: int = 12345) -> dict:
    """Pick and apply the fastest (walkers, regs) for G at tau trees per alpha."""
    key = _key(G, tau)
    cache = _load()
    if key in cache:
        w, r = cache[key]["walkers"], cache[key]["regs"]
        G.set_shape(w, 0, 0, r)
        return dict(cache[key], cached=True)
    probe = probe_trees or max(1, min(tau, 1024 // max(1, G.n_alpha)))
    best = None
    for w, r in CANDIDATES:
        try:
            G.set_shape(w, 0, 0, r)
            G.sample(seed, min(probe, 8), with_C=False)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G.sample(seed, probe, with_C=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        except Exception:
            continue
        if best is None or dt < best[0]:
            best = (dt, w, r, G.last_shape())
    if best is None:
        G.set_shape(0, 0, 0, 0)
        return {"walkers": 0, "regs": 0}
    dt, w, r, shp = best
    G.set_shape(w, 0, 0, r)
    entry = {"walkers": w, "regs": r, "probe_trees": probe, "probe_ms": dt * 1e3, "shape": shp}
    cache[key] = entry
    try:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return entry
