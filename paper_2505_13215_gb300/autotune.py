"""Autotuner of the rasterizer's launch shape for one workload shape.

Chooses the tile-instance capacity (the measured instance count K times a
headroom) and the pixels-per-lane of the two compositing kernels (which sets
how many warps share a 16x16 tile), by timing full training steps of the
actual workload with CUDA events.  The choice is applied to the tuned
rasterizer only (its splat_options), and cached in a JSON file keyed by
(views, resolutions, Gaussian counts, storage dtype).
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional

import torch

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
CANDIDATES = ((8, 8), (8, 4), (4, 8), (4, 4), (2, 4))


def _key(R, G) -> str:
    res = ",".join("%dx%d" % (w, h) for w, h in zip(R.W, R.H))
    return "V%d:%s:n3=%d:n4=%d:%s" % (R.V, res, G.n3, G.n4, str(G.dtype).replace("torch.", ""))


def _load() -> Dict:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save(d: Dict) -> None:
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + ".tmp.%d" % os.getpid()
        with open(tmp, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass


def _time_steps(R, G, target, reps: int) -> float:
    s = torch.cuda.current_stream()
    R.step(G, target)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(s)
    for _ in range(reps):
        R.step(G, target)
    ev[1].record(s)
    torch.cuda.synchronize()
    R.check("autotune")
    return ev[0].elapsed_time(ev[1]) / reps


def tune(R, G, target: torch.Tensor, reps: int = 6, rounds: int = 2, use_cache: bool = True,
         candidates=CANDIDATES) -> Dict:
    """Pick capacity and pixels-per-lane for (R, G); applies them and returns the choice.
    Every candidate is timed in `rounds` interleaved rounds of `reps` steps and
    keeps its fastest round, so that a transient slowdown of one trial does not
    decide the choice."""
    key = _key(R, G)
    cache = _load() if use_cache else {}
    K = R.autotune_capacity(G)
    if key in cache:
        c = cache[key]
        R.set_options(ppl_fwd=c["ppl_fwd"], ppl_bwd=c["ppl_bwd"])
        c = dict(c, K=K, capacity=R.capacity, cached=True)
        return c
    ms = {c: float("inf") for c in candidates}
    for _ in range(rounds):
        for fwd, bwd in candidates:
            R.set_options(ppl_fwd=fwd, ppl_bwd=bwd)
            ms[(fwd, bwd)] = min(ms[(fwd, bwd)], _time_steps(R, G, target, reps))
    (fwd, bwd), t = min(ms.items(), key=lambda kv: kv[1])
    best = {"ppl_fwd": fwd, "ppl_bwd": bwd, "ms": t}
    R.set_options(ppl_fwd=best["ppl_fwd"], ppl_bwd=best["ppl_bwd"])
    cache[key] = best
    if use_cache:
        _save(cache)
    return dict(best, K=K, capacity=R.capacity, cached=False)
