"""Autotuner of the batched persistent kernel's launch configuration.

For a batch of problems it times every candidate (2-D tile shape x resident
blocks per SM) on a throwaway copy of the batch (same problems, same initial
states), with CUDA events around graph replays, and returns the fastest.
Results are cached in a JSON file keyed by a signature of the GPU model and
the workload (precision, counts of 1-D and 2-D problems, and their cell
totals rounded to a power of two), so a workload of the same class on the
same kind of GPU reuses the choice without timing again.
"""
from __future__ import annotations

import json
import math
import os

from . import rhd as R

CANDIDATES = [(t, b) for t in (0, 1, 2) for b in (1, 2)]
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rhd_gb300_autotune.json")


def signature(probs, precision, device: str = "") -> str:
    n1 = [p["n"][0] for p in probs if p["ndim"] == 1]
    n2 = [p["n"][0] * p["n"][1] for p in probs if p["ndim"] == 2]

    def bucket(x):
        return 0 if x <= 0 else int(round(math.log2(x)))
    return "%s%s|1d:%d:%d|2d:%d:%d" % (device + "|" if device else "", precision, len(n1),
                                       bucket(sum(n1)), len(n2), bucket(sum(n2)))


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, cache):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(problems, precision="mixed", nsteps=4, cache_path=DEFAULT_CACHE, force=False,
         stream=None):
    """problems: list of (problem dict, state array).  Returns
    {"tile2d", "blocks_per_sm", "timings_ms", "signature", "cached"}."""
    import torch
    probs = [p for p, _ in problems]
    sig = signature(probs, precision, torch.cuda.get_device_name())
    cache = _load(cache_path) if cache_path else {}
    if not force and sig in cache:
        hit = dict(cache[sig])
        hit["cached"] = True
        return hit
    stream = stream or torch.cuda.Stream()  # a capturable (non-legacy) stream
    timings = {}
    with R.RHDBatch(probs, precision, stream=stream) as b:
        for cfg in CANDIDATES:
            b.configure(*cfg)
            for i, (_, U) in enumerate(problems):
                b.set_state(i, U)
            b.step(nsteps)  # captures the graph; not timed
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(nsteps)
            e1.record(stream)
            torch.cuda.synchronize()
            timings["%d,%d" % cfg] = e0.elapsed_time(e1) / nsteps
    best = min(timings, key=timings.get)
    t, bps = (int(v) for v in best.split(","))
    res = {"tile2d": t, "blocks_per_sm": bps, "timings_ms": timings, "signature": sig}
    if cache_path:
        cache[sig] = res
        _store(cache_path, cache)
    res = dict(res)
    res["cached"] = False
    return res
