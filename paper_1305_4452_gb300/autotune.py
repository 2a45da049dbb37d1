"""Autotuner for the batched solver's launch shape.

The persistent batched kernel is compiled for several launch shapes: 256 threads
per CTA (one resident CTA per SM with up to 255 registers, or two or more with
128) and 512 (128 registers), on a grid of SMs x CTAs per SM.  More threads per
instance put more loads in flight in the memory-bound Krylov phases; fewer
registers spill more in the element kernels.  ``tune(batch, U, opts)``
times one solve per candidate shape, keeps the fastest, applies it with
``iga_batch_set_launch`` and records it in a JSON cache keyed by a signature of
the batch (instance count and the histogram of mesh sizes and degrees), so a
later batch with the same mix starts from the cached shape without re-timing.
"""
import hashlib
import json
import os
import time

# (CTAs per SM, threads per CTA)
CANDIDATES = ((1, 256), (2, 256), (4, 256), (1, 512))


def signature(instances):
    hist = {}
    for ins in instances:
        nel = ins["nel"] if isinstance(ins["nel"], int) else tuple(ins["nel"])
        key = "%s/%d/%d" % (nel, ins["p"], 1 if ins.get("log_kappa") is not None else 0)
        hist[key] = hist.get(key, 0) + 1
    blob = json.dumps(sorted(hist.items()))
    return "%d:%s" % (len(instances), hashlib.sha1(blob.encode()).hexdigest()[:16])


def _cache_path(path=None):
    if path:
        return path
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "paper_1305_4452_gb300", "batch_launch.json")


def load_cache(path=None):
    try:
        with open(_cache_path(path)) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=None):
    p = _cache_path(path)
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def tune(batch, instances, U, opts=None, candidates=CANDIDATES, cache_path=None, retime=False):
    """Choose the launch shape of `batch` (an iga.Batch built from `instances`) by
    timing one solve per candidate (CTAs per SM, threads per CTA) from the initial
    values in U (restored before each timing).  Returns {"ctas_per_sm": c,
    "threads": t, "times_ms": {"c x t": ms}, "cached": bool}."""
    import torch
    sig = signature(instances)
    cache = load_cache(cache_path)
    if not retime and sig in cache and "threads" in cache[sig]:
        best = (int(cache[sig]["ctas_per_sm"]), int(cache[sig]["threads"]))
        batch.set_launch(*best)
        return {"ctas_per_sm": best[0], "threads": best[1], "times_ms": cache[sig].get("times_ms", {}), "cached": True}
    U0 = U.clone()
    times = {}
    for c, t in candidates:
        batch.set_launch(c, t)
        U.copy_(U0)
        batch.solve(U, opts, check=False)  # first call captures the graph for this shape
        U.copy_(U0)
        if U.is_cuda:
            torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch.solve(U, opts, check=False)  # synchronises (it reads the per-instance reports)
        times["%dx%d" % (c, t)] = 1e3 * (time.perf_counter() - t0)
    key = min(times, key=times.get)
    best = tuple(int(v) for v in key.split("x"))
    batch.set_launch(*best)
    U.copy_(U0)
    cache[sig] = {"ctas_per_sm": best[0], "threads": best[1], "times_ms": times}
    save_cache(cache, cache_path)
    return {"ctas_per_sm": best[0], "threads": best[1], "times_ms": times, "cached": False}
