"""Autotuner for the batched solver's launch and work-unit shapes.

The persistent batched kernel is compiled for several launch shapes: 256 threads
per CTA (one resident CTA per SM with up to 255 registers, or two or more with
128) and 512 (128 registers), on a grid of SMs x CTAs per SM.  More threads per
instance put more loads in flight in the memory-bound Krylov phases; fewer
registers spill more in the element kernels.  The Gram-Schmidt dots of its GMRES
have a work-unit shape too: each dot split into R row chunks, one warp per
(dot, chunk) -- one chunk leaves most warps idle while the basis is short, many
chunks add partial sums.  ``tune(batch, U, opts)`` first times one solve per
launch shape, then, on the fastest one, one solve per dot shape (with GMRES; CG
has no such dots), keeps the fastest pair, applies it with
``iga_batch_set_launch`` / ``iga_batch_set_tiles`` and records it in a JSON cache
keyed by a signature of the batch (instance count and the histogram of mesh
sizes and degrees), so a later batch with the same mix starts from the cached
shapes without re-timing.
"""
import hashlib
import json
import os
import time

# (CTAs per SM, threads per CTA)
CANDIDATES = ((1, 256), (2, 256), (4, 256), (1, 512))
# row chunks per Gram-Schmidt dot (0: enough chunks to keep every warp busy)
DOT_CANDIDATES = (1, 2, 4, 0)


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


def _time_solve(batch, U, U0, opts):
    import torch
    U.copy_(U0)
    batch.solve(U, opts, check=False)  # the first call of a launch shape captures its graph
    U.copy_(U0)
    if U.is_cuda:
        torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.solve(U, opts, check=False)  # synchronises (it reads the per-instance reports)
    return 1e3 * (time.perf_counter() - t0)


def tune(batch, instances, U, opts=None, candidates=CANDIDATES, dot_candidates=DOT_CANDIDATES, cache_path=None,
         retime=False):
    """Choose the launch shape and the Gram-Schmidt dot shape of `batch` (an iga.Batch
    built from `instances`) by timing one solve per candidate from the initial values in U
    (restored before each timing): every (CTAs per SM, threads per CTA) first, then every
    row-chunk count of the dots on the fastest launch shape (when opts selects GMRES).
    Returns {"ctas_per_sm": c, "threads": t, "dot_chunks": r, "times_ms": {...},
    "cached": bool}."""
    sig = signature(instances)
    gmres = opts is None or int(getattr(opts, "ksp", 0)) == 0
    key_sig = sig + (":gmres" if gmres else ":cg")
    cache = load_cache(cache_path)
    if not retime and key_sig in cache and "threads" in cache[key_sig]:
        e = cache[key_sig]
        best = (int(e["ctas_per_sm"]), int(e["threads"]))
        batch.set_launch(*best)
        batch.set_tiles(int(e.get("dot_chunks", 1)))
        return {"ctas_per_sm": best[0], "threads": best[1], "dot_chunks": int(e.get("dot_chunks", 1)),
                "times_ms": e.get("times_ms", {}), "cached": True}
    U0 = U.clone()
    times = {}
    batch.set_tiles(1)
    for c, t in candidates:
        batch.set_launch(c, t)
        times["%dx%d/dots1" % (c, t)] = _time_solve(batch, U, U0, opts)
    key = min(times, key=times.get)
    best = tuple(int(v) for v in key.split("/")[0].split("x"))
    batch.set_launch(*best)
    dots = 1
    if gmres:
        base = times["%dx%d/dots1" % best]
        for r in dot_candidates:
            if r == 1:
                continue
            batch.set_tiles(r)
            times["%dx%d/dots%d" % (best[0], best[1], r)] = _time_solve(batch, U, U0, opts)
        # another dot shape replaces one chunk per dot only when it is clearly faster (3 %)
        alt = {int(k.split("/dots")[1]): v for k, v in times.items() if k.startswith("%dx%d/" % best)}
        r_best = min(alt, key=alt.get)
        if alt[r_best] < 0.97 * base:
            dots = r_best
    batch.set_tiles(dots)
    U.copy_(U0)
    cache[key_sig] = {"ctas_per_sm": best[0], "threads": best[1], "dot_chunks": dots, "times_ms": times}
    save_cache(cache, cache_path)
    return {"ctas_per_sm": best[0], "threads": best[1], "dot_chunks": dots, "times_ms": times, "cached": False}
