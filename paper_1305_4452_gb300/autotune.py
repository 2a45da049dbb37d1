"""Autotuner for the batched solver's launch, element-tile and work-unit shapes.

The persistent batched kernel is compiled for several launch shapes: 256 threads
per CTA (one resident CTA per SM with up to 255 registers, or two or more with
128) and 512 (128 registers), on a grid of SMs x CTAs per SM.  More threads per
instance put more loads in flight in the memory-bound Krylov phases; fewer
registers spill more in the element kernels.  The Jacobian's first
sum-factorisation stage runs on element tiles of L Gauss lines staged in shared
memory: a larger L reuses each pair-table value over more lines but gives fewer
tiles to spread over the CTA and more registers per thread.  The Gram-Schmidt dots
of its GMRES have a work-unit shape too: each dot split into R row chunks, one warp
per (dot, chunk) -- one chunk leaves most warps idle while the basis is short, many
chunks add partial sums.  ``tune(batch, U, opts)`` times one solve per launch shape,
then, on the fastest one, one solve per element tile L, then (with GMRES; CG has no
such dots) one per dot shape, keeps the fastest combination, applies it with
``iga_batch_set_launch`` / ``iga_batch_set_tiles`` and records it in a JSON cache
keyed by a signature of the batch (instance count and the histogram of mesh sizes
and degrees), so a later batch with the same mix starts from the cached shapes
without re-timing.  A shape other than the default replaces it only when it is at
least 3 % faster, so that timing noise does not pick between equal shapes.
"""
import hashlib
import json
import os
import time

# (CTAs per SM, threads per CTA)
CANDIDATES = ((1, 256), (2, 256), (4, 256), (1, 512))
# Gauss lines per element tile of the Jacobian's first stage (the first is the default)
LINE_CANDIDATES = (4, 1, 2, 8)
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


def _pick(times, default_key):
    """The fastest key, unless it is within 3 % of the default's time."""
    best = min(times, key=times.get)
    return best if times[best] < 0.97 * times[default_key] else default_key


def tune(batch, instances, U, opts=None, candidates=CANDIDATES, line_candidates=LINE_CANDIDATES,
         dot_candidates=DOT_CANDIDATES, cache_path=None, retime=False):
    """Choose the launch shape, the element tile of the Jacobian and the Gram-Schmidt dot
    shape of `batch` (an iga.Batch built from `instances`) by timing one solve per
    candidate from the initial values in U (restored before each timing): every (CTAs per
    SM, threads per CTA) first, then every element tile on the fastest launch shape, then
    every row-chunk count of the dots (when opts selects GMRES).  Returns
    {"ctas_per_sm": c, "threads": t, "jac_lines": L, "dot_chunks": r, "times_ms": {...},
    "cached": bool}."""
    sig = signature(instances)
    gmres = opts is None or int(getattr(opts, "ksp", 0)) == 0
    key_sig = sig + (":gmres" if gmres else ":cg")
    cache = load_cache(cache_path)
    if not retime and key_sig in cache and "threads" in cache[key_sig]:
        e = cache[key_sig]
        best = (int(e["ctas_per_sm"]), int(e["threads"]))
        lines, dots = int(e.get("jac_lines", line_candidates[0])), int(e.get("dot_chunks", 1))
        batch.set_launch(*best)
        batch.set_tiles(dots, lines)
        return {"ctas_per_sm": best[0], "threads": best[1], "jac_lines": lines, "dot_chunks": dots,
                "times_ms": e.get("times_ms", {}), "cached": True}
    U0 = U.clone()
    times = {}
    lines0 = line_candidates[0]
    batch.set_tiles(1, lines0)
    for c, t in candidates:
        batch.set_launch(c, t)
        times["%dx%d/lines%d/dots1" % (c, t, lines0)] = _time_solve(batch, U, U0, opts)
    key = min(times, key=times.get)
    best = tuple(int(v) for v in key.split("/")[0].split("x"))
    batch.set_launch(*best)
    pre = "%dx%d" % best
    # element tile of the Jacobian's first stage, on the fastest launch shape
    for L in line_candidates[1:]:
        batch.set_tiles(1, L)
        times["%s/lines%d/dots1" % (pre, L)] = _time_solve(batch, U, U0, opts)
    alt = {L: times["%s/lines%d/dots1" % (pre, L)] for L in line_candidates}
    lines = _pick(alt, lines0)
    dots = 1
    if gmres:
        for r in dot_candidates:
            if r == 1:
                continue
            batch.set_tiles(r, lines)
            times["%s/lines%d/dots%d" % (pre, lines, r)] = _time_solve(batch, U, U0, opts)
        alt = {r: times["%s/lines%d/dots%d" % (pre, lines, r)] for r in dot_candidates}
        dots = _pick(alt, 1)
    batch.set_tiles(dots, lines)
    U.copy_(U0)
    cache[key_sig] = {"ctas_per_sm": best[0], "threads": best[1], "jac_lines": lines, "dot_chunks": dots,
                      "times_ms": times}
    save_cache(cache, cache_path)
    return {"ctas_per_sm": best[0], "threads": best[1], "jac_lines": lines, "dot_chunks": dots, "times_ms": times,
            "cached": False}
