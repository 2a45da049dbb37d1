"""Autotuner bookkeeping (CPU): signatures and the JSON cache."""
from paper_1305_4452_gb300 import autotune


def test_signature_depends_on_the_instance_mix_only():
    a = [{"nel": 16, "p": 2, "lam": 1.0}, {"nel": 32, "p": 3, "lam": 2.0}]
    b = [{"nel": 32, "p": 3, "lam": 5.0}, {"nel": 16, "p": 2, "lam": 0.7}]
    c = [{"nel": 16, "p": 2, "lam": 1.0}, {"nel": 33, "p": 3, "lam": 2.0}]
    assert autotune.signature(a) == autotune.signature(b)
    assert autotune.signature(a) != autotune.signature(c)


def test_cache_roundtrip(tmp_path):
    p = str(tmp_path / "x" / "cache.json")
    assert autotune.load_cache(p) == {}
    autotune.save_cache({"k": {"ctas_per_sm": 2}}, p)
    assert autotune.load_cache(p)["k"]["ctas_per_sm"] == 2


class _FakeBatch:
    """Stands in for iga.Batch: a solve takes a fixed time per launch shape, plus a
    change per Gram-Schmidt dot shape and per element tile (negative: a saving)."""

    def __init__(self, cost_ms, dot_delta_ms=None, line_delta_ms=None):
        self.cost_ms = cost_ms
        self.dot_delta_ms = dot_delta_ms if dot_delta_ms is not None else {0: 10.0, 2: 10.0, 4: 10.0}
        self.line_delta_ms = line_delta_ms if line_delta_ms is not None else {1: 10.0, 2: 10.0, 8: 10.0}
        self.shape = None
        self.dots = 1
        self.lines = 4
        self.launches = []

    def set_launch(self, ctas, threads=512):
        self.shape = (ctas, threads)
        self.launches.append(self.shape)

    def set_tiles(self, dots, lines=None):
        self.dots = dots
        if lines is not None:
            self.lines = lines

    def solve(self, U, opts=None, check=True):
        import time
        t = self.cost_ms[self.shape] + self.dot_delta_ms.get(self.dots, 0.0) + self.line_delta_ms.get(self.lines, 0.0)
        time.sleep(max(0.0, t) / 1e3)
        U.add_(1.0)  # the solve changes U; the tuner restores it before each timing
        return {}


def test_tune_picks_the_fastest_shape_restores_u_and_caches_it(tmp_path):
    torch = __import__("pytest").importorskip("torch")
    cost = {s: 30.0 for s in autotune.CANDIDATES}
    cost[(1, 512)] = 5.0
    ins = [{"nel": 16, "p": 2, "lam": 1.0}] * 3
    U = torch.zeros(4, dtype=torch.float64)
    cache = str(tmp_path / "c.json")
    b = _FakeBatch(cost)
    r = autotune.tune(b, ins, U, cache_path=cache)
    assert (r["ctas_per_sm"], r["threads"]) == (1, 512) and not r["cached"]
    assert b.shape == (1, 512) and set(b.launches[:-1]) == set(autotune.CANDIDATES)
    assert torch.equal(U, torch.zeros(4, dtype=torch.float64))
    assert {"%dx%d/lines4/dots1" % s for s in autotune.CANDIDATES} <= set(r["times_ms"])
    assert r["dot_chunks"] == 1 and b.dots == 1 and r["jac_lines"] == 4 and b.lines == 4
    b2 = _FakeBatch(cost)
    r2 = autotune.tune(b2, ins, U, cache_path=cache)
    assert r2["cached"] and (r2["ctas_per_sm"], r2["threads"]) == (1, 512) and b2.launches == [(1, 512)]


def test_tune_picks_the_dot_shape_on_the_best_launch_shape(tmp_path):
    torch = __import__("pytest").importorskip("torch")
    cost = {s: 40.0 for s in autotune.CANDIDATES}
    cost[(2, 256)] = 20.0
    ins = [{"nel": 24, "p": 3, "lam": 2.0}] * 2
    U = torch.zeros(3, dtype=torch.float64)
    b = _FakeBatch(cost, {0: 5.0, 2: 5.0, 4: -12.0})
    r = autotune.tune(b, ins, U, cache_path=str(tmp_path / "c.json"))
    assert (r["ctas_per_sm"], r["threads"], r["dot_chunks"]) == (2, 256, 4)
    assert b.shape == (2, 256) and b.dots == 4
    assert set(r["times_ms"]) >= {"2x256/lines4/dots%d" % d for d in autotune.DOT_CANDIDATES}


def test_tune_picks_the_element_tile_then_the_dot_shape_on_it(tmp_path):
    torch = __import__("pytest").importorskip("torch")
    cost = {s: 40.0 for s in autotune.CANDIDATES}
    cost[(1, 512)] = 20.0
    ins = [{"nel": 40, "p": 2, "lam": 3.0}] * 2
    U = torch.zeros(3, dtype=torch.float64)
    b = _FakeBatch(cost, {0: 5.0, 2: -12.0, 4: 5.0}, {1: 10.0, 2: 4.0, 8: -10.0})
    cache = str(tmp_path / "c.json")
    r = autotune.tune(b, ins, U, cache_path=cache)
    assert (r["ctas_per_sm"], r["threads"], r["jac_lines"], r["dot_chunks"]) == (1, 512, 8, 2)
    assert (b.lines, b.dots) == (8, 2)
    assert set(r["times_ms"]) >= {"1x512/lines%d/dots1" % L for L in autotune.LINE_CANDIDATES}
    assert set(r["times_ms"]) >= {"1x512/lines8/dots%d" % d for d in autotune.DOT_CANDIDATES}
    b2 = _FakeBatch(cost)
    r2 = autotune.tune(b2, ins, U, cache_path=cache)
    assert r2["cached"] and (r2["jac_lines"], r2["dot_chunks"]) == (8, 2) and (b2.lines, b2.dots) == (8, 2)


def test_tune_keeps_the_default_tile_within_the_noise_margin(tmp_path):
    torch = __import__("pytest").importorskip("torch")
    cost = {s: 30.0 for s in autotune.CANDIDATES}
    ins = [{"nel": 20, "p": 2, "lam": 1.0}]
    U = torch.zeros(2, dtype=torch.float64)
    o = type("O", (), {"ksp": 1})()  # CG: no dot stage
    b = _FakeBatch(cost, line_delta_ms={1: 10.0, 2: 10.0, 8: -0.2})  # 8 lines: under 3 % faster
    r = autotune.tune(b, ins, U, o, cache_path=str(tmp_path / "c.json"))
    assert r["jac_lines"] == 4 and r["dot_chunks"] == 1
    assert not any("dots0" in k for k in r["times_ms"])
