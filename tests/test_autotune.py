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
