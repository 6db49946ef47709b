"""Host logic of the autotuner's cache (no GPU needed)."""
from paper_1912_11494_gb300 import tune


def test_cache_key_buckets():
    k1 = tune.cache_key("GB300", "plain", 10000, 4_145_000)
    k2 = tune.cache_key("GB300", "plain", 10000, 4_000_000)
    k3 = tune.cache_key("GB300", "plain", 10000, 100_000)
    k4 = tune.cache_key("GB300", "gemm_bf16", 10000, 4_145_000)
    assert k1 == k2 and k1 != k3 and k1 != k4
    assert "n<=4194304" in k1  # 4,145,000 rounds up to 2^22


def test_cache_roundtrip(tmp_path):
    p = str(tmp_path / "t.json")
    assert tune._load(p) == {}
    tune._store(p, {"a": {"config": 2}})
    assert tune._load(p) == {"a": {"config": 2}}
