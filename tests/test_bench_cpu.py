"""The benchmark's oracle baseline over independent fields (host only): the
single-thread pass and the spawned all-cores pool both run and report."""
import numpy as np


def test_cpu_baseline_fields():
    import bench
    rng = np.random.default_rng(0)
    items = [(np.cumsum(rng.normal(size=(40, 50)), 1).astype(np.float32), 1e-3) for _ in range(5)]
    r = bench.cpu_baseline_fields(items, budget_s=0.2, workers=2)
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["value"] > 0
    assert r["all_cores"]["cores"] == 2 and r["all_cores"]["value"] > 0
    assert r["all_cores"]["sample"].startswith("first ")
