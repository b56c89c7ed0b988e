"""Host-side checks of the benchmark's reporting (no GPU): the stored DRAM
traffic belongs to the current SpMV kernel sources, and the defaults keep at
least three warm-up steps."""
import json
import os

import bench


def test_stored_traffic_matches_the_kernel_sources():
    path = os.path.join(bench.ROOT, "profiles", bench.TRAFFIC_FILE)
    with open(path) as f:
        t = json.load(f)
    assert t["csrc_sha"] == bench.csrc_hash(), "SpMV sources changed since the DRAM capture: re-measure"
    assert set(t["dram_bytes_per_launch"]) >= {"primal_fp32", "dual_fp32"}
    # measured traffic is at least the algorithmic bytes' order (no stale tiny value)
    for kind in ("primal", "dual"):
        ratio = t["dram_bytes_per_launch"][kind + "_fp32"] / bench.spmv_bytes(t["m"], t["n"], t["nnz"], kind, "fp32",
                                                                              t.get("layout"))
        assert 0.9 < ratio < 1.5, (kind, ratio)


def test_default_warmup_is_at_least_three(monkeypatch):
    import argparse
    seen = {}
    real = argparse.ArgumentParser.parse_args

    def capture(self, args=None, namespace=None):
        ns = real(self, [], namespace)
        seen.update(vars(ns))
        raise SystemExit(0)

    monkeypatch.setattr(argparse.ArgumentParser, "parse_args", capture)
    try:
        bench.main()
    except SystemExit:
        pass
    assert seen["warmup"] >= 3 and seen["steps"] >= 1 and seen["gpus"] == 1
