"""bench.py's JSON line, checked on the arm that runs without a GPU: the
reference arm (the oracle on the host cores) prints one line with the
contract's keys and types."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(600)
def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=500)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k, t in (("metric", str), ("value", (int, float)), ("unit", str), ("n_gpus", int), ("steps", int),
                 ("warmup", int), ("ms_per_step", (int, float)), ("higher_is_better", bool), ("scaling", str),
                 ("dtype", str), ("data", str), ("config", dict), ("cpu_baseline", dict), ("e2e", dict)):
        assert isinstance(d[k], t), k
    assert d["steps"] == 1 and d["warmup"] == 0 and d["value"] > 0 and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["host"]["nproc"] == os.cpu_count()
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_gpu_arm_bench_line_is_compact_and_last():
    """The GPU arm's bench line, built from a run's full record: under 4 KB,
    parseable alone, with the contract's keys; the side sections (which can
    be tens of KB) are not folded into it."""
    sys.path.insert(0, ROOT)
    import bench
    big = {"x%d" % i: {"bins_viewed_per_insert": 1.2345, "viewed_by_load": {str(q): 2.5 for q in range(9)},
                       "chain": {"p50": 0, "p99": 12, "p999": 40}} for i in range(60)}
    out = {"metric": bench.METRIC, "value": 5718.25, "unit": "M inserts/s", "n_gpus": 1, "steps": 20,
           "warmup": 5, "ms_per_step": 13.5, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u32 keys/values in u64 slots (integer)", "data": "synthetic",
           "config": {"workload": bench.WORKLOAD, "l2": "no flush", "parallelism": "dp1"},
           "bins_viewed_per_insert": 2.2814, "kicks_per_insert": 0.2794, "claim_aborts_per_insert": 1e-6,
           "m_lookups_per_s": 32800.1, "m_deletes_per_s": 6200.3, "ms": {"fill": 11.1, "lookup": 2.0, "delete": 0.6},
           "exact": {"all_inserted": True, "lookups": True, "lookup_values": True, "deletes": True},
           "roofline": {"kernel": "k_insert<4,QUEUE>", "bound": "hbm", "achieved": 1354.2, "peak": 6683.2,
                        "unit": "GB/s", "frac": 0.2026, "traffic": 518200000,
                        "peak_kind": "measured (MEASURED_PEAKS.json hbm_gbs)", "bytes_per_launch": 247600000,
                        "avg_launch_ms": 0.1828, "vs_random_gather_32B": {"gbs": 1944.0, "frac": 0.7},
                        "random_ops_model": {"frac": 0.58, "note": "x" * 300}},
           "roofline_lookup": {"kernel": "k_lookup2<4>", "bound": "hbm", "achieved": 2396.0, "peak": 6683.2,
                               "unit": "GB/s", "frac": 0.359, "vs_random_gather_32B": {"gbs": 1944.0, "frac": 1.2}},
           "e2e": {"value": 5392.0, "unit": "M inserts/s (fill incl. copies)", "ms_per_step": 11.8,
                   "h2d_bytes_per_step": 510027360, "d2h_bytes_per_step": 63753420, "results_exact": True,
                   "copies": "y" * 200, "whole_step": {"value": 4000.0, "unit": "z" * 100}},
           "gpu_launches": 1260, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 40},
           "cpu_baseline": {"value": 7.3, "unit": "M inserts/s", "cores": 1, "kind": "oracle", "sample": "s" * 300,
                            "m_lookups_per_s": 20.0, "m_deletes_per_s": 15.0,
                            "all_cores": {"cores": 16, "m_lookups_per_s": 200.0, "m_deletes_per_s": 150.0},
                            "host": {"nproc": 16, "machine": "aarch64", "cpu": "c" * 80}},
           "sections": {"policies": big, "transactional": big},
           "section_summary": {"policies": {"queue_vs_random_viewed_at_0.95": [7.5, 18.4], "failed_total": 0,
                                            "failed_beyond_oracle": [], "contents_exact": True,
                                            "lookup_vs_gather": {"b8": 1.0123, "d3": 0.9876, "d4": 0.9765}},
                               "batched_form": {"speedup_vs_per_table": 1.77, "m_inserts_per_s": 900.0,
                                                "all_inserted": True},
                               "serving_form": {"mix_75_20_5": {"results_exact": True, "speedup": 16.7},
                                                "mix_50_25_25": {"results_exact": True, "speedup": 16.9}},
                               "config1": {"m_inserts_per_s": 100.0, "l2_frac": 0.1}}}
    line = bench.headline(out)
    assert len(line.encode()) < 4096
    d = json.loads(line)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "dtype",
              "config", "bins_viewed_per_insert", "m_lookups_per_s", "roofline", "roofline_lookup",
              "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["config"]["workload"] == bench.WORKLOAD
    assert "sections" in d and "policies" not in d and "transactional" not in d
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in d["roofline"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in d["e2e"], k
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in d["cpu_baseline"], k
