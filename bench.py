#!/usr/bin/env python3
"""Benchmark of the GB300 cuckoo-table hot path (arXiv:1605.05236).

One step = fill a 2^24-bin x 4-slot table (2^26 slots, 512 MiB of slots)
from empty to load 0.95 (63,753,420 keys) in 2^20-key insert batches with
queue-kicking, then 2^26 lookups at 50% hit, then 2^22 deletes of present
keys; everything through the C ABI (libck.so) on device-resident inputs.
The table (512 MiB) and key arrays are larger than L2, so no flush is needed
between steps.

Rank 0 prints the side sections first, one JSON line each with a
"section" key (per-policy fills, the batched and serving forms, the
transactional layer, L2-resident small table, probe sweeps), then the bench
line last: one compact JSON line whose `value` is M inserts/s over the
fills, with lookups/s, deletes/s, bins viewed per insertion, the roofline of
the dominant kernel, the end-to-end number through host buffers and the
oracle's CPU baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BINS, B = 1 << 24, 4
LOAD = 0.95
BATCH = 1 << 20
N_LOOKUP = 1 << 26
N_DELETE = 1 << 22
LOOKUP_CHUNKS = 8  # end-to-end whole step: lookups in chunks so result copies overlap
METRIC = "M inserts/s to load 0.95 & bins viewed/insert; M lookups/s; % of HBM roofline"
WORKLOAD = ("2-choice cuckoo, 2^24 bins x 4 slots (2^26 slots, 512 MiB), fill from empty to load 0.95 "
            "(63,753,420 keys) in 2^20-key batches with queue-kicking + claim flags, then 2^26 lookups "
            "(50% hit) and 2^22 deletes of present keys")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-policies", action="store_true", help="skip the per-policy fills")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-multi", action="store_true", help="skip the batched form (4096 tables)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving form")
    ap.add_argument("--no-txn", action="store_true", help="skip the transactional layer's abort counts")
    ap.add_argument("--no-small", action="store_true", help="skip the L2-resident small table")
    ap.add_argument("--policy", action="append",
                    help="with --only policies: fill only the named policy rows (repeatable)")
    ap.add_argument("--only", choices=["serve", "multi", "policies", "txn", "fill"],
                    help="run one side section alone and print its JSON (diagnostics; no bench line); "
                         "fill: one warm-up fill and one timed fill of the step's table, or of a smaller one "
                         "(--fill-bins-log2), for per-launch profiler captures")
    ap.add_argument("--fill-bins-log2", type=int, default=24,
                    help="with --only fill: log2 of the table's bins (4 slots each); the load trajectory and "
                         "the number of launches (61) stay those of the step")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def inputs_values(keys):
    from paper_1605_05236_gb300 import inputs
    return inputs.values_for(keys)


SMALL_BINS = 1 << 14      # the L2-resident small table: 2^14 bins x 4 slots (512 KiB of slots)
SMALL_KEYS = 62259        # floor(0.95 * 2^16)
SMALL_LOOKUPS = 1 << 16


def small_table_workload():
    """Keys (seed 1), values and 50%-present lookups of the small table."""
    from paper_1605_05236_gb300 import inputs
    keys, nxt = inputs.distinct_keys(SMALL_KEYS, 1)
    vals = inputs.values_for(keys)
    lk, expect = inputs.lookup_keys(keys, SMALL_LOOKUPS, 1, 0.5, next_start=nxt)
    return keys, vals, lk, expect


def workload(seed: int):
    from paper_1605_05236_gb300 import inputs
    n = inputs.load_target(BINS * B, LOAD)
    keys, nxt = inputs.distinct_keys(n, seed)
    vals = inputs.values_for(keys)
    lk, expect = inputs.lookup_keys(keys, N_LOOKUP, seed, 0.5, next_start=nxt)
    dk = inputs.delete_keys(keys, N_DELETE, seed)
    return keys, vals, lk, expect, dk


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,clocks.mem")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.environ.get("CK_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), "ck_clocks_gpu%d_%d.csv" % (gpu_index, os.getpid()))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, mem, reasons = [], 0.0, [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
                if len(parts) > 9:
                    mem.append(float(parts[9]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
               "samples": len(sm)}
        if mem:
            out["mem_mhz"] = statistics.median(mem)
        return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def gather_roofline(torch, ck, nbytes, width, n_reads, stream):
    """Measured random-gather bandwidth (GB/s) for `width`-byte records over
    a buffer of `nbytes` (the table's access pattern; bytes counted = reads x
    width): the best launch shape of a sweep over reads in flight per thread,
    block size and grid (one pass, or a grid-stride loop over at most 8, 16
    or 64 blocks per SM), each shape the best of 3 timed launches.  Returns
    (GB/s, best shape, every shape's GB/s)."""
    buf = torch.empty(nbytes // 8, dtype=torch.int64, device="cuda")
    buf.fill_(1)
    sink = torch.zeros(1024, dtype=torch.int64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    results = []
    seed = 100
    for per_thread in (1, 2, 4, 8):
        for block in (128, 256, 512):
            for per_sm in (0, 8, 16, 64):
                max_blocks = per_sm * sms
                try:  # warm (a block too large for the kernel of this width is refused)
                    ck.gather_probe_ex(buf, width, n_reads, 17, per_thread, block, max_blocks, sink, stream)
                except RuntimeError:
                    continue
                best = None
                for _ in range(3):
                    seed += 1
                    e0.record(stream)
                    ck.gather_probe_ex(buf, width, n_reads, seed, per_thread, block, max_blocks, sink, stream)
                    e1.record(stream)
                    e1.synchronize()
                    ms = e0.elapsed_time(e1)
                    best = ms if best is None else min(best, ms)
                results.append(((per_thread, block, per_sm), n_reads * width / (best * 1e-3) / 1e9))
    del buf
    cfg, gbs = max(results, key=lambda r: r[1])
    shape = {"reads_per_thread": cfg[0], "block": cfg[1], "blocks_per_sm": cfg[2] or "one pass"}
    return gbs, shape, [{"shape": list(c), "gbs": round(g, 1)} for c, g in results]


def atomic_rate(torch, ck, nbytes, kind, n_ops, stream):
    """Measured random atomics (G ops/s) of `kind` (ck_atomic_probe) over a
    buffer of `nbytes`."""
    buf = torch.zeros(nbytes // 8, dtype=torch.int64, device="cuda")
    sink = torch.zeros(1024, dtype=torch.int64, device="cuda")
    for i in range(3):
        ck.atomic_probe(buf, kind, n_ops, 17 + i, sink, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for i in range(5):
        e0.record(stream)
        ck.atomic_probe(buf, kind, n_ops, 100 + i, sink, stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del buf
    return n_ops / (best * 1e-3) / 1e9


def fill_once(torch, ck, table, kt, vt, st, stream, batch=BATCH, per_launch=False):
    """Fill from empty in `batch`-key calls; returns (ms, per-launch ms
    list).  The per-launch events (per_launch) sit between the launches and
    keep each from starting while the one before finishes, so they are
    recorded only for the serialised profile."""
    n = kt.numel()
    evs = []
    table.clear(stream)
    start = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for lo in range(0, n, batch):
        hi = min(n, lo + batch)
        if per_launch:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        table.insert_batch(kt[lo:hi], vt[lo:hi], st[lo:hi], stream)
        if per_launch:
            b.record(stream)
            evs.append((a, b))
    end = torch.cuda.Event(enable_timing=True)
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end), [a.elapsed_time(b) for a, b in evs]


def batch_profile(torch, ck, table, kt, vt, st, stream):
    """Diagnostics (outside the timed region): one fill with launches
    serialised and an event pair around each, to show how a batch's time
    grows with the load it starts at (its longest chains)."""
    table.set_param(ck.PARAM_OVERLAP, 0)
    ms, per = fill_once(torch, ck, table, kt, vt, st, stream, per_launch=True)
    table.set_param(ck.PARAM_OVERLAP, 1)
    n = kt.numel()
    idx = sorted(set([0, len(per) // 4, len(per) // 2, (3 * len(per)) // 4, len(per) - 2, len(per) - 1]))
    return {"serialised_fill_ms": round(ms, 3),
            "launch_ms_at_load": {"%.3f" % (min(n, i * BATCH) / (BINS * B)): round(per[i], 4) for i in idx}}


def chain_summary(hist):
    """Median, 99th percentile and mean chain length (kick-outs) from a
    ck_chain_histogram (bucket lower bounds beyond 31)."""
    hist = np.asarray(hist, dtype=np.float64)
    lo = np.array([i if i < 32 else 2 ** (i - 27) for i in range(len(hist))], dtype=np.float64)
    total = hist.sum()
    if total == 0:
        return {}
    cdf = np.cumsum(hist) / total
    return {"p50": int(lo[np.searchsorted(cdf, 0.5)]), "p99": int(lo[np.searchsorted(cdf, 0.99)]),
            "p999": int(lo[np.searchsorted(cdf, 0.999)]), "zero_kick_share": round(float(hist[0] / total), 4)}


def viewed_curve(t, points=(0.5, 0.7, 0.8, 0.9, 0.95)):
    """Bins viewed per insertion at each density (Sec. 3's metric, the
    curves of Figs. A-C): the insertions of the last fill that started in
    the 0.5%-wide load bucket just below the density."""
    v, c = t.load_histogram()
    out = {}
    for q in points:
        b = min(len(c) - 1, max(0, int(round(q * len(c))) - 1))
        out["%.2f" % q] = round(float(v[b]) / float(c[b]), 3) if c[b] else None
    return out


def contents_exact(torch, t, kt, vt, st, stream):
    """The table's key -> value map after a fill is exactly the keys whose
    insertion returned OK, with their values: every such key is found with
    its value, every key reported FAILED is absent, no status other than OK
    or FAILED occurs, and the table's size counter equals the OK count."""
    n = kt.numel()
    v = torch.empty(n, dtype=torch.int32, device="cuda")
    f = torch.empty(n, dtype=torch.uint8, device="cuda")
    t.lookup(kt, v, f, stream)
    torch.cuda.synchronize()
    okm = st == 0
    good = bool(((st == 0) | (st == 1)).all().item())
    good &= bool(torch.equal(f.bool(), okm))
    good &= bool(torch.equal(v[okm], vt.view(torch.int32)[okm]))
    good &= int(t.stats()["size"]) == int(okm.sum().item())
    del v, f
    return good


def oracle_full_size_failures():
    """The serial oracle's failure counts at the full-size fills, written
    by tests/golden/make_full_size_failures.py (name -> row)."""
    p = os.path.join(ROOT, "tests", "golden", "full_size_failures.json")
    return json.load(open(p)) if os.path.exists(p) else {}


def policy_fills(torch, ck, stream, base_keys, only=None):
    """One fill per policy on the same shapes (the policy rows of the path).
    Rows where the GPU fill leaves keys CK_ST_FAILED carry the serial
    oracle's failure count for the same fill (same keys, cap, hash family)."""
    from paper_1605_05236_gb300 import inputs
    ofail = oracle_full_size_failures()
    out = {}
    keys, vals = base_keys
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)
    st = torch.empty(len(keys), dtype=torch.uint8, device="cuda")
    for name, pol in (("random", ck.RANDOM), ("bfs", ck.BFS), ("sorted", ck.SORTED), ("queue", ck.QUEUE),
                      ("random+ghost", ck.RANDOM | ck.GHOST), ("bfs+ghost", ck.BFS | ck.GHOST),
                      ("sorted+ghost", ck.SORTED | ck.GHOST), ("queue+ghost", ck.QUEUE | ck.GHOST),
                      ("hybrid", ck.HYBRID), ("hybrid+ghost", ck.HYBRID | ck.GHOST),
                      ("bfs_k4", ck.BFS | 0x10000), ("sorted_k4", ck.SORTED | 0x10000),
                      ("sorted+ghost_k4", ck.SORTED | ck.GHOST | 0x10000), ("bfs_warp", ck.BFS | 0x20000)):
        # 0x10000 here: searches spawning 4 records a round (Sec. 5 prefetching);
        # 0x20000: breadth-first search by a warp per key (CK_PARAM_SEARCH_WARP)
        if only and name not in only:
            continue
        t = ck.CuckooTable(BINS, B, 2, pol & 0xFFFF, seed=1)
        if pol & 0x10000:
            t.set_param(ck.PARAM_SPAWN_K, 4)
        if pol & 0x20000:
            t.set_param(ck.PARAM_SEARCH_WARP, 1)
        fill_once(torch, ck, t, kt, vt, st, stream)  # warm
        ms, _ = fill_once(torch, ck, t, kt, vt, st, stream)
        s = t.stats()
        exact = contents_exact(torch, t, kt, vt, st, stream)
        out[name] = {"table": "2^24x4", "load": LOAD, "m_inserts_per_s": round(len(keys) / ms / 1e3, 2),
                     "contents_exact": exact,
                     "bins_viewed_per_insert": round(s["bins_viewed_per_insert"], 4),
                     "viewed_by_load": viewed_curve(t),
                     "kicks_per_insert": round(s["kicks"] / max(1, s["inserts_ok"]), 4),
                     "chain_max": s["chain_max"], "chain": chain_summary(t.chain_histogram()),
                     "failed": s["inserts_failed"], "aborted": s["inserts_aborted"],
                     "claim_aborts": s["aborts"], "conflict_views": s["conflict_views"]}
        if name in ofail:
            out[name]["oracle_failed_same_cap"] = ofail[name]["failed"]
        t.close()
        del t
        torch.cuda.empty_cache()
    del kt, vt, st
    # 8-slot bins at 0.99 and the d-ary tables of the same slot count
    lookup_cache = {}
    gathers = {}  # width -> (GB/s, shape) of the measured random gather
    for name, bins, b, d, pol, load, cap in (
            ("queue_b8_0.99", 1 << 23, 8, 2, ck.QUEUE, 0.99, 500),
            ("random_b8_0.99", 1 << 23, 8, 2, ck.RANDOM, 0.99, 500),
            ("random_d3_0.90", 1 << 26, 1, 3, ck.RANDOM, 0.90, 4096),
            ("rattle_d3_0.90", 1 << 26, 1, 3, ck.RATTLE, 0.90, 500),
            ("random_d3_0.90_hash1", 1 << 26, 1, 3, ck.RANDOM | 0x10000, 0.90, 4096),
            ("rattle_d3_0.90_hash1", 1 << 26, 1, 3, ck.RATTLE | 0x10000, 0.90, 500),
            ("random_d4_0.96", 1 << 26, 1, 4, ck.RANDOM, 0.96, 4096),
            ("rattle_d4_0.96", 1 << 26, 1, 4, ck.RATTLE, 0.96, 500),
            ("random_d4_0.96_hash1", 1 << 26, 1, 4, ck.RANDOM | 0x10000, 0.96, 4096),
            ("rattle_d4_0.96_hash1", 1 << 26, 1, 4, ck.RATTLE | 0x10000, 0.96, 500),
            ("sorted_d4_0.96", 1 << 26, 1, 4, ck.SORTED, 0.96, 500),
            ("hybrid_d4_0.96", 1 << 26, 1, 4, ck.HYBRID, 0.96, 500),
            ("sorted_d4_0.96_hash1", 1 << 26, 1, 4, ck.SORTED | 0x10000, 0.96, 500),
            ("hybrid_d4_0.96_hash1", 1 << 26, 1, 4, ck.HYBRID | 0x10000, 0.96, 500)):
        if only and name not in only:
            continue
        n = inputs.load_target(bins * b, load)
        keys, nxt = inputs.distinct_keys(n, 2)
        kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(inputs.values_for(keys))
        st = torch.empty(n, dtype=torch.uint8, device="cuda")
        family = 1 if pol & 0x10000 else 0  # 0x10000 here: the decorrelated hash family
        t = ck.CuckooTable(bins, b, d, pol & 0xFFFF, seed=1)
        t.set_param(ck.PARAM_CHAIN_CAP, cap)
        t.set_param(ck.PARAM_HASH_FAMILY, family)
        ms, _ = fill_once(torch, ck, t, kt, vt, st, stream)
        s = t.stats()
        rec = {"table": "2^%dx%d d=%d" % (int(np.log2(bins)), b, d), "load": load, "cap": cap,
               "hash_family": family, "contents_exact": contents_exact(torch, t, kt, vt, st, stream),
               "m_inserts_per_s": round(n / ms / 1e3, 2),
               "bins_viewed_per_insert": round(s["bins_viewed_per_insert"], 4),
               "viewed_by_load": viewed_curve(t, tuple(q for q in (0.5, 0.7, 0.8, 0.9, 0.95, 0.96, 0.97, 0.99)
                                                       if q <= load)),
               "chain_max": s["chain_max"], "chain": chain_summary(t.chain_histogram()),
               "failed": s["inserts_failed"], "aborted": s["inserts_aborted"]}
        if d > 2 or b == 8:
            ck_key = (bins, d, load)
            if ck_key not in lookup_cache:
                lookup_cache.clear()
                lookup_cache[ck_key] = inputs.lookup_keys(keys, N_LOOKUP, 2, 0.5, next_start=nxt)
            lk, expect = lookup_cache[ck_key]
            lkt = ck.as_u32_tensor(lk)
            v = torch.empty(N_LOOKUP, dtype=torch.int32, device="cuda")
            f = torch.empty(N_LOOKUP, dtype=torch.uint8, device="cuda")
            t.lookup(lkt, v, f, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t.lookup(lkt, v, f, stream)
            e1.record(stream)
            e1.synchronize()
            rec["m_lookups_per_s"] = round(N_LOOKUP / e0.elapsed_time(e1) / 1e3, 1)
            rec["lookups_exact"] = bool(torch.equal(f.cpu(), torch.from_numpy(expect)))
            del lkt, v, f
            # against the measured random gather of the lookup's own width: d
            # single-slot bins of 8 B, or two 8-slot bins of 64 B, per lookup
            width, per_lookup = (8, 8 * d) if d > 2 else (64, 128)
            if width not in gathers:
                gathers[width] = gather_roofline(torch, ck, bins * b * 8, width, 1 << 26, stream)[:2]
            g, shape = gathers[width]
            rb = rec["m_lookups_per_s"] * 1e6 * per_lookup / 1e9
            rec["roofline_lookup"] = {"random_bytes_gbs": round(rb, 1), "bytes_per_lookup": per_lookup,
                                      "vs_random_gather": {"width_bytes": width, "gbs": round(g, 1),
                                                           "shape": shape, "frac": round(rb / g, 4)}}
        if name in ofail:
            rec["oracle_failed_same_cap"] = ofail[name]["failed"]
        out[name] = rec
        t.close()
        del t, kt, vt, st
        torch.cuda.empty_cache()
    return out


def small_table(torch, ck, stream):
    """The L2-resident workload: 2^14 bins x 4 slots (512 KiB of slots, 64
    KiB of metadata: both stay in the 129 MB L2 across repetitions, by
    design), 62,259 keys inserted by one call with random kicking (chain cap
    500), then 65,536 lookups at 50% hits.  Its roofline is L2: the insert
    kernel's algorithmic bytes (as for the large table) over its time,
    against the measured random 32-B gather over a 512 KiB buffer."""
    keys, vals, lk, expect = small_table_workload()
    kt, vt, lkt = ck.as_u32_tensor(keys), ck.as_u32_tensor(vals), ck.as_u32_tensor(lk)
    st = torch.empty(len(keys), dtype=torch.uint8, device="cuda")
    lv = torch.empty(len(lk), dtype=torch.int32, device="cuda")
    lf = torch.empty(len(lk), dtype=torch.uint8, device="cuda")
    t = ck.CuckooTable(SMALL_BINS, B, 2, ck.RANDOM, seed=1)
    t.set_param(ck.PARAM_CHAIN_CAP, 500)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))

    def run(reps):
        fills, looks = [], []
        for r in range(reps + 3):
            t.clear(stream)
            e0.record(stream)
            t.insert_batch(kt, vt, st, stream)
            e1.record(stream)
            t.lookup(lkt, lv, lf, stream)
            e2.record(stream)
            e2.synchronize()
            if r >= 3:
                fills.append(e0.elapsed_time(e1))
                looks.append(e1.elapsed_time(e2))
        return statistics.median(fills), statistics.median(looks)

    # insertions in flight: a small table fills faster with fewer at once
    # (claim conflicts); every setting must leave the same exact table
    inflight = {}
    for m in (0, 16384, 8192, 4096, 2048, 1024):
        t.set_param(ck.PARAM_MAX_INFLIGHT, m)
        f, _ = run(5)
        ok = contents_exact(torch, t, kt, vt, st, stream) and bool((st == 0).all().item())
        inflight[str(m or "all")] = {"fill_ms": round(f, 4), "exact": ok}
    best = min((v["fill_ms"], k) for k, v in inflight.items() if v["exact"])[1]
    t.set_param(ck.PARAM_MAX_INFLIGHT, 0 if best == "all" else int(best))
    fill_ms, look_ms = run(20)
    s = t.stats()
    exact = contents_exact(torch, t, kt, vt, st, stream) and bool((st == 0).all().item())
    exact &= bool(torch.equal(lf.cpu(), torch.from_numpy(expect)))
    n = len(keys)
    ins_bytes = s["bins_viewed"] * 64 + (s["kicks"] + s["inserts_ok"]) * 64 + n * 9
    look_bytes = len(lk) * (2 * 32 + 9)
    l2g, l2_shape, _ = gather_roofline(torch, ck, SMALL_BINS * B * 8, 32, 1 << 24, stream)
    ins_gbs = ins_bytes / (fill_ms * 1e-3) / 1e9
    look_gbs = look_bytes / (look_ms * 1e-3) / 1e9
    t.close()
    return {"table": "2^14 x 4 (512 KiB of slots, L2-resident)", "keys": n, "policy": "random kicking, cap 500",
            "repetitions": 20, "max_inflight": best, "inflight_sweep": inflight,
            "m_inserts_per_s": round(n / fill_ms / 1e3, 2), "fill_ms": round(fill_ms, 4),
            "bins_viewed_per_insert": round(s["bins_viewed_per_insert"], 4), "chain_max": s["chain_max"],
            "m_lookups_per_s": round(len(lk) / look_ms / 1e3, 1), "lookup_ms": round(look_ms, 4),
            "exact": exact,
            "roofline": {"bound": "l2", "unit": "GB/s", "peak": round(l2g, 1),
                         "peak_kind": "measured random 32-B gather over 512 KiB", "peak_shape": l2_shape,
                         "insert_achieved": round(ins_gbs, 1), "insert_frac": round(ins_gbs / l2g, 4),
                         "lookup_achieved": round(look_gbs, 1), "lookup_frac": round(look_gbs / l2g, 4)}}


def multi_form(torch, ck, stream):
    """Batched form: 4096 independent tables (bins log-uniform in [2^10, 2^18],
    4 or 8 slots, keys from seed 8 + table id) filled to 0.95 with
    queue-kicking, as one autotuned persistent launch versus one launch per
    table, each replayed from a CUDA graph."""
    from paper_1605_05236_gb300 import autotune, inputs
    from paper_1605_05236_gb300 import multi as M
    t0 = time.perf_counter()
    bins, slots = inputs.multi_shapes(4096, seed=7)
    keys, vals, n_keys = inputs.multi_keys(bins, slots, 0.95, seed0=8)
    gen_s = time.perf_counter() - t0
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)
    st = torch.empty(len(keys), dtype=torch.uint8, device="cuda")
    mt = M.MultiTable(bins, slots, n_keys, ck.QUEUE, seed=1)
    best, trials = autotune.tune(mt, kt, vt, st, stream)

    def graph_ms(per_table):
        # the product's captured fill (ck_multi_capture): clear + insert,
        # replayed as one CUDA graph
        g = mt.capture(kt, vt, st, per_table=per_table, clear=True, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g.launch(stream)
        torch.cuda.synchronize()
        best_ms = None
        for _ in range(3):
            e0.record(stream)
            g.launch(stream)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best_ms = ms if best_ms is None else min(best_ms, ms)
        ok = bool((st == 0).all().item())
        s = mt.stats()
        g.close()
        return best_ms, ok, s

    ms_b, ok_b, s_b = graph_ms(False)
    ms_p, ok_p, s_p = graph_ms(True)
    n = len(keys)
    out = {"tables": 4096, "keys": n, "slots": int((bins * slots).sum()), "gen_s": round(gen_s, 1),
           "autotuned": best, "tuning": [{"cfg": c, "ms": round(m, 3)} for c, m in trials],
           "batched": {"ms": round(ms_b, 3), "m_inserts_per_s": round(n / ms_b / 1e3, 1), "all_inserted": ok_b,
                       "bins_viewed_per_insert": round(s_b["bins_viewed_per_insert"], 4), "size": s_b["size"]},
           "per_table": {"ms": round(ms_p, 3), "m_inserts_per_s": round(n / ms_p / 1e3, 1), "all_inserted": ok_p,
                         "bins_viewed_per_insert": round(s_p["bins_viewed_per_insert"], 4), "size": s_p["size"],
                         "launches": 4096},
           "speedup": round(ms_p / ms_b, 3)}
    mt.close()
    del kt, vt, st, mt
    torch.cuda.empty_cache()
    return out


# DRAM bytes read + written per insert launch of the step's fill (mean over
# its 61 launches) from an ncu capture of the current kernel build: a
# half-size fill (2^23 x 4, the same 61-launch load trajectory, half the keys
# per launch), scaled by 2; None until captured for this build
INSERT_TRAFFIC_PER_LAUNCH = 382_100_000

SERVE_BINS = 1 << 26
SERVE_PREFILL = 255013683  # floor(0.95 * 2^28)
SERVE_CAP = 1000


def serve_form(torch, ck, stream):
    """Serving form: a 2^26 x 4 table (2 GiB of slots) prefilled to 0.95
    (255,013,683 keys of seed 5) takes a trace of 4096 requests (Poisson
    arrivals at 20k requests/ms, sizes log-uniform 1..2^16 keys, mixes
    lookup/insert/delete 75/20/5 and 50/25/25, seed 11), run (a) as plain
    sequential bulk calls and (b) through the continuous-batching server,
    each at the trace's own rate (a burst far above either's capacity) and
    open-loop at 0.8x the capacity the sequential run showed; the server
    also at 0.8x its own capacity.  The table is refilled before every run, so every
    run starts from the same state, and its results must equal the trace's."""
    from paper_1605_05236_gb300 import inputs, serve
    t0 = time.perf_counter()
    keys, _ = inputs.distinct_keys(SERVE_PREFILL, 5)
    vals = inputs.values_for(keys)
    gen_s = time.perf_counter() - t0
    table = ck.CuckooTable(SERVE_BINS, B, 2, ck.QUEUE, seed=1)
    # chain cap 1000: at 2^28 slots and loads up to 0.965 a few concurrent
    # walks in 10^8 pass 500 kick-outs (the serial fill's longest is ~250),
    # and a failed insert would make the results depend on the interleaving
    table.set_param(ck.PARAM_CHAIN_CAP, SERVE_CAP)
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)
    st = torch.empty(len(keys), dtype=torch.uint8, device="cuda")

    def prefill():
        fill_once(torch, ck, table, kt, vt, st, stream)
        torch.cuda.synchronize()

    def summary(tr, res, scale):
        v, s, lat = res
        arrive = tr["arrive_ns"].astype(np.float64) * scale
        span_s = float(np.max(arrive + lat)) * 1e-9
        n_keys = len(tr["keys"])
        return {"m_keys_per_s": round(n_keys / span_s / 1e6, 1), "k_req_per_s": round(len(lat) / span_s / 1e3, 1),
                "span_ms": round(span_s * 1e3, 3), "p50_us": round(float(np.percentile(lat, 50)) / 1e3, 1),
                "p99_us": round(float(np.percentile(lat, 99)) / 1e3, 1)}

    def check(tr, res):
        """None when every result equals the trace's, else mismatch counts."""
        v, s, _ = res
        op = np.repeat(tr["op"], tr["n_keys"].astype(np.int64))
        look = op == 0
        hit = look & (tr["expect"] == 1)
        want = np.where(look, tr["expect"], np.where(op == 1, 0, 1)).astype(np.uint8)
        bad = s != want
        bad_val = int((v[hit] != tr["vals"][hit]).sum())
        if not bad.any() and not bad_val:
            return None
        out = {"value_mismatch": bad_val}
        for name, k in (("lookup", 0), ("insert", 1), ("delete", 2)):
            sel = bad & (op == k)
            if sel.any():
                st_vals, cnt = np.unique(s[sel], return_counts=True)
                out[name] = {"wrong": int(sel.sum()), "statuses": {int(a): int(b) for a, b in zip(st_vals, cnt)}}
        return out

    cfg = {"wave_keys": 1 << 20, "wave_slots": 4, "load_hi": 0.97}
    out = {"table": "2^26 x 4 prefilled to 0.95 (255,013,683 keys), queue-kicking, chain cap %d" % SERVE_CAP,
           "requests": 4096,
           "sizes": "log-uniform 1..2^16 keys", "arrivals": "Poisson, 20k requests/ms", "server": cfg,
           "gen_s": round(gen_s, 1)}
    for mix in [(75, 20, 5), (50, 25, 25)]:
        tr = inputs.serving_trace(keys, 4096, mix, seed=11, max_log2=16)
        rec = {"keys": int(len(tr["keys"])), "mix": "%d/%d/%d" % mix}
        runs, run_names = [], ["sequential_trace_rate"]
        prefill()
        seq = serve.replay_sequential(table, tr, time_scale=1.0)
        runs.append(seq)
        rec["sequential_trace_rate"] = summary(tr, seq, 1.0)

        def run(name, sc, server):
            prefill()
            if server:
                srv = serve.Server(table, **cfg)
                res = srv.replay(tr, time_scale=sc)
                info = srv.info()
                srv.close()
            else:
                res, info = serve.replay_sequential(table, tr, time_scale=sc), None
            runs.append(res)
            run_names.append(name)
            rec[name] = summary(tr, res, sc)
            if info:
                rec[name]["waves"] = info["waves"]
                rec[name]["busy_rejects"] = info["busy_rejects"]

        def scale_for(rate):  # time scale that makes the trace arrive at `rate` requests/s
            return (len(tr["op"]) / rate * 1e9) / max(1.0, float(tr["arrive_ns"][-1]))

        run("server_trace_rate", 1.0, True)
        cap_seq = len(tr["op"]) / (rec["sequential_trace_rate"]["span_ms"] * 1e-3)  # requests/s
        cap_srv = len(tr["op"]) / (rec["server_trace_rate"]["span_ms"] * 1e-3)
        run("sequential_0.8x_seq_capacity", scale_for(0.8 * cap_seq), False)
        run("server_0.8x_seq_capacity", scale_for(0.8 * cap_seq), True)
        run("server_0.8x_server_capacity", scale_for(0.8 * cap_srv), True)
        rec["capacity_k_req_per_s"] = {"sequential": round(cap_seq / 1e3, 1), "server": round(cap_srv / 1e3, 1)}
        # every run's results equal the trace's, exactly (integer set
        # semantics: no tolerance)
        bad = {name: check(tr, r) for name, r in zip(run_names, runs)}
        rec["results_exact"] = all(b is None for b in bad.values())
        rec["failed_inserts"] = {k: (0 if b is None else b.get("insert", {}).get("wrong", 0)) for k, b in bad.items()}
        if not rec["results_exact"]:
            rec["mismatches"] = {k: b for k, b in bad.items() if b is not None}
        rec["throughput_speedup"] = round(rec["sequential_trace_rate"]["span_ms"] /
                                          rec["server_trace_rate"]["span_ms"], 3)
        out["mix_%d_%d_%d" % mix] = rec
    table.close()
    del kt, vt, st
    torch.cuda.empty_cache()
    return out


TXN_BINS, TXN_B, TXN_WORKERS, TXN_OPS, TXN_TRIALS = 1 << 14, 8, 15, 100, 100
TXN_DENSITIES = (0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 0.95)
TXN_MIXES = (("delete_light", (1, 0, 1, 1)), ("delete_heavy", (2, 1, 2, 2)))


def txn_form(torch, stream):
    """The transactional layer (Sec. 8) on the paper's experiment: tables
    of 2^14 bins x 8 slots, 15 workers each running 100-operation
    transactions (insert:delete:overwrite:read 1:0:1:1 and 2:1:2:2; targets
    drawn among the worker's own earlier inserts, deleted ones included)
    until the table holds 95% of its slots; 100 trials (independent tables,
    salted hash seeds) side by side in one launch per implementation.  For
    each of the six implementations: the mean number of aborts over a
    table's lifetime up to each density (the figures' curves), the share of
    attempts that aborted, abort causes, and the committed transactions per
    second of the whole launch."""
    import numpy as np
    from paper_1605_05236_gb300 import inputs, txn
    cap = TXN_BINS * TXN_B
    fill_to = int(0.95 * cap)
    res = {"table": "2^14 x 8 slots per trial", "workers": TXN_WORKERS, "ops_per_txn": TXN_OPS,
           "trials": TXN_TRIALS, "densities": list(TXN_DENSITIES)}
    for mix_name, mix in TXN_MIXES:
        t_max = 4 * fill_to * sum(mix) // (TXN_WORKERS * TXN_OPS * max(1, mix[0] - mix[1])) + 10
        work = inputs.txn_workload(TXN_WORKERS, t_max, TXN_OPS, mix, seed=13, fill_to=fill_to)
        T = work["txns_per_worker"]
        n = len(work["op"])
        op = torch.from_numpy(work["op"]).cuda()
        key = torch.from_numpy(work["key"].view(np.int32)).cuda()
        val = torch.from_numpy(work["val"].view(np.int32)).cuda()
        section = {"mix": ":".join(map(str, mix)), "txns_per_worker": T, "ops": n}
        for name, flags in txn.VARIANTS:
            tab = txn.TxnTable(TXN_BINS, TXN_B, TXN_TRIALS, seed=21)
            start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            start.record(stream)
            out = tab.run(op, key, val, TXN_WORKERS, T, TXN_OPS, flags, want_values=False, stream=stream)
            end.record(stream)
            end.synchronize()
            ms = start.elapsed_time(end)
            s = tab.stats()
            st = out["status"].cpu().numpy().reshape(TXN_TRIALS, n)
            att = out["attempts"].cpu().numpy().reshape(TXN_TRIALS, -1)
            order = out["order"].cpu().numpy().reshape(TXN_TRIALS, -1)
            ab = np.zeros((TXN_TRIALS, len(TXN_DENSITIES)), dtype=np.float64)
            at = np.zeros_like(ab)
            for r in range(TXN_TRIALS):
                a, t_ = txn.aborts_by_density(st[r], work["op"], att[r], order[r], TXN_OPS, cap, TXN_DENSITIES)
                ab[r], at[r] = a, t_
            reached = (ab >= 0).all(0)
            section[name] = {
                "mean_aborts_by_density": [round(float(ab[:, j].mean()), 2) if reached[j] else None
                                           for j in range(len(TXN_DENSITIES))],
                "abort_pct_by_density": [round(100.0 * float(ab[:, j].sum() / at[:, j].sum()), 4) if reached[j]
                                         else None for j in range(len(TXN_DENSITIES))],
                "abort_pct": round(100.0 * (s["attempts"] - s["commits"]) / max(1, s["attempts"]), 4),
                "statuses_same_in_every_trial": bool((st == st[0]).all()),
                "causes": {k: s[k] for k in ("abort_claimed", "abort_lock", "abort_ws", "abort_rs", "abort_chain",
                                             "abort_overflow")},
                "failed": s["failed"], "local_retries": s["local_retries"], "mini_txns": s["mini_txns"],
                "kicks_per_insert": round(s["kicks"] / max(1, int((work["op"] == txn.TX_INSERT).sum()) * TXN_TRIALS), 4),
                "ms": round(ms, 2),
                "k_txns_per_s": round(s["commits"] / ms, 1),
            }
            tab.close()
        naive, best = section["naive"]["mean_aborts_by_density"], section["claim_system"]["mean_aborts_by_density"]
        section["naive_over_claim_system"] = [round(a / b, 1) if a is not None and b else None
                                              for a, b in zip(naive, best)]
        res[mix_name] = section
        del op, key, val
    return res


def host_info():
    """Core count and CPU model of this host."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "CPU part") and v.strip():
                    model = (k.strip() + " " + v.strip()) if k.strip() == "CPU part" else v.strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "cpu": model}


def cpu_baseline():
    """The oracle, as it stands, on the host cores: a bounded sample of the
    workload (a 2^22-bin x 4-slot table filled to 0.95 with queue-kicking,
    then 2^22 lookups at 50% hits and 2^20 deletes of present keys).  The
    fill is serial (the policies are defined one insertion at a time), so it
    runs on one core; the lookups and deletes run on one core and again on
    all cores (the batch split into one range per core, on a second copy of
    the filled table)."""
    import oracle
    from paper_1605_05236_gb300 import inputs
    bins = 1 << 22
    n = inputs.load_target(bins * B, LOAD)
    keys, nxt = inputs.distinct_keys(n, 1)
    vals = inputs.values_for(keys)
    lk, _ = inputs.lookup_keys(keys, 1 << 22, 1, 0.5, next_start=nxt)
    dk = inputs.delete_keys(keys, 1 << 20, 1)
    t = oracle.OracleTable(bins, B, 2, oracle.QUEUE, rng_seed=1, cap=500)
    t0 = time.perf_counter()
    t.insert(keys, vals)
    dt = time.perf_counter() - t0
    s = t.stats()
    t0 = time.perf_counter()
    t.lookup(lk)
    dl = time.perf_counter() - t0
    t0 = time.perf_counter()
    t.delete(dk)
    dd = time.perf_counter() - t0
    # all cores: a second table filled the same way (the serial fill is
    # deterministic), its lookups and deletes split over every core
    cores = os.cpu_count() or 1
    t2 = oracle.OracleTable(bins, B, 2, oracle.QUEUE, rng_seed=1, cap=500)
    t2.insert(keys, vals)
    t0 = time.perf_counter()
    _, _, used_l = t2.lookup_threads(lk, cores)
    dl_all = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, used_d = t2.delete_threads(dk, cores)
    dd_all = time.perf_counter() - t0
    return {"value": round(n / dt / 1e6, 3), "unit": "M inserts/s", "cores": 1, "kind": "oracle",
            "sample": "serial C oracle, queue-kicking fill of a 2^22-bin x 4-slot table from empty to 0.95 "
                      "(%d keys, %.1f s, 1 core); bins viewed/insert %.4f; then %d lookups (50%% hits) and %d "
                      "deletes of present keys on the filled table, on 1 core and on all %d cores"
                      % (n, dt, s["bins_viewed"] / n, len(lk), len(dk), cores),
            "m_lookups_per_s": round(len(lk) / dl / 1e6, 3), "m_deletes_per_s": round(len(dk) / dd / 1e6, 3),
            "all_cores": {"cores": min(used_l, used_d), "m_lookups_per_s": round(len(lk) / dl_all / 1e6, 3),
                          "m_deletes_per_s": round(len(dk) / dd_all / 1e6, 3)},
            "host": host_info()}


def rank_seed(rank: int) -> int:
    """Key seed of a rank: each rank fills its own table with its own keys
    (independent shards, weak scaling)."""
    return 1 + 1000 * rank


def max_over_ranks(torch, values, world, device):
    """Element-wise maximum of per-rank timings (the slowest rank sets the
    job's time); no-op on one rank."""
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_rate(units_per_rank, steps, ms, world):
    """Whole-job throughput in M units/s: every rank processed
    units_per_rank per step, and the job took `ms` (max over ranks)."""
    return world * units_per_rank * steps / (ms * 1e-3) / 1e6


# A collective that waits longer than this for a rank that is gone fails
# with an error on the ranks still running, instead of holding their GPUs.
PG_TIMEOUT_S = 300


def init_ranks(backend, device=None, timeout_s=PG_TIMEOUT_S):
    """The process group of a multi-rank run (rank and world from the
    environment), with a bounded collective timeout."""
    import datetime
    import torch.distributed as dist
    kw = {"timeout": datetime.timedelta(seconds=timeout_s)}
    if device is not None:
        kw["device_id"] = device
    dist.init_process_group(backend, **kw)


def run_gpu(args, rank, world, local):
    import torch
    from paper_1605_05236_gb300 import ck

    torch.cuda.set_device(local)
    if world > 1:
        init_ranks("nccl", torch.device("cuda", local))
    ck.load()
    stream = torch.cuda.current_stream()
    seed = rank_seed(rank)
    keys, vals, lk, expect, dk = workload(seed)
    n = len(keys)
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)
    lkt, dkt = ck.as_u32_tensor(lk), ck.as_u32_tensor(dk)
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    lv = torch.empty(N_LOOKUP, dtype=torch.int32, device="cuda")
    lf = torch.empty(N_LOOKUP, dtype=torch.uint8, device="cuda")
    df = torch.empty(N_DELETE, dtype=torch.uint8, device="cuda")
    table = ck.CuckooTable(BINS, B, 2, ck.QUEUE, seed=seed)
    n_batches = (n + BATCH - 1) // BATCH
    launches_per_step = n_batches + 2  # inserts, lookup, delete (the clear is a memset)

    def step(rec):
        # no events between the insert launches: consecutive launches overlap
        table.clear(stream)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ins = []
        e[0].record(stream)
        for lo in range(0, n, BATCH):
            hi = min(n, lo + BATCH)
            table.insert_batch(kt[lo:hi], vt[lo:hi], st[lo:hi], stream)
        e[1].record(stream)
        table.lookup(lkt, lv, lf, stream)
        e[2].record(stream)
        table.delete(dkt, df, stream)
        e[3].record(stream)
        return e, ins

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_begin.record(stream)
    recs = [step(True) for _ in range(args.steps)]
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = t_begin.elapsed_time(t_end)
    fill_ms = sum(e[0].elapsed_time(e[1]) for e, _ in recs)
    look_ms = sum(e[1].elapsed_time(e[2]) for e, _ in recs)
    del_ms = sum(e[2].elapsed_time(e[3]) for e, _ in recs)
    s = table.stats()  # counters of the last step (ck_clear zeroes them)

    # correctness of the last step (outside the timed region)
    ok = bool((st == 0).all().item())
    lookups_exact = bool(torch.equal(lf.cpu(), torch.from_numpy(expect)))
    present = torch.from_numpy(expect.astype(bool))
    want = torch.from_numpy(inputs_values(lk).view(np.int32))
    vals_exact = bool(torch.equal(lv.cpu()[present], want[present]))
    deletes_exact = bool((df == 1).all().item())

    total_ms, fill_ms, look_ms, del_ms = max_over_ranks(torch, [total_ms, fill_ms, look_ms, del_ms], world, "cuda")
    K = args.steps
    value = job_rate(n, K, fill_ms, world)
    lookups_mops = job_rate(N_LOOKUP, K, look_ms, world)
    deletes_mops = job_rate(N_DELETE, K, del_ms, world)

    # roofline of the dominant kernel (the insert kernel: it takes most of the step)
    hbm, peak_kind = measured_peaks()
    viewed, kicks, ins_ok = s["bins_viewed"], s["kicks"], s["inserts_ok"]
    # per insertion: each bin viewed = one 32-B slot sector + one 32-B metadata
    # sector; each written slot (kicks + 1) = one slot sector write + one
    # metadata sector atomic; 8 B of key/value in and 1 B of status out
    ins_bytes = viewed * 64 + (kicks + ins_ok) * 64 + n * 9
    bytes_per_launch = ins_bytes / n_batches
    avg_launch_ms = fill_ms / K / n_batches  # launches overlap: fill time per launch
    achieved = bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9
    look_bytes = N_LOOKUP * (2 * 32 + 4 + 4 + 1)
    look_gbs = look_bytes / (look_ms / K * 1e-3) / 1e9  # per GPU, per lookup launch
    # random 32-B reads over a buffer the size of the slots, best launch shape
    g32, g32_shape, g32_sweep = gather_roofline(torch, ck, BINS * B * 8, 32, 1 << 26, stream)
    profile = batch_profile(torch, ck, table, kt, vt, st, stream)
    roofline = {"kernel": "k_insert<4,QUEUE> (one launch per 2^20-key batch)", "bound": "hbm",
                "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": INSERT_TRAFFIC_PER_LAUNCH,
                "traffic_unit": "bytes per launch: mean DRAM read + write over the 61 launches of a half-size fill (2^23 x 4, the same load trajectory, 2^19 keys a launch), times 2 (ncu)",
                "bytes_per_launch": int(bytes_per_launch), "avg_launch_ms": round(avg_launch_ms, 4),
                "vs_random_gather_32B": {"gbs": round(g32, 1), "frac": round(achieved / g32, 4)}}
    gather_section = {"buffer": "512 MiB (the slot array's size)", "width_bytes": 32, "reads": 1 << 26,
                      "best_gbs": round(g32, 1), "best_shape": g32_shape, "sweep": g32_sweep}
    # the random-operation model of a low-load launch: a key reads its two
    # bins' 32-B slot sectors, writes one slot by a 64-bit compare-and-swap
    # and updates its bin's metadata word by a 32-bit add, each class at its
    # measured rate over an array of the table's size
    red = atomic_rate(torch, ck, BINS * 4, 0, 1 << 26, stream)   # metadata words
    cas = atomic_rate(torch, ck, BINS * B * 8, 2, 1 << 26, stream)  # slots
    model_ms = BATCH * (2 * 32 / (g32 * 1e9) + 1 / (cas * 1e9) + 1 / (red * 1e9)) * 1e3
    first_ms = profile["launch_ms_at_load"]["0.000"]
    roofline["random_ops_model"] = {
        "gather32_g_per_s": round(g32 / 32, 2), "cas64_g_per_s": round(cas, 2), "red32_g_per_s": round(red, 2),
        "first_launch_ms": first_ms, "model_ms": round(model_ms, 4), "frac": round(model_ms / first_ms, 4),
        "note": "first 2^20-key launch (load 0 to 0.016, serialised) against 2 random 32-B reads + 1 random "
                "64-bit CAS + 1 random 32-bit add per key at the probes' measured rates"}
    # against the random-gather roofline only the gathered bytes count: two
    # random 32-B sectors per lookup (the key in and the result out stream)
    look_random_gbs = N_LOOKUP * 2 * 32 / (look_ms / K * 1e-3) / 1e9
    roof_lookup = {"kernel": "k_lookup2<4>", "bound": "hbm", "achieved": round(look_gbs, 1), "peak": hbm,
                   "unit": "GB/s", "frac": round(look_gbs / hbm, 4),
                   "bytes_per_lookup": 73, "vs_random_gather_32B": {"gbs": round(g32, 1),
                                                                     "random_bytes_gbs": round(look_random_gbs, 1),
                                                                     "frac": round(look_random_gbs / g32, 4)}}

    # end to end through host buffers (pinned), copies inside the timed region
    e2e = end_to_end(torch, ck, table, keys, vals, lk, dk, stream, K)

    out = {"metric": METRIC, "value": round(value, 2), "unit": "M inserts/s", "n_gpus": world, "steps": K,
           "warmup": args.warmup, "ms_per_step": round(total_ms / K, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u32 keys/values in u64 slots (integer)",
           "data": "synthetic (seeded SplitMix64 uniform distinct uint32 keys)",
           "config": {"workload": WORKLOAD, "l2": "no flush: table (512 MiB) and key arrays exceed the 129 MB L2",
                      "parallelism": "dp%d (independent table per GPU)" % world},
           "bins_viewed_per_insert": round(s["bins_viewed_per_insert"], 4),
           "kicks_per_insert": round(kicks / max(1, ins_ok), 4),
           "claim_aborts_per_insert": round(s["aborts_per_insert"], 6),
           "m_lookups_per_s": round(lookups_mops, 1), "m_deletes_per_s": round(deletes_mops, 1),
           "ms": {"fill": round(fill_ms / K, 3), "lookup": round(look_ms / K, 3), "delete": round(del_ms / K, 3)},
           "exact": {"all_inserted": ok, "lookups": lookups_exact, "lookup_values": vals_exact,
                     "deletes": deletes_exact},
           "roofline": roofline, "roofline_lookup": roof_lookup,
           "e2e": e2e, "gpu_launches": launches_per_step * K, "clocks": clk}
    sections = {"insert_batches": profile, "roofline_detail": {"insert": roofline, "lookup": roof_lookup},
                "e2e_detail": e2e, "random_gather_sweep": gather_section}
    del kt, vt, lkt, dkt, st, lv, lf, df
    table.close()
    torch.cuda.empty_cache()
    summary = {}
    if rank == 0 and world == 1 and not args.no_policies:
        pol = policy_fills(torch, ck, stream, (keys, vals))
        sections["policies"] = pol
        summary["policies"] = {
            # bins viewed by the insertions made at density 0.945-0.95 (the
            # paper's curves), queue-kicking against random kicking
            "queue_vs_random_viewed_at_0.95": [pol["queue"]["viewed_by_load"].get("0.95"),
                                               pol["random"]["viewed_by_load"].get("0.95")],
            "failed_total": sum(int(p.get("failed", 0)) for p in pol.values()),
            # rows whose GPU fill failed keys the serial oracle does not fail
            # at the same cap (none expected)
            "failed_beyond_oracle": sorted(k for k, p in pol.items()
                                           if p.get("failed", 0) > p.get("oracle_failed_same_cap", 0)),
            "contents_exact": all(p.get("contents_exact", True) for p in pol.values()),
            # lookups of the 8-slot and single-slot tables against the random
            # gather of their own width (64 B, 8 B)
            "lookup_vs_gather": {k: pol[r]["roofline_lookup"]["vs_random_gather"]["frac"]
                                 for k, r in (("b8", "queue_b8_0.99"), ("d3", "random_d3_0.90"),
                                              ("d4", "random_d4_0.96")) if "roofline_lookup" in pol.get(r, {})}}
    if rank == 0 and world == 1 and not args.no_small:
        sm = small_table(torch, ck, stream)
        sections["small_table"] = sm
        summary["small_table"] = {"m_inserts_per_s": sm["m_inserts_per_s"], "exact": sm["exact"],
                                  "l2_insert_frac": sm["roofline"]["insert_frac"],
                                  "l2_lookup_frac": sm["roofline"]["lookup_frac"]}
    if rank == 0 and world == 1 and not args.no_multi:
        mf = multi_form(torch, ck, stream)
        sections["batched_form"] = mf
        summary["batched_form"] = {"speedup_vs_per_table": mf["speedup"],
                                   "m_inserts_per_s": mf["batched"]["m_inserts_per_s"],
                                   "all_inserted": mf["batched"]["all_inserted"] and mf["per_table"]["all_inserted"]}
    if rank == 0 and world == 1 and not args.no_serve:
        sf = serve_form(torch, ck, stream)
        sections["serving_form"] = sf
        summary["serving_form"] = {k: {"results_exact": v["results_exact"], "speedup": v["throughput_speedup"]}
                                   for k, v in sf.items() if k.startswith("mix_")}
    if rank == 0 and world == 1 and not args.no_txn:
        sections["transactional"] = txn_form(torch, stream)
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline()
    out["sections"] = sections
    out["section_summary"] = summary
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def end_to_end(torch, ck, table, keys, vals, lk, dk, stream, K):
    """The same metric through the public API from pinned host buffers.

    `value`: the fill alone, as `value` of the bench line counts it, with
    its copies inside the timed region: keys and values come in on a second
    stream in chunks of 1, 2, 4, ... batches while the chunk before is
    inserted, and each chunk's statuses go out once it is inserted.  `whole_step`: the whole step (fill,
    lookups, deletes) the same way, with the lookup and delete keys copied
    in during the fill and every result copied out -- inserts per second of
    the whole step, the same unit over more work.  Both are how a caller of
    the C ABI overlaps transfers with the launches."""
    n = len(keys)
    hk = torch.from_numpy(keys.view(np.int32)).pin_memory()
    hv = torch.from_numpy(vals.view(np.int32)).pin_memory()
    hl = torch.from_numpy(lk.view(np.int32)).pin_memory()
    hd = torch.from_numpy(dk.view(np.int32)).pin_memory()
    hst = torch.empty(n, dtype=torch.uint8).pin_memory()
    hlv = torch.empty(len(lk), dtype=torch.int32).pin_memory()
    hlf = torch.empty(len(lk), dtype=torch.uint8).pin_memory()
    hdf = torch.empty(len(dk), dtype=torch.uint8).pin_memory()
    dkey = torch.empty(n, dtype=torch.int32, device="cuda")
    dval = torch.empty(n, dtype=torch.int32, device="cuda")
    dst = torch.empty(n, dtype=torch.uint8, device="cuda")
    dl = torch.empty(len(lk), dtype=torch.int32, device="cuda")
    dlv = torch.empty(len(lk), dtype=torch.int32, device="cuda")
    dlf = torch.empty(len(lk), dtype=torch.uint8, device="cuda")
    ddk = torch.empty(len(dk), dtype=torch.int32, device="cuda")
    ddf = torch.empty(len(dk), dtype=torch.uint8, device="cuda")
    cs = torch.cuda.Stream()  # copies
    bounds = [(lo, min(n, lo + BATCH)) for lo in range(0, n, BATCH)]
    # batches grouped into chunks of 1, 2, 4, ... batches: the insert stream
    # waits for a chunk's copy once, so consecutive insert launches inside a
    # chunk still overlap, while the first launch waits for one batch only
    chunks, i, size = [], 0, 1
    while i < len(bounds):
        chunks.append(bounds[i:i + size])
        i += size
        size *= 2

    def step(whole):
        cs.wait_stream(stream)
        table.clear(stream)
        copied = []
        with torch.cuda.stream(cs):
            for ch in chunks:  # every chunk in order, each with its own event
                lo, hi = ch[0][0], ch[-1][1]
                dkey[lo:hi].copy_(hk[lo:hi], non_blocking=True)
                dval[lo:hi].copy_(hv[lo:hi], non_blocking=True)
                e = torch.cuda.Event()
                e.record(cs)
                copied.append(e)
            if whole:
                dl.copy_(hl, non_blocking=True)
                ddk.copy_(hd, non_blocking=True)
                keys_in = torch.cuda.Event()
                keys_in.record(cs)
        done = []
        for ch, e in zip(chunks, copied):
            stream.wait_event(e)
            for lo, hi in ch:
                table.insert_batch(dkey[lo:hi], dval[lo:hi], dst[lo:hi], stream)
            d = torch.cuda.Event()
            d.record(stream)
            done.append(d)
        with torch.cuda.stream(cs):  # each chunk's statuses go out once it is inserted
            for ch, d in zip(chunks[:-1], done[:-1]):
                cs.wait_event(d)
                hst[ch[0][0]:ch[-1][1]].copy_(dst[ch[0][0]:ch[-1][1]], non_blocking=True)
        ins_done = done[-1]
        if whole:
            stream.wait_event(keys_in)
            # lookups in 8 chunks: each chunk's results go out while the
            # next chunk (and the deletes) run
            lk_done = []
            for c in range(LOOKUP_CHUNKS):
                lo, hi = c * len(dl) // LOOKUP_CHUNKS, (c + 1) * len(dl) // LOOKUP_CHUNKS
                table.lookup(dl[lo:hi], dlv[lo:hi], dlf[lo:hi], stream)
                e = torch.cuda.Event()
                e.record(stream)
                lk_done.append((lo, hi, e))
            table.delete(ddk, ddf, stream)
            del_done = torch.cuda.Event()
            del_done.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ins_done)
            last = chunks[-1]
            hst[last[0][0]:last[-1][1]].copy_(dst[last[0][0]:last[-1][1]], non_blocking=True)
            if whole:
                for lo, hi, e in lk_done:
                    cs.wait_event(e)
                    hlv[lo:hi].copy_(dlv[lo:hi], non_blocking=True)
                    hlf[lo:hi].copy_(dlf[lo:hi], non_blocking=True)
                cs.wait_event(del_done)
                hdf.copy_(ddf, non_blocking=True)
        stream.wait_stream(cs)

    def timed(whole):
        for _ in range(2):  # warm-up: the first steps from freshly pinned buffers run slow
            step(whole)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            step(whole)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / K

    ms_fill = timed(False)
    fill_ok = bool((hst == 0).all().item())
    ms_whole = timed(True)
    ok = bool((hst == 0).all().item()) and bool((hdf == 1).all().item())
    return {"value": round(n / (ms_fill * 1e-3) / 1e6, 2), "unit": "M inserts/s (fill incl. copies)",
            "ms_per_step": round(ms_fill, 3), "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n,
            "copies": "on a second stream, overlapped with the launches", "results_exact": fill_ok,
            "whole_step": {"value": round(n / (ms_whole * 1e-3) / 1e6, 2),
                           "unit": "M inserts/s (fill + lookups + deletes incl. copies)",
                           "ms_per_step": round(ms_whole, 3),
                           "h2d_bytes_per_step": n * 8 + len(lk) * 4 + len(dk) * 4,
                           "d2h_bytes_per_step": n * 1 + len(lk) * 5 + len(dk) * 1, "results_exact": ok}}


# ---------------------------------------------------------------------------
# reference arm: the oracle, as it stands, on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    from paper_1605_05236_gb300 import inputs
    bins = 1 << 20  # bounded sample: a 2^20-bin x 4-slot table, same load trajectory
    n = inputs.load_target(bins * B, LOAD)
    keys, nxt = inputs.distinct_keys(n, 1)
    vals = inputs.values_for(keys)
    lk, _ = inputs.lookup_keys(keys, 1 << 22, 1, 0.5, next_start=nxt)
    dk = inputs.delete_keys(keys, 1 << 18, 1)

    def step():
        t = oracle.OracleTable(bins, B, 2, oracle.QUEUE, rng_seed=1, cap=500)
        t0 = time.perf_counter()
        t.insert(keys, vals)
        t1 = time.perf_counter()
        t.lookup(lk)
        t.delete(dk)
        t2 = time.perf_counter()
        return t1 - t0, t2 - t0

    for _ in range(args.warmup):
        step()
    fills, totals = [], []
    for _ in range(args.steps):
        f, tot = step()
        fills.append(f)
        totals.append(tot)
    value = n * len(fills) / sum(fills) / 1e6
    sample = ("serial C oracle: queue-kicking fill of a 2^20-bin x 4-slot table to 0.95 (%d keys), "
              "then 2^22 lookups and 2^18 deletes, per step" % n)
    return {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "M inserts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(totals) / len(totals), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32 keys/values in u64 slots (integer)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": round(value, 3), "unit": "M inserts/s", "cores": 1, "kind": "oracle",
                             "sample": sample, "host": host_info()},
            "e2e": {"value": round(value, 3), "unit": "M inserts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def fill_section(bins_log2):
    """One warm-up fill and one timed fill of a 2^bins_log2 x 4 queue-kicking
    table to 0.95 in 61 launches (the step's trajectory at that size)."""
    import torch
    from paper_1605_05236_gb300 import ck, inputs
    ck.load()
    stream = torch.cuda.current_stream()
    bins = 1 << bins_log2
    n = inputs.load_target(bins * B, LOAD)
    keys, _ = inputs.distinct_keys(n, rank_seed(0))
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(inputs.values_for(keys))
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    batch = max(1, (BATCH * bins) // BINS)
    t = ck.CuckooTable(bins, B, 2, ck.QUEUE, seed=rank_seed(0))
    fill_once(torch, ck, t, kt, vt, st, stream, batch)
    ms, _ = fill_once(torch, ck, t, kt, vt, st, stream, batch)
    s = t.stats()
    return {"fill": {"bins": bins, "keys": n, "batch": batch, "launches": (n + batch - 1) // batch, "ms": round(ms, 3),
                     "all_inserted": bool((st == 0).all().item()),
                     "bins_viewed": s["bins_viewed"], "kicks": s["kicks"], "inserts_ok": s["inserts_ok"]}}


def run_section(name, policies=None, fill_bins_log2=24):
    import torch
    from paper_1605_05236_gb300 import ck
    ck.load()
    stream = torch.cuda.current_stream()
    if name == "serve":
        return {"serving_form": serve_form(torch, ck, stream)}
    if name == "multi":
        return {"batched_form": multi_form(torch, ck, stream)}
    if name == "txn":
        return {"transactional": txn_form(torch, stream)}
    if name == "fill":
        return fill_section(fill_bins_log2)
    keys, vals, _, _, _ = workload(rank_seed(0))
    return {"policies": policy_fills(torch, ck, stream, (keys, vals), only=policies)}


def headline(out):
    """The bench line proper: the contract's keys and the headline figures,
    compact (well under 4 KB) so it can be read alone as the last line of
    the output.  The side sections go out on earlier lines."""
    keep = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "bins_viewed_per_insert", "kicks_per_insert",
            "claim_aborts_per_insert", "m_lookups_per_s", "m_deletes_per_s", "ms", "exact", "gpu_launches",
            "clocks")
    h = {k: out[k] for k in keep if k in out}
    r = out.get("roofline")
    if r:
        h["roofline"] = {k: r[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "traffic",
                                           "bytes_per_launch", "avg_launch_ms") if k in r}
        h["roofline"]["peak_kind"] = r.get("peak_kind", "").split(" ")[0]
        if "vs_random_gather_32B" in r:
            h["roofline"]["vs_random_gather_32B"] = r["vs_random_gather_32B"]
        if "random_ops_model" in r:
            h["roofline"]["random_ops_model_frac"] = r["random_ops_model"]["frac"]
    rl = out.get("roofline_lookup")
    if rl:
        h["roofline_lookup"] = {k: rl[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac",
                                                   "vs_random_gather_32B") if k in rl}
    e = out.get("e2e")
    if e:
        h["e2e"] = {k: e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step", "ms_per_step",
                                      "results_exact") if k in e}
        if "whole_step" in e:
            h["e2e"]["whole_step_value"] = e["whole_step"]["value"]
    cb = out.get("cpu_baseline")
    if cb:
        h["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "m_lookups_per_s",
                                                "m_deletes_per_s", "all_cores") if k in cb}
        host = cb.get("host") or {}
        h["cpu_baseline"]["host"] = {"nproc": host.get("nproc"), "machine": host.get("machine")}
    h["sections"] = out.get("section_summary", {})
    line = json.dumps(h)
    # the side summaries are the first thing to go should the line grow
    if len(line) > 3800:
        h["sections"] = {"note": "see the section lines above"}
        line = json.dumps(h)
    return line


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if rank == 0 and out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.only:
        out = run_section(args.only, args.policy, args.fill_bins_log2)
        if rank == 0 and out is not None:
            print(json.dumps(out), flush=True)
        return
    out = run_gpu(args, rank, world, local)
    if rank == 0 and out is not None:
        # side sections first, one line each; the bench line last
        for name, body in out.get("sections", {}).items():
            print(json.dumps({"section": name, **body}), flush=True)
        print(headline(out), flush=True)


if __name__ == "__main__":
    main()
