"""Benchmark of the GB300 stable mergesort: one JSON line on stdout (rank 0).

Default workload (one "step"): the plain GPU mergesort of 2^27 float64 keys with
a uint32 index payload, four patterns from one seed (permuted uniform, heavy
ties, ascending with 1% random transpositions, strictly descending), each at the
100% and at the 50% buffer tier -- eight sorts per step, inputs resident in HBM
(restored from pristine device copies, untimed, before each step; every sort's
working set is 1.5 GiB, larger than L2).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the paper's own algorithms: Knuthsort
for the 100% tier, Frogsort1 for the 50% tier) on a bounded sample of the same
workload.  Multi-GPU runs (torchrun) are replicas: every rank sorts its own
copy, no collective touches the data; value = all ranks' keys / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "stable sort Gkeys/s + HBM roofline fraction; learned/batched vs plain merge"
UNIT = "Gkeys/s"
N_FULL = 1 << 27
TIERS = (1.0, 0.5)
WORKLOAD = ("plain GPU mergesort, 2^27 float64 keys + uint32 index payload, "
            "patterns permut/ties/asc_noise/desc, each at 100% and 50% buffer")
BYTES_PER_ELEM_PASS = 24      # 8 B key + 4 B payload, read and written once per pass


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_FULL, help="keys per sort (default 2^27)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paper-patterns", action="store_true",
                    help="add the paper's pattern suite on both tiers (ratios in the form of its Squidsort table)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 2^31-key low-memory run of the default extras (about 60 GB on the device, 15 s)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the learned-vs-plain and batched-vs-plain comparisons")
    ap.add_argument("--only", default=None,
                    help="diagnostic run of one workload for profiling (no contract line): PATTERN@TIER "
                         "(e.g. permut@100, permut@50), 'segmented' (--nseg segments) or 'learned' "
                         "(the mixture at --n keys, full buffer)")
    ap.add_argument("--variant", default="frog", choices=["frog", "gecko", "squid"],
                    help="with --only PATTERN@TIER below 100: the symmetric variant (gns_sort_symmetric)")
    ap.add_argument("--nseg", type=int, default=4096, help="segments for --only segmented")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(files):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2402_01816_gb300", "csrc")
    for fn in files:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu record, if it was taken on
    the current sources of that kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash(e.get("files", [])):
        return None
    return e.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.lines = []
        self.dev = device_index

    def __enter__(self):
        try:
            import torch
            uuid = "GPU-" + str(torch.cuda.get_device_properties(self.dev).uuid)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", uuid], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "note": "nvidia-smi unavailable"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ reference arm
def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    from paper_2402_01816_gb300 import inputs
    sample = min(args.n, 1 << 20)
    data = {p: inputs.make_keys(p, sample, seed=0) for p in inputs.PATTERNS_C1}
    pay = inputs.index_payload(sample)

    def step():
        t = 0.0
        for p in inputs.PATTERNS_C1:
            for bf in TIERS:
                t0 = time.perf_counter()
                if bf >= 1.0:
                    oracle.knuthsort(data[p], pay)
                else:
                    oracle.frogsort(data[p], pay)
                t += time.perf_counter() - t0
        return t

    for _ in range(args.warmup):
        step()
    times = [step() for _ in range(args.steps)]
    t = statistics.mean(times)
    keys = sample * len(inputs.PATTERNS_C1) * len(TIERS)
    v = keys / t / 1e9
    desc = (f"CPU oracle (Knuthsort for the 100% tier, Frogsort1 for the 50% tier), single thread, "
            f"{sample} keys per pattern x 4 patterns x 2 tiers per step")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "n_per_sort": args.n, "sorts_per_step": 8,
                       "parallelism": "replicas1", "sample_n_per_sort": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ comparisons
def _time_ms(fn, restore, reps=3):
    import torch
    ts = []
    for _ in range(reps):
        restore()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def learned_vs_plain(dev, n=1 << 28):
    """gns_learned_sort against gns_sort (100% tier) on the three-part mixture."""
    import torch
    import paper_2402_01816_gb300 as g
    from paper_2402_01816_gb300 import inputs
    keys = torch.from_numpy(inputs.make_keys("mixture", n, seed=0)).to(dev)
    pay = torch.from_numpy(inputs.index_payload(n).view(np.int32)).to(dev)
    kt, pt = torch.empty_like(keys), torch.empty_like(pay)

    def restore():
        kt.copy_(keys)
        pt.copy_(pay)
    restore()
    rep = g.gns_learned_sort(kt, pt, report=True)          # warm-up + report
    restore()
    g.gns_sort(kt, pt)
    t_learned = _time_ms(lambda: g.gns_learned_sort(kt, pt), restore)
    t_first = _time_ms(lambda: g.gns_learned_sort(kt, pt, train_steps=0), restore)
    t_plain = _time_ms(lambda: g.gns_sort(kt, pt), restore)
    # the same at the 50% tier: the half-buffer learned form against Frogsort1
    restore()
    rep_half = g.gns_learned_sort(kt, pt, buffer_fraction=0.5, report=True)
    t_learned_half = _time_ms(lambda: g.gns_learned_sort(kt, pt, buffer_fraction=0.5), restore)
    t_plain_half = _time_ms(lambda: g.gns_sort(kt, pt, buffer_fraction=0.5), restore)
    ram_half = 1.0 + g.gns_workspace_bytes(n, 0.5, 1) / (12.0 * n)
    ram_plain_half = 1.0 + g.gns_workspace_bytes(n, 0.5, 0) / (12.0 * n)
    if g.gns_stream_status() != 0:
        raise RuntimeError("device status error in learned_vs_plain")
    del keys, pay, kt, pt
    torch.cuda.empty_cache()
    peak, peak_kind = load_peaks()
    part_b = 66 * n                                   # histogram 10, scatter A 28, scan 2, scatter B 26 per key
    mean_bucket = n / 4096.0
    # buckets sorted at global 8192-key tiles: a bucket of L keys touches about
    # L / 8192 + 1 tiles and takes ceil(log2(tiles)) merge levels
    bucket_passes = 1 + max(0, math.ceil(math.log2(mean_bucket / 8192 + 1)))
    bs_b = 24 * n * bucket_passes
    roof = {"bound": "hbm", "peak": peak, "unit": "GB/s", "peak_kind": peak_kind,
            "partition": {"algorithmic_bytes": part_b, "achieved": part_b / (rep["partition_ms"] / 1e3) / 1e9,
                          "frac": part_b / (rep["partition_ms"] / 1e3) / 1e9 / peak,
                          "bytes_model": "66 B per key: bucket pass 10, scatter A 28, digit scan 2, scatter B 26"},
            "bucket_sort": {"algorithmic_bytes": bs_b,
                            "achieved": bs_b / (rep["bucket_sort_ms"] / 1e3) / 1e9,
                            "frac": bs_b / (rep["bucket_sort_ms"] / 1e3) / 1e9 / peak,
                            "bytes_model": f"24 B per key per pass, {bucket_passes} passes of a mean-sized bucket "
                                           "(1 tile pass + ceil(log2(L/8192 + 1)) levels)"}}
    return {"workload": "learned-splitter sort: 2^28 float64 keys (40% log-normal sigma 2, 30% Zipf s=1.2 "
                        "over 2^16 integers, 30% mix of 8 Gaussians) + uint32 index payload, 4096 buckets",
            "roofline": roof,
            "learned_ms": t_learned, "plain_ms": t_plain, "first_stage_only_ms": t_first,
            "learned_gkeys_s": n / t_learned / 1e6, "plain_gkeys_s": n / t_plain / 1e6,
            "speedup_vs_plain": t_plain / t_learned, "speedup_vs_first_stage_only": t_first / t_learned,
            "report": rep,
            "at_50pct": {"learned_ms": t_learned_half, "plain_ms": t_plain_half,
                         "speedup_vs_plain": t_plain_half / t_learned_half,
                         "pct_ram_learned": ram_half, "pct_ram_plain": ram_plain_half,
                         "t_footprint_learned_ms": ram_half * t_learned_half,
                         "t_footprint_plain_ms": ram_plain_half * t_plain_half,
                         "report": rep_half}}


def network_gain(dev, n=1 << 22):
    """What the trained network changes against the first stage alone, on
    log-normal keys (the density changes inside every first-stage interval):
    largest bucket, overfull buckets, fit time and the whole call."""
    import torch
    import paper_2402_01816_gb300 as g
    rng = np.random.default_rng(100)
    keys = torch.from_numpy(np.exp(rng.normal(0.0, 2.0, n))).to(dev)
    pay = torch.arange(n, dtype=torch.int64, device=dev).to(torch.int32)
    kt, pt = torch.empty_like(keys), torch.empty_like(pay)

    def restore():
        kt.copy_(keys)
        pt.copy_(pay)
    out = {"workload": f"{n} log-normal float64 keys (mu 0, sigma 2) + uint32 payload, 4096 buckets"}
    for steps in (0, 32, 256):
        restore()
        rep = g.gns_learned_sort(kt, pt, train_steps=steps, report=True)
        t = _time_ms(lambda: g.gns_learned_sort(kt, pt, train_steps=steps), restore)
        out[f"steps_{steps}"] = {"ms": t, "max_bucket": rep["max_bucket"], "overfull_buckets": rep["overfull_buckets"],
                                 "fit_ms": rep["fit_ms"], "bucket_sort_ms": rep["bucket_sort_ms"],
                                 "final_loss": rep["final_loss"]}
    out["max_bucket_ratio_256_vs_first_stage"] = out["steps_256"]["max_bucket"] / out["steps_0"]["max_bucket"]
    if g.gns_stream_status() != 0:
        raise RuntimeError("device status error in network_gain")
    return out


def batched_vs_plain(dev, nseg=65536, per_segment_sample=2048):
    """gns_segmented_sort (one graph launch) against one gns_sort call per segment
    (timed on the first `per_segment_sample` segments and scaled by key count)
    and against one gns_sort of the whole array (same volume, not segmented)."""
    import torch
    import paper_2402_01816_gb300 as g
    from paper_2402_01816_gb300 import inputs
    keys_h, pay_h, off_h = inputs.segments(nseg, seed=0)
    n = keys_h.size
    keys = torch.from_numpy(keys_h).to(dev)
    pay = torch.from_numpy(pay_h.view(np.int32)).to(dev)
    off = torch.from_numpy(off_h).to(dev)
    kt, pt = torch.empty_like(keys), torch.empty_like(pay)

    def restore():
        kt.copy_(keys)
        pt.copy_(pay)
    restore()
    g.gns_segmented_sort(kt, pt, off)                       # tunes + captures the graph
    launches0 = g.gns_launch_count()
    t_seg = _time_ms(lambda: g.gns_segmented_sort(kt, pt, off), restore)
    kernels_per_call = (g.gns_launch_count() - launches0) // 3
    sched = g.gns_segmented_schedule(n, off)
    t_whole = _time_ms(lambda: g.gns_sort(kt, pt), restore)
    m = min(per_segment_sample, nseg)
    sub_n = int(off_h[m])

    def per_segment():
        for s_ in range(m):
            a, b = int(off_h[s_]), int(off_h[s_ + 1])
            g.gns_sort(kt[a:b], pt[a:b])
    t_sub = _time_ms(per_segment, restore, reps=2)
    t_per_seg = t_sub * nseg / m
    if g.gns_stream_status() != 0:
        raise RuntimeError("device status error in batched_vs_plain")
    del keys, pay, off, kt, pt
    torch.cuda.empty_cache()
    peak, peak_kind = load_peaks()
    alg = segmented_bytes(off_h)
    return {"workload": f"batched segmented sort: {nseg} segments, log-normal lengths (median 2^10, "
                        f"clipped 16..2^20), {n} int64 keys uniform over the full range + uint32 payload",
            "segmented_ms": t_seg, "segmented_gkeys_s": n / t_seg / 1e6, "schedule": sched,
            "roofline": {"bound": "hbm", "algorithmic_bytes": alg, "achieved": alg / (t_seg / 1e3) / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": alg / (t_seg / 1e3) / 1e9 / peak,
                         "bytes_model": "24 B per key per executed pass: 1 tile pass + ceil(log2(L/4096)) "
                                        "merge levels per segment of L keys", "peak_kind": peak_kind},
            "kernels_in_graph": kernels_per_call,
            "per_segment_gns_sort_ms_est": t_per_seg,
            "per_segment_estimate": f"{m} segments timed ({sub_n} keys), scaled by segment count",
            "plain_whole_array_ms": t_whole,
            "speedup_vs_per_segment": t_per_seg / t_seg, "speedup_vs_plain_whole_array": t_whole / t_seg}


# ------------------------------------------------------------------ our arm
def large_low_memory(dev, n=1 << 31):
    """2^31 float64 keys + uint32 index payload at the 50% tier (and the 100%
    tier beside it), plain and learned-splitter: time, %RAM and tFootprint per
    pattern."""
    import torch
    import paper_2402_01816_gb300 as g
    from paper_2402_01816_gb300 import inputs
    out = {"workload": "large low-memory run: 2^31 float64 keys + uint32 index payload (24 GiB), "
                       "patterns permut and presorted_runs (blocks of 2^16, every 10th sorted)"}
    pay = torch.arange(n, dtype=torch.int64, device=dev).to(torch.int32)
    for pattern in ("permut", "presorted_runs"):
        keys = inputs.make_keys_device(pattern, n, seed=0, device=dev)
        kt, pt = torch.empty_like(keys), torch.empty_like(pay)

        def restore():
            kt.copy_(keys)
            pt.copy_(pay)
        for bf in (0.5, 1.0):
            restore()
            g.gns_sort(kt, pt, buffer_fraction=bf)            # warm-up (workspace pool)
            t = _time_ms(lambda: g.gns_sort(kt, pt, buffer_fraction=bf), restore, reps=2)
            ram = 1.0 + g.gns_workspace_bytes(n, bf) / (12.0 * n)
            out[f"{pattern}@{int(bf * 100)}%"] = {"ms": t, "gkeys_s": n / t / 1e6, "pct_ram": ram,
                                                 "t_footprint_ms": ram * t}
        restore()
        rep = g.gns_learned_sort(kt, pt, buffer_fraction=0.5, report=True)
        t = _time_ms(lambda: g.gns_learned_sort(kt, pt, buffer_fraction=0.5), restore, reps=2)
        ram = 1.0 + g.gns_workspace_bytes(n, 0.5, 1) / (12.0 * n)
        out[f"{pattern}@50%-learned"] = {"ms": t, "gkeys_s": n / t / 1e6, "pct_ram": ram,
                                         "t_footprint_ms": ram * t, "fallback": rep["fallback"],
                                         "max_bucket": rep["max_bucket"]}
        if g.gns_stream_status() != 0:
            raise RuntimeError("device status error in large_low_memory")
        del keys, kt, pt
        torch.cuda.empty_cache()
        g.gns_release_workspace_cache()
    return out


def paper_patterns(dev, n=1 << 27):
    """The paper's pattern suite (Methods and measurement section) on both
    tiers: time, %RAM and tFootprint per pattern and tier, and the 50%/100%
    ratios r(%RAM), r(runTime), r(tFootprint) -- the form of the paper's
    Squidsort-vs-Knuthsort table (its numbers are CPU ratios, context only)."""
    import torch
    import paper_2402_01816_gb300 as g
    from paper_2402_01816_gb300 import inputs
    out = {"workload": f"paper patterns, {n} float64 keys + uint32 index payload, 100% and 50% buffer",
           "patterns": {}}
    pay = torch.arange(n, dtype=torch.int64, device=dev).to(torch.int32)
    tot = {1.0: 0.0, 0.5: 0.0, "squid": 0.0, "squid2": 0.0}
    total5 = inputs.PAPER_PATTERNS[:5]       # the TOTAL KPI: permut, tielog2, ascall, asclocal, ascglobal
    for pattern in inputs.PAPER_PATTERNS:
        keys = torch.from_numpy(inputs.make_keys(pattern, n, seed=0)).to(dev)
        kt, pt = torch.empty_like(keys), torch.empty_like(pay)

        def restore():
            kt.copy_(keys)
            pt.copy_(pay)
        row = {}
        for bf in (1.0, 0.5):
            restore()
            g.gns_sort(kt, pt, buffer_fraction=bf)
            t = _time_ms(lambda: g.gns_sort(kt, pt, buffer_fraction=bf), restore)
            ram = 1.0 + g.gns_workspace_bytes(n, bf) / (12.0 * n)
            row[f"{int(bf * 100)}%"] = {"ms": t, "gkeys_s": n / t / 1e6, "pct_ram": ram, "t_footprint_ms": ram * t}
            if pattern in total5:
                tot[bf] += t
        restore()
        g.gns_sort_symmetric(kt, pt, variant=g.SQUIDSORT1)
        t = _time_ms(lambda: g.gns_sort_symmetric(kt, pt, variant=g.SQUIDSORT1), restore)
        row["50%-squidsort1"] = {"ms": t, "gkeys_s": n / t / 1e6, "r_runtime_vs_100": t / row["100%"]["ms"]}
        if pattern in total5:
            tot["squid"] += t
        # Squidsort2 at p = 1/8: %RAM 1.125, r(%RAM) 0.56 against the 100% tier (the paper's
        # Squidsort2 row: 0.57)
        restore()
        g.gns_sort_symmetric(kt, pt, variant=g.SQUIDSORT1, buffer_fraction=0.125)
        t = _time_ms(lambda: g.gns_sort_symmetric(kt, pt, variant=g.SQUIDSORT1, buffer_fraction=0.125), restore)
        ram = 1.0 + g.gns_workspace_bytes(n, 0.125) / (12.0 * n)
        row["12.5%-squidsort2"] = {"ms": t, "gkeys_s": n / t / 1e6, "pct_ram": ram,
                                   "r_pct_ram": ram / row["100%"]["pct_ram"], "r_runtime": t / row["100%"]["ms"],
                                   "r_t_footprint": ram * t / row["100%"]["t_footprint_ms"]}
        if pattern in total5:
            tot["squid2"] += t
        if g.gns_stream_status() != 0:
            raise RuntimeError("device status error in paper_patterns")
        a, b = row["100%"], row["50%"]
        row["r_pct_ram"] = b["pct_ram"] / a["pct_ram"]
        row["r_runtime"] = b["ms"] / a["ms"]
        row["r_t_footprint"] = b["t_footprint_ms"] / a["t_footprint_ms"]
        out["patterns"][pattern] = row
        del keys, kt, pt
        torch.cuda.empty_cache()
    r_ram = (1.0 + g.gns_workspace_bytes(n, 0.5) / (12.0 * n)) / (1.0 + g.gns_workspace_bytes(n, 1.0) / (12.0 * n))
    out["TOTAL"] = {"ms_100": tot[1.0], "ms_50": tot[0.5], "r_pct_ram": r_ram, "r_runtime": tot[0.5] / tot[1.0],
                    "r_t_footprint": r_ram * tot[0.5] / tot[1.0],
                    "patterns": list(total5), "ms_50_squidsort1": tot["squid"],
                    "r_runtime_squidsort1": tot["squid"] / tot[1.0],
                    "ms_12_5_squidsort2": tot["squid2"], "r_runtime_squidsort2": tot["squid2"] / tot[1.0],
                    "r_pct_ram_squidsort2": (1.0 + g.gns_workspace_bytes(n, 0.125) / (12.0 * n))
                    / (1.0 + g.gns_workspace_bytes(n, 1.0) / (12.0 * n))}
    return out


SYM_PATTERNS = ("permut", "asc_noise", "desc_noise", "desc_ties", "desc_runs")


def symmetric_variants(dev, n=1 << 27, host=None):
    """gns_sort_symmetric: Frogsort1, Geckosort1 and Squidsort1 on Frogsort1's
    layout (50% buffer), on random input and on the inputs where the
    orientation of the runs matters (descending with noise, with ties, and in
    long runs)."""
    import torch
    import paper_2402_01816_gb300 as g
    from paper_2402_01816_gb300 import inputs
    names = {g.FROGSORT1: "frogsort1", g.GECKOSORT1: "geckosort1", g.SQUIDSORT1: "squidsort1"}
    out = {"workload": f"symmetric merging variants at 50% buffer: {n} float64 keys + uint32 index payload",
           "patterns": {}}
    pay = torch.arange(n, dtype=torch.int64, device=dev).to(torch.int32)
    for pattern in SYM_PATTERNS:
        src = host[pattern] if host and pattern in host else inputs.make_keys(pattern, n, seed=0)
        keys = torch.from_numpy(src).to(dev)
        kt, pt = torch.empty_like(keys), torch.empty_like(pay)

        def restore():
            kt.copy_(keys)
            pt.copy_(pay)
        row = {}
        for v, nm in names.items():
            restore()
            g.gns_sort_symmetric(kt, pt, variant=v)
            t = _time_ms(lambda: g.gns_sort_symmetric(kt, pt, variant=v), restore)
            row[nm] = {"ms": t, "gkeys_s": n / t / 1e6}
        restore()
        row["plain_100pct_ms"] = _time_ms(lambda: g.gns_sort(kt, pt), restore)
        for nm in ("geckosort1", "squidsort1"):
            row[f"{nm}_speedup_vs_frogsort1"] = row["frogsort1"]["ms"] / row[nm]["ms"]
        if g.gns_stream_status() != 0:
            raise RuntimeError("device status error in symmetric_variants")
        out["patterns"][pattern] = row
        del keys, kt, pt
        torch.cuda.empty_cache()
    return out


def config0(dev, n=1 << 20):
    """The small case (2^20 float64 keys uniform in [0, 1), ascending, 100%
    buffer; L2-resident and launch-bound): the plain call, and the same keys
    as one segment of the segmented engine, whose whole pass chain is one
    CUDA-graph launch after its first call."""
    import torch
    import paper_2402_01816_gb300 as g
    from paper_2402_01816_gb300 import inputs
    keys = torch.from_numpy(inputs.make_keys("uniform", n, seed=0)).to(dev)
    pay = torch.from_numpy(inputs.index_payload(n).view(np.int32)).to(dev)
    off = torch.tensor([0, n], dtype=torch.int64, device=dev)
    kt, pt = torch.empty_like(keys), torch.empty_like(pay)

    def restore():
        kt.copy_(keys)
        pt.copy_(pay)
    restore()
    g.gns_sort(kt, pt)
    t_plain = _time_ms(lambda: g.gns_sort(kt, pt), restore, reps=20)
    restore()
    g.gns_segmented_sort(kt, pt, off)                      # tunes and captures the graph
    t_graph = _time_ms(lambda: g.gns_segmented_sort(kt, pt, off), restore, reps=20)
    if g.gns_stream_status() != 0:
        raise RuntimeError("device status error in config0")
    return {"workload": "2^20 float64 keys uniform in [0,1) + uint32 index payload, ascending, 100% buffer "
                        "(L2-resident, launch-bound)",
            "plain_ms": t_plain, "plain_gkeys_s": n / t_plain / 1e6,
            "one_graph_launch_ms": t_graph, "one_graph_launch_gkeys_s": n / t_graph / 1e6,
            "note": "one_graph_launch: the keys as a single segment of gns_segmented_sort_ex, the whole "
                    "pass chain replayed as one captured CUDA graph"}


def segmented_bytes(off_h, tile=4096):
    """Algorithmic bytes of the batched sort: 24 B per key per executed pass,
    one tile pass plus ceil(log2(L / T)) merge levels for a segment of L keys."""
    L = np.diff(off_h).astype(np.int64)
    L = L[L > 0]
    passes = 1 + np.ceil(np.log2(np.maximum(1.0, L / tile))).astype(np.int64)
    return int(np.sum(24 * L * passes))


def run_only(args):
    """Diagnostic runs for profiling: one workload, warm-up and timed steps,
    a short JSON line (not the benchmark contract)."""
    import torch
    import paper_2402_01816_gb300 as g
    from paper_2402_01816_gb300 import build as cuda_build
    from paper_2402_01816_gb300 import inputs
    if not os.path.exists(cuda_build.LIB):
        cuda_build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n = args.n
    if args.only == "segmented":
        keys_h, pay_h, off_h = inputs.segments(args.nseg, seed=0)
        keys = torch.from_numpy(keys_h).to(dev)
        pay = torch.from_numpy(pay_h.view(np.int32)).to(dev)
        off = torch.from_numpy(off_h).to(dev)
        fn = lambda kt, pt: g.gns_segmented_sort(kt, pt, off)          # noqa: E731
        n = keys_h.size
    elif args.only == "learned":
        keys = torch.from_numpy(inputs.make_keys("mixture", n, seed=0)).to(dev)
        pay = torch.from_numpy(inputs.index_payload(n).view(np.int32)).to(dev)
        fn = lambda kt, pt: g.gns_learned_sort(kt, pt)                  # noqa: E731
    else:
        pattern, tier = args.only.split("@")
        bf = int(tier) / 100.0
        keys = torch.from_numpy(inputs.make_keys(pattern, n, seed=0)).to(dev)
        pay = torch.from_numpy(inputs.index_payload(n).view(np.int32)).to(dev)
        variant = {"frog": g.FROGSORT1, "gecko": g.GECKOSORT1, "squid": g.SQUIDSORT1}[args.variant]
        if args.variant != "frog":
            if bf >= 1.0:
                raise SystemExit("--variant needs an in-place tier (below 100)")
            fn = lambda kt, pt: g.gns_sort_symmetric(kt, pt, variant=variant, buffer_fraction=bf)   # noqa: E731
        else:
            fn = lambda kt, pt: g.gns_sort(kt, pt, buffer_fraction=bf)          # noqa: E731
    kt, pt = torch.empty_like(keys), torch.empty_like(pay)

    def restore():
        kt.copy_(keys)
        pt.copy_(pay)
    for _ in range(args.warmup):
        restore()
        fn(kt, pt)
    torch.cuda.synchronize()
    ts = [_time_ms(lambda: fn(kt, pt), restore, reps=1) for _ in range(args.steps)]
    status = g.gns_stream_status()
    if status != 0:
        raise RuntimeError(f"device status {status}")
    print(json.dumps({"only": args.only, "variant": args.variant, "n": n, "steps": args.steps,
                      "ms": statistics.mean(ts), "gkeys_s": n / statistics.mean(ts) / 1e6,
                      "diagnostic": True}), flush=True)


def cpu_baseline(n_sample=1 << 25):
    import oracle
    from paper_2402_01816_gb300 import inputs
    t, keys = 0.0, 0
    for p in inputs.PATTERNS_C1:
        k = inputs.make_keys(p, n_sample, seed=0)
        pay = inputs.index_payload(n_sample)
        t0 = time.perf_counter()
        oracle.knuthsort(k, pay)
        t += time.perf_counter() - t0
        keys += n_sample
    return {"value": keys / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle Knuthsort (100% buffer), single thread, {n_sample} keys of each of the 4 patterns "
                      f"({keys} keys, {t:.1f} s)"}


def aggregate_replicas(ms: float, keys_per_rank: int, ws: int, device=None):
    """Whole-job throughput of ws independent replicas (no collective touches
    the data): the step time is the maximum over ranks, value = the keys all
    ranks sorted / that time (Gkeys/s).  Returns (ms, value)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, keys_per_rank * ws / (ms / 1e3) / 1e9


def run_ours(args, ws, rank, local):
    import torch
    import paper_2402_01816_gb300 as g
    from paper_2402_01816_gb300 import build as cuda_build
    from paper_2402_01816_gb300 import inputs

    if not os.path.exists(cuda_build.LIB):
        cuda_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    n = args.n
    patterns = inputs.PATTERNS_C1
    host = {p: inputs.make_keys(p, n, seed=0) for p in patterns}
    pay_host = inputs.index_payload(n)
    pristine = {p: torch.from_numpy(host[p]).to(dev) for p in patterns}
    pay_pristine = torch.from_numpy(pay_host.view(np.int32)).to(dev)
    combos = [(p, bf) for p in patterns for bf in TIERS]
    work = {c: (torch.empty(n, dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.int32, device=dev))
            for c in combos}
    stream = torch.cuda.current_stream()

    def restore():
        for (p, bf), (kt, pt) in work.items():
            kt.copy_(pristine[p])
            pt.copy_(pay_pristine)

    def one_step(evs=None, owners=None):
        for i, c in enumerate(combos):
            kt, pt = work[c]
            if evs is not None:
                evs[i][0].record(stream)
            l0 = g.gns_launch_count()
            g.gns_sort(kt, pt, order=0, buffer_fraction=c[1], stream=stream)
            if owners is not None:
                owners.extend([c] * (g.gns_launch_count() - l0))
            if evs is not None:
                evs[i][1].record(stream)

    for _ in range(args.warmup):
        restore()
        one_step()
    torch.cuda.synchronize()
    if g.gns_stream_status() != 0:
        raise RuntimeError("device status error during warm-up")

    step_ms, per_combo = [], {c: [] for c in combos}
    launches0 = g.gns_launch_count()
    prof = []          # (combo, kernel name, ms) of every launch in the timed region
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            restore()
            torch.cuda.synchronize()
            barrier()
            g.gns_profile_read()          # drop records of earlier launches
            g.gns_profile_enable(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in combos]
            owners = []
            e0.record(stream)
            one_step(evs, owners)
            e1.record(stream)
            torch.cuda.synchronize()
            g.gns_profile_enable(False)
            barrier()
            step_ms.append(e0.elapsed_time(e1))
            for c, (a, b) in zip(combos, evs):
                per_combo[c].append(a.elapsed_time(b))
            recs = g.gns_profile_read()
            assert len(recs) == len(owners), (len(recs), len(owners))
            prof.extend((c, name, t) for c, (name, t) in zip(owners, recs))
    launches = g.gns_launch_count() - launches0
    status = g.gns_stream_status()
    if status != 0:
        raise RuntimeError(f"device status {status} during the timed region")
    clocks = clk.summary()

    ms, value = aggregate_replicas(statistics.mean(step_ms), n * len(combos), ws, dev)

    # Roofline of the dominant merge-level kernel, over the sorts that run merge
    # levels (the strictly descending pattern is reversed once and its merge
    # launches return at once, so they are left out of the average).
    peak, peak_kind = load_peaks()
    moving = [c for c in combos if c[0] != "desc"]
    total_kernel_ms = sum(t for _, _, t in prof)

    def roof(name, among):
        ts = [t for c, nm, t in prof if nm == name and c in among]
        if not ts:
            return None
        avg = statistics.mean(ts)
        alg = BYTES_PER_ELEM_PASS * n
        ach = alg / (avg / 1e3) / 1e9
        return {"launches": len(ts), "avg_ms": avg, "algorithmic_bytes_per_launch": alg,
                "achieved_gbs": ach, "frac": ach / peak,
                "share": sum(t for c, nm, t in prof if nm == name) / total_kernel_ms}

    # the roofline object describes the merge-level kernel with the largest share of the step
    level_desc = {"merge_pass": "merge_pass (100% tier merge level over all n; 24 B per element)",
                  "frog_merge": "frog_merge (<=50% tier in-place merge level over all n; 24 B per element)"}
    shares = {nm: sum(t for _, k, t in prof if k == nm) for nm in level_desc}
    dom = max(shares, key=shares.get)
    mp = roof(dom, moving)
    roofline = {"bound": "hbm", "achieved": mp["achieved_gbs"] if mp else None, "peak": peak, "unit": "GB/s",
                "frac": mp["frac"] if mp else None, "traffic": ncu_traffic(dom),
                "kernel": level_desc[dom],
                "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6800 GB/s",
                "note": "frac of measured peak" if peak_kind == "measured" else "frac of fallback peak"}
    kernels = {}
    for name in sorted({nm for _, nm, _ in prof}):
        ts = [t for _, nm, t in prof if nm == name]
        r = roof(name, moving) if name in ("merge_pass", "frog_merge", "tile_sort", "frog_setup") else None
        kernels[name] = r or {"launches": len(ts), "avg_ms": statistics.mean(ts),
                              "share": sum(ts) / total_kernel_ms}

    detail = {}
    for c in combos:
        t = statistics.mean(per_combo[c])
        ram = (12 * n + g.gns_workspace_bytes(n, c[1])) / (12 * n)
        detail[f"{c[0]}@{int(c[1] * 100)}%"] = {"ms": t, "gkeys_s": n / (t / 1e3) / 1e9, "pct_ram": ram,
                                                "t_footprint_ms": ram * t}

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if rank == 0 or ws > 1:
        hk = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        hp = torch.empty(n, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
        for (p, bf) in combos[:2]:         # untimed: the workspace pool grows by the device copies once
            np.copyto(hk, host[p])
            np.copyto(hp, pay_host)
            g.gns_sort_host(hk, hp, order=0, buffer_fraction=bf, stream=stream)
        e2e_times = []
        for _ in range(max(1, args.e2e_steps)):
            tot = 0.0
            for (p, bf) in combos:
                np.copyto(hk, host[p])
                np.copyto(hp, pay_host)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                g.gns_sort_host(hk, hp, order=0, buffer_fraction=bf, stream=stream)
                tot += time.perf_counter() - t0
            e2e_times.append(tot)
        te = statistics.mean(e2e_times)
        e2e = {"value": n * len(combos) / te / 1e9 * ws, "unit": UNIT,
               "h2d_bytes_per_step": n * 12 * len(combos), "d2h_bytes_per_step": n * 12 * len(combos),
               "entry_point": "gns_sort_host (pinned host buffers, copies inside the timed call)"}

    extras = {}
    if not args.no_extras and args.n == N_FULL:
        extras["learned_vs_plain"] = learned_vs_plain(dev)
        extras["batched_vs_plain"] = batched_vs_plain(dev)
        extras["symmetric_variants"] = symmetric_variants(dev, n, host)
        extras["config0"] = config0(dev)
        extras["learned_network_gain"] = network_gain(dev)
    if args.paper_patterns:
        extras["paper_patterns"] = paper_patterns(dev, args.n)
    if not args.no_extras and not args.no_large and args.n == N_FULL:
        extras["large_low_memory"] = large_low_memory(dev)
    if rank != 0:
        return
    cpu = None if args.no_cpu_baseline or ws > 1 else cpu_baseline()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "n_per_sort": n, "sorts_per_step": len(combos), "parallelism": f"replicas{ws}",
                       "l2": "inputs larger than L2 (1.5 GiB per sort), no flush"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "kernels": kernels, "detail": detail, **extras}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.only:
        run_only(args)
        return
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
