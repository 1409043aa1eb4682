"""Host-side logic of the benchmark, on the CPU: the reference arm's JSON line
(the oracle timed on a bounded sample, the contract's keys), the rule that a
recorded ncu traffic figure is reported only for the kernel sources it was
taken on, and the segmented sort's byte model (24 B per key per executed
pass: one tile pass plus ceil(log2(L / T)) merge levels)."""
import importlib.util
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_reference_arm_prints_one_contract_line():
    b = _bench()
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "65536", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == b.METRIC and d["unit"] == b.UNIT and d["higher_is_better"] is True
    assert d["config"]["workload"] == b.WORKLOAD
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # 65,536 keys per pattern, 4 patterns, 2 tiers per step
    assert abs(d["value"] - 65536 * 8 / (d["ms_per_step"] * 1e-3) / 1e9) <= 1e-9 * max(1.0, d["value"])


def test_reference_arm_other_ranks_do_no_work(capsys):
    b = _bench()

    class A:
        n, steps, warmup, gpus = 1 << 16, 1, 0, 2
    assert b.run_reference(A, 2, 1) is None
    assert capsys.readouterr().out == ""


def test_traffic_record_only_for_its_sources(monkeypatch):
    b = _bench()
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    for kernel, e in rec.items():
        assert e["bytes_per_launch"] > 0 and e["files"]
        monkeypatch.setattr(b, "kernel_source_hash", lambda files, h=e["source_hash"]: h)
        assert b.ncu_traffic(kernel) == e["bytes_per_launch"]
        monkeypatch.setattr(b, "kernel_source_hash", lambda files: "0" * 16)
        assert b.ncu_traffic(kernel) is None
    assert b.ncu_traffic("no_such_kernel") is None


def test_source_hash_follows_the_files():
    b = _bench()
    files = ["gns_merge_ws.cuh", "gns_sort.cu"]
    h = b.kernel_source_hash(files)
    assert h == b.kernel_source_hash(list(files))
    assert h != b.kernel_source_hash(files[:1])


def test_segmented_byte_model():
    b = _bench()
    T = 4096
    # segment lengths and their executed passes, by hand
    cases = [(1, 1), (T, 1), (T + 1, 2), (2 * T, 2), (2 * T + 1, 3), (4 * T, 3), (100 * T, 8)]
    for L, passes in cases:
        assert b.segmented_bytes(np.array([0, L], dtype=np.int64), tile=T) == 24 * L * passes
    off = np.cumsum([0] + [L for L, _ in cases] + [0]).astype(np.int64)   # an empty segment adds nothing
    assert b.segmented_bytes(off, tile=T) == sum(24 * L * p for L, p in cases)
