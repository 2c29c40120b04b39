"""Host logic of bench.py: replica aggregation over torch.distributed (gloo,
world size 2) and the reference arm (the FP64 oracle on a bounded sample)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:" + sys.argv[2],
                        rank=int(sys.argv[3]), world_size=2)
r = dist.get_rank()
ms = bench.max_over_ranks(10.0 + 5.0 * r, dist, "cpu")
print(json.dumps({"rank": r, "ms": ms, "value": bench.job_value(1e12, ms, dist.get_world_size())}))
dist.destroy_process_group()
"""


def test_replica_time_is_max_over_ranks_gloo(tmp_path):
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = str(s.getsockname()[1])
    s.close()
    w = tmp_path / "w.py"
    w.write_text(WORKER)
    ps = [subprocess.Popen([sys.executable, str(w), ROOT, port, str(r)], stdout=subprocess.PIPE,
                           stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = [p.communicate(timeout=120) for p in ps]
    for p, (o, e) in zip(ps, outs):
        assert p.returncode == 0, e
    res = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    for d in res:
        assert d["ms"] == 15.0                      # slowest rank
        assert abs(d["value"] - 2 * 1e12 / 15e-3 / 1e12) < 1e-9


def test_reference_arm_prints_one_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_traffic_reported_only_for_the_measured_kernel_source(monkeypatch, tmp_path):
    """A traffic figure is reported only while the kernel source has the hash
    it was measured with (bench.py prints null for a changed kernel)."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    key = ("hubbard6x6_su2_D1024", "k_split_gemm stage1")
    assert key in bench.TRAFFIC
    src = tmp_path / "k.cu"
    src.write_text("// kernel source as measured\n")
    monkeypatch.setattr(bench, "TRAFFIC_SOURCE", str(src))
    monkeypatch.setattr(bench, "TRAFFIC_SHA",
                        hashlib.sha256(src.read_bytes()).hexdigest()[:16])
    assert bench.traffic_of(*key) == bench.TRAFFIC[key]
    assert bench.traffic_of("hubbard6x6_D512", "k_split_gemm stage1") is None
    # any other source text: no traffic figure
    src.write_text("// kernel source as measured\n// changed\n")
    assert bench.traffic_of(*key) is None


def test_peaks_fall_back_without_measured_file(monkeypatch, tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "PEAKS_PATH", str(tmp_path / "absent.json"))
    hbm, bf16, src = bench.peaks()
    assert (hbm, bf16, src) == (6400.0, 1800.0, "fallback")
