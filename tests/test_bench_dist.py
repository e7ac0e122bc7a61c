"""Host logic of bench.py's multi-rank path on CPU: two gloo ranks, each with
its own lattice size and time, must agree on the max-over-ranks time, report
weak-scaling throughput (all ranks' sites / slowest time) and print exactly
one JSON line, from rank 0.  No GPU and no collective on the data path."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_CODE = r"""
import json, os, sys
sys.path.insert(0, %(root)r)
import torch.distributed as dist
import bench
ws, rank, local = bench.dist_env()
dist.init_process_group("gloo")
ms = [2.0, 3.0][rank]                     # rank 1 is the slow one
dist.barrier()
ms_max = bench.reduce_max(ms, dist, "cpu")
value = bench.whole_job_mlups(1000000, ws, ms_max)
bench.emit({"rank_seen": rank, "ms_per_step": ms_max, "value": value, "n_gpus": ws}, rank)
dist.barrier()
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_max_and_single_line():
    pytest.importorskip("torch.distributed")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2",
                   RANK=str(rank), LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_CODE % {"root": ROOT}], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out)
    lines = [l for o in outs for l in o.splitlines() if l.strip()]
    assert len(lines) == 1, lines
    d = json.loads(lines[0])
    assert d["rank_seen"] == 0
    assert d["ms_per_step"] == 3.0
    assert d["n_gpus"] == 2
    assert abs(d["value"] - 2 * 1e6 / 3e-3 / 1e6) < 1e-9


def test_single_rank_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(1.5, None, "cpu") == 1.5
    assert bench.whole_job_mlups(4096 * 4096, 1, 1.0) == pytest.approx(16777.216)


def test_traffic_record_requires_matching_sources(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench._source_hash(bench.FUSED_SOURCES)
    (prof / "k.md").write_text("traffic_bytes_per_launch: 1234\nsource_hash: %s\n" % h)
    (prof / "old.md").write_text("traffic_bytes_per_launch: 1234\nsource_hash: 0000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # sources are read relative to ROOT: point them back at the repository
    monkeypatch.setattr(bench, "FUSED_SOURCES", [os.path.join(ROOT, f) for f in bench.FUSED_SOURCES])
    assert bench.profiled_traffic("k.md", bench.FUSED_SOURCES) == 1234.0
    assert bench.profiled_traffic("old.md", bench.FUSED_SOURCES) is None
    assert bench.profiled_traffic("missing.md", bench.FUSED_SOURCES) is None


def test_clock_records_that_disqualify_a_number():
    sys.path.insert(0, ROOT)
    import bench
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected(dict(ok, reasons=["sw_power_cap"], sm_mhz=1500.0))   # kept, noted
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(ok, reasons=[r]))
    assert bench.clocks_rejected(dict(ok, sm_mhz=1200.0))       # stuck low with no reason: a lock
    assert not bench.clocks_rejected(dict(ok, sm_mhz=None, sm_max_mhz=None, samples=0))
    assert not bench.clocks_rejected(None)
