"""Multi-process host logic of the replica benchmark (two ranks, gloo backend on the
CPU): the whole-job throughput of independent replicas is the summed step count over
the slowest rank's time, for the device-timed loop and the end-to-end loop alike, and
every rank sees the same result.  The reference arm does its work on rank 0 only."""

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank, ws = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=ws)
ms = [1000.0, 1250.0][rank]          # rank 1 is the slow one
e2e_s = [2.0, 1.5][rank]             # rank 0 is slow end to end
agg = bench.replica_throughput(ms, e2e_s, steps=10, e2e_steps=3, ws=ws, device="cpu")
print(json.dumps(agg), flush=True)
dist.destroy_process_group()
"""


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_replica_throughput_two_ranks_gloo():
    pytest.importorskip("torch.distributed")
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out.strip().splitlines()[-1])
    import json

    res = [json.loads(o) for o in outs]
    assert res[0] == res[1]
    assert res[0]["t_max_ms"] == 1250.0
    assert res[0]["value"] == pytest.approx(10 * 2 / 1.25)
    assert res[0]["e2e_value"] == pytest.approx(3 * 2 / 2.0)


def test_single_rank_is_local_time():
    sys.path.insert(0, ROOT)
    import bench

    agg = bench.replica_throughput(500.0, 1.0, steps=10, e2e_steps=3, ws=1, device="cpu")
    assert agg["t_max_ms"] == 500.0 and agg["value"] == pytest.approx(20.0)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class A:
        steps, warmup, chi, cpu_chi, no_ref_full = 1, 0, 4096, 1024, True

    assert bench.reference(A()) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(capsys, monkeypatch):
    """The reference arm's line: the oracle timed on small samples, the same config
    as the GPU arm's line, and one real step at the line's own bond dimension."""
    import json

    sys.path.insert(0, ROOT)
    import bench

    for k, v in (("RANK", "0"), ("WORLD_SIZE", "1"), ("LOCAL_RANK", "0")):
        monkeypatch.setenv(k, v)

    class A:
        steps, warmup, chi, cpu_chi, no_ref_full = 2, 1, 64, 16, False

    bench.reference(A())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2
    assert line["config"] == bench.bench_config(64, 14, 6, 1)
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["full_step_measured"]["chi"] == 64 and line["full_step_measured"]["seconds"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0


FAIL_WORKER = r"""
import os, sys, time
sys.path.insert(0, sys.argv[1])
import bench
rank = int(os.environ["RANK"])
bench.init_dist("gloo")
if rank == 1:
    os._exit(3)                       # a replica dies before the timing all-reduce
t0 = time.time()
try:
    bench.replica_throughput(1000.0, 1.0, steps=10, e2e_steps=1, ws=2, device="cpu")
    print("no error", flush=True)
except Exception as e:
    print("error after %.1f s: %s" % (time.time() - t0, type(e).__name__), flush=True)
    os._exit(7)
"""


def test_dead_replica_fails_the_others_instead_of_hanging():
    """Host-side failure detection of the replica run: a rank that exits before the
    all-reduce makes the survivor's collective raise within the process group's bounded
    timeout (MPS_BENCH_PG_TIMEOUT_S), so the job ends with an error, not a hang."""
    pytest.importorskip("torch.distributed")
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   MPS_BENCH_PG_TIMEOUT_S="10")
        procs.append(subprocess.Popen([sys.executable, "-c", FAIL_WORKER, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    out0, _ = procs[0].communicate(timeout=120)
    procs[1].communicate(timeout=120)
    assert procs[1].returncode == 3
    assert procs[0].returncode == 7, out0
    assert "error after" in out0
