"""The benchmark's multi-process host logic on the CPU (gloo, world size 2):
the path shards by nothing (every rank runs a full replica, `scaling: weak`),
so what runs across processes is the timing reduction (every rank takes
the slowest rank's time, the value counts every rank's units) and the
reference arm's rank handling (rank 0 alone runs the oracle and prints one
line; the other ranks exit 0 without work).  No GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    t = [0.25, 0.75][rank]
    got = bench.max_over_ranks(t, dist, torch.device("cpu"), torch)
    out.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res == {0: 0.75, 1: 0.75}


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.5, None, torch.device("cpu"), torch) == 0.5


def test_reference_arm_under_torchrun():
    """`bench.py --impl reference` launched under torchrun with two ranks
    (the multi-GPU launch): one JSON line (from rank 0), both ranks exit 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_sweep_and_chain_label():
    """The reference arm on the paper's timing grid names both filters, and
    on a fixed workload the chain it actually runs."""
    for wl, want in [("paper_sweep", None), ("table4_chain", "2 SOS + 2 SOS + 2 SOS + 2 SOS")]:
        r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", wl,
                            "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        d = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
        assert d["impl"] == "reference" and d["value"] > 0
        if want is None:
            assert d["config"]["workload"] == "paper_sweep_44k1"
            assert d["config"]["filters"] == {"fir": "FIR 101", "iir": "2 SOS"}
        else:
            assert d["config"]["chain"] == want
