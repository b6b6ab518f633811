"""The N > 1 host path of bench.py on CPU: world size 2 over gloo.  Each rank
evaluates its own replica (no collective on the data path), so what needs
checking is the host logic around it: the max-over-ranks timing, the
barrier, and that only rank 0 prints the result line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    bench.barrier(2)
    m = bench.max_over_ranks(1.5 + rank, 2)  # per-rank times 1.5 and 2.5
    bench.barrier(2)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"max": m}, fh)
    dist.destroy_process_group()


def test_max_over_ranks_and_barrier_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = free_port()
    mp.start_processes(_rank_main, args=(port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = [json.load(open(tmp_path / f"r{r}.json"))["max"] for r in range(2)]
    assert got == [2.5, 2.5]


def test_reference_arm_two_ranks_prints_once():
    # launched as the driver launches N > 1 runs; the reference arm (the
    # oracle on the host cores) runs on rank 0 alone
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--cpu-sample-n", "10", "--qubits", "12", "--layers", "2"]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["cores"] == 1 and d["e2e"]["h2d_bytes_per_step"] == 0
