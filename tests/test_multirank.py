"""The multi-process (N > 1) host path of bench.py on CPU with the gloo backend,
world size 2, rendezvous on 127.0.0.1 (no GPU).

bench.py shards by replica: every rank integrates its own copy of the mesh
(elements are independent units, weak scaling), with no collective on the
data path.  What runs across ranks is harness: the process-group set-up, the
barrier around the timed region and the max-over-ranks reduction of the
timed duration; and for the reference arm, rank 0 alone runs and prints."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world)})
    sys.path.insert(0, ROOT)
    import torch

    import bench
    ws, r, local, pg = bench.dist_setup(world)
    assert (ws, r, local) == (world, rank, rank) and pg is not None
    bench.barrier(pg)
    m = bench.max_over_ranks(pg, 1.5 * (rank + 1), torch.device("cpu"))
    bench.barrier(pg)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"max": m, "backend": pg.get_backend()}, f)
    pg.destroy_process_group()


def test_dist_helpers_gloo_world2(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        d = json.load(open(tmp_path / f"rank{r}.json"))
        assert d["max"] == 3.0 and d["backend"] == "gloo"


def test_reference_arm_under_torchrun_prints_once():
    """--impl reference launched like the N = 2 bench: rank 0 alone times the
    oracle and prints one JSON line; the other rank exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--mesh-n", "8", "--ref-sample", "2000"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
