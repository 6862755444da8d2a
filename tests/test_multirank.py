"""The multi-process (N > 1) host paths on CPU with the gloo backend, world
sizes 2 and 3, rendezvous on 127.0.0.1 (no GPU): bench.py's harness, and the
exchange step of one mesh split across ranks by elements.

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


def test_element_ranges_partition_the_mesh():
    from paper_1103_0066_gb300.shard import element_range
    for n in (0, 1, 31, 32, 33, 1000, 12582912):
        for world in (1, 2, 3, 4, 8):
            rs = [element_range(n, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[r][1] == rs[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0
    with pytest.raises(ValueError):
        element_range(10, 2, 2)


def _shard_main(rank, world, port, out_dir):
    """One rank of the sharded adjoint on CPU: the oracle's reverse mode over
    this rank's element slice stands in for the slice's kernels, and the
    package's exchange adds the ranks' partial vertex gradients."""
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world)})
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1103_0066_gb300 import meshgen as mg
    from paper_1103_0066_gb300.shard import element_range, exchange_dcoords
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mesh = mg.cube_tet_mesh(4, 0.15, mg.rng_for(81), 0.05, np.float32)
    dA = mg.upstream(mg.rng_for(82), mesh.n_elem, 4)
    w = mg.lognormal_coef(mg.rng_for(83), mesh.n_elem)
    e0, e1 = element_range(mesh.n_elem, world, rank)
    gx, gw = oracle.integrate_vjp(3, 0, mesh.conn[e0:e1], mesh.coords, dA[e0:e1], w[e0:e1])
    dx = exchange_dcoords(torch.from_numpy(gx))
    np.save(os.path.join(out_dir, f"dx{rank}.npy"), dx.numpy())
    np.save(os.path.join(out_dir, f"dw{rank}.npy"), gw)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_adjoint_exchange_gloo(tmp_path, world):
    """world ranks, one mesh split by elements: after the exchange every rank
    holds the whole mesh's vertex gradient (the single-process oracle's, up to
    the order of the FP64 sums), and each rank's coefficient gradient is its
    rows."""
    import numpy as np
    import torch.multiprocessing as mp

    import oracle
    from paper_1103_0066_gb300 import meshgen as mg
    oracle.build()
    port = _free_port()
    mp.start_processes(_shard_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    mesh = mg.cube_tet_mesh(4, 0.15, mg.rng_for(81), 0.05, np.float32)
    dA = mg.upstream(mg.rng_for(82), mesh.n_elem, 4)
    w = mg.lognormal_coef(mg.rng_for(83), mesh.n_elem)
    gx, gw = oracle.integrate_vjp(3, 0, mesh.conn, mesh.coords, dA, w)
    dx = [np.load(tmp_path / f"dx{r}.npy") for r in range(world)]
    assert all(np.array_equal(dx[0], d) for d in dx[1:])
    assert np.abs(dx[0] - gx).max() <= 1e-12 * np.abs(gx).max()
    shared = np.intersect1d(mesh.conn[: mesh.n_elem // 2], mesh.conn[mesh.n_elem // 2:])
    assert shared.size > 0  # the split does cut through vertices: the exchange is needed
    assert np.array_equal(np.concatenate([np.load(tmp_path / f"dw{r}.npy") for r in range(world)]), gw)


def _sharded_class_main(rank, world, port, out_dir):
    """One rank running the ShardedMesh class itself on CPU tensors: its slice
    kernels (integrate_fwd, Workspace, integrate_bwd of the package) are
    replaced by the oracle, so the class's own logic -- the element range, the
    slice of the connectivity and of the per-element arrays, the workspace kept
    between calls and the exchange over the process group -- runs as it does
    on GPUs."""
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world)})
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1103_0066_gb300 import meshgen as mg
    from paper_1103_0066_gb300 import shard
    calls = {"ws": 0}

    class CpuWorkspace:
        def __init__(self, coords, conn, form):
            calls["ws"] += 1

    def cpu_fwd(coords, conn, form, coef=None, **kw):
        A, _ = oracle.integrate(3, form, conn.numpy(), coords.numpy(), None if coef is None else coef.numpy())
        return torch.from_numpy(A)

    def cpu_bwd(coords, conn, form, dA, coef=None, ws=None, reduce=0, need_dcoef=True, **kw):
        assert isinstance(ws, CpuWorkspace) and reduce == 0
        gx, gw = oracle.integrate_vjp(3, form, conn.numpy(), coords.numpy(), dA.numpy(),
                                      None if coef is None else coef.numpy())
        return torch.from_numpy(gx), (torch.from_numpy(gw) if need_dcoef else None)
    shard.Workspace, shard.integrate_fwd, shard.integrate_bwd = CpuWorkspace, cpu_fwd, cpu_bwd
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mesh = mg.cube_tet_mesh(4, 0.15, mg.rng_for(84), 0.05, np.float32)
    dA = torch.from_numpy(mg.upstream(mg.rng_for(85), mesh.n_elem, 4).astype(np.float64))
    w = torch.from_numpy(mg.lognormal_coef(mg.rng_for(86), mesh.n_elem).astype(np.float64))
    sm = shard.ShardedMesh(torch.from_numpy(mesh.coords.astype(np.float64)), torch.from_numpy(mesh.conn), 0)
    assert (sm.world, sm.rank) == (world, rank)
    A = sm.integrate_fwd(sm.local(w))
    for _ in range(2):  # the workspace is built once and kept
        dx, dw = sm.integrate_bwd(sm.local(dA).contiguous(), sm.local(w))
    assert calls["ws"] == 1
    np.save(os.path.join(out_dir, f"cA{rank}.npy"), A.numpy())
    np.save(os.path.join(out_dir, f"cdx{rank}.npy"), dx.numpy())
    np.save(os.path.join(out_dir, f"cdw{rank}.npy"), dw.numpy())
    dist.destroy_process_group()


def test_sharded_mesh_class_runs_at_world_size_2(tmp_path):
    """ShardedMesh over two gloo ranks: the forward rows and coefficient
    gradients of the ranks concatenate to the whole mesh's, and after the
    exchange both ranks hold the whole mesh's vertex gradient."""
    import numpy as np
    import torch.multiprocessing as mp

    import oracle
    from paper_1103_0066_gb300 import meshgen as mg
    oracle.build()
    world = 2
    port = _free_port()
    mp.start_processes(_sharded_class_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    mesh = mg.cube_tet_mesh(4, 0.15, mg.rng_for(84), 0.05, np.float32)
    dA = mg.upstream(mg.rng_for(85), mesh.n_elem, 4).astype(np.float64)
    w = mg.lognormal_coef(mg.rng_for(86), mesh.n_elem).astype(np.float64)
    A, _ = oracle.integrate(3, 0, mesh.conn, mesh.coords, w)
    gx, gw = oracle.integrate_vjp(3, 0, mesh.conn, mesh.coords, dA, w)
    assert np.array_equal(np.concatenate([np.load(tmp_path / f"cA{r}.npy") for r in range(world)]), A)
    assert np.array_equal(np.concatenate([np.load(tmp_path / f"cdw{r}.npy") for r in range(world)]), gw)
    dx = [np.load(tmp_path / f"cdx{r}.npy") for r in range(world)]
    assert np.array_equal(dx[0], dx[1])
    assert np.abs(dx[0] - gx).max() <= 1e-12 * np.abs(gx).max()


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
