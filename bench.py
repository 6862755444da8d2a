"""Benchmark: finite element integration by tensor contraction on GB300.

Default workload: 3D P1 Laplacian on the 128^3 Kuhn cube (12,582,912 tets,
2,775,835 vertices, 5% sliver elements), FP32 coordinates and element
matrices, compensated-FP32 Jacobian.  One step = the whole hot path over the
mesh: forward integration (gather, Jacobian, G, G:K, coalesced stores) and
the adjoint for an upstream dA ~ N(0,1) (element pass + deterministic
segmented vertex reduction).

Prints ONE JSON line (rank 0).  Timing: W untimed warm-up steps, then timed
regions of exactly K steps, each bracketed by barrier + synchronize, CUDA
events on the launching stream, max over ranks; the region is repeated until
the repeats span at least one second of device time (nvidia-smi clocks are
sampled throughout), and the line reports the median per-step time with its
spread.  The working set (~2.7 GB) is far larger than L2, so no L2 flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload tet128|tet128_shuffled|batch96|elastic128|adjoint64|coef_p1|
                              tri64_fp64|assemble128|multiphysics128|iso128] [--shard]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "elements/s & HBM GB/s vs peak, fwd and fwd+adjoint, at stated error vs FP64"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (context beside the measured copy bandwidth)

# Sources each timed kernel is compiled from; a traffic figure is reported only
# while the hash of its kernel's sources equals the one it was captured with.
KERNEL_SOURCES = {
    "fem_fwd_kernel<3,LAPLACE_P1,JAC_COMP>": ("fem_fwd.cuh", "fem_fwd_d3_lap.cu", "fem_core.cuh", "fem_forms.cuh",
                                              "fem_pipe.cuh", "fem_internal.h", "fem_geometry.cu"),
    "fem_bwd_elem_kernel<3,LAPLACE_P1,JAC_SAVED>": ("fem_bwd.cuh", "fem_bwd.cu", "fem_fwd.cuh", "fem_core.cuh",
                                                   "fem_forms.cuh", "fem_pipe.cuh", "fem_internal.h",
                                                   "fem_geometry.cu"),
    "vertex_reduce_kernel<3>": ("fem_incidence.cu", "fem_reduce.cuh", "fem_internal.h"),
    "fem_assemble<LAPLACE_P1>": ("fem_assembly.cu", "fem_pipe.cuh", "fem_internal.h"),
}

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# 128^3 sliver cube (12,582,912 tets).  A capture with DRAM counters stays on a
# smaller case, so these are the 96^3 cube's figures (one ncu capture of one
# launch each after three warm-up steps, 5,308,416 tets, 4,852,051 records)
# scaled by the elements per launch (x 2.370): records and vertices grow in the
# same proportion.  The
# forward's and the reduction's scaled figures are lower bounds: the part of
# their output still dirty in L2 when the kernel ends does not grow with it.
NCU_TRAFFIC = {
    "fem_bwd_elem_kernel<3,LAPLACE_P1,JAC_SAVED>": {"bytes_per_launch": 1321.0e6, "src": "4a6c95b7dc30da51"},
    "fem_fwd_kernel<3,LAPLACE_P1,JAC_COMP>": {"bytes_per_launch": 962.3e6, "src": "7c0682f050b938ea"},
    "vertex_reduce_kernel<3>": {"bytes_per_launch": 149.3e6, "src": "2fda9ba9be91ca76"},
    # tile pass + entry pass of one call, 96^3 capture scaled by the elements (records grow alike)
    "fem_assemble<LAPLACE_P1>": {"bytes_per_launch": 2232.3e6, "src": "2fcf5baed442a38c"},
}


def ncu_traffic(name: str):
    """Captured DRAM bytes per launch of `name`, or None once its sources changed."""
    tr = NCU_TRAFFIC.get(name)
    return tr["bytes_per_launch"] if tr and tr.get("src") == kernel_src_hash(name) else None


def kernel_src_hash(name: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[name]:
        with open(os.path.join(ROOT, "paper_1103_0066_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001 - file absent on some machines
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.out = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:  # noqa: BLE001 - no nvidia-smi: clocks reported as unknown
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.out.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ distributed

def dist_setup(gpus: int):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return ws, rank, local, pg


def barrier(pg, dev=None):
    if pg is not None:
        if dev is not None:
            pg.barrier(device_ids=[dev.index])
        else:
            pg.barrier()


def max_over_ranks(pg, x: float, dev) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ timing

MIN_TIMED_MS = 1000.0  # repeats of the K-step timed region span at least this much device time


def measure(step, K, stream, dev, pg=None, min_ms=None, max_repeats=400, label=None):
    """Times exactly K calls of step(rep, k) per timed region: barrier and
    synchronize, an event on `stream`, the K steps, an event, synchronize and
    barrier; the region's duration is the max over ranks.  The region is
    repeated until the repeats span at least min_ms of device time, with
    nvidia-smi clock samples taken throughout.  Returns the median, min and
    max ms per step over the repeats, the repeat count and the clocks."""
    import torch
    if min_ms is None:
        min_ms = MIN_TIMED_MS
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    time.sleep(0.3)
    per, total = [], 0.0
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    while len(per) < max_repeats and (total < min_ms or len(per) < 3):
        rep = len(per)
        barrier(pg, dev)
        torch.cuda.synchronize()
        s0.record(stream)
        for k in range(K):
            step(rep, k)
        s1.record(stream)
        torch.cuda.synchronize()
        barrier(pg, dev)
        ms = max_over_ranks(pg, s0.elapsed_time(s1), dev)
        per.append(ms / K)
        total += ms
    clk = clocks.stop()
    out = {"ms_per_step": statistics.median(per), "ms_min": min(per), "ms_max": max(per), "repeats": len(per),
           "timed_ms": total, "clocks": clk}
    if label:
        out["label"] = label
    return out


# ------------------------------------------------------------------ workloads

def tet_workload(n=128, k=2):
    from paper_1103_0066_gb300 import meshgen as mg
    mesh = mg.workload_tet_slivers(n, k)
    dA = mg.upstream(mg.rng_for(k + 10), mesh.n_elem, 4)
    return mesh, dA


def algorithmic_bytes(E, V, R, n, dim, coef, saved_det=True, nn=None):
    """Bytes each kernel must move (every input read once, every output written
    once, vertex arrays once).  R = records of the deterministic reduction (one
    per distinct vertex of each 32-element tile).  saved_det: the forward
    writes det J (4 B per element) and the adjoint reads it."""
    nv = dim + 1
    sd = 4 if saved_det else 0
    nn = n * n if nn is None else nn  # entries of one element block (rows x cols)
    fwd = E * (4 * nv + 4 * nn + (4 if coef else 0) + sd) + V * 4 * dim
    # dA, connectivity, the slot ranks (one 4-byte word per element); record
    # spans (2 B) and destinations (4 B) read, record sums (4 d B) written
    bwd_elem = E * (4 * nn + 4 * nv + 4 + (8 if coef else 0) + sd) + R * (2 + 4 + 4 * dim) + V * 4 * dim
    # vertex-major record sums and the vertex offsets read, dcoords written
    reduce = R * 4 * dim + V * (4 + 4 * dim)
    return {"fwd": fwd, "bwd_elem": bwd_elem, "reduce": reduce}


def cpu_baseline_leg(mesh, dA, A_gpu, dcoords_gpu, sample_elems):
    """Times the FP64 oracle (as it stands) on a bounded sample on the host
    cores and, untimed, measures the GPU results' error on that sample."""
    import oracle
    oracle.build()
    S = min(sample_elems, mesh.n_elem)
    conn = mesh.conn[:S]
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    Ar, fl = oracle.integrate(3, oracle.LAPLACE_P1, conn, mesh.coords)
    gx, _ = oracle.integrate_vjp(3, oracle.LAPLACE_P1, conn, mesh.coords, dA[:S])
    dt = time.perf_counter() - t0
    # error of the GPU outputs on the sample
    Ag = A_gpu[:S].double().cpu().numpy()
    num = np.abs(Ag - Ar).reshape(S, -1).max(1)
    den = np.abs(Ar).reshape(S, -1).max(1)
    fwd_err = float((num / den).max())
    # dcoords is comparable where every incident element lies in the sample
    inc_all = np.bincount(mesh.conn.ravel(), minlength=mesh.n_vert)
    inc_s = np.bincount(conn.ravel(), minlength=mesh.n_vert)
    full = (inc_s == inc_all) & (inc_all > 0)
    gg = dcoords_gpu.double().cpu().numpy()[full]
    bwd_err = float(np.abs(gg - gx[full]).max() / np.abs(gx[full]).max())
    return {"value": S / dt, "unit": "elements/s", "cores": cores, "kind": "oracle",
            "sample": f"first {S:,} elements of the mesh (cell-major, slivers included): FP64 "
                      f"quadrature forward + reverse mode, {dt:.1f} s wall on {cores} threads",
            "seconds": dt}, {"fwd_max_rel": fwd_err, "dcoords_max_rel": bwd_err,
                             "sample_elements": S, "dcoords_vertices_checked": int(full.sum())}


def run_ours(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_0066_gb300 as fem

    ws_n, rank, local, pg = dist_setup(args.gpus)
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    shuffled = args.workload == "tet128_shuffled"
    shard = args.shard and ws_n > 1

    if shuffled:
        from paper_1103_0066_gb300 import meshgen as mg
        mesh = mg.workload_tet_shuffled(args.mesh_n)
        dA_h = mg.upstream(mg.rng_for(12), mesh.n_elem, 4)
    else:
        mesh, dA_h = tet_workload(args.mesh_n)
    E_all, V = mesh.n_elem, mesh.n_vert
    coords = torch.from_numpy(mesh.coords).to(dev)
    conn_all = torch.from_numpy(mesh.conn).to(dev)
    dA_all = torch.from_numpy(dA_h).to(dev)
    if shard:  # this rank's contiguous element range of the one mesh
        from paper_1103_0066_gb300.shard import element_range, exchange_dcoords
        e0, e1 = element_range(E_all, ws_n, rank)
    else:
        e0, e1 = 0, E_all
    conn = conn_all[e0:e1].contiguous()
    dA = dA_all[e0:e1].contiguous()
    E = e1 - e0
    A = torch.empty((E, 4, 4), dtype=torch.float32, device=dev)
    dcoords = torch.empty((V, 3), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ws = fem.Workspace(coords, conn)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3

    det = torch.empty(E, dtype=torch.float32, device=dev)  # det J kept from the forward for the adjoint
    ev_store = []  # per-kernel events of the timed steps (fwd | bwd_elem | reduce | exchange)

    # launch shapes of the forward and the adjoint element pass chosen by the
    # autotuner on this mesh (fem_tune_fwd / fem_tune_bwd), before any timing
    shapes = {"fwd": (0, 0, None), "bwd_elem": (0, 0, None)}
    if not args.no_tune:
        shapes["fwd"] = fem.tune_fwd(coords, conn, fem.LAPLACE_P1, out=A, det_out=det)
        shapes["bwd_elem"] = fem.tune_bwd(coords, conn, fem.LAPLACE_P1, dA, ws=ws, reduce=fem.REDUCE_DEFERRED,
                                          det=det, dcoords=dcoords)
    (wf, cf, _), (wb, cb, _) = shapes["fwd"], shapes["bwd_elem"]

    def step(rep=None, k=None):
        evs = None
        if rep is not None and len(ev_store) < 4000:
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(5 if shard else 4)]
            ev_store.append(evs)
        if evs is not None:
            evs[0].record(stream)
        fem.integrate_fwd(coords, conn, fem.LAPLACE_P1, out=A, det_out=det, warps_per_cta=wf, ctas_per_sm=cf)
        if evs is not None:
            evs[1].record(stream)
        fem.integrate_bwd(coords, conn, fem.LAPLACE_P1, dA, ws=ws, reduce=fem.REDUCE_DEFERRED,
                          dcoords=dcoords, need_dcoef=False, det=det, warps_per_cta=wb, ctas_per_sm=cb)
        if evs is not None:
            evs[2].record(stream)
        fem.adjoint_reduce(coords, conn, ws, dcoords)
        if evs is not None:
            evs[3].record(stream)
        if shard:  # the path's one exchange: the partial vertex gradients summed over the ranks
            exchange_dcoords(dcoords)
            if evs is not None:
                evs[4].record(stream)

    for _ in range(args.warmup):
        step()
    K = args.steps
    m = measure(step, K, stream, dev, pg)
    torch.cuda.synchronize()
    names = ("fwd", "bwd_elem", "reduce") + (("exchange",) if shard else ())
    per = {name: float(np.mean([e[i].elapsed_time(e[i + 1]) for e in ev_store]))
           for i, name in enumerate(names)}
    ms_step = m["ms_per_step"]

    R = ws.n_records()
    byts = algorithmic_bytes(E, V, R, 4, 3, False)
    peak, peak_kind = hbm_peak()
    dom = max(("fwd", "bwd_elem", "reduce"), key=per.get)
    kname = {"fwd": "fem_fwd_kernel<3,LAPLACE_P1,JAC_COMP>", "bwd_elem": "fem_bwd_elem_kernel<3,LAPLACE_P1,JAC_SAVED>",
             "reduce": "vertex_reduce_kernel<3>"}
    h = {k: kernel_src_hash(v) for k, v in kname.items()}
    traffic = None if (shuffled or shard) else ncu_traffic(kname[dom])  # captured on the cell-major mesh
    ach = byts[dom] / (per[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": kname[dom], "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                "frac_of_nominal": ach / NOMINAL_HBM_GBS, "nominal_gbs": NOMINAL_HBM_GBS,
                "traffic": traffic, "algorithmic_bytes": byts[dom],
                "duration_ms": per[dom], "timing": "CUDA events around the kernel on its launching stream, "
                                                    f"mean over {len(ev_store)} timed steps"}
    kernels = {k: {"ms": per[k], "GB/s": byts[k] / (per[k] * 1e-3) / 1e9,
                   "frac_of_peak": byts[k] / (per[k] * 1e-3) / 1e9 / peak,
                   "frac_of_nominal": byts[k] / (per[k] * 1e-3) / 1e9 / NOMINAL_HBM_GBS} for k in byts}
    if shard:
        kernels["exchange"] = {"ms": per["exchange"], "bytes": V * 12, "what": "all-reduce of dcoords [V][3]"}
    fwd_eps = E / (per["fwd"] * 1e-3)
    value = (E_all if shard else ws_n * E_all) / (ms_step * 1e-3)

    # end to end through the public API: pinned host buffers, copies in the timed region
    e2e = None
    if not args.no_e2e and not shard:
        coords_h = torch.from_numpy(mesh.coords).pin_memory()
        conn_h = torch.from_numpy(mesh.conn).pin_memory()
        dA_hp = torch.from_numpy(dA_h).pin_memory()
        A_h = torch.empty_like(A, device="cpu").pin_memory()
        dc_h = torch.empty_like(dcoords, device="cpu").pin_memory()
        # HostStep (the C ABI's fem_host_step_run): per slice of elements, the
        # copies in, the forward, the adjoint element pass and the copies out
        # overlap on three streams
        hs = fem.HostStep(V, E, 3, fem.LAPLACE_P1, device=dev)

        def e2e_step(rep=None, k=None):
            hs.run(coords_h, conn_h, dA_hp, A_h, dc_h)
        e2e_step()
        torch.cuda.synchronize()
        e2e_steps = max(3, min(K, 10))
        me = measure(e2e_step, e2e_steps, stream, dev, pg)
        match = bool(torch.equal(A_h, A.cpu()) and torch.equal(dc_h, dcoords.cpu()))
        # the connectivity went in with the first (building) run; each timed
        # step copies the coordinates and dA in, A and dcoords out
        h2d = coords_h.numel() * 4 + dA_hp.numel() * 4
        d2h = A_h.numel() * 4 + dc_h.numel() * 4
        e2e = {"value": ws_n * E / (me["ms_per_step"] * 1e-3), "unit": "elements/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": me["ms_per_step"], "ms_min": me["ms_min"],
               "ms_max": me["ms_max"], "steps": e2e_steps, "repeats": me["repeats"], "clocks": me["clocks"],
               "path": f"fem_host_step_run (C ABI) through HostStep.run: pinned host buffers, {hs.chunk:,}-element "
                       "slices; coordinates and dA in (the connectivity and the incidence stay on the device "
                       "from the first, building run), forward, adjoint element pass and A out overlapped on "
                       "three streams, then the reduction and dcoords out",
               "bitwise_equal_to_device_path": match}

    # the shuffled mesh renumbered by fem_mesh_order / fem_mesh_renumber (setup,
    # once per mesh), then the same step in the new numbering
    renumbered = None
    if shuffled and not shard:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ep, vp = fem.mesh_order(coords, conn)
        c2, k2 = fem.renumber(coords, conn, ep, vp)
        torch.cuda.synchronize()
        order_ms = (time.perf_counter() - t0) * 1e3
        ws2 = fem.Workspace(c2, k2)
        epl, vpl = ep.long(), vp.long()
        dA2 = dA[epl].contiguous()  # dA in the new element numbering
        A2 = torch.empty_like(A)
        det2 = torch.empty_like(det)
        dc2 = torch.empty_like(dcoords)
        ev2 = []

        def step2(rep=None, k=None):
            evs = None
            if rep is not None and len(ev2) < 4000:
                evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                ev2.append(evs)
                evs[0].record(stream)
            fem.integrate_fwd(c2, k2, fem.LAPLACE_P1, out=A2, det_out=det2)
            if evs is not None:
                evs[1].record(stream)
            fem.integrate_bwd(c2, k2, fem.LAPLACE_P1, dA2, ws=ws2, reduce=fem.REDUCE_DEFERRED, dcoords=dc2,
                              need_dcoef=False, det=det2)
            if evs is not None:
                evs[2].record(stream)
            fem.adjoint_reduce(c2, k2, ws2, dc2)
            if evs is not None:
                evs[3].record(stream)
        for _ in range(args.warmup):
            step2()
        m2 = measure(step2, K, stream, dev, pg)
        torch.cuda.synchronize()
        per2 = {name: float(np.mean([e[i].elapsed_time(e[i + 1]) for e in ev2]))
                for i, name in enumerate(("fwd", "bwd_elem", "reduce"))}
        R2 = ws2.n_records()
        byts2 = algorithmic_bytes(E, V, R2, 4, 3, False)
        renumbered = {
            "what": "the shuffled mesh renumbered by fem_mesh_order + fem_mesh_renumber (Z-order of vertex "
                    "positions and element centroids), then the same step",
            "ms_per_step": m2["ms_per_step"], "ms_min": m2["ms_min"], "ms_max": m2["ms_max"],
            "repeats": m2["repeats"], "clocks": m2["clocks"], "value": E / (m2["ms_per_step"] * 1e-3),
            "kernels_ms": per2, "records": R2,
            "record_layout": {0: "vertex-major", 1: "tile order"}.get(ws2.record_layout(), "?"),
            "frac_of_peak": sum(byts2.values()) / (m2["ms_per_step"] * 1e-3) / 1e9 / hbm_peak()[0],
            "setup_ms": {"order_and_renumber": order_ms},
            "A_bitwise_equal_permuted": bool(torch.equal(A2, A[epl])),
            "dcoords_max_rel_diff": float((dc2 - dcoords[vpl]).abs().max() / dcoords.abs().max()),
        }
        del A2, dA2, det2, dc2, ws2, c2, k2

    order = "elements in random order, vertices renumbered at random" if shuffled else "cell-major element order"
    par = (f"{ws_n} ranks each integrating a contiguous element range of the one mesh; dcoords summed by an "
           "NCCL all-reduce inside each step" if shard else
           f"{ws_n} independent replicas (elements shard with no collective)")
    out = {
        "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": ws_n, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"3D P1 Laplacian, {args.mesh_n}^3 Kuhn cube, 6 tets/cell, jitter 0.15h, "
                               f"5% slivers ({E_all:,} tets, {V:,} vertices), {order}; FP32 coords and 4x4 FP32 "
                               "element matrices, compensated-FP32 Jacobian; step = forward (saving det J) + "
                               "adjoint (deterministic segmented reduction), dA ~ N(0,1)",
                   "elements": E_all, "vertices": V, "form": "laplace_p1", "dim": 3,
                   "element_order": "random" if shuffled else "cell-major",
                   "l2": "no flush: inputs/outputs (~2.7 GB per step) far exceed the 129 MB L2",
                   "parallelism": par},
        "timing": {"repeats": m["repeats"], "ms_per_step_min": m["ms_min"], "ms_per_step_max": m["ms_max"],
                   "timed_ms": m["timed_ms"], "statistic": "median over repeats of K-step timed regions"},
        "roofline": roofline,
        "kernels": kernels,
        "fwd": {"elements_per_s": fwd_eps, "gflops_paper_convention": fwd_eps * 288 / 1e9,
                "GB/s": kernels["fwd"]["GB/s"], "frac_of_peak": kernels["fwd"]["frac_of_peak"]},
        "fwd_adjoint": {"elements_per_s": E / (ms_step * 1e-3),
                        "GB/s": sum(byts.values()) / (ms_step * 1e-3) / 1e9,
                        "frac_of_peak": sum(byts.values()) / (ms_step * 1e-3) / 1e9 / peak,
                        "frac_of_nominal": sum(byts.values()) / (ms_step * 1e-3) / 1e9 / NOMINAL_HBM_GBS},
        "setup": {"incidence_build_ms": setup_ms, "records": R, "slots": 4 * E,
                  "record_layout": {0: "vertex-major", 1: "tile order"}.get(ws.record_layout(), "?"),
                  "launch_shapes": {k: {"warps_per_cta": v[0], "ctas_per_sm": v[1], "tuned_ms": v[2],
                                        "chosen_by": "default (--no-tune)" if v[2] is None else
                                        "fem_tune_fwd / fem_tune_bwd on this mesh"}
                                    for k, v in shapes.items()}},
        "e2e": e2e,
        **({"renumbered": renumbered} if renumbered is not None else {}),
        "gpu_launches": 3 * K,  # per K-step timed region: forward, element pass, reduction
        "gpu_launches_all_repeats": 3 * K * m["repeats"],
        "clocks": m["clocks"],
        "kernel_src_hash": h,
    }
    if rank == 0 and ws_n == 1 and not args.no_cpu and not shuffled:
        cpu, err = cpu_baseline_leg(mesh, dA_h, A, dcoords, args.cpu_sample)
        out["cpu_baseline"] = cpu
        out["error_vs_fp64"] = err
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def batch_bytes(items):
    """Algorithmic bytes of forward + adjoint + reduction summed over a batch."""
    total = 0
    for it in items:
        m = it["src"].mesh
        n = int(it["A"].shape[1])
        R = it.get("records", 0)
        b = algorithmic_bytes(m.n_elem, m.n_vert, R, n, m.dim, True, saved_det=False)
        total += b["fwd"] + b["bwd_elem"] + b["reduce"]
    return total


def run_batch(args):
    """96 meshes of log-uniform size in [1e3, 2e6] elements, six (shape, form)
    kinds, forward + adjoint: per-mesh eager launches, the same launches in one
    CUDA graph, each batched mode in a CUDA graph, and the tuned batched launch
    in a CUDA graph.  Every variant does the same work (each adjoint takes det J
    from its forward); the tuned launch's outputs are compared with the
    per-mesh ones bit for bit outside the timed regions."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_0066_gb300 as fem
    from paper_1103_0066_gb300 import meshgen as mg

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    batch_src = mg.mixed_batch(scale=args.batch_scale)
    items = []
    for b in batch_src:
        m = b.mesh
        n = mg.form_n(b.form, m.dim)
        items.append({"coords": torch.from_numpy(m.coords).to(dev), "conn": torch.from_numpy(m.conn).to(dev),
                      "form": b.form, "coef": torch.from_numpy(b.coef).to(dev),
                      "A": torch.empty((m.n_elem, n, n), device=dev), "dA": torch.from_numpy(b.dA).to(dev),
                      "dcoords": torch.empty((m.n_vert, m.dim), device=dev),
                      "dcoef": torch.empty(m.n_elem, device=dev), "src": b})
    E = sum(it["src"].mesh.n_elem for it in items)
    wss = [fem.Workspace(it["coords"], it["conn"], it["form"]) for it in items]
    dets = [torch.empty(it["src"].mesh.n_elem, device=dev) for it in items]
    for it, ws in zip(items, wss):
        it["records"] = ws.n_records()
    stream = torch.cuda.Stream(dev)

    def per_mesh(rep=None, k=None):  # det J kept from each forward for its adjoint, as the batch does
        for it, ws, det in zip(items, wss, dets):
            fem.integrate_fwd(it["coords"], it["conn"], it["form"], it["coef"], out=it["A"], stream=stream,
                              det_out=det)
            fem.integrate_bwd(it["coords"], it["conn"], it["form"], it["dA"], it["coef"], ws=ws,
                              dcoords=it["dcoords"], dcoef=it["dcoef"], stream=stream, det=det)

    def timed(fn, label):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        return measure(lambda rep, k: fn(), args.steps, stream, dev, label=label)

    with torch.cuda.stream(stream):
        eager = timed(per_mesh, "per-mesh eager")
        torch.cuda.synchronize()
        ref = [(it["A"].clone(), it["dcoords"].clone(), it["dcoef"].clone()) for it in items]
        g1 = torch.cuda.CUDAGraph()
        per_mesh()
        torch.cuda.synchronize()
        with torch.cuda.graph(g1, stream=stream):
            per_mesh()
        graph = timed(g1.replay, "per-mesh graph")
        bt = fem.Batch(items, stream=stream)
        cfg = bt.tune(stream=stream)
        mode_names = {fem.BATCH_SINGLE: "single", fem.BATCH_GROUPED: "grouped",
                      fem.BATCH_GROUPED_CONCURRENT: "grouped_concurrent", fem.BATCH_PER_ITEM: "per_item",
                      fem.BATCH_PER_ITEM_CONCURRENT: "per_item_concurrent", fem.BATCH_PHASED: "phased"}
        per_mode = {}
        for mode in mode_names:  # each mode at full occupancy, chunk 1, in a CUDA graph
            bt.set_config(32, 1, mode)
            bt.run(stream=stream)
            torch.cuda.synchronize()
            gm = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gm, stream=stream):
                bt.run(stream=stream)
            r = timed(gm.replay, mode_names[mode])
            per_mode[mode_names[mode]] = {"ms": r["ms_per_step"], "ms_min": r["ms_min"], "ms_max": r["ms_max"],
                                          "clocks": r["clocks"]}
            del gm
        bt.set_config(*cfg)
        for it in items:  # outputs poisoned, then written by the tuned launch alone
            it["A"].fill_(float("nan"))
            it["dcoords"].fill_(float("nan"))
            it["dcoef"].fill_(float("nan"))
        bt.run(stream=stream)
        torch.cuda.synchronize()
        g2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g2, stream=stream):
            bt.run(stream=stream)
        tuned = timed(g2.replay, "tuned batch graph")
        torch.cuda.synchronize()
        err = bt.errors(stream=stream)
    bitwise = all(torch.equal(it["A"], a) and torch.equal(it["dcoords"], x) and torch.equal(it["dcoef"], w)
                  for it, (a, x, w) in zip(items, ref))
    batch_ms = tuned["ms_per_step"]
    peak, peak_kind = hbm_peak()
    kinds = {(it["src"].mesh.dim, it["form"]) for it in items if it["src"].mesh.n_elem > 0}
    launches = {fem.BATCH_SINGLE: 1, fem.BATCH_PER_ITEM: 3 * len(items),
                fem.BATCH_PER_ITEM_CONCURRENT: 3 * len(items),
                fem.BATCH_PHASED: 3 * len(kinds)}.get(cfg[2], len(kinds))
    byts = batch_bytes(items)
    ach = byts / (batch_ms * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": E / (batch_ms * 1e-3), "unit": "elements/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": batch_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"96 meshes, element counts log-uniform in [1e3, 2e6] x {args.batch_scale}, "
                               "tri/tet x P1/P2 Laplacian/P1 elasticity, lognormal coefficient, forward + "
                               "adjoint (deterministic, det J kept from the forward in every variant), tuned "
                               "batched launch in a CUDA graph",
                   "elements": E, "meshes": len(items),
                   "l2": "no flush: ~%.1f GB moved per step" % (byts / 1e9)},
        "timing": {"repeats": tuned["repeats"], "ms_per_step_min": tuned["ms_min"],
                   "ms_per_step_max": tuned["ms_max"], "statistic": "median over repeats of K-step timed regions"},
        "roofline": {"bound": "hbm", "kernel": {fem.BATCH_SINGLE: "fem_batch_kernel",
                                                fem.BATCH_PER_ITEM: "per-mesh kernels",
                                                fem.BATCH_PER_ITEM_CONCURRENT: "per-mesh kernels on ten streams",
                                                fem.BATCH_PHASED: "multi-mesh fwd/adjoint/reduction kernels per kind"}.get(
                         cfg[2], "fem_batch_kind_kernel (all kinds)"), "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": ach / peak, "peak_kind": f"{peak_kind} copy bandwidth", "traffic": None,
                     "algorithmic_bytes": byts},
        "comparison_ms": {"per_mesh_eager": eager["ms_per_step"], "per_mesh_graph": graph["ms_per_step"],
                          "batched_graph": batch_ms, "batched_mode_untuned": per_mode},
        "comparison_clocks": {"per_mesh_eager": eager["clocks"], "per_mesh_graph": graph["clocks"]},
        "speedup_vs_eager": eager["ms_per_step"] / batch_ms, "speedup_vs_graph": graph["ms_per_step"] / batch_ms,
        "tuned_config": {"ctas_per_sm": cfg[0], "chunk": cfg[1], "mode": mode_names[cfg[2]]},
        "bitwise_equal_to_per_mesh": bitwise,
        "gpu_launches": launches * args.steps, "device_errors": err, "clocks": tuned["clocks"],
    }
    print(json.dumps(out), flush=True)


def _sample_err(orc, dim, form, mesh, coef, A_dev, idx):
    Ar, _ = orc.integrate(dim, form, mesh.conn[idx], mesh.coords, None if coef is None else coef[idx])
    import torch
    Ag = A_dev[torch.from_numpy(idx).to(A_dev.device)].double().cpu().numpy()
    num = np.abs(Ag - Ar).reshape(len(idx), -1).max(1)
    return float((num / np.abs(Ar).reshape(len(idx), -1).max(1)).max())


def run_elastic(args):
    """Symmetric-gradient elasticity on the 128^3 sliver cube with a lognormal
    coefficient: FP32 sparse contraction vs split-BF16 tensor-core contraction."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_1103_0066_gb300 as fem
    from paper_1103_0066_gb300 import meshgen as mg

    dev = torch.device("cuda:0")
    mesh = mg.workload_tet_slivers(args.mesh_n, 2)
    coef_h = mg.lognormal_coef(mg.rng_for(3), mesh.n_elem)
    E, V = mesh.n_elem, mesh.n_vert
    coords, conn = torch.from_numpy(mesh.coords).to(dev), torch.from_numpy(mesh.conn).to(dev)
    coef = torch.from_numpy(coef_h).to(dev)
    A = torch.empty((E, 12, 12), device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    for name, contract in (("fp32_sparse", fem.CONTRACT_F32), ("bf16x3_tensor_core", fem.CONTRACT_BF16X3)):
        def step():
            fem.integrate_fwd(coords, conn, fem.ELASTIC_P1, coef, out=A, contract=contract)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        r = measure(lambda rep, k: step(), args.steps, stream, dev)
        ms = r["ms_per_step"]
        rng = np.random.default_rng(7)
        idx = np.unique(np.concatenate([rng.choice(np.where(mesh.sliver)[0], 20000, replace=False),
                                        rng.choice(E, 20000, replace=False), np.arange(E - 40, E)]))
        err = _sample_err(oracle, 3, fem.ELASTIC_P1, mesh, coef_h, A, idx)
        res[name] = {"ms": ms, "ms_min": r["ms_min"], "ms_max": r["ms_max"], "repeats": r["repeats"],
                     "clocks": r["clocks"], "elements_per_s": E / (ms * 1e-3), "max_rel_err_vs_fp64": err}
    byts = algorithmic_bytes(E, V, 0, 12, 3, True, saved_det=False)["fwd"]
    peak, peak_kind = hbm_peak()
    best = min(res, key=lambda k: res[k]["ms"])
    for k in res:
        res[k]["GB/s"] = byts / (res[k]["ms"] * 1e-3) / 1e9
        res[k]["frac_of_peak"] = res[k]["GB/s"] / peak
    out = {"metric": METRIC, "value": E / (res[best]["ms"] * 1e-3), "unit": "elements/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": res[best]["ms"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"P1 symmetric-gradient elasticity, {args.mesh_n}^3 Kuhn cube with 5% slivers "
                                  f"({E:,} tets), lognormal coefficient, 12x12 FP32 element matrices, forward",
                      "elements": E, "l2": "no flush: 7.5 GB moved per step"},
           "roofline": {"bound": "hbm", "kernel": best, "achieved": res[best]["GB/s"], "peak": peak, "unit": "GB/s",
                        "frac": res[best]["frac_of_peak"], "peak_kind": f"{peak_kind} copy bandwidth",
                        "traffic": None, "algorithmic_bytes": byts},
           "paths": res, "gpu_launches": args.steps, "clocks": res[best]["clocks"]}
    print(json.dumps(out), flush=True)


def run_coef_p1(args):
    """P2 Laplacian with a P1 coefficient (vertex values, Eqs. 20-23) on the
    128^3 sliver cube, forward; the per-element-coefficient P2 Laplacian timed
    beside it on the same mesh."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_1103_0066_gb300 as fem
    from paper_1103_0066_gb300 import meshgen as mg

    dev = torch.device("cuda:0")
    mesh = mg.workload_tet_slivers(args.mesh_n, 2)
    E, V = mesh.n_elem, mesh.n_vert
    wv_h = mg.lognormal_coef(mg.rng_for(6), V)
    we_h = mg.lognormal_coef(mg.rng_for(7), E)
    coords, conn = torch.from_numpy(mesh.coords).to(dev), torch.from_numpy(mesh.conn).to(dev)
    wv, we = torch.from_numpy(wv_h).to(dev), torch.from_numpy(we_h).to(dev)
    A = torch.empty((E, 10, 10), device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    for name, form, coef, contract in (("p1_coefficient", fem.LAPLACE_P2_W1, wv, fem.CONTRACT_F32),
                                       ("p0_coefficient", fem.LAPLACE_P2, we, fem.CONTRACT_F32),
                                       ("p1_coefficient_tensor_core", fem.LAPLACE_P2_W1, wv, fem.CONTRACT_BF16X3)):
        def step():
            fem.integrate_fwd(coords, conn, form, coef, out=A, contract=contract)
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        r = measure(lambda rep, k: step(), args.steps, stream, dev)
        ms = r["ms_per_step"]
        res[name] = {"ms": ms, "ms_min": r["ms_min"], "ms_max": r["ms_max"], "repeats": r["repeats"],
                     "clocks": r["clocks"], "elements_per_s": E / (ms * 1e-3)}
        if name != "p0_coefficient":
            rng = np.random.default_rng(8)
            idx = np.unique(np.concatenate([rng.choice(np.where(mesh.sliver)[0], 20000, replace=False),
                                            rng.choice(E, 20000, replace=False), np.arange(E - 40, E)]))
            Ar, _ = oracle.integrate_w1(3, oracle.LAPLACE_P2, mesh.conn[idx], mesh.coords, wv_h)
            Ag = A[torch.from_numpy(idx).to(dev)].double().cpu().numpy()
            num = np.abs(Ag - Ar).reshape(len(idx), -1).max(1)
            res[name]["max_rel_err_vs_fp64"] = float((num / np.abs(Ar).reshape(len(idx), -1).max(1)).max())
            res[name]["error_sample"] = f"{len(idx):,} elements (20,000 slivers, 20,000 uniform, the last 40)"
    # forward + adjoint of the P1-coefficient form: coordinate gradient and the
    # gradient of the coefficient's vertex values (deterministic, det J kept)
    dA = torch.randn((E, 10, 10), device=dev, generator=torch.Generator(device=dev).manual_seed(13))
    det = torch.empty(E, device=dev)
    dx = torch.empty((V, 3), device=dev)
    dwv = torch.empty(V, device=dev)
    ws = fem.Workspace(coords, conn, fem.LAPLACE_P2_W1)
    R = ws.n_records()

    def step_adj():
        fem.integrate_fwd(coords, conn, fem.LAPLACE_P2_W1, wv, out=A, det_out=det)
        fem.integrate_bwd(coords, conn, fem.LAPLACE_P2_W1, dA, wv, ws=ws, dcoords=dx, dcoef=dwv, det=det)
    for _ in range(max(3, args.warmup)):
        step_adj()
    torch.cuda.synchronize()
    ra = measure(lambda rep, k: step_adj(), args.steps, stream, dev)
    res["p1_coefficient_fwd_adjoint"] = {"ms": ra["ms_per_step"], "ms_min": ra["ms_min"], "ms_max": ra["ms_max"],
                                         "repeats": ra["repeats"], "clocks": ra["clocks"],
                                         "elements_per_s": E / (ra["ms_per_step"] * 1e-3)}
    rng = np.random.default_rng(14)
    verts = rng.choice(V, 300, replace=False)
    hit = np.zeros(V, bool)
    hit[verts] = True
    el = np.where(hit[mesh.conn].any(1))[0]
    gx, gw = oracle.integrate_w1_vjp(3, oracle.LAPLACE_P2, mesh.conn[el], mesh.coords, wv_h,
                                     dA[torch.from_numpy(el).to(dev)].cpu().numpy())
    res["p1_coefficient_fwd_adjoint"]["max_rel_err_vs_fp64"] = {
        "dcoords": float(np.abs(dx.cpu().numpy()[verts] - gx[verts]).max() / np.abs(gx[verts]).max()),
        "dcoef_vertex_values": float(np.abs(dwv.cpu().numpy()[verts] - gw[verts]).max() / np.abs(gw[verts]).max()),
        "sample": "300 random vertices, against the oracle's reverse mode over all their incident elements"}
    byts = {"p1_coefficient": E * (16 + 400) + V * (12 + 4), "p0_coefficient": E * (16 + 400 + 4) + V * 12}
    byts["p1_coefficient_tensor_core"] = byts["p1_coefficient"]
    # forward (saving det J) + element pass (dA, conn, slot positions, det J; per
    # record span, destination and a 16-byte record) + reduction (records,
    # vertex offsets; dcoords and the coefficient gradient written)
    byts["p1_coefficient_fwd_adjoint"] = (E * (16 + 400 + 4) + V * (12 + 4) + E * (400 + 16 + 4 + 4) + R * (2 + 4 + 16)
                                          + V * (12 + 4) + R * 16 + V * (4 + 12 + 4))
    peak, peak_kind = hbm_peak()
    for k in res:
        res[k]["GB/s"] = byts[k] / (res[k]["ms"] * 1e-3) / 1e9
        res[k]["frac_of_peak"] = res[k]["GB/s"] / peak
    r = res["p1_coefficient"]
    out = {"metric": METRIC, "value": r["elements_per_s"], "unit": "elements/s", "n_gpus": 1,
           "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": r["ms"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"P2 Laplacian with a P1 coefficient (vertex values ~ lognormal), {args.mesh_n}^3 "
                                  f"Kuhn cube with 5% slivers ({E:,} tets), 10x10 FP32 element matrices, forward",
                      "elements": E, "l2": "no flush: 5.2 GB moved per step"},
           "roofline": {"bound": "hbm", "kernel": "fem_fwd_kernel<3,LAPLACE_P2_W1,JAC_COMP>", "achieved": r["GB/s"],
                        "peak": peak, "unit": "GB/s", "frac": r["frac_of_peak"],
                        "peak_kind": f"{peak_kind} copy bandwidth", "traffic": None,
                        "algorithmic_bytes": byts["p1_coefficient"]},
           "paths": res, "gpu_launches": args.steps, "clocks": r["clocks"]}
    print(json.dumps(out), flush=True)


def run_tri64_fp64(args):
    """The 64x64 jittered square (8,192 triangles), FP64 coordinates and FP64
    3x3 element matrices: launch-bound, reported in microseconds per launch
    (eager) and per replay of a CUDA graph of 100 launches."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_1103_0066_gb300 as fem
    from paper_1103_0066_gb300 import meshgen as mg

    dev = torch.device("cuda:0")
    mesh = mg.workload_tri_p1_fp64()
    coords, conn = torch.from_numpy(mesh.coords).to(dev), torch.from_numpy(mesh.conn).to(dev)
    A = torch.empty((mesh.n_elem, 3, 3), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(dev)

    def step():
        fem.integrate_fwd(coords, conn, fem.LAPLACE_P1, out=A, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        re = measure(lambda rep, k: step(), args.steps, stream, dev, min_ms=200.0)
        eager_us = re["ms_per_step"] * 1e3
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(100):
                step()
        g.replay()
        torch.cuda.synchronize()
        rg = measure(lambda rep, k: g.replay(), max(1, args.steps // 100), stream, dev)
        graph_us = rg["ms_per_step"] / 100 * 1e3
    Ar, _ = oracle.integrate(2, oracle.LAPLACE_P1, mesh.conn, mesh.coords)
    Ag = A.cpu().numpy()
    err = float((np.abs(Ag - Ar).reshape(mesh.n_elem, -1).max(1) / np.abs(Ar).reshape(mesh.n_elem, -1).max(1)).max())
    E = mesh.n_elem
    out = {"metric": METRIC, "value": E / (graph_us * 1e-6), "unit": "elements/s", "n_gpus": 1,
           "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": graph_us * 1e-3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "2D P1 Laplacian, 64x64 jittered square (8,192 triangles), FP64 coordinates "
                                  "and 3x3 FP64 element matrices, forward; launch-bound",
                      "elements": E, "l2": "inputs and outputs (0.8 MB) are L2-resident"},
           "us_per_launch": {"eager": eager_us, "cuda_graph": graph_us,
                             "eager_spread_us": [re["ms_min"] * 1e3, re["ms_max"] * 1e3],
                             "cuda_graph_spread_us": [rg["ms_min"] * 10, rg["ms_max"] * 10]},
           "timing": {"eager_repeats": re["repeats"], "graph_repeats": rg["repeats"],
                      "statistic": "median over repeats of timed regions"},
           "max_rel_err_vs_fp64_oracle": err, "roofline": None, "gpu_launches": args.steps,
           "clocks": rg["clocks"], "eager_clocks": re["clocks"]}
    print(json.dumps(out), flush=True)


def run_assemble(args):
    """Global assembly of the 128^3 sliver cube's P1 Laplacian element matrices
    into CSR (vertex graph), deterministic: element integration then assembly,
    each timed."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_1103_0066_gb300 as fem

    dev = torch.device("cuda:0")
    mesh, _ = tet_workload(args.mesh_n)
    E, V = mesh.n_elem, mesh.n_vert
    coords, conn = torch.from_numpy(mesh.coords).to(dev), torch.from_numpy(mesh.conn).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    asm = fem.Assembly(coords, conn, fem.LAPLACE_P1)
    build_ms = (time.perf_counter() - t0) * 1e3
    A = fem.integrate_fwd(coords, conn, fem.LAPLACE_P1)
    vals = torch.empty(asm.nnz, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        return measure(lambda rep, k: fn(), args.steps, stream, dev)

    ra = timed(lambda: asm.assemble(A, out=vals))
    rf = timed(lambda: fem.integrate_fwd(coords, conn, fem.LAPLACE_P1, out=A))
    asm_ms, fwd_ms = ra["ms_per_step"], rf["ms_per_step"]
    # rows checked against the FP64 oracle: every row of a sample of vertices
    rng = np.random.default_rng(9)
    rows = np.unique(rng.choice(V, 2000, replace=False))
    rp = asm.row_ptr.cpu().numpy()
    ci = asm.col_idx.cpu().numpy()
    vh = vals.cpu().numpy()
    inc = np.zeros(V, bool)
    inc[rows] = True
    el = np.where(inc[mesh.conn].any(1))[0]
    Ar, _ = oracle.integrate(3, oracle.LAPLACE_P1, mesh.conn[el], mesh.coords)
    Mr = oracle.assemble(3, oracle.LAPLACE_P1, mesh.conn[el], V, Ar)
    elmax = np.abs(Ar).reshape(len(el), -1).max(1)
    bound = np.zeros(V)
    for i in range(4):
        np.add.at(bound, mesh.conn[el, i], elmax)
    err = 0.0
    for v in rows:
        ref = dict(zip(Mr.indices[Mr.indptr[v]:Mr.indptr[v + 1]], Mr.data[Mr.indptr[v]:Mr.indptr[v + 1]]))
        got = dict(zip(ci[rp[v]:rp[v + 1]], vh[rp[v]:rp[v + 1]]))
        if not ref:
            continue
        err = max(err, max(abs(got.get(k, 0.0) - ref[k]) for k in ref) / bound[v])
    nnz, R2 = asm.nnz, asm.n_records
    T = (E + 31) // 32
    # tile pass: A, run words, record cells, tile offsets/runs, record slots read, records written;
    # entry pass: entry offsets, records read (contiguous), values written
    byts = E * 64 + E * 4 + R2 * 2 + T * 6 + R2 * 4 + (nnz + 1) * 4 + R2 * 4 + R2 * 4 + nnz * 4
    peak, peak_kind = hbm_peak()
    gbs = byts / (asm_ms * 1e-3) / 1e9
    out = {"metric": METRIC, "value": E / (asm_ms * 1e-3), "unit": "elements/s", "n_gpus": 1,
           "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": asm_ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"global CSR assembly of the P1 Laplacian element matrices, {args.mesh_n}^3 "
                                  f"Kuhn cube with 5% slivers ({E:,} tets, {V:,} vertices, {nnz:,} nonzeros, "
                                  f"{R2:,} tile records), "
                                  "deterministic (per 32-element tile in element order, then in tile order)",
                      "elements": E, "nnz": nnz, "l2": f"no flush: {byts / 1e9:.1f} GB moved per step"},
           "roofline": {"bound": "hbm", "kernel": "fem_assemble<LAPLACE_P1> (tile pass + entry pass, one call)",
                        "achieved": gbs, "peak": peak,
                        "unit": "GB/s", "frac": gbs / peak, "peak_kind": f"{peak_kind} copy bandwidth",
                        "traffic": ncu_traffic("fem_assemble<LAPLACE_P1>"), "algorithmic_bytes": byts},
           "forward_ms": fwd_ms, "build_ms": build_ms, "max_row_err_vs_fp64": err,
           "error_metric": "per row v: max |a - a_fp64| / (sum over the elements at v of max |A_e|)",
           "error_sample": f"all entries of {len(rows):,} random rows",
           "timing": {"repeats": ra["repeats"], "ms_per_step_min": ra["ms_min"], "ms_per_step_max": ra["ms_max"],
                      "statistic": "median over repeats of K-step timed regions"},
           "clocks": ra["clocks"], "forward_clocks": rf["clocks"],
           "gpu_launches": 2 * args.steps}  # tile pass + entry pass per call
    # the P2 Laplacian over its vertex and edge unknowns (row kernel, element order)
    del A, vals
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    asm2 = fem.Assembly(coords, conn, fem.LAPLACE_P2)
    build2_ms = (time.perf_counter() - t0) * 1e3
    A2 = fem.integrate_fwd(coords, conn, fem.LAPLACE_P2)
    vals2 = torch.empty(asm2.nnz, device=dev)
    r2 = timed(lambda: asm2.assemble(A2, out=vals2))
    ms2 = r2["ms_per_step"]
    R = asm2.n_rows
    # A read, the unknowns' incidences, positions and row offsets, values written
    byts2 = E * 400 + (R + 1) * 4 + E * 10 * 4 + E * 100 + (R + 1) * 4 + asm2.nnz * 4
    dofs = asm2.dofs.cpu().numpy()
    rp2, ci2, vh2 = asm2.row_ptr.cpu().numpy(), asm2.col_idx.cpu().numpy(), vals2.cpu().numpy()
    rows2 = np.unique(rng.choice(V, 500, replace=False))
    el2 = np.where(np.isin(mesh.conn, rows2).any(1))[0]
    Ar2, _ = oracle.integrate(3, oracle.LAPLACE_P2, mesh.conn[el2], mesh.coords)
    err2 = 0.0
    for v in rows2:
        ref, bnd = {}, 0.0
        for k, e in enumerate(el2):
            i = np.flatnonzero(dofs[e] == v)
            if len(i) == 0:
                continue
            bnd += np.abs(Ar2[k]).max()
            for j in range(10):
                ref[dofs[e, j]] = ref.get(dofs[e, j], 0.0) + Ar2[k, i[0], j]
        got = dict(zip(ci2[rp2[v]:rp2[v + 1]], vh2[rp2[v]:rp2[v + 1]]))
        if ref:
            err2 = max(err2, max(abs(got.get(c, 0.0) - x) for c, x in ref.items()) / bnd)
    gbs2 = byts2 / (ms2 * 1e-3) / 1e9
    out["p2"] = {"ms": ms2, "ms_min": r2["ms_min"], "ms_max": r2["ms_max"], "repeats": r2["repeats"],
                 "clocks": r2["clocks"], "build_ms": build2_ms, "unknowns": R, "nnz": asm2.nnz,
                 "elements_per_s": E / (ms2 * 1e-3), "GB/s": gbs2, "frac_of_peak": gbs2 / peak,
                 "algorithmic_bytes": byts2, "max_row_err_vs_fp64": err2,
                 "error_sample": f"all entries of {len(rows2)} vertex rows, against the FP64 oracle's element "
                                 "matrices summed over the library's unknowns",
                 "kernel": "assemble_rows_kernel<10> (a row per 10-lane group, 3 rows per warp, incidences in element order)"}
    print(json.dumps(out), flush=True)


def run_multiphysics(args):
    """The blocks of a coupled thermo-elastic system on the 128^3 sliver cube
    (Sec. 6: coupled systems broken into blocks): P1 elasticity for the
    displacement u, the P1 Laplacian for the temperature T, their coupling
    block int T div v (DIV_P1P1), and a second scalar field's P2 Laplacian;
    forward + adjoint, as four items of one tuned batched launch in a CUDA
    graph, against the same blocks launched per form.  The batch's outputs are
    compared with the per-form ones bit for bit outside the timed regions."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_0066_gb300 as fem
    from paper_1103_0066_gb300 import meshgen as mg

    dev = torch.device("cuda:0")
    mesh = mg.workload_tet_slivers(args.mesh_n, 2)
    E, V = mesh.n_elem, mesh.n_vert
    coords, conn = torch.from_numpy(mesh.coords).to(dev), torch.from_numpy(mesh.conn).to(dev)
    coef = torch.from_numpy(mg.lognormal_coef(mg.rng_for(3), E)).to(dev)
    gen = torch.Generator(device=dev).manual_seed(5)
    items, wss = [], []
    forms = (fem.ELASTIC_P1, fem.LAPLACE_P1, fem.DIV_P1P1, fem.LAPLACE_P2)
    for form in forms:
        rows, cols = fem.form_shape(form, 3)
        items.append({"coords": coords, "conn": conn, "form": form, "coef": coef,
                      "A": torch.empty((E, rows, cols), device=dev),
                      "dA": torch.randn((E, rows, cols), device=dev, generator=gen),
                      "dcoords": torch.empty((V, 3), device=dev), "dcoef": torch.empty(E, device=dev)})
        wss.append(fem.Workspace(coords, conn, form))
    stream = torch.cuda.Stream(dev)

    dets = [torch.empty(E, device=dev) for _ in items]

    def per_form():  # det J kept from each forward for its adjoint, as the batch does
        for it, ws, det in zip(items, wss, dets):
            fem.integrate_fwd(coords, conn, it["form"], coef, out=it["A"], stream=stream, det_out=det)
            fem.integrate_bwd(coords, conn, it["form"], it["dA"], coef, ws=ws, dcoords=it["dcoords"],
                              dcoef=it["dcoef"], stream=stream, det=det)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        return measure(lambda rep, k: fn(), args.steps, stream, dev)

    with torch.cuda.stream(stream):
        re = timed(per_form)
        eager_ms = re["ms_per_step"]
        torch.cuda.synchronize()
        ref = [(it["A"].clone(), it["dcoords"].clone(), it["dcoef"].clone()) for it in items]
        bt = fem.Batch(items, stream=stream)
        cfg = bt.tune(stream=stream)
        for it in items:
            it["A"].fill_(float("nan"))
            it["dcoords"].fill_(float("nan"))
        bt.run(stream=stream)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            bt.run(stream=stream)
        rb = timed(g.replay)
        batch_ms = rb["ms_per_step"]
        err = bt.errors(stream=stream)
    bitwise = all(torch.equal(it["A"], a) and torch.equal(it["dcoords"], x) and torch.equal(it["dcoef"], w)
                  for it, (a, x, w) in zip(items, ref))
    R = wss[0].n_records()  # the records depend on the connectivity only
    byts = 0
    for it in items:
        rows, cols = it["A"].shape[1], it["A"].shape[2]
        b = algorithmic_bytes(E, V, R, 0, 3, True, saved_det=False, nn=rows * cols)
        byts += b["fwd"] + b["bwd_elem"] + b["reduce"]
    peak, peak_kind = hbm_peak()
    gbs = byts / (batch_ms * 1e-3) / 1e9
    mode_names = {fem.BATCH_SINGLE: "single", fem.BATCH_GROUPED: "grouped",
                  fem.BATCH_GROUPED_CONCURRENT: "grouped_concurrent", fem.BATCH_PER_ITEM: "per_item",
                  fem.BATCH_PER_ITEM_CONCURRENT: "per_item_concurrent", fem.BATCH_PHASED: "phased"}
    out = {"metric": METRIC, "value": len(items) * E / (batch_ms * 1e-3), "unit": "elements/s", "n_gpus": 1,
           "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": batch_ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"four blocks of a coupled thermo-elastic system on the {args.mesh_n}^3 sliver "
                                  f"cube ({E:,} tets): P1 elasticity, P1 Laplacian, the coupling block int T div v "
                                  "(4 x 12), and a P2 Laplacian; lognormal coefficient, forward + adjoint, one "
                                  "tuned batched launch in a CUDA graph",
                      "elements": E, "blocks": len(items), "l2": "no flush"},
           "roofline": {"bound": "hbm", "kernel": "per-item kernels of the tuned batch", "achieved": gbs,
                        "peak": peak, "unit": "GB/s", "frac": gbs / peak, "peak_kind": f"{peak_kind} copy bandwidth",
                        "traffic": None, "algorithmic_bytes": byts},
           "comparison_ms": {"per_form_eager": eager_ms, "batched_graph": batch_ms},
           "timing": {"repeats": rb["repeats"], "ms_per_step_min": rb["ms_min"], "ms_per_step_max": rb["ms_max"],
                      "statistic": "median over repeats of K-step timed regions"},
           "clocks": rb["clocks"], "per_form_clocks": re["clocks"],
           "tuned_config": {"ctas_per_sm": cfg[0], "chunk": cfg[1], "mode": mode_names.get(cfg[2], cfg[2])},
           "bitwise_equal_to_per_form": bitwise, "device_errors": err,
           "gpu_launches": args.steps * 4 * len(items)}
    print(json.dumps(out), flush=True)


def run_iso(args):
    """The Laplacian on non-affine (quadratic-geometry) elements, Eqs. 16-19:
    the 128^3 jittered cube warped into curved tets, P1 and P2, forward, and
    forward + adjoint."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_1103_0066_gb300 as fem
    from paper_1103_0066_gb300 import meshgen as mg

    dev = torch.device("cuda:0")
    mesh, mid_h = mg.workload_curved_tets(args.mesh_n)
    E, V = mesh.n_elem, mesh.n_vert
    coords, conn = torch.from_numpy(mesh.coords).to(dev), torch.from_numpy(mesh.conn).to(dev)
    mid = torch.from_numpy(mid_h).to(dev)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = hbm_peak()
    res = {}
    for name, form, n, contract in (("p1", fem.LAPLACE_P1_ISO, 4, fem.CONTRACT_F32),
                                    ("p2", fem.LAPLACE_P2_ISO, 10, fem.CONTRACT_F32),
                                    ("p2_tensor_core", fem.LAPLACE_P2_ISO, 10, fem.CONTRACT_BF16X3)):
        A = torch.empty((E, n, n), device=dev)

        def step():
            fem.integrate_fwd_iso(coords, conn, mid, form, out=A, contract=contract)
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        r = measure(lambda rep, k: step(), args.steps, stream, dev)
        ms = r["ms_per_step"]
        rng = np.random.default_rng(11)
        idx = np.unique(np.concatenate([rng.choice(E, 20000, replace=False), np.arange(E - 40, E)]))
        Ar, _ = oracle.integrate_iso(3, form - 5, mesh.conn[idx], mesh.coords, mid_h[idx])
        Ag = A[torch.from_numpy(idx).to(dev)].double().cpu().numpy()
        num = np.abs(Ag - Ar).reshape(len(idx), -1).max(1)
        byts = E * (16 + 72 + 4 * n * n) + V * 12
        res[name] = {"ms": ms, "ms_min": r["ms_min"], "ms_max": r["ms_max"], "repeats": r["repeats"],
                     "clocks": r["clocks"], "elements_per_s": E / (ms * 1e-3), "GB/s": byts / (ms * 1e-3) / 1e9,
                     "frac_of_peak": byts / (ms * 1e-3) / 1e9 / peak, "algorithmic_bytes": byts,
                     "max_rel_err_vs_fp64": float((num / np.abs(Ar).reshape(len(idx), -1).max(1)).max())}
        del A
    # forward + adjoint (fem_integrate_bwd_iso: vertex gradients through the
    # deterministic reduction, edge-node gradients per element)
    ws = fem.Workspace(coords, conn, fem.LAPLACE_P1_ISO)
    R = ws.n_records()
    dx = torch.empty((V, 3), device=dev)
    dm = torch.empty_like(mid)
    for name, form, n, contract in (("p1_fwd_adjoint", fem.LAPLACE_P1_ISO, 4, fem.CONTRACT_F32),
                                    ("p2_fwd_adjoint", fem.LAPLACE_P2_ISO, 10, fem.CONTRACT_F32),
                                    ("p2_fwd_adjoint_tensor_core", fem.LAPLACE_P2_ISO, 10, fem.CONTRACT_BF16X3)):
        A = torch.empty((E, n, n), device=dev)
        dA_h = mg.upstream(mg.rng_for(13), E, n)
        dA = torch.from_numpy(dA_h).to(dev)

        def step():
            fem.integrate_fwd_iso(coords, conn, mid, form, out=A, contract=contract)
            fem.integrate_bwd_iso(coords, conn, mid, form, dA, ws=ws, dcoords=dx, dmid=dm, contract=contract)
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        r = measure(lambda rep, k: step(), args.steps, stream, dev)
        ms = r["ms_per_step"]
        # algorithmic bytes: the forward's, the element pass's (dA, conn, edge
        # nodes in, edge-node gradients out, slot ranks, coordinates; per record
        # its span, destination and sum) and the reduction's
        fwd_b = E * (16 + 72 + 4 * n * n) + V * 12
        bwd_b = E * (4 * n * n + 16 + 72 + 72 + 4) + R * (2 + 4 + 12) + V * 12
        red_b = R * 12 + V * 16
        byts = fwd_b + bwd_b + red_b
        # errors against the oracle's reverse mode: edge-node gradients on a
        # sample of elements, vertex gradients where every incident element is evaluated
        rng = np.random.default_rng(14)
        verts = rng.choice(V, 30, replace=False)
        els = np.unique(np.concatenate([np.flatnonzero(np.isin(mesh.conn, verts).any(1)),
                                        rng.choice(E, 3000, replace=False)]))
        rx, rm, _ = oracle.integrate_iso_vjp(3, form - 5, mesh.conn[els], mesh.coords, mid_h[els], dA_h[els])
        gm = dm[torch.from_numpy(els).to(dev)].double().cpu().numpy()
        gx = dx.double().cpu().numpy()[verts]
        # a vertex gradient is a small difference of its elements' node gradients
        # (coefficients summing to zero): its error is measured against them
        s_e = np.abs(rm).reshape(len(els), -1).max(1)
        node_scale = np.abs(rx).max(1)
        np.maximum.at(node_scale, mesh.conn[els].ravel(), np.repeat(s_e, 4))
        res[name] = {"ms": ms, "ms_min": r["ms_min"], "ms_max": r["ms_max"], "repeats": r["repeats"],
                     "clocks": r["clocks"], "elements_per_s": E / (ms * 1e-3), "GB/s": byts / (ms * 1e-3) / 1e9,
                     "frac_of_peak": byts / (ms * 1e-3) / 1e9 / peak, "algorithmic_bytes": byts,
                     "max_rel_err_vs_fp64": {"dmid": float(np.abs(gm - rm).max() / np.abs(rm).max()),
                                             "dcoords": float((np.abs(gx - rx[verts]).max(1)
                                                               / node_scale[verts]).max()),
                                             "dcoords_metric": "per vertex, relative to the largest node "
                                                               "gradient of its elements",
                                             "sample": f"{len(els):,} elements, 30 vertices with all their elements"}}
        del A, dA
    r = res["p1"]
    out = {"metric": METRIC, "value": r["elements_per_s"], "unit": "elements/s", "n_gpus": 1,
           "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": r["ms"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"Laplacian on quadratic-geometry tets (Eqs. 16-19): {args.mesh_n}^3 jittered "
                                  f"cube warped by a smooth map ({E:,} tets), P1 and P2 (FP32 contraction; P2 also "
                                  "split-BF16 on the tensor cores), forward; and forward + adjoint (vertex and "
                                  "edge-node gradients)",
                      "elements": E, "l2": "no flush"},
           "roofline": {"bound": "hbm", "kernel": "fem_fwd_iso_kernel<3,LAPLACE_P1_ISO>", "achieved": r["GB/s"],
                        "peak": peak, "unit": "GB/s", "frac": r["frac_of_peak"],
                        "peak_kind": f"{peak_kind} copy bandwidth", "traffic": None,
                        "algorithmic_bytes": r["algorithmic_bytes"]},
           "paths": res, "gpu_launches": args.steps, "clocks": r["clocks"]}
    print(json.dumps(out), flush=True)


def run_adjoint64(args):
    """Forward + adjoint of the P1 Laplacian on the 64^3 sliver cube with a
    lognormal coefficient (dcoords and dcoef), both reductions."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_0066_gb300 as fem
    from paper_1103_0066_gb300 import meshgen as mg

    dev = torch.device("cuda:0")
    mesh = mg.workload_tet_slivers(64, k=4)
    E, V = mesh.n_elem, mesh.n_vert
    coords, conn = torch.from_numpy(mesh.coords).to(dev), torch.from_numpy(mesh.conn).to(dev)
    coef = torch.from_numpy(mg.lognormal_coef(mg.rng_for(50), E)).to(dev)
    dA = torch.from_numpy(mg.upstream(mg.rng_for(51), E, 4)).to(dev)
    A = torch.empty((E, 4, 4), device=dev)
    dx = torch.empty((V, 3), device=dev)
    dw = torch.empty(E, device=dev)
    ws = fem.Workspace(coords, conn)
    R = ws.n_records()
    det = torch.empty(E, device=dev)  # det J kept from the forward for the adjoint
    stream = torch.cuda.current_stream(dev)
    res = {}
    for name, reduce in (("deterministic", fem.REDUCE_DETERMINISTIC), ("atomic", fem.REDUCE_ATOMIC)):
        def step():
            fem.integrate_fwd(coords, conn, fem.LAPLACE_P1, coef, out=A, det_out=det)
            fem.integrate_bwd(coords, conn, fem.LAPLACE_P1, dA, coef, ws=ws, reduce=reduce, dcoords=dx, dcoef=dw,
                              det=det)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        r = measure(lambda rep, k: step(), args.steps, stream, dev)
        ms = r["ms_per_step"]
        # the same step captured once in a CUDA graph and replayed: no host
        # launch work between the kernels
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            step()  # warm on the capturing stream
        stream.wait_stream(side)
        with torch.cuda.graph(g):
            step()
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        rg = measure(lambda rep, k: g.replay(), args.steps, stream, dev)
        graph_ms = rg["ms_per_step"]
        b = algorithmic_bytes(E, V, R if reduce == 0 else 0, 4, 3, True)
        byts = b["fwd"] + (b["bwd_elem"] + b["reduce"] if reduce == 0 else
                           E * (64 + 16 + 4 + 4 + 4) + V * 12 * 2)
        res[name] = {"ms": ms, "ms_min": r["ms_min"], "ms_max": r["ms_max"], "repeats": r["repeats"],
                     "clocks": r["clocks"], "elements_per_s": E / (ms * 1e-3), "GB/s": byts / (ms * 1e-3) / 1e9,
                     "graph_ms": graph_ms, "graph_ms_min": rg["ms_min"], "graph_ms_max": rg["ms_max"],
                     "graph_clocks": rg["clocks"], "graph_GB/s": byts / (graph_ms * 1e-3) / 1e9}
    peak, peak_kind = hbm_peak()
    d = res["deterministic"]
    out = {"metric": METRIC, "value": d["elements_per_s"], "unit": "elements/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": d["ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"P1 Laplacian forward + adjoint (dcoords, dcoef), 64^3 Kuhn cube with 5% "
                                  f"slivers ({E:,} tets), lognormal coefficient, dA ~ N(0,1)",
                      "elements": E, "l2": "working set ~0.5 GB, L2 not flushed"},
           "roofline": {"bound": "hbm", "kernel": "step", "achieved": d["GB/s"], "peak": peak, "unit": "GB/s",
                        "frac": d["GB/s"] / peak, "peak_kind": f"{peak_kind} copy bandwidth", "traffic": None},
           "reductions": res, "gpu_launches": 3 * args.steps, "clocks": d["clocks"]}
    print(json.dumps(out), flush=True)


def run_reference(args):
    """The FP64 oracle timed on the host cores, bounded sample per step."""
    ws_n = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    mesh, dA = tet_workload(args.mesh_n)
    S = args.ref_sample
    nwin = max(1, mesh.n_elem // S)

    def step(k):
        w = k % nwin
        conn = mesh.conn[w * S:(w + 1) * S]
        oracle.integrate(3, oracle.LAPLACE_P1, conn, mesh.coords)
        oracle.integrate_vjp(3, oracle.LAPLACE_P1, conn, mesh.coords, dA[w * S:(w + 1) * S])

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    dt = time.perf_counter() - t0
    v = S * args.steps / dt
    cores = oracle.max_threads()
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "elements/s", "n_gpus": ws_n,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "3D P1 Laplacian, 128^3 Kuhn cube, 5% slivers (12,582,912 tets); "
                                  "step = forward + adjoint, FP64 oracle by direct quadrature",
                      "elements": mesh.n_elem, "vertices": mesh.n_vert, "form": "laplace_p1", "dim": 3},
           "cpu_baseline": {"value": v, "unit": "elements/s", "cores": cores, "kind": "oracle",
                            "sample": f"{S:,} consecutive elements per step (rotating window)"},
           "e2e": {"value": v, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    global MIN_TIMED_MS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the timed oracle leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-tune", action="store_true",
                    help="default launch shapes instead of the autotuner's (tet128 workloads)")
    ap.add_argument("--mesh-n", type=int, default=128, help="cells per cube edge (128 = the benchmark mesh)")
    ap.add_argument("--cpu-sample", type=int, default=12_582_912)
    ap.add_argument("--workload", choices=["tet128", "tet128_shuffled", "batch96", "elastic128", "adjoint64",
                                           "coef_p1", "tri64_fp64", "assemble128", "multiphysics128", "iso128"],
                    default="tet128",
                    help="tet128: the headline 128^3 sliver cube (forward + adjoint); tet128_shuffled: the same "
                         "mesh with its elements in random order and its vertices renumbered; batch96: the mixed "
                         "96-mesh batch; elastic128: elasticity FP32 vs tensor cores; adjoint64: 64^3 adjoint; "
                         "coef_p1: P2 Laplacian with a P1 coefficient; tri64_fp64: the FP64 triangle mesh; "
                         "assemble128: global CSR assembly; multiphysics128: three blocks on one mesh; "
                         "iso128: non-affine elements")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="element-count scale of the batch96 meshes")
    ap.add_argument("--min-timed-ms", type=float, default=MIN_TIMED_MS,
                    help="repeat the K-step timed region until it spans this much device time (at least 3 repeats)")
    ap.add_argument("--shard", action="store_true",
                    help="N > 1: the ranks split ONE mesh by element ranges and sum dcoords with an all-reduce "
                         "inside each step (strong scaling); default: N independent replicas (weak scaling)")
    ap.add_argument("--ref-sample", type=int, default=262_144)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    MIN_TIMED_MS = args.min_timed_ms
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch96":
        run_batch(args)
    elif args.workload == "elastic128":
        run_elastic(args)
    elif args.workload == "adjoint64":
        run_adjoint64(args)
    elif args.workload == "coef_p1":
        run_coef_p1(args)
    elif args.workload == "tri64_fp64":
        run_tri64_fp64(args)
    elif args.workload == "assemble128":
        run_assemble(args)
    elif args.workload == "multiphysics128":
        run_multiphysics(args)
    elif args.workload == "iso128":
        run_iso(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
