"""Benchmark of the fused coupled step (one JSON line on stdout, rank 0).

Workload: 1-DOF vortex-induced vibration of a cylinder (m* 10, zeta 0, V_R 5,
Re 100, Ma 0.2) on an O-grid of 512 radial x 256 angular nodes deformed by the
blending polynomial, FP32 populations with FP64 loads, RK4 and blend
displacement; a batch of independent solves per GPU (default 16, a
302 MB ping-pong population set, larger than the 129 MB L2).  A step is one
coupled time step of every solve of the batch: one launch of the fused kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B]
  python bench.py --impl reference ...   (the FP64 oracle on the host cores)

Under torchrun every rank runs its own batch (replicas: the solves are
independent, no data-path collective); the timed region is bracketed by a
barrier and a synchronize, the time is the max over ranks and the value is the
node updates of all ranks divided by it.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
if "reference" in sys.argv:
    # the oracle baseline runs single-threaded; set before numpy loads
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np  # noqa: E402

from paper_2107_01370_gb300 import inputs, replicas  # noqa: E402

METRIC = "fused-step MLUPS"
UNIT = "MLUPS"
BYTES_PER_NODE_FP32 = 144   # 18 populations read + 18 written, 4 bytes each
KERNEL = "k_step<float>"


def workload_name(batch):
    return (f"1-DOF VIV cylinder, O-grid 512x256 (131072 nodes) blended mesh, m* 10, V_R 5, "
            f"Re 100, Ma 0.2, FP32 populations / FP64 loads+RK4; batch of {batch} solves per GPU")


# The sources the step kernel is compiled from (a profile taken on them stays
# valid while they are unchanged).
KERNEL_SOURCES = ("lbfsi_device.cuh", "lbfsi_internal.h", "lbfsi_step.cu")


def source_sha():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2107_01370_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_per_node():
    """DRAM bytes per node update of the step kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "k_step_fp32_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha") != source_sha():
        return None
    return float(d["dram_bytes_per_node"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_worker(args):
    """One independent oracle solve of the bench workload (run in a spawned
    process): a warm-up step, then 'steps' timed steps."""
    root, seed, steps = args
    import time as _time
    sys.path.insert(0, root)
    from paper_2107_01370_gb300 import inputs as _inputs
    import oracle.mesh as OM
    import oracle.solver as OS
    c = _inputs.viv_cylinder_512x256()
    M0 = _inputs.initial_field(c.nr, c.ntheta, c.flow, seed=seed)
    s = OS.Solver.from_case(OM.ogrid_mesh(c.r, c.e), c, M0)
    s.step()
    t = _time.perf_counter()
    for _ in range(steps):
        s.step()
    return _time.perf_counter() - t, c.nodes


def cpu_baseline_sample(solves=16, steps=2):
    """Time the FP64 oracle on the host cores: the bench's batch of
    independent 512x256 solves, one per core (spawned processes, one BLAS
    thread each), a few steps each; the slowest worker's time is the
    batch's time (a bounded sample of the workload)."""
    import multiprocessing as mp
    cores = max(1, min(solves, os.cpu_count() or 1))
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            res = pool.map(_oracle_worker, [(ROOT, k, steps) for k in range(cores)])
    except Exception as ex:   # report, do not fail the bench
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"failed: {ex}"[:300]}
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    secs = max(r[0] for r in res)
    nodes = sum(r[1] for r in res)
    return {"value": nodes * steps / secs / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} independent 512x256 solves in {cores} spawned processes "
                      f"(FP64 numpy, 1 thread each), {steps} timed steps each after one warm-up "
                      f"step; slowest worker {secs:.1f} s"}


REF_ROWS = 33   # odd: the truncated radial table stays subparametric


def reference_sample_case(rows=REF_ROWS):
    """Bounded sample of the bench workload for the oracle: the first 'rows'
    (odd) radial rows, all 256 angular nodes, of the 512x256 VIV mesh, with
    the same body, blend region, flow and time step."""
    case = inputs.viv_cylinder_512x256()
    case.r = case.r[:rows].copy()
    case.nr = rows
    return case


REF_BUDGET_S = 150.0   # wall-time target of the whole reference run


def reference_rows(steps, warmup):
    """Radial rows of the reference sample such that warm-up plus timed steps
    take about REF_BUDGET_S: one calibration step of the 33-row sample, then
    the rows scaled down (odd, at least 5) when the step count needs it."""
    import oracle.mesh as OM
    import oracle.solver as OS
    case = reference_sample_case(REF_ROWS)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    s = OS.Solver.from_case(OM.ogrid_mesh(case.r, case.e), case, M0)
    s.step()
    t = time.perf_counter()
    s.step()
    t_step = time.perf_counter() - t
    # the workers run in parallel and share the memory system: about half the
    # single-process rate
    budget = 0.5 * REF_BUDGET_S / max(1, steps + warmup)
    rows = int(REF_ROWS * min(1.0, budget / max(t_step, 1e-6)))
    rows = max(5, rows - (1 - rows % 2))   # odd: the truncated table stays subparametric
    return min(rows, REF_ROWS)


SERVING_POOL = 1 << 30   # 1 GiB: about half of what the 256 requests need at once


def serving_bench(stream):
    """Serving workload: 256 cylinder-VIV requests (O-grid sizes uniform over
    64x32 .. 512x256, V_R in [3, 8], m* in [2, 20], seed 0, 2000 steps each,
    FP32) admitted into a 1 GiB device pool.  Capacity: all requests at t = 0;
    then a Poisson stream at 90% of capacity for p50/p99 time-to-solution;
    baseline: the same requests one after another as plain solves."""
    from paper_2107_01370_gb300 import serving
    cache = serving.CaseCache()
    schedule = serving.tune_schedule(SERVING_POOL, stream=stream, cache=cache)
    reqs = serving.viv_requests(256, 2000, seed=0)
    done_c, loads_c, wall_c, peak_c = serving.run_batched(reqs, SERVING_POOL, chunk=50,
                                                          stream=stream, cache=cache,
                                                          schedule=schedule)
    capacity = len(reqs) / wall_c
    reqs_p = serving.poisson_arrivals(serving.viv_requests(256, 2000, seed=0), 0.9 * capacity,
                                      seed=1)
    done_p, loads_p, wall_p, peak_p = serving.run_batched(reqs_p, SERVING_POOL, chunk=50,
                                                          stream=stream, cache=cache,
                                                          schedule=schedule)
    p50, p99 = serving.latency_stats(done_p)
    done_s, loads_s, wall_s = serving.run_sequential(reqs, stream=stream, cache=cache, schedule=schedule)
    same = all(np.array_equal(loads_p[k], loads_s[k]) for k in loads_s)
    return {"metric": "batched solves/s", "solves_per_s": round(len(reqs_p) / wall_p, 3),
            "p50_s": round(p50, 4), "p99_s": round(p99, 4),
            "capacity_solves_per_s": round(capacity, 3),
            "sequential_solves_per_s": round(len(reqs) / wall_s, 3),
            "speedup_vs_sequential": round(wall_s / wall_c, 2),
            "requests": len(reqs), "steps_per_request": 2000, "arrival_rate": round(0.9 * capacity, 3),
            "pool_bytes": SERVING_POOL, "peak_active": peak_p,
            "schedule": {"variant": schedule[0], "order": schedule[1]},
            "results_equal_alone_and_in_mix": bool(same)}


# single-solve O-grids of 1, 4 and 16.8 M nodes (radial x angular, far-field
# radius): 512 angular nodes (the impulsive start stays physical; at 1024 the
# wall temperature of the uniform initial state goes negative within five
# steps in the oracle and on the GPU alike), radial rows grown with the far
# field pushed out as far as the geometric radial table needs
SWEEP = ((2048, 512, 20.0), (8192, 512, 80.0), (32768, 512, 320.0))


def roofline_sweep(stream, schedule, peak, steps=50):
    """HBM roofline sweep: one 1-DOF VIV solve on O-grids of 1-16.8 M nodes
    (the ping-pong populations, 151 MB - 2.4 GB, exceed L2), same schedule as
    the main measurement; MLUPS and algorithmic GB/s per size."""
    import torch
    from paper_2107_01370_gb300 import lbfsi
    out = []
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.5, m_star=10.0, v_r=5.0)
    for nr, nt, r_far in SWEEP:
        case = inputs.cylinder_case(nr, nt, r_far=r_far, body=body)
        M0 = inputs.initial_field(nr, nt, case.flow, seed=0)
        row = {"mesh": f"{nr}x{nt}", "nodes": case.nodes, "r_far": r_far}
        m = lbfsi.Mesh(case.r, case.e, case.bodies, precision=lbfsi.FP32, stream=stream.cuda_stream)
        try:
            m.set_schedule(*schedule)
            m.init_fields(case.flow, M0[None])
            m.step(5)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            m.synchronize()
            ms = e0.elapsed_time(e1) / steps
            gbs = BYTES_PER_NODE_FP32 * case.nodes / (ms * 1e-3) / 1e9
            row.update({"ms_per_step": round(ms, 4), "MLUPS": round(case.nodes / ms / 1e3, 1),
                        "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4)})
        except lbfsi.LbfsiError as ex:
            row["error"] = str(ex)
        finally:
            m.close()
        out.append(row)
        del M0
    return out


def small_case_graphs(stream, steps=1000, graph_steps=100):
    """The fixed cylinder on the 128 x 64 O-grid (FP64, 1000 steps): a
    launch-bound case, timed with plain launches and with CUDA-graph replay."""
    import torch
    from paper_2107_01370_gb300 import lbfsi
    case = inputs.fixed_cylinder_128x64(steps)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    res = {"workload": case.name + ", FP64", "nodes": case.nodes, "steps": steps}
    for label, g in (("plain", 0), ("graph", graph_steps)):
        m = lbfsi.Mesh(case.r, case.e, case.bodies, precision=lbfsi.FP64, stream=stream.cuda_stream)
        m.init_fields(case.flow, M0[None])
        # the tile shape (8, 4 or 2 rows: few tiles leave SMs idle) by the tuner
        v, o, _ = m.autotune(20)
        res["schedule"] = {"variant": v, "order": o}
        m.set_graph_steps(g)
        m.step(2 * max(g, 1))   # warm-up (captures the graph)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        m.synchronize()
        ms = e0.elapsed_time(e1)
        m.close()
        res[label] = {"ms_per_step": round(ms / steps, 5), "MLUPS": round(case.nodes * steps / ms / 1e3, 1)}
    res["graph_steps"] = graph_steps
    return res


def general_mesh_cases():
    """General-mesh workloads (FP32, inputs above L2): an elliptic cylinder
    on a 512 x 256 O-grid given by node coordinates (1-DOF, batch 8); the
    airfoil case, a NACA 0012 section on a 192 x 769 C-grid (147,648 nodes,
    wake cut 128 nodes per side), 2-DOF pitch-plunge (m* 100, w_h/w_a 0.3,
    x_a 1.8, r_a 1.87, V_R 0.5025, elastic axis half a chord ahead of the
    leading edge), Ma 0.8, T_inf 0.2, Re 1e5, 1 degree forced pitching for
    two periods then free (batch 8); two cylinders in tandem on a 512 x 2049
    C-grid, rigidly linked on one DOF (one solve) and as two independent
    1-DOF bodies swept over six reduced velocities (six solves)."""
    from paper_2107_01370_gb300 import lbfsi
    ell = inputs.xy_case(inputs.ellipse_wall(256, 0.6, 0.35), 512, r_far=20.0, length=1.2,
                         body=inputs.BodySpec(dof=1, r_in=0.75, r_out=2.5, m_star=10.0, v_r=5.0,
                                              length=1.2),
                         name="elliptic cylinder (0.6 x 0.35) O-grid 512x256 by node coordinates, 1-DOF")
    cg = inputs.naca0012_flutter_case()
    linked = inputs.BodySpec(dof=1, xc=2.0, yc=0.0, xp=2.0, yp=0.0, r_in=2.7, r_out=4.5, m_star=4.0,
                             v_r=5.0, length=1.0)
    tc = inputs.tandem_case(257, 257, 255, 256, 512, body=linked,
                            name="two cylinders in tandem 4 D apart, rigidly linked (1 DOF, V_R 5), "
                                 "C-grid 512x2049 with three wall chains, Re 100, Ma 0.2")
    # the same mesh and flow, the cylinders as independent 1-DOF bodies, one
    # solve per reduced velocity of the sweep
    ti = inputs.tandem_1m_independent()
    ti.name += ", V_R swept " + "/".join(f"{v:g}" for v in inputs.TANDEM_VR_SWEEP) + " (one solve each)"
    sweep = inputs.TANDEM_VR_SWEEP
    return ((ell, lambda prec, nb, st: lbfsi.Mesh.xy(ell.X, ell.bodies * nb, precision=prec, stream=st)),
            (cg, lambda prec, nb, st: lbfsi.Mesh.cgrid(cg.X, cg.n_cut, cg.bodies * nb, precision=prec,
                                                       stream=st)),
            (tc, lambda prec, nb, st: lbfsi.Mesh.cgrid_walls(tc.X, tc.walls, tc.bodies * nb, precision=prec,
                                                             stream=st)),
            (ti, lambda prec, nb, st: lbfsi.Mesh.cgrid_walls(
                ti.X, ti.walls, [inputs.tandem_independent_pair(sweep[k % len(sweep)]) for k in range(nb)],
                precision=prec, stream=st, wall_body=ti.wall_body)))


def general_mesh_throughput(stream, peak, steps=200, warmup=5, batch=(8, 8, 1, 6), only=None):
    """MLUPS of the general-mesh step (Newton departure points, cached for
    the nodes no blend moves; stored metric) on the workloads of
    general_mesh_cases, timed with CUDA events on the library's stream; the
    C-grid step is two launches (the collision of the rows next to the cut,
    then the step).  HBM fraction against the algorithmic 144 B per node
    update."""
    import torch
    from paper_2107_01370_gb300 import lbfsi
    out = []
    for k, (case, make) in enumerate(general_mesh_cases()):
        if only is not None and k != only:
            continue
        nb = batch[k] if isinstance(batch, tuple) else batch
        M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
        m = make(lbfsi.FP32, nb, stream.cuda_stream)
        m.init_fields(case.flow, np.ascontiguousarray(np.broadcast_to(M0, (nb,) + M0.shape)))
        m.step(warmup)
        m.synchronize()
        ls = m.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        m.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ok = True
        try:
            m.synchronize()
        except lbfsi.LbfsiError as e:
            ok = str(e)
        launches = m.launch_count() - ls
        m.close()
        nodes = case.nodes * nb
        gbs = BYTES_PER_NODE_FP32 * nodes * steps / (ms * 1e-3) / 1e9
        out.append({"workload": case.name, "nodes": case.nodes, "batch": nb, "steps": steps,
                    "launches_per_step": launches // steps, "ms_per_step": round(ms / steps, 4),
                    "MLUPS": round(nodes * steps / ms / 1e3, 1),
                    "hbm_frac_of_measured": round(gbs / peak, 4), "physical": ok})
    return out


def element_mesh_throughput(stream, peak, steps=100, warmup=5, batch=8):
    """MLUPS of the step on an unstructured Q2 element list: the 1-DOF VIV
    cylinder of the bench workload on a 513 x 256 O-grid (odd radial count,
    so its 3 x 3 windows tile it) renumbered into a shuffled element list,
    FP32, gradients of the element average (reading R33); four launches per
    step, timed with CUDA events on the library's stream.  HBM fraction
    against the algorithmic 144 B per node update."""
    import torch
    from paper_2107_01370_gb300 import lbfsi
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.5, m_star=10.0, v_r=5.0)
    case = inputs.cylinder_case(513, 256, body=body)
    X = np.stack([case.r[:, None] * case.e[None, :, 0], case.r[:, None] * case.e[None, :, 1]], axis=-1)
    el = inputs.ogrid_element_list(X, seed=0)
    M0 = el.to_list(inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0))
    m = lbfsi.ElementMesh(el.X, el.elements, el.wall, el.far, case.bodies * batch, precision=lbfsi.FP32,
                          stream=stream.cuda_stream)
    m.init_fields(case.flow, np.ascontiguousarray(np.broadcast_to(M0, (batch,) + M0.shape)))
    m.step(warmup)
    m.synchronize()
    l0 = m.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    m.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ok = True
    try:
        m.synchronize()
    except lbfsi.LbfsiError as e:
        ok = str(e)
    launches = m.launch_count() - l0
    m.close()
    nodes = case.nodes * batch
    gbs = BYTES_PER_NODE_FP32 * nodes * steps / (ms * 1e-3) / 1e9
    return {"workload": "1-DOF VIV cylinder (m* 10, V_R 5, Re 100, Ma 0.2), O-grid 513x256 renumbered "
                        "into a shuffled Q2 element list, FP32, reading R33 gradients",
            "nodes": case.nodes, "batch": batch, "steps": steps, "launches_per_step": launches // steps,
            "ms_per_step": round(ms / steps, 4), "MLUPS": round(nodes * steps / ms / 1e3, 1),
            "hbm_frac_of_measured": round(gbs / peak, 4), "physical": ok}


def issue_roofline(nodes, kernel_s, sm_mhz):
    """Instruction-issue ceiling of the step kernel: warp instructions per
    node from the committed ncu capture (current source only) against one
    warp instruction per scheduler per cycle (152 SMs x 4 schedulers)."""
    p = os.path.join(ROOT, "profiles", "k_step_fp32_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha") != source_sha() or "warp_inst_per_node" not in d:
        return None
    achieved = d["warp_inst_per_node"] * nodes / kernel_s / 1e9
    peak = 152 * 4 * sm_mhz * 1e6 / 1e9
    return {"bound": "issue", "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "G warp-instructions/s", "frac": round(achieved / peak, 4),
            "warp_inst_per_node": d["warp_inst_per_node"],
            "fp32_flop_per_node": d.get("fp32_flop_per_node"),
            "peak_kind": "152 SMs x 4 schedulers x median SM clock of the timed region"}


def _reference_worker(args):
    """One oracle solve of the bounded reference sample in a spawned process:
    'warmup' untimed steps, then 'steps' timed steps."""
    root, seed, warmup, steps, rows = args
    import time as _time
    sys.path.insert(0, root)
    from paper_2107_01370_gb300 import inputs as _inputs
    import oracle.mesh as OM
    import oracle.solver as OS
    import bench as _bench
    case = _bench.reference_sample_case(rows)
    M0 = _inputs.initial_field(case.nr, case.ntheta, case.flow, seed=seed)
    s = OS.Solver.from_case(OM.ogrid_mesh(case.r, case.e), case, M0)
    for _ in range(warmup):
        s.step()
    t = _time.perf_counter()
    for _ in range(steps):
        s.step()
    return _time.perf_counter() - t, case.nodes


def run_reference(args):
    """The oracle timed on the host cores, same metric and workload: one
    independent oracle solve of the bounded sample (reference_sample_case)
    per core, as the GPU arm runs a batch of independent solves; the slowest
    worker's time is the batch's time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp
    cores = max(1, min(16, os.cpu_count() or 1))
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    rows = reference_rows(args.steps, args.warmup)
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_reference_worker, [(ROOT, k, args.warmup, args.steps, rows) for k in range(cores)])
    dt = max(r[0] for r in res)
    nodes = sum(r[1] for r in res)
    value = nodes * args.steps / dt / 1e6
    sample = (f"{cores} independent oracle solves (FP64 numpy, one spawned process and one thread "
              f"each) of the first {rows} radial rows x 256 angular nodes ({rows * 256} "
              f"nodes) of the 512x256 VIV solve (rows sized to the step count); "
              f"{args.steps} timed steps each")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": workload_name(cores) + " (oracle sample)", "l2": "host run"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default tile shape and CTA order")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 1-16 M-node roofline sweep and the small FP64 case")
    ap.add_argument("--schedule", default=None,
                    help="'variant,order': fixed tile shape and CTA order instead of the autotuner")
    ap.add_argument("--general-only", type=int, default=None, choices=[0, 1, 2, 3],
                    help="time only one general-mesh workload (0: O-grid by coordinates, 1: NACA C-grid, "
                         "2: linked tandem cylinders, 3: independent tandem cylinders) "
                         "with --steps, --warmup and --batch, print its JSON and exit")
    ap.add_argument("--elements-only", action="store_true",
                    help="time only the unstructured element-list workload with --steps, --warmup and "
                         "--batch, print its JSON and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    from paper_2107_01370_gb300 import build, lbfsi
    if not os.path.exists(lbfsi.LIB_PATH):
        build.build()
    lbfsi.load()

    if args.general_only is not None:
        peak, _ = measured_peaks()
        res = general_mesh_throughput(torch.cuda.Stream(device=dev), peak, steps=args.steps,
                                      warmup=args.warmup, batch=args.batch, only=args.general_only)
        print(json.dumps(res[0]), flush=True)
        return

    if args.elements_only:
        peak, _ = measured_peaks()
        res = element_mesh_throughput(torch.cuda.Stream(device=dev), peak, steps=args.steps,
                                      warmup=args.warmup, batch=args.batch)
        print(json.dumps(res), flush=True)
        return

    case = inputs.viv_cylinder_512x256()
    B = args.batch
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=rank)
    M0b = np.ascontiguousarray(np.broadcast_to(M0, (B,) + M0.shape))
    stream = torch.cuda.Stream(device=dev)
    mesh = lbfsi.Mesh(case.r, case.e, case.bodies * B, precision=lbfsi.FP32,
                      stream=stream.cuda_stream)
    mesh.init_fields(case.flow, M0b)
    # untimed: the autotuner picks the tile shape and CTA order on this GPU
    # (its trial steps are real steps of the solves, so they count as warm-up)
    tuned = None
    if args.schedule:
        mesh.set_schedule(*[int(x) for x in args.schedule.split(",")])
    elif not args.no_tune:
        v, o, ms = mesh.autotune(steps_per_trial=20)
        tuned = {"variant": v, "order": o, "ms_per_step_by_variant_order": np.round(ms, 4).tolist()}
    mesh.step(args.warmup)
    mesh.synchronize()
    variant, order = mesh.schedule()

    sampler = ClockSampler(dev)
    sampler.start()
    time.sleep(0.4)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = mesh.launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        mesh.step(1)
        ev[k][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = mesh.launch_count() - l0
    mesh.synchronize()   # raises if the kernels flagged an error
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    region_ms = t_start.elapsed_time(t_end)
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    # replicas: every rank advanced its own batch; the time is the slowest
    # rank's, the work is that of all ranks
    region_ms = replicas.max_over_ranks(region_ms, dist, device="cuda")
    nodes = case.nodes * B
    value = replicas.aggregate_mlups(replicas.sum_over_ranks(nodes * args.steps, dist, device="cuda"),
                                     region_ms * 1e-3)
    kavg_s = statistics.mean(kern_ms) * 1e-3
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_NODE_FP32 * nodes / kavg_s / 1e9
    tpn = traffic_per_node()
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": None if tpn is None else round(tpn * nodes),
                "peak_kind": peak_kind, "kernel": KERNEL,
                "algorithmic_bytes_per_launch": BYTES_PER_NODE_FP32 * nodes,
                "kernel_ms": round(kavg_s * 1e3, 4)}

    e2e = None
    if not args.no_e2e:
        # end to end through the C ABI with host buffers: upload the initial
        # fields, K coupled steps with the loads read back to the host after
        # every step, download the final fields.
        K = args.steps
        m2 = lbfsi.Mesh(case.r, case.e, case.bodies * B, precision=lbfsi.FP32,
                        stream=stream.cuda_stream)
        m2.set_schedule(variant, order)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        m2.init_fields(case.flow, M0b)
        hist, states = m2.step_record(K, states=True)
        fields = m2.get_fields()
        t1 = time.perf_counter()
        el = replicas.max_over_ranks(t1 - t0, dist, device="cuda")
        per_step_d2h = hist[0].nbytes + states[0].nbytes
        e2e = {"value": nodes * world * K / el / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(M0b.nbytes / K),
               "d2h_bytes_per_step": int(fields.nbytes / K + per_step_d2h),
               "note": "init_fields upload, every step's loads and body states copied to the host "
                       "behind its launch (lbfsi_step_record), final get_fields"}
        m2.close()
        del fields

    sweep = small = general = elements = None
    if not args.no_sweep and world == 1:
        sweep = roofline_sweep(stream, (variant, order), peak)
        small = small_case_graphs(stream)
        general = general_mesh_throughput(stream, peak)
        elements = element_mesh_throughput(stream, peak)
    issue = issue_roofline(nodes, kavg_s, clocks.get("sm_mhz") or 2070.0) if clocks else None

    serving_out = None
    if not args.no_serving and world == 1:
        serving_out = serving_bench(stream.cuda_stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample()

    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": round(region_ms / args.steps, 4), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": workload_name(B), "nodes_per_gpu": nodes, "batch": B,
                          "mesh": "O-grid 512x256, r 0.5..20 D", "steps_per_solve": case.steps,
                          "l2": "inputs larger than L2 (ping-pong populations "
                                f"{BYTES_PER_NODE_FP32 * nodes / 1e6:.0f} MB)",
                          "parallelism": f"replicas x{world}",
                          "schedule": {"variant": variant, "order": order, "autotuner": tuned}},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "clocks": clocks, "serving": serving_out,
               "issue_roofline": issue, "roofline_sweep": sweep, "small_case": small,
               "general_meshes": general, "element_mesh": elements,
               "solves_per_s": round(B * world / (case.steps * region_ms / args.steps * 1e-3), 4)}
        print(json.dumps(out), flush=True)
    mesh.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
