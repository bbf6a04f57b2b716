"""Request loop of the batch runtime: FSI solves arrive over time, are
admitted into the device memory pool as room frees up, advance together (one
launch per step covering every active solve), and leave when finished.

The loop itself is host bookkeeping only: admission, stepping and retirement
are calls of the C ABI (lbfsi_batch_*); every step of the method runs in the
library's kernels.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import inputs, lbfsi

SIZES = ((64, 32), (128, 64), (256, 128), (512, 256))


@dataclass
class Request:
    rid: int
    nr: int
    ntheta: int
    v_r: float
    m_star: float
    steps: int
    arrival: float = 0.0


def viv_requests(n=256, steps=2000, seed=0):
    """Independent cylinder-VIV requests: O-grid size uniform over SIZES,
    reduced velocity uniform in [3, 8], mass ratio uniform in [2, 20]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nr, nt = SIZES[rng.integers(len(SIZES))]
        out.append(Request(k, nr, nt, float(rng.uniform(3.0, 8.0)), float(rng.uniform(2.0, 20.0)),
                           steps))
    return out


class CaseCache:
    """Mesh tables, flow and initial field per request (tables shared per size)."""

    def __init__(self):
        self._meshes = {}

    def case(self, req: Request):
        key = (req.nr, req.ntheta)
        if key not in self._meshes:
            self._meshes[key] = inputs.cylinder_case(req.nr, req.ntheta)
        base = self._meshes[key]
        body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.5, m_star=req.m_star, v_r=req.v_r)
        M0 = inputs.initial_field(req.nr, req.ntheta, base.flow, seed=req.rid)
        return base, body, M0


def tune_schedule(pool_bytes, precision=lbfsi.FP32, stream=None, cache=None, steps_per_trial=10,
                  seed=12345):
    """Tile shape and CTA order for the serving mix, from the batch
    autotuner run on a small mix of the request sizes (two of each)."""
    cache = cache or CaseCache()
    batch = lbfsi.Batch(pool_bytes, precision=precision, stream=stream)
    rng = np.random.default_rng(seed)
    trial_steps = 2 * lbfsi.step_variants(precision) * (1 + steps_per_trial) + 1
    for k, (nr, nt) in enumerate(SIZES * 2):
        req = Request(10 ** 6 + k, nr, nt, float(rng.uniform(3, 8)), float(rng.uniform(2, 20)), trial_steps)
        base, body, M0 = cache.case(req)
        if batch.add(base.r, base.e, body, base.flow, req.steps, M0) is None:
            break
    v, o, _ = batch.autotune(steps_per_trial)
    batch.close()
    return v, o


def run_batched(reqs, pool_bytes, precision=lbfsi.FP32, chunk=50, stream=None, cache=None,
                clock=time.perf_counter, schedule=None):
    """Serve the requests in arrival order with continuous batching (tile
    shape and CTA order 'schedule', else the default).  Returns per-request
    (arrival, completion) times relative to the start, the final loads of
    each request and the wall time."""
    cache = cache or CaseCache()
    batch = lbfsi.Batch(pool_bytes, precision=precision, stream=stream)
    if schedule is not None:
        batch.set_schedule(*schedule)
    pending = sorted(reqs, key=lambda r: r.arrival)
    active = {}
    done = {}
    loads = {}
    peak_active = 0
    t0 = clock()
    i = 0
    while i < len(pending) or active:
        now = clock() - t0
        while i < len(pending) and pending[i].arrival <= now:
            req = pending[i]
            base, body, M0 = cache.case(req)
            slot = batch.add(base.r, base.e, body, base.flow, req.steps, M0)
            if slot is None:
                break                     # no room: wait for a solve to leave
            active[slot] = req
            i += 1
        peak_active = max(peak_active, len(active))
        if not active:
            if i < len(pending):
                time.sleep(max(0.0, min(pending[i].arrival - now, 0.01)))
            continue
        batch.step(chunk)
        for slot in list(active):
            _, fin = batch.poll(slot)
            if fin:
                _, ld, _ = batch.get(slot, fields=False)
                req = active.pop(slot)
                done[req.rid] = (req.arrival, clock() - t0)
                loads[req.rid] = ld
                batch.remove(slot)
    wall = clock() - t0
    batch.close()
    return done, loads, wall, peak_active


def run_sequential(reqs, precision=lbfsi.FP32, stream=None, cache=None, clock=time.perf_counter,
                   schedule=None):
    """The same requests one at a time, each a plain single-mesh solve (with
    the tile shape of 'schedule' when given)."""
    cache = cache or CaseCache()
    done = {}
    loads = {}
    t0 = clock()
    for req in reqs:
        base, body, M0 = cache.case(req)
        mesh = lbfsi.Mesh(base.r, base.e, [body], precision=precision, stream=stream)
        if schedule is not None:
            mesh.set_schedule(*schedule)
        mesh.init_fields(base.flow, M0[None])
        mesh.step(req.steps)
        loads[req.rid] = mesh.body_forces()[0]
        mesh.close()
        done[req.rid] = (0.0, clock() - t0)
    return done, loads, clock() - t0


def poisson_arrivals(reqs, rate, seed=1):
    rng = np.random.default_rng(seed)
    t = 0.0
    for r in reqs:
        t += rng.exponential(1.0 / rate)
        r.arrival = t
    return reqs


def latency_stats(done):
    lat = np.array([c - a for a, c in done.values()])
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))
