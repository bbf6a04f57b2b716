"""Writes fixed128_steps.json: the oracle's run of the fixed-cylinder workload
(O-grid 128 x 64, Re 100, Ma 0.2, seeded noise) over its full 1000 steps,
against which the GPU tests state the FP32 path's accuracy at several step
counts.  Calls only the oracle and the seeded input generators; about four
minutes of one CPU core.

    python tests/golden/make_fixed128_steps.py

Stored: every step's load (F_x, F_y, M_z); the moment field at sampled
nodes after steps CHECK; the field's scales (max
|rho|, max |u|, max |T| over the whole mesh) at those steps."""
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))

import oracle.mesh as OM  # noqa: E402
import oracle.solver as OS  # noqa: E402
from paper_2107_01370_gb300 import inputs  # noqa: E402

STEPS = 1000
CHECK = (60, 150, 300, 600, 1000)


def samples(nr, nt):
    rng = np.random.default_rng(22)
    pts = {(int(i), int(j)) for i, j in zip(rng.integers(0, nr, 400), rng.integers(0, nt, 400))}
    pts |= {(0, j) for j in range(0, nt, 2)} | {(1, j) for j in range(0, nt, 8)}
    pts |= {(i, 0) for i in range(0, nr, 8)} | {(i, nt // 2) for i in range(0, nr, 8)}
    pts |= {(nr - 1, j) for j in range(0, nt, 4)} | {(nr - 2, j) for j in range(0, nt, 8)}
    return sorted(pts)


def main():
    case = inputs.fixed_cylinder_128x64()
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    s = OS.Solver.from_case(OM.ogrid_mesh(case.r, case.e), case, M0)
    pts = samples(case.nr, case.ntheta)
    ii = np.array([p[0] for p in pts])
    jj = np.array([p[1] for p in pts])
    loads, states, fields, scales = [], [], {}, {}
    t0 = time.time()
    for n in range(1, STEPS + 1):
        r = s.step()
        loads.append([float(v) for v in r.force])
        states.append([float(s.S[0]["h"]), float(s.S[0]["hdot"])])
        if n in CHECK:
            M = r.M
            fields[str(n)] = M[:, ii, jj].T.tolist()
            scales[str(n)] = [float(np.abs(M[0]).max()), float(np.hypot(M[1], M[2]).max()),
                              float(np.abs(M[3]).max())]
        if n % 50 == 0:
            print(f"step {n}: {time.time() - t0:.0f} s", flush=True)
    data = {
        "workload": case.name,
        "what": "oracle (FP64) steps of the fixed cylinder from the seeded initial field (seed 0)",
        "command": "python tests/golden/make_fixed128_steps.py",
        "steps": STEPS,
        "check": list(CHECK),
        "samples": pts,
        "fields": fields,
        "scale": scales,
        "loads": loads,
        "states": states,
        "q_inf_d": 0.5 * case.flow.rho_inf * case.flow.u_inf ** 2 * case.flow.length,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fixed128_steps.json")
    with open(path, "w") as fh:
        json.dump(data, fh, indent=0)
    print(path, len(pts), "samples")


if __name__ == "__main__":
    main()
