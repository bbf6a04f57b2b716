"""Writes tandem_1m_step1.json: the oracle's first coupled step on the full-size
tandem workload (two cylinders 4 D apart as independent 1-DOF bodies on the
512 x 2049 C-grid, readings R31-R32), sampled.  Calls only the oracle and the
seeded input generators; about two minutes of CPU.

    python tests/golden/make_tandem_1m_step1.py

Stored: the sample nodes, the moment field there after the step, the field's
scales (max |rho|, max |u|, max |T| over the whole mesh), each body's load and,
for every reduced velocity of the sweep, the bodies' states after the RK4
update with those loads (the flow of the step does not depend on V_R)."""
import json
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))

import oracle.mesh as OM  # noqa: E402
import oracle.solver as OS  # noqa: E402
import oracle.structure as ST  # noqa: E402
from paper_2107_01370_gb300 import inputs  # noqa: E402

# initial body states (front, rear) and the states one step earlier (V_G)
STATES = [{"h": 0.01, "alpha": 0.0, "hdot": 0.002, "adot": 0.0},
          {"h": -0.005, "alpha": 0.0, "hdot": -0.001, "adot": 0.0}]


def prev_states(dt):
    return [dict(s, h=s["h"] - s["hdot"] * dt) for s in STATES]


def samples(nr, nt, walls):
    rng = np.random.default_rng(2107)
    pts = {(int(i), int(j)) for i, j in zip(rng.integers(0, nr, 448), rng.integers(0, nt, 448))}
    pts |= {(0, j) for j in range(0, nt, 32)}
    pts |= {(0, a) for a, b in walls} | {(0, b) for a, b in walls}
    pts |= {(1, a) for a, b in walls} | {(nr - 1, j) for j in range(0, nt, 256)}
    return sorted(pts)


def main():
    case = inputs.tandem_1m_independent()
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    mesh = OM.CGridMesh(case.X, walls=case.walls, wall_body=case.wall_body)
    s = OS.Solver.from_case(mesh, case, M0)
    s.S = [dict(x) for x in STATES]
    s.S_prev = prev_states(case.flow.dt)
    r = s.step()
    pts = samples(case.nr, case.ntheta, case.walls)
    M = r.M
    u_inf = case.flow.ma * math.sqrt(case.flow.gamma * case.flow.t_inf)
    states = {}
    for v in inputs.TANDEM_VR_SWEEP:
        out = []
        for spec, st, F in zip(inputs.tandem_independent_pair(v), STATES, r.forces):
            b = OS.body_dict(spec, case.flow.rho_inf, u_inf)
            h, hdot = ST.advance_one_dof(st["h"], st["hdot"], F[1], b["m"], b["k"], b["c"], case.flow.dt)
            out.append([h, 0.0, hdot, 0.0])
        states[repr(v)] = out
    data = {
        "workload": case.name,
        "what": "oracle (FP64) after one coupled step from the seeded initial field (seed 0) with the "
                "body states below; readings R31-R32 (Sec. II D blended maps, Sec. III loads and RK4)",
        "command": "python tests/golden/make_tandem_1m_step1.py",
        "initial_states": STATES,
        "samples": pts,
        "M": [[float(M[c, i, j]) for c in range(4)] for i, j in pts],
        "scale": [float(np.abs(M[0]).max()), float(np.hypot(M[1], M[2]).max()), float(np.abs(M[3]).max())],
        "loads": [list(map(float, F)) for F in r.forces],
        "states": states,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tandem_1m_step1.json")
    with open(path, "w") as fh:
        json.dump(data, fh, indent=0)
    print(path, len(pts), "samples")


if __name__ == "__main__":
    main()
