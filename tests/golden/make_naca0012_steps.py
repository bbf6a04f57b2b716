"""Writes naca0012_steps.json: the oracle's first three coupled steps on the
full-size transonic flutter workload (NACA 0012 on the 192 x 769 C-grid,
2-DOF pitch-plunge with forced pitching, Ma 0.8; readings R28-R30), sampled.
Calls only the oracle and the seeded input generators; about a minute of CPU.

    python tests/golden/make_naca0012_steps.py

Stored: the sample nodes, the moment field there after the third step, the
field's scales (max |rho|, max |u|, max |T| over the whole mesh), the load of
every step and the body state after the third step."""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))

import oracle.mesh as OM  # noqa: E402
import oracle.solver as OS  # noqa: E402
from paper_2107_01370_gb300 import inputs  # noqa: E402

STEPS = 3


def samples(nr, nt, n_cut):
    rng = np.random.default_rng(12)
    pts = {(int(i), int(j)) for i, j in zip(rng.integers(0, nr, 448), rng.integers(0, nt, 448))}
    pts |= {(0, j) for j in range(0, nt, 16)}
    pts |= {(0, n_cut), (0, nt - 1 - n_cut), (1, n_cut), (2, n_cut), (0, (nt - 1) // 2)}
    pts |= {(nr - 1, j) for j in range(0, nt, 128)} | {(i, 0) for i in range(0, nr, 32)}
    return sorted(pts)


def main():
    case = inputs.naca0012_flutter_case()
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    s = OS.Solver.from_case(OM.CGridMesh(case.X, case.n_cut), case, M0)
    loads = []
    for _ in range(STEPS):
        r = s.step()
        loads.append(list(map(float, r.force)))
    pts = samples(case.nr, case.ntheta, case.n_cut)
    M = r.M
    data = {
        "workload": case.name,
        "what": "oracle (FP64) after three coupled steps from the seeded initial field (seed 0), the "
                "body at rest with its pitch forced; readings R28-R30 (C-grid), Sec. IV D forcing",
        "command": "python tests/golden/make_naca0012_steps.py",
        "steps": STEPS,
        "samples": pts,
        "M": [[float(M[c, i, j]) for c in range(4)] for i, j in pts],
        "scale": [float(np.abs(M[0]).max()), float(np.hypot(M[1], M[2]).max()), float(np.abs(M[3]).max())],
        "loads": loads,
        "state": [float(s.S[0][k]) for k in ("h", "alpha", "hdot", "adot")],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "naca0012_steps.json")
    with open(path, "w") as fh:
        json.dump(data, fh, indent=0)
    print(path, len(pts), "samples")


if __name__ == "__main__":
    main()
