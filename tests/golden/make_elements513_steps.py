"""Writes elements513_steps.json: the oracle's first STEPS coupled steps on the
element-list workload of the bench (the 1-DOF VIV cylinder, m* 10, V_R 5,
Re 100, Ma 0.2, on a 513 x 256 O-grid renumbered into a shuffled Q2 element
list, seed 0; gradients of reading R33).  Calls only the oracle and the
seeded input generators; about two minutes of one CPU core.

    python tests/golden/make_elements513_steps.py

Stored: every step's load (F_x, F_y, M_z) and body state (h, hdot); the
moment field at sampled nodes (indices of the element list) after steps
CHECK; the field's scales (max |rho|, max |u|, max |T| over the whole mesh)
at those steps."""
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))

import oracle.unstructured as OU  # noqa: E402
from paper_2107_01370_gb300 import inputs  # noqa: E402

STEPS = 20
CHECK = (5, 20)


def workload():
    """The element list, the case and the initial field of the bench's
    element-list workload (list numbering)."""
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.5, m_star=10.0, v_r=5.0)
    case = inputs.cylinder_case(513, 256, body=body)
    X = np.stack([case.r[:, None] * case.e[None, :, 0], case.r[:, None] * case.e[None, :, 1]], axis=-1)
    el = inputs.ogrid_element_list(X, seed=0)
    M0 = el.to_list(inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0))
    return case, el, M0


def samples(el):
    """Sampled list indices: random nodes, the wall and far-field chains
    (every 8th / 16th node) and the rows next to them."""
    rng = np.random.default_rng(23)
    N = el.X.shape[0]
    pts = set(int(v) for v in rng.integers(0, N, 400))
    pts |= set(int(v) for v in np.asarray(el.wall)[::8]) | set(int(v) for v in np.asarray(el.far)[::16])
    nr, nt = el.nr, el.nt
    grid = np.asarray(el.grid_ij)
    for row in (1, 2, nr - 2):
        at = np.nonzero(grid[:, 0] == row)[0]
        pts |= set(int(v) for v in at[::16])
    return sorted(pts)


def main():
    case, el, M0 = workload()
    um = OU.UnstructuredQ2Mesh(el.X, el.elements)
    s = OU.UnstructuredSolver.from_case(um, el.wall, el.far, case, M0)
    pts = samples(el)
    loads, states, fields, scales = [], [], {}, {}
    t0 = time.time()
    for n in range(1, STEPS + 1):
        r = s.step()
        loads.append([float(v) for v in r.force])
        states.append([float(s.S[0]["h"]), float(s.S[0]["hdot"])])
        if n in CHECK:
            M = r.M
            fields[str(n)] = M[:, pts].T.tolist()
            scales[str(n)] = [float(np.abs(M[0]).max()), float(np.hypot(M[1], M[2]).max()),
                              float(np.abs(M[3]).max())]
        print(f"step {n}: {time.time() - t0:.0f} s", flush=True)
    flow = case.flow
    data = {
        "workload": "1-DOF VIV cylinder (m* 10, V_R 5, Re 100, Ma 0.2), O-grid 513x256 renumbered into a "
                    "shuffled Q2 element list (seed 0), reading R33 gradients",
        "what": "oracle (FP64) coupled steps on the element list from the seeded initial field (seed 0), "
                "the body at rest",
        "steps": STEPS,
        "check": list(CHECK),
        "samples": pts,
        "q_inf_d": 0.5 * flow.rho_inf * flow.u_inf ** 2 * flow.length,
        "loads": loads,
        "states": states,
        "fields": fields,
        "scale": scales,
    }
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "elements513_steps.json")
    with open(out, "w") as fh:
        json.dump(data, fh)
    print("wrote", out)


if __name__ == "__main__":
    main()
