"""Accuracy of the FP32 path (FP32 populations and collision; FP64 for the
wall-load reduction, the body ODE and the blended maps) against the FP64
oracle over long runs, in the units the result is used in:

  fields   max over the sampled nodes of |gpu - oracle| / max |oracle| for
           rho and T, the Euclidean norm of the velocity difference over
           max |u| for the velocity (the scales are the oracle's, over the
           whole mesh);
  C_D      |dC_D| / |C_D| at every step;
  C_L      |dC_L| / max_t |C_L|, the lift's amplitude so far;
  h        |dh| / max_t |h|, the displacement's amplitude so far;
  M_z      like C_L.

The expected values are stored oracle runs (tests/golden/, written by
committed scripts that call only the oracle): the fixed cylinder's full
1000 steps on the 128 x 64 O-grid, and the first 1000 steps of the 1-DOF VIV
workload on the 512 x 256 O-grid.  The FP64 path is held to the oracle as
well over the same runs.
"""
import json
import os

import numpy as np
import pytest

from paper_2107_01370_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def lbfsi():
    from paper_2107_01370_gb300 import build, lbfsi as L
    build.build()
    L.load()
    return L


def _load(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def _sample_err(M, gold, n):
    """Relative errors (rho, |u|, T) of the GPU field M [4, nr, nt] at the
    golden's sampled nodes after step n."""
    pts = np.array(gold["samples"])
    ref = np.array(gold["fields"][str(n)])          # [npts, 4]
    got = M[:, pts[:, 0], pts[:, 1]].T
    s_rho, s_u, s_T = gold["scale"][str(n)]
    return (np.abs(got[:, 0] - ref[:, 0]).max() / s_rho,
            np.hypot(got[:, 1] - ref[:, 1], got[:, 2] - ref[:, 2]).max() / s_u,
            np.abs(got[:, 3] - ref[:, 3]).max() / s_T)


def _coefficient_errors(loads, gold_loads, qd):
    """|dC_D|/|C_D| (max over steps), |dC_L| / max|C_L| and the moment's
    likewise, over the steps given."""
    a = np.asarray(loads) / qd
    b = np.asarray(gold_loads) / qd
    cd = np.abs(a[:, 0] - b[:, 0]) / np.abs(b[:, 0])
    cl = np.abs(a[:, 1] - b[:, 1]).max() / np.abs(b[:, 1]).max()
    return cd.max(), cl


def _run(L, case, precision, checks, nbatch=1):
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    mesh = L.Mesh(case.r, case.e, case.bodies * nbatch, precision=precision)
    mesh.init_fields(case.flow, np.ascontiguousarray(np.broadcast_to(M0, (nbatch,) + M0.shape)))
    loads, states, fields = [], [], {}
    done = 0
    for n in checks:
        ld, st = mesh.step_record(n - done, states=True)
        loads.append(ld)
        states.append(st)
        fields[n] = mesh.get_fields()
        done = n
    mesh.close()
    return np.concatenate(loads), np.concatenate(states), fields


def test_fixed_cylinder_full_run_fp32_and_fp64(lbfsi):
    """Fixed cylinder, O-grid 128 x 64, Re 100, Ma 0.2: the workload's whole
    1000 steps.  FP32: fields within 1e-5 at every checkpoint up to 1000
    steps, C_D within 1e-4 relative at every step.  FP64: fields within
    1e-11 and loads within 1e-11 p_inf D after 1000 steps."""
    gold = _load("fixed128_steps.json")
    case = inputs.fixed_cylinder_128x64()
    qd = gold["q_inf_d"]
    checks = gold["check"]
    for prec in (lbfsi.FP32, lbfsi.FP64):
        loads, _, fields = _run(lbfsi, case, prec, checks)
        for n in checks:
            e = _sample_err(fields[n][0], gold, n)
            if prec == lbfsi.FP32:
                assert max(e) < 1e-5, (n, e)
            else:
                assert max(e) < 1e-11, (n, e)
        if prec == lbfsi.FP32:
            cd, _ = _coefficient_errors(loads[:, 0], gold["loads"], qd)
            assert cd < 1e-4, cd
        else:
            assert np.abs(loads[:, 0] - np.array(gold["loads"])).max() < 1e-11 / 3.0
