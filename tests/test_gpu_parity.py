"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs.

Tolerances (relative error of a field = max over nodes of |gpu - oracle|
divided by max over nodes of |oracle|, for rho and T; for the velocity the
Euclidean norm of the vector u at each node is used in both places):
  FP64 path   fields, populations <= 1e-12 (and the velocity of the four
              rows next to the wall within 1e-10 of its own magnitude at
              every node); loads: |dF| <= 1e-12 * p_inf * D
              (the scale of the pressure terms whose sum the load is, so
              cancellation in small lift values does not inflate a relative
              error); body states 1e-12 relative to their scale.
  FP32 path   fields <= 1e-5 after 60 and 150 steps of the impulsive start
              of the 128 x 64 cylinder (longer runs: test_gpu_fp32_accuracy.py);
              loads <= 1e-4 * p_inf * D.
"""
import numpy as np
import pytest

import oracle.mesh as OM
import oracle.solver as OS
from paper_2107_01370_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbfsi():
    from paper_2107_01370_gb300 import build, lbfsi as L
    build.build()
    L.load()
    return L


def field_err(a, b):
    """max of the relative errors of rho, |u| (vector) and T."""
    e_rho = np.abs(a[0] - b[0]).max() / np.abs(b[0]).max()
    e_u = np.hypot(a[1] - b[1], a[2] - b[2]).max() / np.hypot(b[1], b[2]).max()
    e_T = np.abs(a[3] - b[3]).max() / np.abs(b[3]).max()
    return max(e_rho, e_u, e_T)


def near_wall_velocity_err(a, b, rows=4):
    """Node-wise relative error of the velocity vector on the first rows
    (the wall and the three rows above it), where the speed is far below
    the free stream's and the field-wide scale would hide an error: max over
    those nodes of |u_gpu - u_oracle| / |u_oracle| (nodes slower than 1e-9
    excluded)."""
    du = np.hypot(a[1, :rows] - b[1, :rows], a[2, :rows] - b[2, :rows])
    sp = np.hypot(b[1, :rows], b[2, :rows])
    ok = sp > 1e-9
    return (du[ok] / sp[ok]).max()


def run_oracle(case, M0, steps, state=None, prev=None):
    s = OS.Solver.from_case(OM.ogrid_mesh(case.r, case.e), case, M0)
    if state is not None:
        s.S = [dict(state)]
        s.S_prev = [dict(prev if prev is not None else state)]
    hist = []
    for _ in range(steps):
        r = s.step()
        hist.append(r.force)
    return s, r, np.array(hist)


def run_gpu(L, case, M0, steps, precision, state=None, prev=None, per_step_loads=False):
    mesh = L.Mesh(case.r, case.e, case.bodies, precision=precision)
    mesh.init_fields(case.flow, M0[None])
    if state is not None:
        to = lambda d: (d["h"], d["alpha"], d["hdot"], d["adot"])
        mesh.blend_mesh([to(state)], None if prev is None else [to(prev)])
    hist = []
    if per_step_loads:
        for _ in range(steps):
            mesh.step(1)
            hist.append(mesh.body_forces()[0].copy())
    else:
        mesh.step(steps)
        hist.append(mesh.body_forces()[0].copy())
    return mesh, np.array(hist)


P_SCALE = 1.0 / 3.0   # p_inf * D


def test_fp64_fixed_cylinder_128x64(lbfsi):
    """Fixed cylinder, O-grid 128 x 64, Re 100, Ma 0.2, seeded noise: every
    field, the post-propagation and post-collision populations and the loads
    of every step match the oracle."""
    case = inputs.fixed_cylinder_128x64(steps=12)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    s, r, hist = run_oracle(case, M0, case.steps)
    mesh, ghist = run_gpu(lbfsi, case, M0, case.steps, lbfsi.FP64, per_step_loads=True)
    assert field_err(mesh.get_fields()[0], r.M) < 1e-12
    assert near_wall_velocity_err(mesh.get_fields()[0], r.M) < 1e-10
    f0, g0 = mesh.get_populations(0)
    last = case.nr - 1
    assert np.abs(f0[0, :, :last] - r.f_pre[:, :last]).max() < 1e-12 * np.abs(r.f_pre).max()
    assert np.abs(g0[0, :, :last] - r.g_pre[:, :last]).max() < 1e-12 * np.abs(r.g_pre).max()
    f1, g1 = mesh.get_populations(1)
    assert np.abs(f1[0] - r.f_post).max() < 1e-12 * np.abs(r.f_post).max()
    assert np.abs(g1[0] - r.g_post).max() < 1e-12 * np.abs(r.g_post).max()
    assert np.abs(ghist - hist).max() < 1e-12 * P_SCALE
    assert mesh.launch_count() >= case.steps


@pytest.mark.parametrize("dof", [1, 2])
def test_fp64_moving_body_blended_mesh(lbfsi, dof):
    """Moving body from the first step (initial plunge/pitch and rates), so the
    blended map, V_G, g != I, the moving-wall Grad targets, the rotated wall
    loads and the RK4 of the 1-DOF / 2-DOF models are all exercised."""
    if dof == 1:
        body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=2.0, v_r=4.0)
        state = {"h": 0.02, "alpha": 0.0, "hdot": 0.004, "adot": 0.0}
        prev = {"h": 0.0199, "alpha": 0.0, "hdot": 0.004, "adot": 0.0}
    else:
        body = inputs.BodySpec(dof=2, xp=-0.25, yp=0.0, r_in=0.75, r_out=2.0, m_star=5.0, v_r=2.0,
                               x_alpha=0.3, r_alpha=0.6, wh_wa=0.5)
        state = {"h": -0.01, "alpha": 0.03, "hdot": 0.0, "adot": 0.01}
        prev = {"h": -0.0101, "alpha": 0.0299, "hdot": 0.0, "adot": 0.01}
    case = inputs.cylinder_case(48, 64, r_far=8.0, body=body, steps=10)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=3)
    s, r, hist = run_oracle(case, M0, case.steps, state, prev)
    mesh, ghist = run_gpu(lbfsi, case, M0, case.steps, lbfsi.FP64, state, prev, per_step_loads=True)
    assert field_err(mesh.get_fields()[0], r.M) < 1e-12
    assert near_wall_velocity_err(mesh.get_fields()[0], r.M) < 1e-10
    f1, g1 = mesh.get_populations(1)
    assert np.abs(f1[0] - r.f_post).max() < 1e-12 * np.abs(r.f_post).max()
    assert np.abs(ghist - hist).max() < 1e-12 * P_SCALE
    st = mesh.body_state()[0]
    for k in ("h", "alpha", "hdot", "adot"):
        assert abs(st[k] - s.S[0][k]) < 1e-12 * (1 + abs(s.S[0][k])), k


@pytest.mark.parametrize("nr,nt", [(21, 40), (16, 8), (33, 96)])
def test_fp64_ragged_and_tiny_meshes(lbfsi, nr, nt):
    """Odd radial count (no clamped window), angular counts that are not a
    multiple of the 32-node tile and a ring smaller than one tile."""
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=3.0, v_r=5.0)
    case = inputs.cylinder_case(nr, nt, r_far=10.0, body=body, steps=5)
    M0 = inputs.initial_field(nr, nt, case.flow, seed=nr + nt)
    state = {"h": 0.01, "alpha": 0.0, "hdot": 0.0, "adot": 0.0}
    s, r, hist = run_oracle(case, M0, case.steps, state)
    mesh, ghist = run_gpu(lbfsi, case, M0, case.steps, lbfsi.FP64, state)
    assert field_err(mesh.get_fields()[0], r.M) < 1e-12
    assert np.abs(ghist[-1] - hist[-1]).max() < 1e-12 * P_SCALE


def test_fp64_batch_equals_individual_runs(lbfsi):
    """Independent solves batched in one launch give each solve's own result."""
    bodies = [inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=ms, v_r=vr)
              for ms, vr in ((2.0, 3.0), (10.0, 5.0), (5.0, 8.0))]
    case = inputs.cylinder_case(24, 32, r_far=8.0, steps=6)
    M0s = [inputs.initial_field(24, 32, case.flow, seed=10 + k) for k in range(3)]
    mesh = lbfsi.Mesh(case.r, case.e, bodies, precision=lbfsi.FP64)
    mesh.init_fields(case.flow, np.stack(M0s))
    mesh.step(case.steps)
    fields = mesh.get_fields()
    loads = mesh.body_forces()
    states = mesh.body_state()
    for k in range(3):
        case.bodies = [bodies[k]]
        s, r, hist = run_oracle(case, M0s[k], case.steps)
        assert field_err(fields[k], r.M) < 1e-12
        assert np.abs(loads[k] - hist[-1]).max() < 1e-12 * P_SCALE
        assert abs(states[k]["h"] - s.S[0]["h"]) < 1e-12


def test_fp32_fixed_cylinder_within_stated_tolerance(lbfsi):
    case = inputs.fixed_cylinder_128x64()
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    s = OS.Solver.from_case(OM.ogrid_mesh(case.r, case.e), case, M0)
    mesh = lbfsi.Mesh(case.r, case.e, case.bodies, precision=lbfsi.FP32)
    mesh.init_fields(case.flow, M0[None])
    done = 0
    for steps, tol in ((60, 1e-5), (150, 1e-5)):
        for _ in range(steps - done):
            r = s.step()
        mesh.step(steps - done)
        done = steps
        assert field_err(mesh.get_fields()[0], r.M) < tol, steps
        assert np.abs(mesh.body_forces()[0] - np.array(r.force)).max() < 1e-4 * P_SCALE


def test_fp32_viv_512x256_full_size_bench_launch(lbfsi):
    """The bench workload at full size (O-grid 512 x 256, 1-DOF VIV, FP32
    populations) in the bench's launch configuration (a batch of identical
    solves): the first steps match the oracle run on the full mesh."""
    case = inputs.viv_cylinder_512x256(steps=3)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    state = {"h": 0.01, "alpha": 0.0, "hdot": 0.002, "adot": 0.0}
    s, r, hist = run_oracle(case, M0, case.steps, state)
    nb = 16
    mesh = lbfsi.Mesh(case.r, case.e, case.bodies * nb, precision=lbfsi.FP32)
    mesh.init_fields(case.flow, np.broadcast_to(M0, (nb,) + M0.shape))
    to = (state["h"], state["alpha"], state["hdot"], state["adot"])
    mesh.blend_mesh([to] * nb)
    mesh.step(case.steps)
    fields = mesh.get_fields()
    loads = mesh.body_forces()
    for k in (0, nb - 1):
        assert field_err(fields[k], r.M) < 1e-5
        assert np.abs(loads[k] - hist[-1]).max() < 1e-4 * P_SCALE
    assert np.array_equal(fields[0], fields[nb - 1])


def test_cfl_violation_reported(lbfsi):
    """A time step far above the near-wall CFL puts departure points outside
    the adjacent cells: the kernel flags it (no out-of-bounds access, the
    lookup only ever touches the four adjacent cells) and the host returns
    EDEPARTURE."""
    case = inputs.cylinder_case(24, 32, r_far=8.0, steps=1)
    case.flow.dt *= 12.0
    mesh = lbfsi.Mesh(case.r, case.e, case.bodies, precision=lbfsi.FP64)
    mesh.init_fields(case.flow)
    mesh.step(1)
    with pytest.raises(lbfsi.LbfsiError) as ei:
        mesh.synchronize()
    assert ei.value.code == lbfsi.EDEPARTURE
