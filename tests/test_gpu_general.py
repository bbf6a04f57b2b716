"""Parity of the general-geometry path (O-grids given by node coordinates,
departure points by Newton's method on the bilinear element, Eq. depPnt)
with the FP64 oracle on the same meshes and seeded inputs: an elliptic
cylinder and a thin elliptic section, fixed and moving (1-DOF plunge, 2-DOF
pitch-plunge with rotation), plus agreement with the closed-form path on a
circular O-grid given as coordinates.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

import oracle.mesh as OM
import oracle.solver as OS
from paper_2107_01370_gb300 import inputs

pytestmark = pytest.mark.gpu

P_SCALE = 1.0 / 3.0   # p_inf * length


@pytest.fixture(scope="module")
def L():
    from paper_2107_01370_gb300 import build, lbfsi
    build.build()
    lbfsi.load()
    return lbfsi


def field_err(a, b):
    e_rho = np.abs(a[0] - b[0]).max() / np.abs(b[0]).max()
    e_u = np.hypot(a[1] - b[1], a[2] - b[2]).max() / np.hypot(b[1], b[2]).max()
    e_T = np.abs(a[3] - b[3]).max() / np.abs(b[3]).max()
    return max(e_rho, e_u, e_T)


def to_tuple(d):
    return (d["h"], d["alpha"], d["hdot"], d["adot"])


def run_both(L, case, M0, steps, precision, state=None, prev=None):
    s = OS.Solver.from_case(OM.Q2Mesh(case.X, periodic_i=False, periodic_j=True), case, M0)
    if state is not None:
        s.S = [dict(state)]
        s.S_prev = [dict(prev if prev is not None else state)]
    hist = []
    for _ in range(steps):
        r = s.step()
        hist.append(r.force)
    m = L.Mesh.xy(case.X, case.bodies, precision=precision, centre=case.centre)
    m.init_fields(case.flow, M0[None])
    if state is not None:
        m.blend_mesh([to_tuple(state)], None if prev is None else [to_tuple(prev)])
    ghist = []
    for _ in range(steps):
        m.step(1)
        ghist.append(m.body_forces()[0].copy())
    out = (m.get_fields()[0], np.array(ghist), m.body_state()[0])
    m.close()
    return s, r, np.array(hist), out


ELLIPSE_BODIES = {
    0: (inputs.BodySpec(dof=0), None, None),
    1: (inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=2.0, v_r=4.0, length=1.2),
        {"h": 0.02, "alpha": 0.0, "hdot": 0.004, "adot": 0.0},
        {"h": 0.0199, "alpha": 0.0, "hdot": 0.004, "adot": 0.0}),
    2: (inputs.BodySpec(dof=2, xp=-0.2, yp=0.0, r_in=0.75, r_out=2.0, m_star=5.0, v_r=2.0,
                        x_alpha=0.3, r_alpha=0.6, wh_wa=0.5, length=1.2),
        {"h": -0.01, "alpha": 0.03, "hdot": 0.0, "adot": 0.01},
        {"h": -0.0101, "alpha": 0.0299, "hdot": 0.0, "adot": 0.01}),
}


@pytest.mark.parametrize("dof", [0, 1, 2])
def test_fp64_elliptic_cylinder_matches_oracle(L, dof):
    body, state, prev = ELLIPSE_BODIES[dof]
    case = inputs.xy_case(inputs.ellipse_wall(64, 0.6, 0.35), 48, r_far=8.0, length=1.2, body=body)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=11 + dof)
    s, r, hist, (f, ghist, st) = run_both(L, case, M0, 10, L.FP64, state, prev)
    assert field_err(f, r.M) < 1e-12
    assert np.abs(ghist - hist).max() < 1e-12 * P_SCALE
    for k in ("h", "alpha", "hdot", "adot"):
        assert abs(st[k] - s.S[0][k]) < 1e-12 * (1 + abs(s.S[0][k])), k


def test_fp64_thin_section_pitch_plunge_matches_oracle(L):
    """2-DOF pitch-plunge of a 12%-thick elliptic section (chord 1, elastic
    axis a quarter chord ahead of mid-chord) on an algebraic O-grid: skewed
    cells near the tips, rotation of the blended mesh from the first step."""
    body = inputs.BodySpec(dof=2, xp=-0.25, yp=0.0, r_in=0.6, r_out=2.0, m_star=8.0, v_r=1.2,
                           x_alpha=0.2, r_alpha=0.5, wh_wa=0.4, length=1.0)
    case = inputs.xy_case(inputs.ellipse_wall(96, 0.5, 0.06), 40, r_far=8.0, body=body)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=21)
    state = {"h": 0.0, "alpha": 0.02, "hdot": 0.0, "adot": 0.004}
    prev = {"h": 0.0, "alpha": 0.019997, "hdot": 0.0, "adot": 0.004}
    s, r, hist, (f, ghist, st) = run_both(L, case, M0, 8, L.FP64, state, prev)
    assert field_err(f, r.M) < 1e-12
    assert np.abs(ghist - hist).max() < 1e-12 * P_SCALE
    for k in ("h", "alpha", "hdot", "adot"):
        assert abs(st[k] - s.S[0][k]) < 1e-12 * (1 + abs(s.S[0][k])), k


def test_fp32_elliptic_cylinder_within_stated_tolerance(L):
    body, state, prev = ELLIPSE_BODIES[1]
    case = inputs.xy_case(inputs.ellipse_wall(64, 0.6, 0.35), 48, r_far=8.0, length=1.2, body=body)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=13)
    s, r, hist, (f, ghist, st) = run_both(L, case, M0, 40, L.FP32, state, prev)
    assert field_err(f, r.M) < 1e-5
    assert np.abs(ghist - hist).max() < 1e-4 * P_SCALE


def test_general_path_agrees_with_closed_form_on_a_circle(L):
    """The circular O-grid given as coordinates runs the Newton departure
    solve and the stored metric; the separable handle the closed forms and
    row/column tables.  FP64 results agree to round-off."""
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=3.0, v_r=4.0)
    case = inputs.cylinder_case(40, 64, r_far=8.0, body=body)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=4)
    X = np.empty((case.nr, case.ntheta, 2))
    X[..., 0] = case.r[:, None] * case.e[None, :, 0]
    X[..., 1] = case.r[:, None] * case.e[None, :, 1]
    a = L.Mesh(case.r, case.e, case.bodies, precision=L.FP64)
    b = L.Mesh.xy(X, case.bodies, precision=L.FP64)
    for m in (a, b):
        m.init_fields(case.flow, M0[None])
        m.blend_mesh([(0.01, 0.0, 0.002, 0.0)])
        m.step(12)
    assert field_err(b.get_fields()[0], a.get_fields()[0]) < 1e-12
    assert np.abs(b.body_forces() - a.body_forces()).max() < 1e-12 * P_SCALE
    a.close()
    b.close()


def test_general_path_reports_cfl_violation(L):
    case = inputs.xy_case(inputs.ellipse_wall(32, 0.6, 0.35), 24, r_far=6.0, length=1.2)
    case.flow.dt *= 8.0
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=1)
    m = L.Mesh.xy(case.X, case.bodies, precision=L.FP32)
    m.init_fields(case.flow, M0[None])
    m.step(2)
    with pytest.raises(L.LbfsiError) as ei:
        m.synchronize()
    assert ei.value.code == L.EDEPARTURE
    m.close()


def test_fp64_forced_then_free_pitching_matches_oracle(L):
    """Forced pitching (Sec. IV D): alpha = A sin(w_alpha t) prescribed over
    the first steps, the plunge driven by the load and the pitch
    acceleration, then the free pitch-plunge system; the switch falls between
    steps 4 and 5 of the run, on the thin section's general O-grid."""
    base = inputs.BodySpec(dof=2, xp=-0.25, yp=0.0, r_in=0.6, r_out=2.0, m_star=8.0, v_r=1.2,
                           x_alpha=0.2, r_alpha=0.5, wh_wa=0.4, length=1.0)
    case = inputs.xy_case(inputs.ellipse_wall(96, 0.5, 0.06), 40, r_far=8.0, body=base)
    u_inf = case.flow.ma * np.sqrt(case.flow.gamma * case.flow.t_inf)
    w_a = u_inf / (base.v_r * 0.5 * np.sqrt(base.m_star))
    base.pitch_amp = 0.2
    base.forced_periods = 5.5 * case.flow.dt * w_a / (2.0 * np.pi)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=23)
    s, r, hist, (f, ghist, st) = run_both(L, case, M0, 10, L.FP64)
    assert field_err(f, r.M) < 1e-12
    assert np.abs(ghist - hist).max() < 1e-12 * P_SCALE
    for k in ("h", "alpha", "hdot", "adot"):
        assert abs(st[k] - s.S[0][k]) < 1e-12 * (1 + abs(s.S[0][k])), k
    # the pitch is free after the switch: not the prescribed sine any more
    t = 10 * case.flow.dt
    assert abs(s.S[0]["alpha"] - 0.2 * np.sin(w_a * t)) > 1e-9


def test_tensor_copy_staging_is_bit_identical_on_a_general_mesh(L, monkeypatch):
    """The general kernel stages the populations and moments of a tile whose
    columns do not wrap by tensor copies (TMA); LBFSI_TMA=0 at handle creation
    stages every tile by per-thread copies.  An elliptic O-grid with
    Ntheta = 128 (two such tiles of four per tile row), two solves with a
    2-DOF body moving from the first step: the same bits either way."""
    body, state, prev = ELLIPSE_BODIES[2]
    case = inputs.xy_case(inputs.ellipse_wall(128, 0.6, 0.35), 40, r_far=8.0, length=1.2, body=body)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=17)

    def run():
        m = L.Mesh.xy(case.X, case.bodies * 2, precision=L.FP32, centre=case.centre)
        m.init_fields(case.flow, np.ascontiguousarray(np.broadcast_to(M0, (2,) + M0.shape)))
        m.blend_mesh([to_tuple(state)] * 2, [to_tuple(prev)] * 2)
        m.step(20)
        out = (m.get_fields(), m.body_forces(), m.body_state())
        m.close()
        return out

    monkeypatch.setenv("LBFSI_TMA", "0")
    ref = run()
    monkeypatch.delenv("LBFSI_TMA")
    got = run()
    assert np.array_equal(ref[0], got[0])
    assert np.array_equal(ref[1], got[1])
    assert ref[2] == got[2]
