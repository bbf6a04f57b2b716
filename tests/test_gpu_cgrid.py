"""Parity of the C-grid path (a wake cut with mirrored cells across it,
outlet columns, an open wall chain; readings R28-R30) with the FP64 oracle on
the same meshes and seeded inputs: an elliptic section fixed, in 1-DOF
plunge, in 2-DOF pitch-plunge with rotation, and across the switch from forced
to free pitching.  A C-grid step is two launches (the collision of the rows
next to the cut into a post-collision buffer, then the stream of the tiles
next to the cut from it and a fused collide-and-stream of the others); graph
replay and checkpoint / resume keep it bit for bit.  Tolerances as in test_gpu_parity."""
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
    walls = getattr(case, "walls", None)
    mesh = OM.CGridMesh(case.X, walls=walls) if walls else OM.CGridMesh(case.X, case.n_cut)
    s = OS.Solver.from_case(mesh, case, M0)
    if state is not None:
        s.S = [dict(state)]
        s.S_prev = [dict(prev if prev is not None else state)]
    hist = []
    for _ in range(steps):
        r = s.step()
        hist.append(r.force)
    if walls:
        m = L.Mesh.cgrid_walls(case.X, walls, case.bodies, precision=precision, centre=case.centre)
    else:
        m = L.Mesh.cgrid(case.X, case.n_cut, case.bodies, precision=precision, centre=case.centre)
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


def _case(body, n_wall=49, n_cut=8, nr=32, **kw):
    return inputs.cgrid_case(n_wall, n_cut, nr, 0.6, 0.35, r_far=6.0, wake=4.0, length=1.2, body=body, **kw)


BODIES = {
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
def test_fp64_cgrid_matches_oracle(L, dof):
    body, state, prev = BODIES[dof]
    case = _case(body)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=31 + dof)
    s, r, hist, (f, ghist, st) = run_both(L, case, M0, 10, L.FP64, state, prev)
    assert field_err(f, r.M) < 1e-12
    assert np.abs(ghist - hist).max() < 1e-12 * P_SCALE
    for k in ("h", "alpha", "hdot", "adot"):
        assert abs(st[k] - s.S[0][k]) < 1e-12 * (1 + abs(s.S[0][k])), k
    # the second copies of the cut nodes hold the first copies' values
    jc, nt = case.n_cut, case.ntheta
    assert np.array_equal(f[:, 0, nt - 1 - jc:], f[:, 0, :jc + 1][:, ::-1])


def test_fp64_cgrid_forced_then_free_pitching_matches_oracle(L):
    base = inputs.BodySpec(dof=2, xp=-0.25, yp=0.0, r_in=0.75, r_out=2.0, m_star=8.0, v_r=1.2,
                           x_alpha=0.2, r_alpha=0.5, wh_wa=0.4, length=1.2)
    case = _case(base)
    u_inf = case.flow.ma * np.sqrt(case.flow.gamma * case.flow.t_inf)
    w_a = u_inf / (base.v_r * 0.6 * np.sqrt(base.m_star))
    base.pitch_amp = 0.2
    base.forced_periods = 5.5 * case.flow.dt * w_a / (2.0 * np.pi)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=41)
    s, r, hist, (f, ghist, st) = run_both(L, case, M0, 10, L.FP64)
    assert field_err(f, r.M) < 1e-12
    assert np.abs(ghist - hist).max() < 1e-12 * P_SCALE
    for k in ("h", "alpha", "hdot", "adot"):
        assert abs(st[k] - s.S[0][k]) < 1e-12 * (1 + abs(s.S[0][k])), k


def test_fp32_cgrid_within_stated_tolerance(L):
    body, state, prev = BODIES[1]
    case = _case(body)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=43)
    s, r, hist, (f, ghist, st) = run_both(L, case, M0, 40, L.FP32, state, prev)
    assert field_err(f, r.M) < 1e-5
    assert np.abs(ghist - hist).max() < 1e-4 * P_SCALE


def _state(m):
    return m.get_fields(), m.body_forces(), m.body_state()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cgrid_graph_replay_and_resume_are_bit_identical(L, precision):
    prec = L.FP32 if precision == "fp32" else L.FP64
    body = BODIES[2][0]
    case = _case(body)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=47)
    M2 = np.ascontiguousarray(np.broadcast_to(M0, (2,) + M0.shape))

    def fresh():
        m = L.Mesh.cgrid(case.X, case.n_cut, case.bodies * 2, precision=prec)
        m.init_fields(case.flow, M2)
        return m

    a = fresh()
    a.step(9)
    ckpt = a.checkpoint()
    a.step(14)
    ref = _state(a)
    n_launch = a.launch_count()
    a.close()
    b = fresh()
    b.set_graph_steps(4)
    b.step(23)
    got = _state(b)
    b.close()
    for x, y in zip(ref[:2], got[:2]):
        assert np.array_equal(x, y)
    assert ref[2] == got[2]
    c = fresh()
    c.restore(ckpt)
    c.step(14)
    got = _state(c)
    c.close()
    for x, y in zip(ref[:2], got[:2]):
        assert np.array_equal(x, y)
    assert ref[2] == got[2]
    assert n_launch >= 2 * 23


def test_cgrid_reports_cfl_violation(L):
    """A time step eight times the C-grid's CFL step: departure points leave
    the cells adjacent to their nodes; the kernel records it and the next
    synchronising call reports EDEPARTURE (the oracle raises likewise)."""
    case = _case(BODIES[0][0], n_wall=33, n_cut=8, nr=24)
    case.flow.dt *= 8.0
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=3)
    with pytest.raises(OM.DepartureError):
        OS.Solver.from_case(OM.CGridMesh(case.X, case.n_cut), case, M0).step()
    m = L.Mesh.cgrid(case.X, case.n_cut, case.bodies, precision=L.FP32)
    m.init_fields(case.flow, M0[None])
    m.step(2)
    with pytest.raises(L.LbfsiError) as ei:
        m.synchronize()
    assert ei.value.code == L.EDEPARTURE
    m.close()


def _naca_case(nr=32, n_wall=97, n_cut=24, ma=0.8, t_inf=0.2):
    body = inputs.BodySpec(dof=2, xp=-1.0, yp=0.0, r_in=0.6, r_out=2.0, m_star=100.0, v_r=0.5025,
                           x_alpha=1.8, r_alpha=1.87, wh_wa=0.3, length=1.0)
    case = inputs.cgrid_case(n_wall, n_cut, nr, 0.5, 0.06, r_far=6.0, wake=4.0, length=1.0, ma=ma,
                             t_inf=t_inf, re=1e5, body=body, naca=0.12)
    u_inf = case.flow.ma * np.sqrt(case.flow.gamma * case.flow.t_inf)
    w_a = u_inf / (body.v_r * 0.5 * np.sqrt(body.m_star))
    body.pitch_amp = np.pi / 180.0
    body.forced_periods = 4.5 * case.flow.dt * w_a / (2.0 * np.pi)
    return case


def test_fp64_naca0012_cgrid_matches_oracle(L):
    """NACA 0012 (public thickness formula, closed trailing edge) on a C-grid,
    the airfoil case's flow (Ma 0.8, T_inf 0.2, Re 1e5) and structure (2-DOF,
    m* 100, w_h/w_a 0.3, x_a 1.8, r_a 1.87, V_R 0.5025), 1-degree forced
    pitching that ends between steps 4 and 5: the sharp trailing edge is the
    point where the wall meets the cut."""
    case = _naca_case()
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=61)
    s, r, hist, (f, ghist, st) = run_both(L, case, M0, 8, L.FP64)
    assert field_err(f, r.M) < 1e-12
    assert np.abs(ghist - hist).max() < 1e-12 * P_SCALE
    for k in ("h", "alpha", "hdot", "adot"):
        assert abs(st[k] - s.S[0][k]) < 1e-12 * (1 + abs(s.S[0][k])), k


def test_fp32_naca0012_cgrid_within_stated_tolerance(L):
    case = _naca_case()
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=62)
    s, r, hist, (f, ghist, st) = run_both(L, case, M0, 30, L.FP32)
    assert field_err(f, r.M) < 1e-5
    assert np.abs(ghist - hist).max() < 1e-4 * P_SCALE


LINKED = inputs.BodySpec(dof=1, xc=2.0, yc=0.0, xp=2.0, yp=0.0, r_in=2.7, r_out=4.5, m_star=4.0, v_r=5.0,
                         length=1.0)


@pytest.mark.parametrize("moving", [False, True])
def test_fp64_linked_tandem_cylinders_match_oracle(L, moving):
    """Two cylinders in tandem (4 D apart) rigidly linked on one transverse
    DOF (reading R31): a C-grid with three wall chains (the front body, the
    rear body's upper and lower halves), the cut through the gap and the wake;
    one rigid zone holds both walls and the load is their sum."""
    case = inputs.tandem_case(34, 17, 11, 16, 33, body=LINKED)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=71)
    state = {"h": 0.02, "alpha": 0.0, "hdot": 0.004, "adot": 0.0} if moving else None
    prev = {"h": 0.0199, "alpha": 0.0, "hdot": 0.004, "adot": 0.0} if moving else None
    s, r, hist, (f, ghist, st) = run_both(L, case, M0, 10, L.FP64, state, prev)
    assert field_err(f, r.M) < 1e-12
    assert np.abs(ghist - hist).max() < 1e-12 * P_SCALE
    for k in ("h", "hdot"):
        assert abs(st[k] - s.S[0][k]) < 1e-12 * (1 + abs(s.S[0][k])), k


def test_fp32_linked_tandem_within_stated_tolerance(L):
    case = inputs.tandem_case(34, 17, 11, 16, 33, body=LINKED)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=72)
    s, r, hist, (f, ghist, st) = run_both(L, case, M0, 30, L.FP32)
    assert field_err(f, r.M) < 1e-5
    assert np.abs(ghist - hist).max() < 1e-4 * P_SCALE


# ----- independent bodies (reading R32) -----------------------------------
FRONT = inputs.BodySpec(dof=1, xc=0.0, yc=0.0, xp=0.0, yp=0.0, r_in=0.7, r_out=1.8, m_star=2.0, v_r=4.0,
                        length=1.0)
REAR = inputs.BodySpec(dof=2, xc=4.0, yc=0.0, xp=3.9, yp=0.0, r_in=0.7, r_out=1.8, m_star=5.0, v_r=2.0,
                       x_alpha=0.3, r_alpha=0.6, wh_wa=0.5, length=1.0)
WALL_BODY = [1, 0, 1]   # chains: rear lower half, front, rear upper half
IND_STATE = [{"h": 0.02, "alpha": 0.0, "hdot": 0.004, "adot": 0.0},
             {"h": -0.01, "alpha": 0.02, "hdot": -0.002, "adot": 0.01}]
IND_PREV = [{"h": 0.0199, "alpha": 0.0, "hdot": 0.004, "adot": 0.0},
            {"h": -0.0099, "alpha": 0.0199, "hdot": -0.002, "adot": 0.01}]


def _independent(L, precision, steps, seed, moving=True):
    case = inputs.tandem_case(34, 17, 11, 16, 33)
    case.bodies = [FRONT, REAR]
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=seed)
    s = OS.Solver.from_case(OM.CGridMesh(case.X, walls=case.walls, wall_body=WALL_BODY), case, M0)
    if moving:
        s.S = [dict(x) for x in IND_STATE]
        s.S_prev = [dict(x) for x in IND_PREV]
    hist = []
    for _ in range(steps):
        r = s.step()
        hist.append(r.forces)
    m = L.Mesh.cgrid_walls(case.X, case.walls, [[FRONT, REAR]], precision=precision, wall_body=WALL_BODY)
    m.init_fields(case.flow, M0[None])
    if moving:
        m.blend_mesh([to_tuple(x) for x in IND_STATE], [to_tuple(x) for x in IND_PREV])
    ghist = []
    for _ in range(steps):
        m.step(1)
        ghist.append(m.body_forces()[0].copy())
    out = (m.get_fields()[0], np.array(ghist), m.body_state()[0])
    m.close()
    return s, r, np.array(hist), out


def test_fp64_independent_tandem_bodies_match_oracle(L):
    """The two cylinders as independent bodies: the front one in transverse
    VIV, the rear one in pitch-plunge about its own elastic axis, each with
    its own blended region, load (its chains only) and RK4 update."""
    s, r, hist, (f, ghist, st) = _independent(L, L.FP64, 10, 73)
    assert field_err(f, r.M) < 1e-12
    assert ghist.shape == (10, 2, 3)
    assert np.abs(ghist - hist).max() < 1e-12 * P_SCALE
    # each body carries a load of its own (not a copy of the other's)
    assert np.abs(ghist[:, 0] - ghist[:, 1]).max() > 1e-4 * P_SCALE
    for b in range(2):
        for k in ("h", "alpha", "hdot", "adot"):
            assert abs(st[b][k] - s.S[b][k]) < 1e-12 * (1 + abs(s.S[b][k])), (b, k)
    assert st[0]["alpha"] == 0.0   # the transverse body does not rotate


def test_fp64_independent_fixed_bodies_match_oracle(L):
    s, r, hist, (f, ghist, st) = _independent(L, L.FP64, 6, 74, moving=False)
    assert field_err(f, r.M) < 1e-12
    assert np.abs(ghist - hist).max() < 1e-12 * P_SCALE


def test_fp32_independent_tandem_bodies_within_stated_tolerance(L):
    s, r, hist, (f, ghist, st) = _independent(L, L.FP32, 30, 75)
    assert field_err(f, r.M) < 1e-5
    assert np.abs(ghist - hist).max() < 1e-4 * P_SCALE


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_independent_bodies_graph_replay_resume_and_record(L, precision):
    """Two solves of the independent pair: graph replay and checkpoint /
    resume are bit for bit, and lbfsi_step_record's per-(solve, body)
    records equal body_forces / body_state after each step."""
    prec = L.FP32 if precision == "fp32" else L.FP64
    case = inputs.tandem_case(34, 17, 11, 16, 33)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=76)
    M2 = np.ascontiguousarray(np.broadcast_to(M0, (2,) + M0.shape))
    rear_b = inputs.BodySpec(**{**REAR.__dict__, "m_star": 3.0})

    def fresh():
        m = L.Mesh.cgrid_walls(case.X, case.walls, [[FRONT, REAR], [FRONT, rear_b]], precision=prec,
                               wall_body=WALL_BODY)
        m.init_fields(case.flow, M2)
        m.blend_mesh([to_tuple(x) for x in IND_STATE] * 2, [to_tuple(x) for x in IND_PREV] * 2)
        return m

    a = fresh()
    a.step(7)
    ckpt = a.checkpoint()
    loads, states = a.step_record(9, states=True)
    assert loads.shape == (9, 2, 2, 3) and states.shape == (9, 2, 2, 4)
    ref = (a.get_fields(), a.body_forces(), a.body_state())
    assert np.array_equal(loads[-1], ref[1])
    assert states[-1, 1, 1, 0] == ref[2][1][1]["h"]
    # the two solves differ only in the rear body's mass: the rear bodies'
    # states part, their loads follow
    assert states[-1, 0, 1, 0] != states[-1, 1, 1, 0]
    a.close()
    b = fresh()
    b.set_graph_steps(4)
    b.step(16)
    got = (b.get_fields(), b.body_forces(), b.body_state())
    b.close()
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1]) and ref[2] == got[2]
    c = fresh()
    c.restore(ckpt)
    c.step(9)
    got = (c.get_fields(), c.body_forces(), c.body_state())
    c.close()
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1]) and ref[2] == got[2]


def test_fp32_tandem_1m_independent_sweep_full_size_bench_launch(L):
    """The tandem workload at full size (512 x 2049 C-grid, two independent
    1-DOF bodies) in the bench's launch configuration (one solve per reduced
    velocity of the sweep, FP32): after one step every solve matches the
    oracle's stored first step at the sampled nodes (FP32 tolerance), each
    body's load matches, and each solve's RK4 update matches the oracle's
    for its reduced velocity (tests/golden/make_tandem_1m_step1.py)."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tandem_1m_step1.json")))
    case = inputs.tandem_1m_independent()
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    sweep = inputs.TANDEM_VR_SWEEP
    nb = len(sweep)
    m = L.Mesh.cgrid_walls(case.X, case.walls, [inputs.tandem_independent_pair(v) for v in sweep],
                           precision=L.FP32, wall_body=case.wall_body)
    m.init_fields(case.flow, np.broadcast_to(M0, (nb,) + M0.shape))
    st = [to_tuple(x) for x in gold["initial_states"]]
    pv = [(h - hd * case.flow.dt, a, hd, ad) for h, a, hd, ad in st]
    m.blend_mesh(st * nb, pv * nb)
    m.step(1)
    fields = m.get_fields()
    loads = m.body_forces()
    states = m.body_state()
    m.close()
    ii, jj = np.array(gold["samples"]).T
    ref = np.array(gold["M"])
    s_rho, s_u, s_T = gold["scale"]
    for k, v in enumerate(sweep):
        got = fields[k][:, ii, jj].T
        err = max(np.abs(got[:, 0] - ref[:, 0]).max() / s_rho,
                  np.hypot(got[:, 1] - ref[:, 1], got[:, 2] - ref[:, 2]).max() / s_u,
                  np.abs(got[:, 3] - ref[:, 3]).max() / s_T)
        assert err < 1e-5, (v, err)
        assert np.abs(loads[k] - np.array(gold["loads"])).max() < 1e-4 * P_SCALE
        for b in range(2):
            want = gold["states"][repr(v)][b]
            assert abs(states[k][b]["h"] - want[0]) < 1e-9 and abs(states[k][b]["hdot"] - want[2]) < 1e-8
    # the flow of the step does not depend on the reduced velocity
    assert np.array_equal(fields[0], fields[nb - 1])


def test_fp32_naca0012_full_size_bench_launch(L):
    """The transonic flutter workload at full size (NACA 0012 on the
    192 x 769 C-grid, 2-DOF with forced pitching, Ma 0.8) in the bench's
    launch configuration (a batch of eight identical solves, FP32): after
    three steps the sampled nodes match the oracle's stored run
    (tests/golden/make_naca0012_steps.py) within the FP32 tolerance, every
    step's load within 1e-4 p_inf c and the body state to round-off."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "naca0012_steps.json")))
    case = inputs.naca0012_flutter_case()
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    nb = 8
    m = L.Mesh.cgrid(case.X, case.n_cut, case.bodies * nb, precision=L.FP32)
    m.init_fields(case.flow, np.broadcast_to(M0, (nb,) + M0.shape))
    loads, states = m.step_record(gold["steps"], states=True)
    fields = m.get_fields()
    m.close()
    ii, jj = np.array(gold["samples"]).T
    ref = np.array(gold["M"])
    s_rho, s_u, s_T = gold["scale"]
    p_scale = case.flow.rho_inf * case.flow.t_inf * 1.0   # p_inf times the chord
    for k in (0, nb - 1):
        got = fields[k][:, ii, jj].T
        err = max(np.abs(got[:, 0] - ref[:, 0]).max() / s_rho,
                  np.hypot(got[:, 1] - ref[:, 1], got[:, 2] - ref[:, 2]).max() / s_u,
                  np.abs(got[:, 3] - ref[:, 3]).max() / s_T)
        assert err < 1e-5, err
        assert np.abs(loads[:, k] - np.array(gold["loads"])).max() < 1e-4 * p_scale
        assert np.abs(states[-1, k] - np.array(gold["state"])).max() < 1e-9
    assert np.array_equal(fields[0], fields[nb - 1])
