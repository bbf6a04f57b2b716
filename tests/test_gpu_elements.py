"""The step on unstructured Q2 element lists (lbfsi_create_mesh_elements)
against the oracle's element-list step (oracle/unstructured.py) on the same
seeded inputs, through the C ABI.

Meshes: cylinder O-grids (odd radial count, so the grid's 3 x 3 windows tile
it) renumbered into shuffled element lists; a plunging 1-DOF body moves the
mesh through the blending function; flow from the left (inlet and outlet
far field).  Tolerances as in test_gpu_parity.py: FP64 1e-12 relative in
fields and populations, 1e-12 p_inf D in loads; FP32 1e-5 in fields and
1e-4 p_inf D in loads."""
import numpy as np
import pytest

import oracle.mesh as OM
import oracle.solver as OS
import oracle.unstructured as OU
from paper_2107_01370_gb300 import inputs

pytestmark = pytest.mark.gpu

P_SCALE = 1.0 / 3.0


@pytest.fixture(scope="module")
def lbfsi():
    from paper_2107_01370_gb300 import build, lbfsi as L
    build.build()
    L.load()
    return L


def field_err(a, b):
    e_rho = np.abs(a[0] - b[0]).max() / np.abs(b[0]).max()
    e_u = np.hypot(a[1] - b[1], a[2] - b[2]).max() / np.hypot(b[1], b[2]).max()
    e_T = np.abs(a[3] - b[3]).max() / np.abs(b[3]).max()
    return max(e_rho, e_u, e_T)


STATE = {"h": 0.02, "alpha": 0.0, "hdot": 0.004, "adot": 0.0}
PREV = {"h": 0.0199, "alpha": 0.0, "hdot": 0.004, "adot": 0.0}


def _case(nr=25, nt=48, seed=3):
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=2.0, v_r=4.0)
    case = inputs.cylinder_case(nr, nt, r_far=8.0, body=body)
    sm = OM.ogrid_mesh(case.r, case.e)
    el = inputs.ogrid_element_list(sm.X, seed=seed)
    M0 = inputs.initial_field(nr, nt, case.flow, seed=seed, noise=1e-2)
    return case, sm, el, M0


def _gpu(L, case, el, M0, precision, grid=False, nbatch=1):
    m = L.ElementMesh(el.X, el.elements, el.wall, el.far, case.bodies * nbatch, precision=precision,
                      grid_ij=el.grid_ij if grid else None, grid=(el.nr, el.nt))
    m.init_fields(case.flow, np.broadcast_to(el.to_list(M0), (nbatch, 4, el.X.shape[0])))
    to = (STATE["h"], STATE["alpha"], STATE["hdot"], STATE["adot"])
    tp = (PREV["h"], PREV["alpha"], PREV["hdot"], PREV["adot"])
    m.blend_mesh([to] * nbatch, [tp] * nbatch)
    return m


def _oracle_unstructured(case, el, M0):
    um = OU.UnstructuredQ2Mesh(el.X, el.elements)
    s = OU.UnstructuredSolver.from_case(um, el.wall, el.far, case, el.to_list(M0))
    s.S, s.S_prev = [dict(STATE)], [dict(PREV)]
    return s


def test_fp64_element_list_matches_the_oracle(lbfsi):
    """Reading R33 gradients on both sides: fields, pre- and post-collision
    populations, every step's load and the body state after 8 steps."""
    case, sm, el, M0 = _case()
    s = _oracle_unstructured(case, el, M0)
    m = _gpu(lbfsi, case, el, M0, lbfsi.FP64)
    for _ in range(8):
        r = s.step()
        m.step(1)
        assert np.abs(m.body_forces()[0] - np.array(r.force)).max() < 1e-12 * P_SCALE
    assert field_err(m.get_fields()[0], r.M) < 1e-12
    f0, g0 = m.get_populations(0)
    inner = ~np.isin(np.arange(el.X.shape[0]), el.far)
    assert np.abs(f0[0][:, inner] - r.f_pre[:, inner]).max() < 1e-12 * np.abs(r.f_pre).max()
    assert np.abs(g0[0][:, inner] - r.g_pre[:, inner]).max() < 1e-12 * np.abs(r.g_pre).max()
    f1, g1 = m.get_populations(1)
    assert np.abs(f1[0] - r.f_post).max() < 1e-12 * np.abs(r.f_post).max()
    assert np.abs(g1[0] - r.g_post).max() < 1e-12 * np.abs(r.g_post).max()
    st = m.body_state()[0]
    for k in ("h", "hdot"):
        assert abs(st[k] - s.S[0][k]) < 1e-12 * (1 + abs(s.S[0][k])), k
    assert m.launch_count() >= 4 * 8
    m.close()


def test_fp64_renumbered_grid_steps_as_the_structured_mesh(lbfsi):
    """With the grid's index map (reading R18 gradients) the shuffled element
    list is the structured O-grid: the structured oracle and the structured
    GPU path give the same fields, loads and body state to 1e-12."""
    case, sm, el, M0 = _case(nr=21, nt=40, seed=5)
    s = OS.Solver.from_case(sm, case, M0)
    s.S, s.S_prev = [dict(STATE)], [dict(PREV)]
    m = _gpu(lbfsi, case, el, M0, lbfsi.FP64, grid=True)
    ms = lbfsi.Mesh(case.r, case.e, case.bodies, precision=lbfsi.FP64)
    ms.init_fields(case.flow, M0[None])
    ms.blend_mesh([(STATE["h"], 0.0, STATE["hdot"], 0.0)], [(PREV["h"], 0.0, PREV["hdot"], 0.0)])
    for _ in range(6):
        r = s.step()
        m.step(1)
        ms.step(1)
        assert np.abs(m.body_forces()[0] - np.array(r.force)).max() < 1e-12 * P_SCALE
    got = el.to_grid(m.get_fields()[0])
    assert field_err(got, r.M) < 1e-12
    assert field_err(got, ms.get_fields()[0]) < 1e-12
    assert np.abs(m.body_forces()[0] - ms.body_forces()[0]).max() < 1e-12 * P_SCALE
    m.close()
    ms.close()


def test_fp32_element_list_within_tolerance(lbfsi):
    case, sm, el, M0 = _case(nr=25, nt=48, seed=7)
    s = _oracle_unstructured(case, el, M0)
    m = _gpu(lbfsi, case, el, M0, lbfsi.FP32)
    for _ in range(40):
        r = s.step()
    m.step(40)
    assert field_err(m.get_fields()[0], r.M) < 1e-5
    assert np.abs(m.body_forces()[0] - np.array(r.force)).max() < 1e-4 * P_SCALE
    m.close()


def test_batch_of_solves_equals_each_alone(lbfsi):
    """Two solves in one handle (one launch per kernel for both) end
    bit-identical to the same solve alone."""
    case, sm, el, M0 = _case(nr=17, nt=32, seed=9)
    a = _gpu(lbfsi, case, el, M0, lbfsi.FP32, nbatch=2)
    b = _gpu(lbfsi, case, el, M0, lbfsi.FP32, nbatch=1)
    a.step(20)
    b.step(20)
    fa, fb = a.get_fields(), b.get_fields()
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[0])
    assert np.array_equal(a.body_forces()[1], b.body_forces()[0])
    a.close()
    b.close()


def test_cfl_violation_reported_on_element_list(lbfsi):
    case, sm, el, M0 = _case(nr=13, nt=24, seed=1)
    case.flow.dt *= 12.0
    m = lbfsi.ElementMesh(el.X, el.elements, el.wall, el.far, case.bodies, precision=lbfsi.FP64)
    m.init_fields(case.flow)
    m.step(1)
    with pytest.raises(lbfsi.LbfsiError) as ei:
        m.synchronize()
    assert ei.value.code == lbfsi.EDEPARTURE
    m.close()


def test_fp64_cgrid_element_list_with_a_pitching_section(lbfsi):
    """A C-grid around an elliptic section as an element list, its wake cut
    merged (the two sides share the cut's nodes), shuffled; a pitch-plunge
    body about an axis ahead of the section, already pitched and moving, so
    that g != I and the wall's normals rotate: fields, every step's load and
    the body state match the oracle's element-list step to 1e-12."""
    body = inputs.BodySpec(dof=2, xp=-0.2, yp=0.0, r_in=0.7, r_out=2.5, m_star=20.0, v_r=2.0,
                           x_alpha=0.3, r_alpha=0.5, wh_wa=0.5)
    case = inputs.cgrid_case(33, 8, 17, 0.5, 0.25, r_far=5.0, wake=4.0, body=body)
    el = inputs.cgrid_element_list(case.X, case.n_cut, seed=4)
    N = el.X.shape[0]
    rng = np.random.default_rng(4)
    M0 = np.empty((4, N))
    M0[0] = 1.0
    M0[1] = case.flow.u_inf * (1 + 1e-2 * rng.uniform(-1, 1, N))
    M0[2] = 1e-2 * case.flow.u_inf * rng.uniform(-1, 1, N)
    M0[3] = case.flow.t_inf
    st = {"h": 0.01, "alpha": 0.04, "hdot": 0.002, "adot": 0.01}
    pv = {"h": 0.00998, "alpha": 0.03996, "hdot": 0.002, "adot": 0.01}
    um = OU.UnstructuredQ2Mesh(el.X, el.elements)
    s = OU.UnstructuredSolver.from_case(um, el.wall, el.far, case, M0)
    s.S, s.S_prev = [dict(st)], [dict(pv)]
    m = lbfsi.ElementMesh(el.X, el.elements, el.wall, el.far, case.bodies, precision=lbfsi.FP64)
    m.init_fields(case.flow, M0[None])
    m.blend_mesh([tuple(st[k] for k in ("h", "alpha", "hdot", "adot"))],
                 [tuple(pv[k] for k in ("h", "alpha", "hdot", "adot"))])
    for _ in range(8):
        r = s.step()
        m.step(1)
        assert np.abs(m.body_forces()[0] - np.array(r.force)).max() < 1e-12 * P_SCALE
    assert field_err(m.get_fields()[0], r.M) < 1e-12
    st_g = m.body_state()[0]
    for k in ("h", "alpha", "hdot", "adot"):
        assert abs(st_g[k] - s.S[0][k]) < 1e-12 * (1 + abs(s.S[0][k])), k
    m.close()


def _golden_elements():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "elements513_steps.json")
    with open(path) as fh:
        return json.load(fh)


def _bench_element_run(L, precision, nbatch, gold):
    """The bench's element-list workload (tests/golden/make_elements513_steps.py
    builds the same inputs) stepped gold['steps'] times; every step's load
    and body state of solve 0 and the fields after the checked steps."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "make_el", os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_elements513_steps.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    case, el, M0 = mk.workload()
    m = L.ElementMesh(el.X, el.elements, el.wall, el.far, case.bodies * nbatch, precision=precision)
    m.init_fields(case.flow, np.ascontiguousarray(np.broadcast_to(M0, (nbatch,) + M0.shape)))
    loads, states, fields = [], [], {}
    for n in range(1, gold["steps"] + 1):
        m.step(1)
        loads.append(m.body_forces()[0].copy())
        st = m.body_state()[0]
        states.append((st["h"], st["hdot"]))
        if n in gold["check"]:
            fields[n] = m.get_fields()
    m.close()
    return np.array(loads), np.array(states), fields


def _sampled_err(M, gold, n):
    pts = np.array(gold["samples"])
    ref = np.array(gold["fields"][str(n)])
    got = M[:, pts].T
    s_rho, s_u, s_T = gold["scale"][str(n)]
    return max(np.abs(got[:, 0] - ref[:, 0]).max() / s_rho,
               np.hypot(got[:, 1] - ref[:, 1], got[:, 2] - ref[:, 2]).max() / s_u,
               np.abs(got[:, 3] - ref[:, 3]).max() / s_T)


def test_bench_element_workload_fp32_against_stored_oracle(lbfsi):
    """The bench's element-list workload at full size (513 x 256 O-grid as a
    shuffled element list, 131,328 nodes) in the bench's launch
    configuration (eight solves, FP32), against the oracle's stored first 20
    steps: sampled fields within 1e-5, every step's C_D within 1e-4
    relative, C_L within 1e-4 of its amplitude, the displacement within
    1e-6 D; the eight solves bit-identical.  Measured on a GB300: fields
    6.5e-7, C_D 1.2e-7, C_L 7.2e-6, h 2e-12 D."""
    gold = _golden_elements()
    loads, states, fields = _bench_element_run(lbfsi, lbfsi.FP32, 8, gold)
    errs = {n: _sampled_err(fields[n][0], gold, n) for n in gold["check"]}
    for n in gold["check"]:
        for b in range(1, 8):
            assert np.array_equal(fields[n][b], fields[n][0])
    qd = gold["q_inf_d"]
    a, g = loads / qd, np.array(gold["loads"]) / qd
    cd = (np.abs(a[:, 0] - g[:, 0]) / np.abs(g[:, 0])).max()
    cl = np.abs(a[:, 1] - g[:, 1]).max() / np.abs(g[:, 1]).max()
    dh = np.abs(states[:, 0] - np.array(gold["states"])[:, 0]).max()
    assert max(errs.values()) < 1e-5, errs
    assert cd < 1e-4, cd
    assert cl < 1e-4, cl
    assert dh < 1e-6, dh


def test_bench_element_workload_fp64_against_stored_oracle(lbfsi):
    """The same workload, one FP64 solve: sampled fields within 1e-12 and
    every step's load within 1e-12 p_inf D of the oracle's stored run
    (measured: 4.5e-14 and 7e-15 p_inf D)."""
    gold = _golden_elements()
    loads, states, fields = _bench_element_run(lbfsi, lbfsi.FP64, 1, gold)
    errs = {n: _sampled_err(fields[n][0], gold, n) for n in gold["check"]}
    dl = np.abs(loads - np.array(gold["loads"])).max()
    assert max(errs.values()) < 1e-12, errs
    assert dl < 1e-12 * P_SCALE, dl


def test_node_order_round_trip(lbfsi):
    """The handle numbers nodes along a Z-order curve internally; the caller
    sees its own order: fields given to init_fields come back unchanged from
    get_fields (FP64), and after one step the shuffled list's fields equal
    the same mesh's unshuffled list's fields node by node."""
    case, sm, el, M0 = _case(nr=25, nt=48, seed=13)
    rng = np.random.default_rng(13)
    Mr = el.to_list(M0) * (1 + 1e-3 * rng.uniform(-1, 1, (4, el.X.shape[0])))
    m = lbfsi.ElementMesh(el.X, el.elements, el.wall, el.far, case.bodies, precision=lbfsi.FP64)
    m.init_fields(case.flow, Mr[None])
    assert np.array_equal(m.get_fields()[0], Mr)
    m.step(1)
    shuffled = el.to_grid(m.get_fields()[0])
    m.close()
    plain = inputs.ogrid_element_list(sm.X, seed=13, shuffle=False)
    m = lbfsi.ElementMesh(plain.X, plain.elements, plain.wall, plain.far, case.bodies, precision=lbfsi.FP64)
    m.init_fields(case.flow, plain.to_list(el.to_grid(Mr))[None])
    m.step(1)
    unshuffled = plain.to_grid(m.get_fields()[0])
    m.close()
    assert np.abs(shuffled - unshuffled).max() < 1e-13 * np.abs(unshuffled).max()
