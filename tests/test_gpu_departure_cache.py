"""The step on meshes given by node coordinates and on element lists solves
the departure points of the nodes the blend does not move once per handle (they are the same every step: g = I, V_G = 0,
displacement -dt c_q) and reads them back each step.  Solving them every step
instead (LBFSI_NO_DEPARTURE_CACHE=1 at handle creation) gives bit-identical
fields, loads and body states: an O-grid given by coordinates with a moving
body, a C-grid with a pitch-plunge body, the independent tandem bodies, a
periodic box and unstructured element lists (their interior nodes), in
FP32 and FP64."""
import os

import numpy as np
import pytest

from paper_2107_01370_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2107_01370_gb300 import build, lbfsi
    build.build()
    lbfsi.load()
    return lbfsi


def _tuple(d):
    return (d["h"], d["alpha"], d["hdot"], d["adot"])


def _run(L, make, flow, M0, states, prev, steps, cache):
    old = os.environ.pop("LBFSI_NO_DEPARTURE_CACHE", None)
    if not cache:
        os.environ["LBFSI_NO_DEPARTURE_CACHE"] = "1"
    try:
        m = make()
    finally:
        os.environ.pop("LBFSI_NO_DEPARTURE_CACHE", None)
        if old is not None:
            os.environ["LBFSI_NO_DEPARTURE_CACHE"] = old
    m.init_fields(flow, M0[None])
    if states is not None:
        m.blend_mesh(states, prev)
    loads = m.step_record(steps, states=True)
    out = (m.get_fields(), loads[0], loads[1], m.launch_count())
    m.close()
    return out


def _same(L, make, flow, M0, steps, states=None, prev=None):
    a = _run(L, make, flow, M0, states, prev, steps, True)
    b = _run(L, make, flow, M0, states, prev, steps, False)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert a[3] == b[3] + 1   # the one pass that fills the cache
    return a


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cache_same_on_general_ogrid_and_cgrid(L, precision):
    prec = L.FP32 if precision == "fp32" else L.FP64
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=2.0, v_r=4.0, length=1.2)
    st = [(0.02, 0.0, 0.004, 0.0)]
    pv = [(0.0199, 0.0, 0.004, 0.0)]
    case = inputs.xy_case(inputs.ellipse_wall(64, 0.6, 0.35), 48, r_far=8.0, length=1.2, body=body)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=81)
    _same(L, lambda: L.Mesh.xy(case.X, case.bodies, precision=prec), case.flow, M0, 12, st, pv)
    pp = inputs.BodySpec(dof=2, xp=-0.2, yp=0.0, r_in=0.75, r_out=2.0, m_star=5.0, v_r=2.0,
                         x_alpha=0.3, r_alpha=0.6, wh_wa=0.5, length=1.2)
    cg = inputs.cgrid_case(49, 8, 32, 0.6, 0.35, r_far=6.0, wake=4.0, length=1.2, body=pp)
    M0 = inputs.initial_field(cg.nr, cg.ntheta, cg.flow, seed=82)
    _same(L, lambda: L.Mesh.cgrid(cg.X, cg.n_cut, cg.bodies, precision=prec), cg.flow, M0, 12,
          [(-0.01, 0.03, 0.0, 0.01)], [(-0.0101, 0.0299, 0.0, 0.01)])


def test_cache_same_on_independent_tandem_and_box(L):
    tc = inputs.tandem_case(34, 17, 11, 16, 33)
    pair = [inputs.BodySpec(dof=1, xc=x, yc=0.0, xp=x, yp=0.0, r_in=0.7, r_out=1.8, m_star=2.0, v_r=4.0)
            for x in (0.0, 4.0)]
    M0 = inputs.initial_field(tc.nr, tc.ntheta, tc.flow, seed=83)
    st = [(0.02, 0.0, 0.004, 0.0), (-0.01, 0.0, -0.002, 0.0)]
    pv = [(0.0199, 0.0, 0.004, 0.0), (-0.0099, 0.0, -0.002, 0.0)]
    _same(L, lambda: L.Mesh.cgrid_walls(tc.X, tc.walls, [pair], precision=L.FP64, wall_body=[1, 0, 1]),
          tc.flow, M0, 10, st, pv)
    X, si, sj = inputs.box_mesh(24, 16, 24.0, 16.0, skew=0.3)
    rng = np.random.default_rng(4)
    Mb = np.empty((4, 24, 16))
    Mb[0] = 1.0 + 0.01 * rng.uniform(-1, 1, (24, 16))
    Mb[1] = 0.03 * rng.uniform(-1, 1, (24, 16))
    Mb[2] = 0.03 * rng.uniform(-1, 1, (24, 16))
    Mb[3] = 1.0 / 3.0 + 0.005 * rng.uniform(-1, 1, (24, 16))
    flow = inputs.FlowSpec(ma=0.1, re=0.1 * np.sqrt(1.4 / 3.0) / (0.1 / 3.0 * 0.5), dt=0.5, length=1.0)
    _same(L, lambda: L.Mesh.box(X, si, sj, precision=L.FP32), flow, Mb, 10)


def _element_run(L, el, bodies, flow, M0, states, prev, steps, precision, cache):
    old = os.environ.pop("LBFSI_NO_DEPARTURE_CACHE", None)
    if not cache:
        os.environ["LBFSI_NO_DEPARTURE_CACHE"] = "1"
    try:
        m = L.ElementMesh(el.X, el.elements, el.wall, el.far, bodies, precision=precision)
    finally:
        os.environ.pop("LBFSI_NO_DEPARTURE_CACHE", None)
        if old is not None:
            os.environ["LBFSI_NO_DEPARTURE_CACHE"] = old
    m.init_fields(flow, M0[None])
    m.blend_mesh(states, prev)
    loads = []
    for _ in range(steps):
        m.step(1)
        loads.append(m.body_forces()[0].copy())
    out = (m.get_fields(), np.array(loads), m.body_state()[0], m.launch_count())
    m.close()
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cache_same_on_element_lists(L, precision):
    """Unstructured element lists: a shuffled cylinder O-grid list under a
    plunging body (interior nodes inside and outside the blend) and a
    shuffled C-grid list with its cut merged, under a pitching body."""
    prec = L.FP32 if precision == "fp32" else L.FP64
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=2.0, v_r=4.0)
    case = inputs.cylinder_case(25, 48, r_far=8.0, body=body)
    import oracle.mesh as OM
    sm = OM.ogrid_mesh(case.r, case.e)
    el = inputs.ogrid_element_list(sm.X, seed=86)
    M0 = el.to_list(inputs.initial_field(25, 48, case.flow, seed=86, noise=1e-2))
    st, pv = [(0.02, 0.0, 0.004, 0.0)], [(0.0199, 0.0, 0.004, 0.0)]
    a = _element_run(L, el, case.bodies, case.flow, M0, st, pv, 10, prec, True)
    b = _element_run(L, el, case.bodies, case.flow, M0, st, pv, 10, prec, False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
    assert a[3] == b[3] + 1   # the one pass that fills the cache
    pp = inputs.BodySpec(dof=2, xp=-0.2, yp=0.0, r_in=0.7, r_out=2.5, m_star=20.0, v_r=2.0,
                         x_alpha=0.3, r_alpha=0.5, wh_wa=0.5)
    cg = inputs.cgrid_case(33, 8, 17, 0.5, 0.25, r_far=5.0, wake=4.0, body=pp)
    el = inputs.cgrid_element_list(cg.X, cg.n_cut, seed=87)
    N = el.X.shape[0]
    rng = np.random.default_rng(87)
    M0 = np.empty((4, N))
    M0[0] = 1.0
    M0[1] = cg.flow.u_inf * (1 + 1e-2 * rng.uniform(-1, 1, N))
    M0[2] = 1e-2 * cg.flow.u_inf * rng.uniform(-1, 1, N)
    M0[3] = cg.flow.t_inf
    st, pv = [(0.01, 0.04, 0.002, 0.01)], [(0.00998, 0.03996, 0.002, 0.01)]
    a = _element_run(L, el, cg.bodies, cg.flow, M0, st, pv, 8, prec, True)
    b = _element_run(L, el, cg.bodies, cg.flow, M0, st, pv, 8, prec, False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
