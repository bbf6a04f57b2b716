"""Pins of the oracle's C-grid (readings R28-R30) against facts that do not
come from the oracle itself:
- along the wake cut the generated elements are parallelograms (every cut
  column's grid line has the same direction), so Q2 interpolation reproduces
  any quadratic exactly, also at points in the mirrored cells across the cut;
  the index-space gradient stencil across the cut gives a closed-form value;
- wall normals of the open wall chain: unit, out of the ellipse, (1, 0) at the
  rear point, where the chain's two ends meet;
- wall force of the open chain: zero for a uniform stress, -A grad p for a
  linear pressure (divergence theorem, A the area of the wall polygon);
- a mirror-symmetric C-grid with a mirror-symmetric initial field stays
  mirror-symmetric (f_q(i, j) = f_q'(i, Nj-1-j), q' the reflected velocity);
- independent bodies (reading R32): fixed bodies' loads transfer to the
  linked pair's (forces add, moments by M + (r_b - r) x F_b), relabelling
  the bodies permutes their loads, and on a symmetric flow neither body has
  lift or moment and a free body stays at rest."""
import numpy as np
import pytest

import oracle.boundary as OB
import oracle.forces as OF
import oracle.mesh as OM
import oracle.solver as OS
from paper_2107_01370_gb300 import inputs


def _case(n_wall=33, n_cut=8, nr=24, **kw):
    return inputs.cgrid_case(n_wall, n_cut, nr, 0.6, 0.35, r_far=6.0, wake=4.0, **kw)


def _quad(P):
    x, y = P[..., 0], P[..., 1]
    return 0.7 + 1.3 * x - 0.4 * y + 0.9 * x * x - 1.1 * x * y + 0.6 * y * y


def _quad_grad(P):
    x, y = P[..., 0], P[..., 1]
    return 1.3 + 1.8 * x - 1.1 * y, -0.4 - 1.1 * x + 1.2 * y


def test_generated_cgrid_shape_and_cut():
    case = _case()
    X = case.X
    nt, jc = case.ntheta, case.n_cut
    assert nt % 2 == 1 and X.shape == (case.nr, nt, 2)
    for j in range(jc + 1):
        assert np.array_equal(X[0, j], X[0, nt - 1 - j])
    assert np.all(X[0, :jc + 1, 1] == 0.0)
    # rear point is where the wall starts and ends
    assert np.array_equal(X[0, jc], [0.6, 0.0])
    m = OM.CGridMesh(X, jc)
    x_xi, y_xi, x_eta, y_eta = m.metrics()
    assert np.all(x_xi * y_eta - y_xi * x_eta > 0)
    with pytest.raises(ValueError):
        OM.CGridMesh(X, jc + 2)       # nodes jc+1.. of the two sides do not coincide


@pytest.mark.parametrize("row", [0, 1, 2])
def test_quadratic_reproduced_across_the_cut(row):
    """Departure-type points around cut nodes in every direction, some of
    them in the mirrored cells below row 0, interpolate a quadratic exactly."""
    case = _case()
    X = case.X
    nt, jc = case.ntheta, case.n_cut
    m = OM.CGridMesh(X, jc)
    field = _quad(X)
    cols = [j for j in range(1, nt - 1) if j < jc or j > nt - 1 - jc]
    h = 0.3 * np.min(np.hypot(*(X[0, 1:jc + 1] - X[0, :jc]).T))
    worst = 0.0
    used_ghost = False
    for j in cols:
        for ang in np.linspace(0.0, 2.0 * np.pi, 16, endpoint=False):
            P = X[row, j] + h * np.array([np.cos(ang), np.sin(ang)])
            wa, wb, xi, eta, found = m.locate(P[None], np.array([row]), np.array([j]))
            assert found[0], (row, j, ang)
            used_ghost |= bool(wa[0] < 0)
            v = m.interpolate(field, wa, wb, xi, eta)[0]
            worst = max(worst, abs(v - _quad(P)))
    assert worst < 1e-12
    if row == 0:
        assert used_ghost


def test_gradient_across_the_cut():
    """At a row-0 cut node (x, 0) the i-stencil differences the field between
    its first rows on both sides of the cut, (x + h, h) and (x + h, -h) on the
    45-degree grid lines, the j-stencil along the cut.  For F = y^2 + x y the
    stencil gives exactly (dF/dX, dF/dY) = (0, x + h), the y-derivative at
    the shifted point, which a wrong mirrored row would not.  Linear fields
    are exact everywhere, the rear point included."""
    case = _case()
    X = case.X
    nt, jc = case.ntheta, case.n_cut
    m = OM.CGridMesh(X, jc)
    dX, dY = m.grad_X(X[..., 1] ** 2 + X[..., 0] * X[..., 1])
    for j in list(range(1, jc)) + list(range(nt - jc, nt - 1)):
        assert abs(dX[0, j]) < 1e-12
        assert abs(dY[0, j] - X[1, j, 0]) < 1e-12
    lx, ly = m.grad_X(0.7 + 1.3 * X[..., 0] - 0.4 * X[..., 1])
    assert np.abs(lx - 1.3).max() < 1e-11 and np.abs(ly + 0.4).max() < 1e-11


def test_wrong_mirror_breaks_the_quadratic():
    """Planted mistake: ghost rows read their values one column off.  The
    quadratic across the cut is no longer reproduced, so the pin above has
    teeth."""
    case = _case()
    X = case.X
    m = OM.CGridMesh(X, case.n_cut)
    bad = OM.CGridMesh(X, case.n_cut)
    good = bad.window_node

    def shifted(wa, wb, a, b):
        i, j = good(wa, wb, a, b)
        return i, np.where(np.asarray(wa) < 0, np.maximum(j - 1, 0), j)

    bad.window_node = shifted
    j = 3
    P = X[0, j] - np.array([0.0, 0.3 * X[1, j, 1]])   # below the cut, within the first row
    wa, wb, xi, eta, found = m.locate(P[None], np.array([0]), np.array([j]))
    assert found[0] and wa[0] < 0
    assert abs(m.interpolate(_quad(X), wa, wb, xi, eta)[0] - _quad(P)) < 1e-12
    assert abs(bad.interpolate(_quad(X), wa, wb, xi, eta)[0] - _quad(P)) > 1e-6


def test_wall_normals_of_the_open_chain():
    case = _case()
    m = OM.CGridMesh(case.X, case.n_cut)
    n = OB.wall_normals_cgrid(m)
    jc, nt = case.n_cut, case.ntheta
    wall = np.arange(jc, nt - jc)
    assert np.allclose(np.hypot(n[wall, 0], n[wall, 1]), 1.0, atol=1e-14)
    P = case.X[0, wall]
    grad = np.stack([2 * P[:, 0] / 0.6 ** 2, 2 * P[:, 1] / 0.35 ** 2], axis=1)
    assert np.all(np.sum(n[wall] * grad, axis=1) > 0)
    assert np.allclose(n[jc], [1.0, 0.0], atol=1e-14)
    assert np.array_equal(n[jc], n[nt - 1 - jc])
    assert np.all(n[:jc] == 0.0) and np.all(n[nt - jc:] == 0.0)


def test_open_chain_force_closed_forms():
    case = _case()
    jc, nt = case.n_cut, case.ntheta
    P = case.X[0, jc:nt - jc]
    k = P.shape[0]
    F = OF.wall_force(P, np.full(k, -2.0), np.full(k, 0.3), np.full(k, -0.7), np.zeros(2),
                      closed=False)
    assert max(abs(F[0]), abs(F[1]), abs(F[2])) < 1e-13
    # linear pressure p = a . x: sigma = -p I; F = -sum p n ds = -A a (the
    # outward normal of the fluid region is -n)
    a = np.array([0.4, -0.25])
    p = P @ a
    F = OF.wall_force(P, -p, np.zeros(k), -p, np.zeros(2), closed=False)
    V = P[0:-1:2]
    area = 0.5 * np.sum(V[:, 0] * np.roll(V[:, 1], -1) - np.roll(V[:, 0], -1) * V[:, 1])
    assert abs(F[0] + area * a[0]) < 1e-13 and abs(F[1] + area * a[1]) < 1e-13


REFLECT = np.array([0, 1, 4, 3, 2, 8, 7, 6, 5])   # c_q -> (c_x, -c_y)


def test_mirror_symmetric_flow_stays_symmetric():
    case = _case(n_wall=29, n_cut=6, nr=16)
    X = case.X
    nt, jc = case.ntheta, case.n_cut
    # the generator mirrors the two sides up to the round-off of cos/sin
    assert np.allclose(X[:, ::-1, 0], X[:, :, 0], atol=1e-14)
    assert np.allclose(X[:, ::-1, 1], -X[:, :, 1], atol=1e-14)
    Xs = X.copy()
    Xs[:, nt // 2 + 1:, 0] = X[:, :nt // 2, 0][:, ::-1]
    Xs[:, nt // 2 + 1:, 1] = -X[:, :nt // 2, 1][:, ::-1]
    Xs[:, nt // 2, 1] = 0.0
    M0 = inputs.initial_field(case.nr, nt, case.flow, noise=1e-2, seed=7)
    M = M0.copy()
    M[0] = 0.5 * (M0[0] + M0[0, :, ::-1])
    M[1] = 0.5 * (M0[1] + M0[1, :, ::-1])
    M[2] = 0.5 * (M0[2] - M0[2, :, ::-1])
    M[3] = 0.5 * (M0[3] + M0[3, :, ::-1])
    M[2, 0, :jc + 1] = 0.0
    M[2, 0, nt - 1 - jc:] = 0.0
    m = OM.CGridMesh(Xs, jc)
    s = OS.Solver.from_case(m, case, M)
    for _ in range(4):
        r = s.step()
    f = r.f_post
    scale = np.abs(f).max()
    assert np.abs(f - f[REFLECT][:, :, ::-1]).max() < 1e-12 * scale
    assert abs(r.force[1]) < 1e-12 and abs(r.force[2]) < 1e-12
    # the lower copies of the cut nodes hold the upper copies' values
    assert np.array_equal(r.M[:, 0, nt - 1 - jc:], r.M[:, 0, :jc + 1][:, ::-1])


# ----- several wall chains: two cylinders in tandem (reading R31) ---------
def _tandem(nr=17):
    return inputs.tandem_cgrid(34, 17, 11, 16, nr)


def test_tandem_mesh_chains_and_normals():
    X, walls = _tandem()
    nt = X.shape[1]
    assert walls == [(16, 32), (44, nt - 1 - 44), (nt - 1 - 32, nt - 1 - 16)]
    m = OM.CGridMesh(X, walls=walls)
    x_xi, y_xi, x_eta, y_eta = m.metrics()
    assert np.all(x_xi * y_eta - y_xi * x_eta > 0)
    n = OB.wall_normals_cgrid(m)
    for (a, b), c in zip(walls, ((4.0, 0.0), (0.0, 0.0), (4.0, 0.0))):
        cols = np.arange(a, b + 1)
        assert np.allclose(np.hypot(n[cols, 0], n[cols, 1]), 1.0, atol=1e-14)
        out = X[0, cols] - np.array(c)
        assert np.all(np.sum(n[cols] * out, axis=1) > 0)        # out of each cylinder
    # junctions: the rear points face downstream, the rear body's front upstream
    assert np.allclose(n[16], [1.0, 0.0], atol=1e-14) and np.allclose(n[44], [1.0, 0.0], atol=1e-14)
    assert np.allclose(n[32], [-1.0, 0.0], atol=1e-14)
    assert m.junction_dir[16] == -1 and m.junction_dir[32] == 1 and m.junction_dir[44] == -1
    # the one-chain form of the constructor is the single C-grid
    Xc = inputs.cgrid_ellipse(17, 4, 9, 0.6, 0.35, r_far=4.0, wake=3.0)
    a1, a2 = OM.CGridMesh(Xc, 4), OM.CGridMesh(Xc, walls=[(4, Xc.shape[1] - 5)])
    assert np.array_equal(a1.junction, a2.junction) and np.array_equal(a1.metrics()[0], a2.metrics()[0])


def test_tandem_forces_closed_forms():
    """Summed over the three chains: zero for a uniform stress; -(A_f + A_r) a
    for a linear pressure a . x (both cylinders' polygon areas)."""
    X, walls = _tandem()
    P0 = X[0]
    a = np.array([0.4, -0.25])
    tot_u = np.zeros(3)
    tot_p = np.zeros(3)
    for s_, e_ in walls:
        P = P0[s_:e_ + 1]
        k = P.shape[0]
        tot_u += OF.wall_force(P, np.full(k, -2.0), np.full(k, 0.3), np.full(k, -0.7), np.zeros(2),
                               closed=False)
        p = P @ a
        tot_p += OF.wall_force(P, -p, np.zeros(k), -p, np.zeros(2), closed=False)
    assert np.abs(tot_u).max() < 1e-13

    def area(V):
        return 0.5 * np.sum(V[:, 0] * np.roll(V[:, 1], -1) - np.roll(V[:, 0], -1) * V[:, 1])

    (r0, r1), (f0, f1), (l0, l1) = walls
    A_front = area(P0[f0:f1 + 1:2][:-1])
    A_rear = area(np.concatenate([P0[r0:r1 + 1:2], P0[l0:l1 + 1:2][1:-1]]))
    assert abs(tot_p[0] + (A_front + A_rear) * a[0]) < 1e-13
    assert abs(tot_p[1] + (A_front + A_rear) * a[1]) < 1e-13


def test_tandem_linear_fields_reproduced_across_the_gap():
    """Points around the gap's and the wake's cut nodes, many of them in the
    mirrored cells below row 0, interpolate a linear field exactly (it lies in
    the Q2 space of every bilinear element); a window read one column off
    below row 0 does not."""
    X, walls = _tandem()
    m = OM.CGridMesh(X, walls=walls)
    field = 0.3 + 1.7 * X[..., 0] - 0.9 * X[..., 1]
    cut = [j for j in range(1, (X.shape[1] - 1) // 2) if m.cut_columns()[j]]
    ghost = 0
    for j in cut:
        h = 0.3 * abs(X[1, j, 1])
        for ang in np.linspace(0.0, 2.0 * np.pi, 12, endpoint=False):
            P = X[0, j] + h * np.array([np.cos(ang), np.sin(ang)])
            wa, wb, xi, eta, found = m.locate(P[None], np.array([0]), np.array([j]))
            assert found[0], (j, ang)
            ghost += int(wa[0] < 0)
            v = m.interpolate(field, wa, wb, xi, eta)[0]
            assert abs(v - (0.3 + 1.7 * P[0] - 0.9 * P[1])) < 1e-12
    assert ghost > 0


def test_tandem_symmetric_flow_stays_symmetric():
    X, walls = _tandem(nr=13)
    nt = X.shape[1]
    flow = inputs.FlowSpec(ma=0.2, re=100.0, dt=float(np.hypot(*(X[0, 45] - X[0, 44]))) / 3.0)
    case = inputs.CGridCase(nr=X.shape[0], ntheta=nt, n_cut=None, X=X, centre=(0.0, 0.0), flow=flow,
                            bodies=[inputs.BodySpec(dof=0)])
    M0 = inputs.initial_field(case.nr, nt, flow, noise=1e-2, seed=9)
    M = M0.copy()
    M[0] = 0.5 * (M0[0] + M0[0, :, ::-1])
    M[1] = 0.5 * (M0[1] + M0[1, :, ::-1])
    M[2] = 0.5 * (M0[2] - M0[2, :, ::-1])
    M[3] = 0.5 * (M0[3] + M0[3, :, ::-1])
    m = OM.CGridMesh(X, walls=walls)
    M[2, 0, m.cut_columns() | m.junction] = 0.0
    s = OS.Solver.from_case(m, case, M)
    for _ in range(4):
        r = s.step()
    f = r.f_post
    assert np.abs(f - f[REFLECT][:, :, ::-1]).max() < 1e-12 * np.abs(f).max()
    assert abs(r.force[1]) < 1e-12 and abs(r.force[2]) < 1e-12


# ----- independent bodies on one C-grid (reading R32) ----------------------
def _tandem_flow(X):
    return inputs.FlowSpec(ma=0.2, re=100.0, dt=float(np.hypot(*(X[0, 45] - X[0, 44]))) / 3.0)


def _run(X, walls, bodies, M, steps, wall_body=None):
    flow = _tandem_flow(X)
    case = inputs.CGridCase(nr=X.shape[0], ntheta=X.shape[1], n_cut=None, X=X, centre=(0.0, 0.0), flow=flow,
                            bodies=bodies)
    s = OS.Solver.from_case(OM.CGridMesh(X, walls=walls, wall_body=wall_body), case, M)
    out = [s.step() for _ in range(steps)]
    return s, out


def _cross(r, F):
    return r[0] * F[1] - r[1] * F[0]


def test_independent_fixed_bodies_transfer_to_the_linked_load():
    """Two fixed cylinders as independent bodies see the flow of the linked
    pair (fixed walls: the same step), so their loads add up to the linked
    load: the forces sum, and the moments about each body's own reference
    point, moved to the linked reference point (M + (r_b - r) x F_b), sum to
    the linked moment.  Relabelling the bodies permutes the loads exactly."""
    X, walls = _tandem(nr=13)
    M0 = inputs.initial_field(X.shape[0], X.shape[1], _tandem_flow(X), noise=1e-2, seed=21)
    r_lin, r_f, r_r = np.array([1.0, 0.2]), np.array([0.0, 0.1]), np.array([4.0, -0.3])
    _, lin = _run(X, walls, [inputs.BodySpec(dof=0, xp=r_lin[0], yp=r_lin[1])], M0, 3)
    front = inputs.BodySpec(dof=0, xp=r_f[0], yp=r_f[1])
    rear = inputs.BodySpec(dof=0, xp=r_r[0], yp=r_r[1])
    _, ind = _run(X, walls, [front, rear], M0, 3, wall_body=[1, 0, 1])
    _, swp = _run(X, walls, [rear, front], M0, 3, wall_body=[0, 1, 0])
    for a, b, c in zip(lin, ind, swp):
        assert np.array_equal(a.f_post, b.f_post)
        Ff, Fr = np.array(b.forces[0]), np.array(b.forces[1])
        F = np.array(a.force)
        scale = np.abs(F[:2]).max()
        assert np.abs(Ff[:2] + Fr[:2] - F[:2]).max() < 1e-13 * scale
        m_t = Ff[2] + _cross(r_f - r_lin, Ff[:2]) + Fr[2] + _cross(r_r - r_lin, Fr[:2])
        assert abs(m_t - F[2]) < 1e-13 * scale
        # each body takes a share of its own (the rear body's drag sign is
        # not the front's: it sits in the front body's wake)
        assert np.abs(Ff).max() > 1e-3 * scale and np.abs(Fr).max() > 1e-3 * scale
        assert c.forces[0] == b.forces[1] and c.forces[1] == b.forces[0]


def test_independent_bodies_symmetric_flow_no_lift_on_either():
    """A mirror-symmetric field on the symmetric tandem mesh: each body's
    lift and its moment about a reference point on the axis vanish, and a
    free transverse body next to a fixed one is not driven (its state stays
    at rest); the fixed body's state never changes."""
    X, walls = _tandem(nr=13)
    flow = _tandem_flow(X)
    M0 = inputs.initial_field(X.shape[0], X.shape[1], flow, noise=1e-2, seed=9)
    M = M0.copy()
    M[0] = 0.5 * (M0[0] + M0[0, :, ::-1])
    M[1] = 0.5 * (M0[1] + M0[1, :, ::-1])
    M[2] = 0.5 * (M0[2] - M0[2, :, ::-1])
    M[3] = 0.5 * (M0[3] + M0[3, :, ::-1])
    m = OM.CGridMesh(X, walls=walls)
    M[2, 0, m.cut_columns() | m.junction] = 0.0
    free = inputs.BodySpec(dof=1, xc=0.0, yc=0.0, xp=0.0, yp=0.0, r_in=0.7, r_out=1.8, m_star=2.0, v_r=4.0)
    fixed = inputs.BodySpec(dof=0, xp=4.0, yp=0.0)
    s, out = _run(X, walls, [free, fixed], M, 3, wall_body=[1, 0, 1])
    for r in out:
        for Fb in r.forces:
            assert abs(Fb[1]) < 1e-12 and abs(Fb[2]) < 1e-12
        assert abs(r.forces[0][0]) > 1e-6 and abs(r.forces[1][0]) > 1e-6
    assert abs(s.S[0]["h"]) < 1e-15 and abs(s.S[0]["hdot"]) < 1e-13
    assert all(v == 0.0 for v in s.S[1].values())


def test_departure_on_a_thin_wake_cell_edge():
    """Reading R8's second pass: in the wake of the NACA 0012 C-grid the
    cells behind the clustered trailing-edge columns are ~5000 times longer
    than wide and far from the origin, so a departure point on the edge two
    of them share comes out of the bilinear inverse ~1e-12 outside both.  It
    is taken (a linear field interpolates exactly), while a point a
    millionth of the cell width beyond the adjacent cells is still refused."""
    case = inputs.naca0012_flutter_case()
    m = OM.CGridMesh(case.X, case.n_cut)
    X = case.X
    i, j = 182, 642
    d = case.flow.dt * np.array([1.0, -1.0])
    P = X[i, j] - d
    strict = [m.locate_in_cell(np.array([a]), np.array([b]), P[None])[4][0]
              for a in (i - 1, i) for b in (j - 1, j)]
    assert not any(strict)                        # outside every cell at 1e-12
    wa, wb, xi, eta, found = m.locate(P[None], np.array([i]), np.array([j]))
    assert found[0]
    lin = 0.4 + 1.3 * X[..., 0] - 0.7 * X[..., 1]
    v = m.interpolate(lin, wa, wb, xi, eta)[0]
    assert abs(v - (0.4 + 1.3 * P[0] - 0.7 * P[1])) < 1e-9
    # the middle of the far edge of the adjacent cells is taken; a millionth
    # of the cell width beyond it is not
    w = np.hypot(*(X[i, j + 1] - X[i, j]))
    e = (X[i, j + 1] - X[i, j]) / w
    M_edge = 0.5 * (X[i, j + 1] + X[i + 1, j + 1])
    assert m.locate(M_edge[None], np.array([i]), np.array([j]))[4][0]
    Q = M_edge + 1e-6 * w * e
    assert not m.locate(Q[None], np.array([i]), np.array([j]))[4][0]
