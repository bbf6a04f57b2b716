"""Pins of the oracle's boundary conditions (Sec. III A) against what the
geometry and the mathematics fix, each chosen so that a plausible mistake
fails it:

- wall normals and the missing set on a circle: closed forms from the node
  angles, and for nodes on an edge the brute-force test whether the
  departure point lies inside the body polygon;
- wall targets (reading R19): on fields linear in space the Q2 value at
  B = A + dt n0 and the FE wall gradients are exact, so the point B (not
  A - dt n0), the frame mapping of the gradient and the field that is
  interpolated are all fixed; a coupled step takes them from the previous
  step's moment field;
- far field (reading R20): the inlet set against the outward direction of
  the boundary computed from the mesh generator's closed form; the targets
  against the linear field at B = A - dt n_out (not the inner neighbour),
  the inlet's velocity and temperature against the free stream, on an
  O-grid and on a C-grid (last row and outlet columns).
"""
import math

import numpy as np
import pytest

from oracle import boundary as BC, kinetics as K, mesh as OM, solver as OS
from oracle.ale import physical_gradient  # noqa: F401  (the mapping under test)
from paper_2107_01370_gb300 import inputs

C = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)],
             dtype=np.float64)


def _linear(coef, X):
    """a0 + a1 x + a2 y at points X[..., 2]."""
    return coef[0] + coef[1] * X[..., 0] + coef[2] * X[..., 1]


LIN = {0: (1.1, 0.03, -0.02),      # rho
       1: (0.05, 0.011, 0.007),     # u_x
       2: (-0.02, -0.004, 0.013),   # u_y
       3: (0.33, 0.006, -0.009)}    # T


def _linear_moments(X):
    return np.stack([_linear(LIN[c], X) for c in range(4)])


def _circle_case(nr=12, nt=32, r_far=6.0):
    case = inputs.cylinder_case(nr, nt, r_far=r_far)
    mesh = OM.ogrid_mesh(case.r, case.e)
    theta = 2.0 * np.pi * np.arange(nt) / nt
    return case, mesh, theta


# ----- wall normals and the missing set --------------------------------------
def test_wall_normals_of_a_circle_are_radial():
    """On the polygon of a circle's even nodes the normal at a vertex (the
    bisector of its edges) and at an edge midpoint (the edge normal) both
    point along the node's polar angle 2 pi j / N."""
    _, mesh, theta = _circle_case()
    n0 = BC.wall_normals(mesh)
    np.testing.assert_allclose(n0, np.stack([np.cos(theta), np.sin(theta)], axis=1), atol=1e-14)


def _inside_polygon(P, poly):
    """Winding-number point-in-polygon test (brute force, no mesh code)."""
    wn = 0
    n = len(poly)
    for k in range(n):
        a, b = poly[k], poly[(k + 1) % n]
        cross = (b[0] - a[0]) * (P[1] - a[1]) - (P[0] - a[0]) * (b[1] - a[1])
        if a[1] <= P[1] < b[1] and cross > 0:
            wn += 1
        elif b[1] <= P[1] < a[1] and cross < 0:
            wn -= 1
    return wn != 0


def test_missing_set_of_a_static_wall():
    """A fixed wall (c_hat = c): the missing populations are exactly those
    with c . n0 > 0, n0 the radial direction of the node; at the nodes on an
    edge (odd j) these are exactly the directions whose departure point
    X - dt c lies inside the body polygon."""
    case, mesh, theta = _circle_case()
    nt = mesh.Nj
    u_inf = case.flow.u_inf
    M0 = np.empty((4, mesh.Ni, nt))
    M0[0], M0[1], M0[2], M0[3] = 1.0, u_inf, 0.0, case.flow.t_inf
    s = OS.Solver.from_case(mesh, case, M0)
    r = s.step()
    expect = (C[:, 0, None] * np.cos(theta)[None] + C[:, 1, None] * np.sin(theta)[None]) > 1e-12
    np.testing.assert_array_equal(r.missing[:, 0], expect)
    assert not r.missing[:, 1:].any()
    poly = mesh.X[0, 0::2]
    dt = case.flow.dt
    for j in range(1, nt, 2):
        for q in range(1, 9):
            P = mesh.X[0, j] - dt * C[q]
            assert _inside_polygon(P, poly) == expect[q, j], (q, j)


# ----- wall targets -------------------------------------------------------------
def _mesh_variants():
    case, mesh, _ = _circle_case()
    yield "circle", mesh, case.flow.dt
    wall = inputs.ellipse_wall(48, 0.6, 0.35)
    X = inputs.algebraic_ogrid(wall, 14, 6.0, 0.02)
    yield "ellipse", OM.Q2Mesh(X, periodic_i=False, periodic_j=True), 0.006


@pytest.mark.parametrize("which", ["circle", "ellipse"])
def test_wall_targets_on_linear_fields(which):
    """rho_B, T_B are the field at B = A + dt n0 (exact for a field linear in
    X: Q2 reproduces it on subparametric elements); the wall gradients of a
    field linear in the physical frame x = R(alpha) X come back exactly as
    its physical gradient through F = R(alpha) (a transposed or missing
    mapping fails)."""
    mesh = dt = None
    for name, m_, dt_ in _mesh_variants():
        if name == which:
            mesh, dt = m_, dt_
    n0 = BC.wall_normals(mesh)
    alpha = 0.3
    R = np.array([[math.cos(alpha), -math.sin(alpha)], [math.sin(alpha), math.cos(alpha)]])
    x = np.einsum("ab,ijb->ija", R, mesh.X)     # physical positions of a rigid rotation
    M_prev = _linear_moments(x)
    Fw = np.broadcast_to(R, (mesh.Nj, 2, 2)).copy()
    rho_b, T_b, grads = BC.wall_targets(mesh, M_prev, n0, dt, Fw)
    B = np.einsum("ab,jb->ja", R, mesh.X[0] + dt * n0)
    np.testing.assert_allclose(rho_b, _linear(LIN[0], B), rtol=0, atol=1e-13)
    np.testing.assert_allclose(T_b, _linear(LIN[3], B), rtol=0, atol=1e-13)
    # B lies one time step from A (a wrong point, A - dt n0, is 2 dt away)
    A = x[0]
    np.testing.assert_allclose(np.hypot(*(B - A).T), dt, rtol=1e-12)
    for comp, (gx, gy) in zip((1, 2, 3), grads):
        np.testing.assert_allclose(gx, LIN[comp][1], rtol=0, atol=1e-12)
        np.testing.assert_allclose(gy, LIN[comp][2], rtol=0, atol=1e-12)


def test_wall_targets_of_a_step_come_from_the_previous_field():
    """Inside a coupled step the missing populations are Grad's populations
    at the targets built from the moment field of the previous step (reading
    R19), not from the field the step produces."""
    case, mesh, _ = _circle_case()
    M0 = inputs.initial_field(mesh.Ni, mesh.Nj, case.flow, seed=3, noise=2e-2)
    s = OS.Solver.from_case(mesh, case, M0)
    r1 = s.step()
    r2 = s.step()
    dt, Cv = case.flow.dt, 1.0 / (case.flow.gamma - 1.0)
    n0 = BC.wall_normals(mesh)
    Fw = np.broadcast_to(np.eye(2), (mesh.Nj, 2, 2)).copy()
    zero = np.zeros(mesh.Nj)

    def grad_pops(Mf):
        rho_b, T_b, grads = BC.wall_targets(mesh, Mf, n0, dt, Fw)
        return BC.grad_populations(rho_b, zero, zero, T_b, grads, Cv, s.mu, dt, s.Pr)

    miss = r2.missing[:, 0]
    f_prev, g_prev = grad_pops(r1.M)
    np.testing.assert_allclose(r2.f_pre[:, 0][miss], f_prev[miss], rtol=1e-14, atol=0)
    np.testing.assert_allclose(r2.g_pre[:, 0][miss], g_prev[miss], rtol=1e-14, atol=0)
    f_cur, _ = grad_pops(r2.M)
    assert np.abs(f_cur[miss] - f_prev[miss]).max() > 1e-9   # the two readings differ here


# ----- far field -----------------------------------------------------------------
@pytest.mark.parametrize("beta", [0.0, 0.7, math.pi])
def test_far_field_targets_on_an_ogrid(beta):
    """Inlet exactly where the free stream enters through the far-field
    circle, U . (cos theta, sin theta) < 0.  At B = A - dt (cos theta,
    sin theta): the inlet's density and every outlet quantity equal the
    linear field there; the inlet's velocity and temperature are the free
    stream's."""
    case, mesh, theta = _circle_case()
    dt = case.flow.dt
    U = 0.08
    u_inf = (U * math.cos(beta), U * math.sin(beta))
    M_prev = _linear_moments(mesh.X)
    rho, ux, uy, T, inlet = BC.far_field_targets(mesh, M_prev, u_inf, 1.0 / 3.0, dt)
    un = np.cos(theta - beta)
    sure = np.abs(un) > 1e-9
    np.testing.assert_array_equal(inlet[sure], (un < 0)[sure])
    assert inlet.any() and (~inlet).any()
    n = np.stack([np.cos(theta), np.sin(theta)], axis=1)
    B = mesh.X[-1] - dt * n
    for comp, v in enumerate((rho, ux, uy, T)):
        free = (None, u_inf[0], u_inf[1], 1.0 / 3.0)[comp]
        at_b = ~inlet if free is not None else np.ones_like(inlet)
        if free is not None:
            np.testing.assert_array_equal(v[inlet], free)
        np.testing.assert_allclose(v[at_b], _linear(LIN[comp], B[at_b]), rtol=0, atol=1e-13)


@pytest.mark.parametrize("beta", [0.0, math.pi])
def test_far_field_targets_on_a_cgrid(beta):
    """C-grid from straight grid lines W_j -> C_j (the generator's closed
    form): the last row's outward direction is C_j - W_j, the outlet
    columns' is +x.  Inlet sets and targets as on an O-grid, on the last
    row and on both outlet columns (row 0 included)."""
    n_wall, n_cut, nr = 33, 8, 12
    X = inputs.cgrid_ellipse(n_wall, n_cut, nr, 0.6, 0.3, r_far=6.0)
    mesh = OM.CGridMesh(X, n_cut)
    Ni, Nj = mesh.Ni, mesh.Nj
    dt = 0.004
    U = 0.08
    u_inf = (U * math.cos(beta), U * math.sin(beta))
    M_prev = _linear_moments(X)
    rho, ux, uy, T, inlet = BC.far_field_targets_cgrid(mesh, M_prev, u_inf, 1.0 / 3.0, dt)
    far = BC.far_field_mask_cgrid(mesh)
    n = np.zeros((Ni, Nj, 2))
    n[:, 0] = (1.0, 0.0)
    n[:, Nj - 1] = (1.0, 0.0)
    d = X[-1] - X[0]
    n[-1] = d / np.hypot(d[:, 0], d[:, 1])[:, None]
    un = u_inf[0] * n[..., 0] + u_inf[1] * n[..., 1]
    np.testing.assert_array_equal(inlet[far], (un < 0)[far])
    assert inlet[far].any() and (~inlet[far]).any()
    outlet = far & ~inlet
    B = X - dt * n
    for comp, v in enumerate((rho, ux, uy, T)):
        free = (None, u_inf[0], u_inf[1], 1.0 / 3.0)[comp]
        at_b = outlet if free is not None else far
        if free is not None:
            np.testing.assert_array_equal(v[far & inlet], free)
        np.testing.assert_allclose(v[at_b], _linear(LIN[comp], B[at_b]), rtol=0, atol=1e-13)
    # the outlet columns are outlets for a stream along +x, inlets against it
    assert (not inlet[: Ni - 1, 0].any()) if beta == 0.0 else inlet[: Ni - 1, 0].all()


def test_outlet_targets_inside_a_step_use_the_previous_field():
    """A coupled step's far-field outlet nodes take, as moments, the targets
    built from the previous step's field (reading R20), and their
    post-collision populations are the equilibria there."""
    case, mesh, _ = _circle_case()
    M0 = inputs.initial_field(mesh.Ni, mesh.Nj, case.flow, seed=4, noise=2e-2)
    s = OS.Solver.from_case(mesh, case, M0)
    r1 = s.step()
    r2 = s.step()
    t = BC.far_field_targets(mesh, r1.M, s.u_inf, s.T_inf, case.flow.dt)
    for c in range(4):
        np.testing.assert_array_equal(r2.M[c, -1], t[c])
    np.testing.assert_allclose(r2.f_post[:, -1], K.f_eq(t[0], t[1], t[2], t[3]), rtol=1e-15)
    outlet = ~t[4]
    # the outlet value is not the inner neighbour's (the earlier reading)
    assert np.abs(r2.M[0, -1][outlet] - r1.M[0, -2][outlet]).max() > 1e-9
