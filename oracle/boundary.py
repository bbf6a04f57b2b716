"""Boundary conditions of the oracle (Sec. III A: wall by Grad's
approximation, Eqs. fnoneq, gnoneq, strainrate and the zero-normal-gradient
targets; inlet and outlet by equilibrium).

Test infrastructure only (see the package docstring).

Wall rows are i = 0 of an O-grid; far-field rows are i = Ni - 1.
"""
from __future__ import annotations

import numpy as np

from . import kinetics as K
from .ale import physical_gradient

MISSING_TOL = 1e-12


def wall_normals(mesh):
    """Unit normal n0 at every wall node (row 0), pointing out of the body
    into the fluid, in the undeformed frame.  The wall is the polygon of the
    elements' straight wall edges (even-indexed wall nodes are its vertices):
    an odd node takes its edge's normal, an even node the normalised sum of
    the normals of its two edges."""
    Nj = mesh.Nj
    P = mesh.X[0]
    n_edge = np.empty((Nj // 2, 2))
    for k in range(Nj // 2):
        a = P[2 * k]
        b = P[(2 * k + 2) % Nj]
        t = b - a
        n_edge[k] = np.array([t[1], -t[0]]) / np.hypot(t[0], t[1])
    n = np.empty((Nj, 2))
    for j in range(Nj):
        if j % 2:
            n[j] = n_edge[j // 2]
        else:
            v = n_edge[j // 2] + n_edge[(j // 2 - 1) % (Nj // 2)]
            n[j] = v / np.hypot(v[0], v[1])
    return n


def missing_mask(chat_wall, n0):
    """Populations of a wall node whose departure point lies inside the body:
    c_hat_i . n0 > 0 (reading R10; the departure point X - c_hat dt then lies
    behind the supporting line of the convex wall polygon).  chat_wall has
    shape [9, Nj, 2]."""
    dot = chat_wall[..., 0] * n0[None, :, 0] + chat_wall[..., 1] * n0[None, :, 1]
    return dot > MISSING_TOL


def wall_targets(mesh, M_prev, n0, dt, F_wall):
    """rho_tgt, T_tgt from the zero-normal-gradient condition: the values at
    B = A + dt n0 (the largest distance the paper allows), interpolated with
    second-order elements (Sec. III A).  Reading R19: the interpolated field is
    the previous step's moment field.  Also returns grad u and grad T at the
    wall nodes from the same field (first-order FE derivative, Eq. ddx+fem,
    one-sided along the wall-normal index), mapped to the physical frame."""
    Nj = mesh.Nj
    j = np.arange(Nj)
    i = np.zeros(Nj, dtype=np.int64)
    B = mesh.X[0] + dt * n0
    wa, wb, xi, eta, found = mesh.locate(B, i, j)
    if not np.all(found):
        raise RuntimeError("wall target point B outside the first element row")
    rho_b = mesh.interpolate(M_prev[0], wa, wb, xi, eta)
    T_b = mesh.interpolate(M_prev[3], wa, wb, xi, eta)
    grads = []
    for comp in (1, 2, 3):
        dX, dY = mesh.grad_X(M_prev[comp])
        gx, gy = physical_gradient(F_wall, dX[0], dY[0])
        grads.append((gx, gy))
    return rho_b, T_b, grads


def grad_populations(rho, ux, uy, T, grads, Cv, mu, dt, Pr):
    """Grad's approximation f^eq + dt f^(1), g^eq + dt g^(1) at the targets."""
    (dudx, dudy), (dvdx, dvdy), (dTdx, dTdy) = grads
    feq = K.f_eq(rho, ux, uy, T)
    geq = K.g_eq(rho, ux, uy, T, Cv)
    f1, g1 = K.grad_f1(rho, ux, uy, T, Cv, dudx, dudy, dvdx, dvdy, dTdx, dTdy, mu, dt, Pr)
    return feq + f1, geq + g1


def _outlet_values(mesh, M_prev, A, n_hat, i, j, dt):
    """rho, u_x, u_y, T of the previous step's moment field at
    B = A - dt n_hat, one time step inside the far field along its outward
    unit direction, by Q2 interpolation in the cells of node (i, j) (reading
    R20: the wall's zero-gradient construction of Sec. III A applied to the
    far field)."""
    B = A - dt * n_hat
    wa, wb, xi, eta, found = mesh.locate(B, i, j)
    if not np.all(found):
        raise RuntimeError("far-field point B outside the cells next to the far field")
    return [mesh.interpolate(M_prev[c], wa, wb, xi, eta) for c in range(4)]


def _unit(v):
    return v / np.hypot(v[..., 0], v[..., 1])[..., None]


def far_field_targets(mesh, M_prev, u_inf, T_inf, dt):
    """Inlet / outlet targets at the far-field row (Sec. III A 2).  Reading
    R20: a far-field node is an inlet where the free stream enters
    (U_inf . n_out < 0, n_out the outward direction of the grid line that
    ends there, X[last] - X[last-1]), else an outlet.  Targets are built the
    way the wall's are (Sec. III A 2 refers the outlet to the wall's
    zero-gradient construction): a quantity the boundary does not prescribe
    takes a zero normal gradient, imposed through the point B one time step
    inside the boundary along the outward unit direction, B = A - dt n_out,
    whose value is the Q2 interpolation of the previous step's moment field
    (as for the wall targets, reading R19).  The outlet prescribes nothing:
    rho, u and T all take the value at B.  The inlet prescribes the free
    stream's velocity and temperature (the paper does not list the inlet's
    target values); its density takes the value at B, which leaves the one
    outgoing acoustic wave of a subsonic inflow free (imposing rho as well
    over-specifies the inflow: with it the gas in the domain is compressed
    until the run turns non-physical after about a hundred convective
    times)."""
    last = mesh.Ni - 1
    Nj = mesh.Nj
    n_out = _unit(mesh.X[last] - mesh.X[last - 1])
    inlet = (u_inf[0] * n_out[:, 0] + u_inf[1] * n_out[:, 1]) < 0.0
    ob = _outlet_values(mesh, M_prev, mesh.X[last], n_out, np.full(Nj, last), np.arange(Nj), dt)
    rho = ob[0]
    ux = np.where(inlet, u_inf[0], ob[1])
    uy = np.where(inlet, u_inf[1], ob[2])
    T = np.where(inlet, T_inf, ob[3])
    return rho, ux, uy, T, inlet


# ----- C-grid (reading R29): open wall chain, outlet columns ---------------
def wall_normals_cgrid(mesh):
    """Unit normals of the wall nodes of a C-grid (its wall chains, each
    counterclockwise around its body, out of the body), zero on the cut.  A
    chain is the open polygon of straight edges between its even-offset
    nodes; interior nodes as on a closed wall.  A chain's end is a junction,
    one point with the mirrored column's node, which ends the mirrored chain
    (the same chain for a body that row 0 wraps around): its normal is the
    normalised sum of the normals of the two edges that meet there."""
    Nj = mesh.Nj
    P = mesh.X[0]

    def edge_normal(a, b):
        t = P[b] - P[a]
        return np.array([t[1], -t[0]]) / np.hypot(t[0], t[1])

    n = np.zeros((Nj, 2))
    for a, b in mesh.walls:
        for j in range(a, b + 1):
            m = j - a
            if m % 2:
                n[j] = edge_normal(j - 1, j + 1)
                continue
            if a < j < b:
                v = edge_normal(j - 2, j) + edge_normal(j, j + 2)
            else:
                # the junction: this chain's end edge and the mirrored chain's
                k = Nj - 1 - j
                mine = edge_normal(j, j + 2) if j == a else edge_normal(j - 2, j)
                other = edge_normal(k - 2, k) if j == a else edge_normal(k, k + 2)
                v = mine + other
            n[j] = v / np.hypot(v[0], v[1])
    return n


def far_field_mask_cgrid(mesh):
    """Far-field nodes of a C-grid: the last row and the outlet columns."""
    far = np.zeros((mesh.Ni, mesh.Nj), dtype=bool)
    far[mesh.Ni - 1, :] = True
    far[:, 0] = True
    far[:, mesh.Nj - 1] = True
    return far


def far_field_targets_cgrid(mesh, M_prev, u_inf, T_inf, dt):
    """Inlet / outlet targets on the far field of a C-grid (reading R20 on
    each boundary): on the last row the outward direction is that of the
    grid line along i, on the outlet columns (rows below the last) along j;
    the values at B = A - dt n_out as on an O-grid (the inlet prescribes the
    free stream's u and T, its density and every outlet quantity take the
    value at B).  Returns rho, ux, uy,
    T on the whole [Ni, Nj] grid (meaningful on the far-field mask only) and
    the inlet mask."""
    Ni, Nj = mesh.Ni, mesh.Nj
    X = mesh.X
    n_out = np.zeros((Ni, Nj, 2))
    n_out[..., 0] = 1.0          # placeholder off the far field
    n_out[:, 0] = _unit(X[:, 0] - X[:, 1])
    n_out[:, Nj - 1] = _unit(X[:, Nj - 1] - X[:, Nj - 2])
    n_out[Ni - 1] = _unit(X[Ni - 1] - X[Ni - 2])
    inlet = (u_inf[0] * n_out[..., 0] + u_inf[1] * n_out[..., 1]) < 0.0
    far = far_field_mask_cgrid(mesh)
    ii, jj = np.nonzero(far)
    ob = _outlet_values(mesh, M_prev, X[ii, jj], n_out[ii, jj], ii, jj, dt)
    out = []
    for c, free in enumerate((None, u_inf[0], u_inf[1], T_inf)):
        v = np.zeros((Ni, Nj))
        v[ii, jj] = ob[c]
        out.append(v if free is None else np.where(inlet, free, v))
    return out[0], out[1], out[2], out[3], inlet & far
