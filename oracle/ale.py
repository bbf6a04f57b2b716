"""ALE kinematics and the blended mesh of the oracle (Sec. II A, Eqs. dx_ref,
DboltzmannEqn_ALE; Sec. II D, Eq. blendPol and the blended map).

Test infrastructure only (see the package docstring).

A body b carries a region of influence centred at (xc, yc) with a rigid zone
|X - Xc| < r_in and a blended zone r_in <= |X - Xc| <= r_out; its rigid map is
G'_b(X) = Xp + R(alpha)(X - Xp) + (0, h)  (plunge h, pitch alpha about Xp).

Reading R6: s_R = (|X - Xc| - r_in) / (r_out - r_in), radial distance from
the centre of the region; r_blend = 0 moves a node rigidly, r_blend = 1 keeps
it fixed.  With several bodies (non-overlapping regions, Sec. II D) the
displacements add: x = X + sum_b (1 - r_b(X)) (G'_b(X) - X), which is the
paper's x = r X + (1 - r) G'(X) for one body.
"""
from __future__ import annotations

import numpy as np

from .kinetics import C


def r5(s):
    """r5(s) = 10 s^3 - 15 s^4 + 6 s^5 (Eq. blendPol)."""
    return 10.0 * s ** 3 - 15.0 * s ** 4 + 6.0 * s ** 5


def dr5(s):
    """d r5 / ds = 30 s^2 - 60 s^3 + 30 s^4."""
    return 30.0 * s ** 2 - 60.0 * s ** 3 + 30.0 * s ** 4


def blend(X, body):
    """s_R, r_blend and d r_blend / dX (both components) at points X[..., 2]."""
    dx = X[..., 0] - body["xc"]
    dy = X[..., 1] - body["yc"]
    dist = np.sqrt(dx * dx + dy * dy)
    width = body["r_out"] - body["r_in"]
    s = (dist - body["r_in"]) / width
    rb = np.where(s < 0.0, 0.0, np.where(s > 1.0, 1.0, r5(np.clip(s, 0.0, 1.0))))
    inside = (s >= 0.0) & (s <= 1.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        ds_dx = np.where(inside, dx / (dist * width), 0.0)
        ds_dy = np.where(inside, dy / (dist * width), 0.0)
    d = np.where(inside, dr5(np.clip(s, 0.0, 1.0)), 0.0)
    return s, rb, d * ds_dx, d * ds_dy


def rotation(alpha):
    ca, sa = np.cos(alpha), np.sin(alpha)
    return np.array([[ca, -sa], [sa, ca]])


def rigid_displacement(X, body, state):
    """d_b(X) = G'_b(X) - X = Xp + R(alpha)(X - Xp) + (0, h) - X."""
    R = rotation(state["alpha"])
    px = X[..., 0] - body["xp"]
    py = X[..., 1] - body["yp"]
    gx = body["xp"] + R[0, 0] * px + R[0, 1] * py
    gy = body["yp"] + R[1, 0] * px + R[1, 1] * py + state["h"]
    return gx - X[..., 0], gy - X[..., 1]


def mesh_displacement(X, bodies, states):
    """x - X = sum_b (1 - r_b)(G'_b(X) - X)."""
    d = np.zeros_like(X)
    for body, st in zip(bodies, states):
        if body["dof"] == 0:
            continue
        _, rb, _, _ = blend(X, body)
        ux, uy = rigid_displacement(X, body, st)
        d[..., 0] = d[..., 0] + (1.0 - rb) * ux
        d[..., 1] = d[..., 1] + (1.0 - rb) * uy
    return d


def mesh_position(X, bodies, states):
    """x = X + sum_b (1 - r_b)(G'_b(X) - X)."""
    return X + mesh_displacement(X, bodies, states)


def deformation_gradient(X, bodies, states):
    """F_jk = d x_j / d X_k of the blended map, evaluated analytically
    (reading R5):
      F = I + sum_b [(1 - r_b)(R_b - I) - d_b (grad r_b)^T].
    The paper's ALE Jacobian is g = F^T (g_ij = d x_j / d X_i, reading R2), so
    that grad_x = g^{-1} grad_X (Eq. dx_ref)."""
    F = np.zeros(X.shape[:-1] + (2, 2))
    F[..., 0, 0] = 1.0
    F[..., 1, 1] = 1.0
    for body, st in zip(bodies, states):
        if body["dof"] == 0:
            continue
        _, rb, drx, dry = blend(X, body)
        R = rotation(st["alpha"])
        ux, uy = rigid_displacement(X, body, st)
        w = 1.0 - rb
        F[..., 0, 0] += w * (R[0, 0] - 1.0) - ux * drx
        F[..., 0, 1] += w * R[0, 1] - ux * dry
        F[..., 1, 0] += w * R[1, 0] - uy * drx
        F[..., 1, 1] += w * (R[1, 1] - 1.0) - uy * dry
    return F


def mesh_velocity(X, bodies, states, states_prev, dt):
    """V_G = (x^n - x^{n-1}) / dt: first-order backward difference of the
    blended map in time at fixed X (Sec. II D; reading R4), formed as the
    difference of the two displacements x - X, the same quantity without
    the round-off of X itself (which 1/dt would amplify)."""
    dn = mesh_displacement(X, bodies, states)
    dp = mesh_displacement(X, bodies, states_prev)
    return (dn - dp) / dt


def inverse2(F):
    det = F[..., 0, 0] * F[..., 1, 1] - F[..., 0, 1] * F[..., 1, 0]
    inv = np.empty_like(F)
    inv[..., 0, 0] = F[..., 1, 1] / det
    inv[..., 0, 1] = -F[..., 0, 1] / det
    inv[..., 1, 0] = -F[..., 1, 0] / det
    inv[..., 1, 1] = F[..., 0, 0] / det
    return inv


def transformed_velocities(F, VG):
    """c_hat_i = g^{-T} c_i - V_G with g^{-T} = F^{-1}
    (Eq. DboltzmannEqn_ALE and the line after it).  Reading R3: the printed
    form is used.  Returns an array [9, ..., 2]."""
    Fi = inverse2(F)
    out = np.empty((9,) + F.shape[:-2] + (2,))
    for i, (cx, cy) in enumerate(C):
        out[i, ..., 0] = Fi[..., 0, 0] * cx + Fi[..., 0, 1] * cy - VG[..., 0]
        out[i, ..., 1] = Fi[..., 1, 0] * cx + Fi[..., 1, 1] * cy - VG[..., 1]
    return out


def physical_gradient(F, dX, dY):
    """grad_x C = g^{-1} grad_X C = F^{-T} grad_X C (Eq. dx_ref)."""
    Fi = inverse2(F)
    return Fi[..., 0, 0] * dX + Fi[..., 1, 0] * dY, Fi[..., 0, 1] * dX + Fi[..., 1, 1] * dY
