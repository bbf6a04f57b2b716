"""Wall force and moment of the oracle (Sec. III, force on the wall elements
with the fluid stress and Eq. fnoneq1).

Test infrastructure only (see the package docstring).

Reading R21: the stress uses the post-propagation populations of the wall
nodes (including the reconstructed ones) and the local omega; each straight
wall edge is integrated with Simpson's rule over its three nodes (exact for a
quadratic nodal stress on a straight edge); the normal of an edge is constant
and the edge moves rigidly with the body; the moment is taken about the
body's reference point in the deformed frame.
"""
from __future__ import annotations

import numpy as np

from . import kinetics as K


def node_stress(f, g, Cv, mu, dt, Pr):
    """sigma = -p I - (1 - omega/2) P^(1), P^(1) = sum_i (f_i - f_i^eq) c_i c_i
    (Sec. III, Eq. fnoneq1).  f, g: [9, n]; returns sxx, sxy, syy."""
    rho, ux, uy, E, T = K.moments(f, g, Cv)
    om, _ = K.relaxation(rho, T, mu, dt, Pr)
    fneq = f - K.f_eq(rho, ux, uy, T)
    pxx, pxy, pyy = K.second_moment(fneq)
    p = rho * T
    a = 1.0 - 0.5 * om
    return -p - a * pxx, -a * pxy, -p - a * pyy


def wall_force(x_wall, sxx, sxy, syy, x_ref, closed=True):
    """F = sum_j sigma . n ds over the wall edges j, and the moment
    M = sum_j (x - x_ref) x (sigma . n) ds, with Simpson weights (1, 4, 1)/6
    over the three nodes of each edge.  x_wall[Nj, 2] are the deformed wall
    node positions, ordered counter-clockwise (body on the left of increasing
    j reversed, i.e. n = (t_y, -t_x)/|t| points out of the body).
    closed=False: an open chain of Nj (odd) nodes whose two ends are the same
    point (the wall of a C-grid), (Nj-1)/2 edges."""
    Nj = x_wall.shape[0]
    Fx = Fy = Mz = 0.0
    for k in range(Nj // 2):
        ids = (2 * k, 2 * k + 1, (2 * k + 2) % Nj if closed else 2 * k + 2)
        t = x_wall[ids[2]] - x_wall[ids[0]]
        ds = float(np.hypot(t[0], t[1]))
        n = np.array([t[1], -t[0]]) / ds
        for w, idx in zip((1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0), ids):
            tx = sxx[idx] * n[0] + sxy[idx] * n[1]
            ty = sxy[idx] * n[0] + syy[idx] * n[1]
            rx = x_wall[idx, 0] - x_ref[0]
            ry = x_wall[idx, 1] - x_ref[1]
            Fx += w * ds * tx
            Fy += w * ds * ty
            Mz += w * ds * (rx * ty - ry * tx)
    return Fx, Fy, Mz
