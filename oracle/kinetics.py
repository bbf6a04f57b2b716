"""Kinetic model of the oracle: D2Q9 two-population equilibria, correction
terms and collision (Sec. II C, Eqs. f_boltz, feq, geq, gstar and the
definitions that follow them).

Test infrastructure only (see the package docstring).

Arrays of populations carry the 9 discrete velocities on axis 0; all other
axes are nodes.  Everything is float64.
"""
from __future__ import annotations

import numpy as np

# D2Q9 discrete velocities c_i = (c_ix, c_iy), c_ia in {-1, 0, 1} (Sec. II C).
C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1],
              [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.float64)
Q = 9


def _bcast(v, like):
    return np.asarray(v, dtype=np.float64) * np.ones_like(like, dtype=np.float64)


def phi_1d(c: int, u, T):
    """Phi_{c}(u_alpha) of the product-form equilibrium (Eq. feq):
    Phi_0 = 1 - (u^2 + T),  Phi_{+-1} = (+-u + u^2 + T) / 2."""
    if c == 0:
        return 1.0 - (u * u + T)
    return 0.5 * (c * u + u * u + T)


def f_eq(rho, ux, uy, T):
    """f_i^eq = rho Phi_{c_ix}(u_x) Phi_{c_iy}(u_y)  (Eq. feq)."""
    rho = np.asarray(rho, dtype=np.float64)
    return np.stack([rho * phi_1d(int(cx), ux, T) * phi_1d(int(cy), uy, T) for cx, cy in C])


def w_1d(c: int, T):
    """W_0 = 1 - T, W_{+-1} = T / 2  (weights under Eq. gstar)."""
    return (1.0 - T) if c == 0 else 0.5 * T


def weights(T):
    """W_i = W_{c_ix} W_{c_iy}."""
    T = np.asarray(T, dtype=np.float64)
    return np.stack([w_1d(int(cx), T) * w_1d(int(cy), T) for cx, cy in C])


def energy(ux, uy, T, Cv):
    """E = Cv T + u^2 / 2 (inverse of the temperature definition, Sec. II C)."""
    return Cv * T + 0.5 * (ux * ux + uy * uy)


def heat_flux_eq(rho, ux, uy, T, Cv):
    """q^eq = 2 rho u H with the enthalpy H = Cp T + u^2/2 = E + T.
    Reading R11: the printed 'H = (Cv+1)/T + u^2/2' is read as (Cv+1) T + u^2/2
    (dimensional consistency; q^eq then is the energy flux 2(rho E + p) u)."""
    E = energy(ux, uy, T, Cv)
    H = E + T
    return 2.0 * rho * ux * H, 2.0 * rho * uy * H


def r_eq(rho, ux, uy, T, Cv):
    """R^eq = 2 rho E (T I + u u) + 2 rho T (T I + 2 u u); returns xx, xy, yy."""
    E = energy(ux, uy, T, Cv)
    rxx = 2.0 * rho * E * (T + ux * ux) + 2.0 * rho * T * (T + 2.0 * ux * ux)
    rxy = 2.0 * rho * E * (ux * uy) + 2.0 * rho * T * (2.0 * ux * uy)
    ryy = 2.0 * rho * E * (T + uy * uy) + 2.0 * rho * T * (T + 2.0 * uy * uy)
    return rxx, rxy, ryy


def psi_vector(rho, ux, uy, T, Cv):
    """The vector rho (1 - 3T)(T^2 + 2 (u.u) T + E (u.u)) / T of the energy
    correction Psi_i (component-wise products, Sec. II C)."""
    E = energy(ux, uy, T, Cv)
    pre = rho * (1.0 - 3.0 * T) / T
    xx = pre * (T * T + 2.0 * ux * ux * T + E * ux * ux)
    xy = pre * (T * T + 2.0 * uy * uy * T + E * uy * uy)
    return xx, xy


# Reading R13: the paper leaves B_i undefined.  B_0 = (1, 1), B_1 = B_3 =
# (-1/2, 0), B_2 = B_4 = (0, -1/2), diagonal velocities 0.  This is the
# minimal-support choice with sum Psi = 0, sum Psi c = 0 and
# sum Psi c_a c_b = -X_a delta_ab, which is exactly the lattice deficit of the
# Hermite term (so that sum g^eq c c = R^eq holds for every T).
B_PSI = np.array([[1.0, 1.0], [-0.5, 0.0], [0.0, -0.5], [-0.5, 0.0], [0.0, -0.5],
                  [0.0, 0.0], [0.0, 0.0], [0.0, 0.0], [0.0, 0.0]])


def psi(rho, ux, uy, T, Cv):
    """Psi_i = B_i . X  (Sec. II C, reading R13 for B_i)."""
    xx, xy = psi_vector(rho, ux, uy, T, Cv)
    return np.stack([B_PSI[i, 0] * xx + B_PSI[i, 1] * xy for i in range(Q)])


def g_hermite(rho, ux, uy, T, Cv, qx, qy):
    """W_i (2 rho E + q.c_i / T + (R^eq - 2 rho E T I):(c_i c_i - T I)/(2 T^2)) + Psi_i
    (Eqs. geq, gstar).  Reading R12: the printed 'R^eq - rho E T I' is read as
    R^eq - 2 rho E T I, the only form with sum_i g_i c_i c_i = R^eq."""
    E = energy(ux, uy, T, Cv)
    rxx, rxy, ryy = r_eq(rho, ux, uy, T, Cv)
    axx = rxx - 2.0 * rho * E * T
    ayy = ryy - 2.0 * rho * E * T
    axy = rxy
    W = weights(T)
    ps = psi(rho, ux, uy, T, Cv)
    out = []
    for i, (cx, cy) in enumerate(C):
        herm = (axx * (cx * cx - T) + 2.0 * axy * (cx * cy) + ayy * (cy * cy - T)) / (2.0 * T * T)
        out.append(W[i] * (2.0 * rho * E + (qx * cx + qy * cy) / T + herm) + ps[i])
    return np.stack(out)


def g_eq(rho, ux, uy, T, Cv):
    """g_i^eq of Eq. geq with q = q^eq."""
    qx, qy = heat_flux_eq(rho, ux, uy, T, Cv)
    return g_hermite(rho, ux, uy, T, Cv, qx, qy)


def moments(f, g, Cv):
    """rho = sum f, rho u = sum f c, 2 rho E = sum g, T = (E - u^2/2)/Cv
    (Sec. II C)."""
    rho = f.sum(axis=0)
    jx = np.tensordot(C[:, 0], f, axes=(0, 0))
    jy = np.tensordot(C[:, 1], f, axes=(0, 0))
    ux = jx / rho
    uy = jy / rho
    E = g.sum(axis=0) / (2.0 * rho)
    T = (E - 0.5 * (ux * ux + uy * uy)) / Cv
    return rho, ux, uy, E, T


def second_moment(f):
    """P = sum_i f_i c_i c_i; returns xx, xy, yy."""
    pxx = np.tensordot(C[:, 0] * C[:, 0], f, axes=(0, 0))
    pxy = np.tensordot(C[:, 0] * C[:, 1], f, axes=(0, 0))
    pyy = np.tensordot(C[:, 1] * C[:, 1], f, axes=(0, 0))
    return pxx, pxy, pyy


def first_moment(g):
    return np.tensordot(C[:, 0], g, axes=(0, 0)), np.tensordot(C[:, 1], g, axes=(0, 0))


def relaxation(rho, T, mu, dt, Pr):
    """omega and omega_1 from mu = (1/omega - 1/2) p dt and
    kappa = Cp (1/omega_1 - 1/2) p dt with Pr = Cp mu / kappa (Sec. II C).
    Reading R16: mu is fixed by Re, omega is local through p = rho T."""
    p = rho * T
    tau = 0.5 + mu / (p * dt)
    tau1 = 0.5 + (tau - 0.5) / Pr
    return 1.0 / tau, 1.0 / tau1


def delta_q(rho, ux, uy, T):
    """Deviation of the lattice third moment, rho u (1 - 3T) - rho u (.) u (.) u,
    the argument of the momentum correction phi_i (Sec. II C)."""
    return (rho * ux * (1.0 - 3.0 * T) - rho * ux ** 3,
            rho * uy * (1.0 - 3.0 * T) - rho * uy ** 3)


def phi_correction(yx, yy):
    """phi_i = -(1/2) c_i . Y on the four axis velocities, zero on the rest and
    diagonal velocities.  Y_a = d_a[(1/omega - 1/2) dt d_a dQ_a] (component-wise
    divergence of the paper's phi).  Reading R14: the support is the axis set,
    which makes the printed factor 1/2 give sum_i phi_i c_i = -Y; dt is restored
    inside the bracket so the scheme is invariant under X -> sX, dt -> s dt,
    mu -> s mu."""
    zero = np.zeros_like(np.asarray(yx, dtype=np.float64))
    out = []
    for i, (cx, cy) in enumerate(C):
        if 1 <= i <= 4:
            out.append(-0.5 * (cx * yx + cy * yy))
        else:
            out.append(zero.copy())
    return np.stack(out)


def quasi_heat_flux(f, rho, ux, uy, T, Cv):
    """q* of the quasi-equilibrium g* (Eq. gstar).  Reading R15: the paper does
    not print q*.  q* = q^eq + 2 u . (P - P^eq), P = sum f c c,
    P^eq = rho (u u + T I): the part of the heat flux carried by the viscous
    stress relaxes with omega and the Fourier part with omega_1, which is what
    kappa = Cp (1/omega_1 - 1/2) p dt states (pinned by the thermal-diffusion
    decay test)."""
    qx, qy = heat_flux_eq(rho, ux, uy, T, Cv)
    pxx, pxy, pyy = second_moment(f)
    dxx = pxx - rho * (ux * ux + T)
    dxy = pxy - rho * (ux * uy)
    dyy = pyy - rho * (uy * uy + T)
    return qx + 2.0 * (ux * dxx + uy * dxy), qy + 2.0 * (ux * dxy + uy * dyy)


def collide(f, g, yx, yy, mu, dt, Cv, Pr):
    """Two-population update at a node (Eq. f_boltz):
      f* = f + omega (f^eq - f) + dt phi
      g* = g + omega (g^eq - g) + (omega_1 - omega)(g^qe - g)
    with f, g the post-propagation populations at the node (reading R1:
    collide at the node, store post-collision populations, pull next step)."""
    rho, ux, uy, E, T = moments(f, g, Cv)
    om, om1 = relaxation(rho, T, mu, dt, Pr)
    feq = f_eq(rho, ux, uy, T)
    geq = g_eq(rho, ux, uy, T, Cv)
    qsx, qsy = quasi_heat_flux(f, rho, ux, uy, T, Cv)
    gqe = g_hermite(rho, ux, uy, T, Cv, qsx, qsy)
    ph = phi_correction(yx, yy)
    fs = f + om * (feq - f) + dt * ph
    gs = g + om * (geq - g) + (om1 - om) * (gqe - g)
    return fs, gs


def grad_f1(rho, ux, uy, T, Cv, dudx, dudy, dvdx, dvdy, dTdx, dTdy, mu, dt, Pr):
    """Non-equilibrium parts of Grad's approximation (Eqs. fnoneq, gnoneq,
    strainrate), already multiplied by dt:
      P1 = -(1/omega) rho T [S - (1/Cv)(div u) I],  S = grad u + grad u^T
      f1_i = W_i P1:(c c - T I) / (2 T^2)
      q1 = -(2/omega_1) rho Cp T grad T + 2 u . P1
      R1 = -(2/omega_1) rho T [S (E + 2T) + u grad E^T + grad E u^T]
      g1_i = W_i (q1.c / T + R1:(c c - T I) / (2 T^2))
    Reading R19: the garbled parentheses of P1 are read as
    [S - (1/Cv)(div u) I], the stress of the target Navier-Stokes equations.
    (grad u)_ab = d_a u_b;  dudx = d u_x / dx, dvdx = d u_y / dx, ..."""
    Cp = Cv + 1.0
    om, om1 = relaxation(rho, T, mu, dt, Pr)
    E = energy(ux, uy, T, Cv)
    sxx = 2.0 * dudx
    syy = 2.0 * dvdy
    sxy = dvdx + dudy
    div = dudx + dvdy
    p1xx = -(1.0 / om) * rho * T * (sxx - div / Cv)
    p1yy = -(1.0 / om) * rho * T * (syy - div / Cv)
    p1xy = -(1.0 / om) * rho * T * sxy
    # grad E = Cv grad T + (grad u) . u
    dEdx = Cv * dTdx + ux * dudx + uy * dvdx
    dEdy = Cv * dTdy + ux * dudy + uy * dvdy
    q1x = -(2.0 / om1) * rho * Cp * T * dTdx + 2.0 * (ux * p1xx + uy * p1xy)
    q1y = -(2.0 / om1) * rho * Cp * T * dTdy + 2.0 * (ux * p1xy + uy * p1yy)
    r1xx = -(2.0 / om1) * rho * T * (sxx * (E + 2.0 * T) + 2.0 * ux * dEdx)
    r1yy = -(2.0 / om1) * rho * T * (syy * (E + 2.0 * T) + 2.0 * uy * dEdy)
    r1xy = -(2.0 / om1) * rho * T * (sxy * (E + 2.0 * T) + ux * dEdy + dEdx * uy)
    W = weights(T)
    f1, g1 = [], []
    for i, (cx, cy) in enumerate(C):
        hp = (p1xx * (cx * cx - T) + 2.0 * p1xy * cx * cy + p1yy * (cy * cy - T)) / (2.0 * T * T)
        hr = (r1xx * (cx * cx - T) + 2.0 * r1xy * cx * cy + r1yy * (cy * cy - T)) / (2.0 * T * T)
        f1.append(dt * W[i] * hp)
        g1.append(dt * W[i] * ((q1x * cx + q1y * cy) / T + hr))
    return np.stack(f1), np.stack(g1)
