"""Rigid-body structural models of the oracle (Sec. III, Eqs. 1dofSM,
2dofSM; Sec. IV A, Eqs. 1dofSM_nonDim, fN1; Sec. IV D).

Test infrastructure only (see the package docstring).

Both models are integrated with the classical fourth-order Runge-Kutta method
(Sec. III B).  Reading R22: the fluid load of the current step is held
constant over the four stages (weak, staggered coupling of Sec. III).
"""
from __future__ import annotations

import math

import numpy as np


def one_dof_parameters(m_star, v_r, zeta, D, rho_inf, u_inf):
    """Dimensional m, k_h, c_h of Eq. 1dofSM from the nondimensional groups of
    Sec. IV A:  m* = 4 m / (rho pi D^2),  V_R = U / (f_N D),
    f_N = sqrt(k_h / m) / (2 pi).  zeta is a damping ratio (0 in the paper:
    undamped)."""
    m = m_star * rho_inf * math.pi * D * D / 4.0
    f_n = u_inf / (v_r * D)
    w_n = 2.0 * math.pi * f_n
    return m, m * w_n * w_n, 2.0 * zeta * m * w_n


def two_dof_parameters(m_star, v_r, x_alpha, r_alpha, wh_wa, b, rho_inf, u_inf):
    """Dimensional m, S_alpha, I_alpha, k_h, k_alpha of Eq. 2dofSM from
    m* = m / (pi rho b^2), V_R = U / (b omega_alpha sqrt(m*)),
    x_alpha = S_alpha / (m b), r_alpha^2 = I_alpha / (m b^2),
    omega_alpha^2 = k_alpha / I_alpha, omega_h^2 = k_h / m (Sec. IV D)."""
    m = m_star * math.pi * rho_inf * b * b
    w_a = u_inf / (v_r * b * math.sqrt(m_star))
    w_h = wh_wa * w_a
    s_a = x_alpha * m * b
    i_a = r_alpha * r_alpha * m * b * b
    return m, s_a, i_a, m * w_h * w_h, i_a * w_a * w_a


def rk4(rhs, y, dt):
    k1 = rhs(y)
    k2 = rhs(y + 0.5 * dt * k1)
    k3 = rhs(y + 0.5 * dt * k2)
    k4 = rhs(y + dt * k3)
    return y + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def advance_one_dof(h, hdot, fy, m, k, c, dt):
    """m h'' + c h' + k h = F_y (Eq. 1dofSM, damping added as an option)."""
    def rhs(y):
        return np.array([y[1], (fy - k * y[0] - c * y[1]) / m])
    y = rk4(rhs, np.array([h, hdot], dtype=np.float64), dt)
    return float(y[0]), float(y[1])


def advance_plunge_forced_pitch(h, hdot, fy, m, s_a, k_h, amp, w, n, dt):
    """Step n (from t = n dt to (n + 1) dt) of the pitch-plunge model (Eq.
    2dofSM) with the pitch prescribed, alpha(t) = amp sin(w t) (the forced
    pitching that starts the paper's flutter runs, Sec. IV D): the plunge row
    m h'' + S_alpha alpha''(t) + k_h h = F_y integrated by RK4 with alpha''
    evaluated at the stage times n dt, (n + 1/2) dt, (n + 1) dt; alpha and
    its rate at (n + 1) dt are the prescribed values.  Returns h, alpha,
    hdot, adot."""
    def rhs(t, y):
        acc_a = -amp * w * w * math.sin(w * t)
        return np.array([y[1], (fy - k_h * y[0] - s_a * acc_a) / m])
    t0, tm, t1 = n * dt, (n + 0.5) * dt, (n + 1) * dt
    y = np.array([h, hdot], dtype=np.float64)
    k1 = rhs(t0, y)
    k2 = rhs(tm, y + 0.5 * dt * k1)
    k3 = rhs(tm, y + 0.5 * dt * k2)
    k4 = rhs(t1, y + dt * k3)
    y = y + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return float(y[0]), amp * math.sin(w * t1), float(y[1]), amp * w * math.cos(w * t1)


def advance_two_dof(h, alpha, hdot, adot, fy, m_ea, m, s_a, i_a, k_h, k_a, dt):
    """[m S; S I] [h''; a''] + [k_h h; k_a a] = [F_y; M_EA]  (Eq. 2dofSM).
    Sign convention of this oracle: h positive up, alpha positive
    counter-clockwise, M_EA the counter-clockwise moment about the elastic
    axis; S_alpha enters with the sign that makes the mass centre lie
    downstream of the axis for x_alpha > 0."""
    Mm = np.array([[m, s_a], [s_a, i_a]], dtype=np.float64)
    Minv = np.linalg.inv(Mm)

    def rhs(y):
        acc = Minv @ np.array([fy - k_h * y[0], m_ea - k_a * y[1]])
        return np.array([y[2], y[3], acc[0], acc[1]])
    y = rk4(rhs, np.array([h, alpha, hdot, adot], dtype=np.float64), dt)
    return float(y[0]), float(y[1]), float(y[2]), float(y[3])
