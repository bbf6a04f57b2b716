"""Pins of the oracle's whole step against what the target equations fix
(Sec. II C: Navier-Stokes-Fourier with mu = (1/omega - 1/2) p dt and
kappa = Cp (1/omega_1 - 1/2) p dt): Taylor-Green shear decay, thermal
diffusion of an entropy mode, the adiabatic sound speed; plus the invariants
of the boundary conditions and of the ALE step (rest state around a wall,
free stream on a moving blended mesh, scale invariance)."""
import math

import numpy as np
import pytest

from oracle import kinetics as K, mesh as OM, solver as OS
from paper_2107_01370_gb300 import inputs


def _box_solver(n_i, n_j, h, dt, M0, tau=0.6, gamma=1.4, Pr=0.71, skew=0.0, bodies=()):
    m = OM.periodic_box_mesh(n_i, n_j, n_i * h, n_j * h, skew=skew)
    T0 = float(np.mean(M0[3]))
    rho0 = float(np.mean(M0[0]))
    mu = (tau - 0.5) * rho0 * T0 * dt
    return OS.Solver(m, gamma=gamma, Pr=Pr, mu=mu, dt=dt, rho_inf=rho0, u_inf=(0.0, 0.0),
                     T_inf=T0, bodies=list(bodies), M0=M0, walls=False), m, mu


def _decay_rate(amps, t):
    a = np.log(np.abs(np.asarray(amps)))
    return -np.polyfit(t, a, 1)[0]


def test_taylor_green_shear_decay_rate():
    """u = U (sin kx cos ky, -cos kx sin ky) decays as exp(-2 nu k^2 t),
    nu = mu / rho (Sec. II C)."""
    n = 32
    x = np.arange(n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    k = 2 * np.pi / n
    U = 0.02
    M0 = np.empty((4, n, n))
    M0[0] = 1.0
    M0[1] = U * np.sin(k * X) * np.cos(k * Y)
    M0[2] = -U * np.cos(k * X) * np.sin(k * Y)
    M0[3] = 1.0 / 3.0
    s, m, mu = _box_solver(n, n, 1.0, 1.0, M0, tau=0.6)
    basis = np.sin(k * X) * np.cos(k * Y)
    amps, ts = [], []
    for step in range(1, 161):
        r = s.step()
        if step >= 20:
            amps.append((r.M[1] * basis).sum())
            ts.append(step)
    nu = mu / 1.0
    rate = _decay_rate(amps, ts)
    assert abs(rate / (2 * nu * k * k) - 1) < 0.02


def test_thermal_diffusion_uses_omega1():
    """An isobaric temperature wave decays as exp(-chi k^2 t) with
    chi = kappa / (rho Cp) = (1/omega_1 - 1/2) T dt.  With Pr = 0.5 this rate is
    twice the one omega alone would give, which pins reading R15 (q*)."""
    n = 64
    x = np.arange(n)
    k = 2 * np.pi / n
    T0, dT = 1.0 / 3.0, 0.01
    M0 = np.empty((4, n, 4))
    M0[3] = (T0 + dT * np.sin(k * x))[:, None]
    M0[0] = (1.0 / 3.0) / M0[3]
    M0[1] = 0.0
    M0[2] = 0.0
    Pr = 0.5
    s, m, mu = _box_solver(n, 4, 1.0, 1.0, M0, tau=0.6, Pr=Pr)
    basis = np.sin(k * x)[:, None]
    amps, ts = [], []
    for step in range(1, 401):
        r = s.step()
        if step >= 40:
            amps.append(((r.M[3] - T0) * basis).sum())
            ts.append(step)
    chi = (0.6 - 0.5) / Pr * T0
    rate = _decay_rate(amps, ts)
    assert abs(rate / (chi * k * k) - 1) < 0.04


def test_adiabatic_sound_speed():
    """A standing acoustic wave oscillates with c_s = sqrt(gamma T)
    (Sec. II C), not with the isothermal sqrt(T)."""
    n = 64
    x = np.arange(n)
    k = 2 * np.pi / n
    gamma, T0, eps = 1.4, 1.0 / 3.0, 1e-3
    M0 = np.empty((4, n, 4))
    M0[0] = (1 + eps * np.cos(k * x))[:, None]
    M0[3] = (T0 * (1 + (gamma - 1) * eps * np.cos(k * x)))[:, None]
    M0[1] = 0.0
    M0[2] = 0.0
    s, m, mu = _box_solver(n, 4, 1.0, 1.0, M0, tau=0.55, gamma=gamma)
    basis = np.cos(k * x)[:, None]
    amps = [((M0[0] - 1) * basis).sum()]
    for _ in range(150):
        amps.append(((s.step().M[0] - 1) * basis).sum())
    amps = np.array(amps)
    z = [i + amps[i] / (amps[i] - amps[i + 1]) for i in range(len(amps) - 1)
         if amps[i] * amps[i + 1] < 0]
    half_period = z[1] - z[0]
    cs = np.pi / (k * half_period)
    assert abs(cs / math.sqrt(gamma * T0) - 1) < 0.01


def test_rest_state_around_wall_is_fixed_point():
    """Gas at rest around a fixed cylinder: the wall (Grad's approximation at
    zero gradients), the far field and the collision keep every population at
    its equilibrium."""
    case = inputs.cylinder_case(16, 16, r_far=8.0)
    m = OM.ogrid_mesh(case.r, case.e)
    M0 = np.empty((4, 16, 16))
    M0[0], M0[1], M0[2], M0[3] = 1.0, 0.0, 0.0, 1.0 / 3.0
    s = OS.Solver(m, gamma=1.4, Pr=0.71, mu=1e-3, dt=case.flow.dt, rho_inf=1.0,
                  u_inf=(0.0, 0.0), T_inf=1.0 / 3.0, bodies=[OS.body_dict(case.bodies[0], 1.0, 0.1)],
                  M0=M0)
    feq = K.f_eq(1.0, 0.0, 0.0, 1.0 / 3.0)
    for _ in range(4):
        r = s.step()
    np.testing.assert_allclose(r.f_post, np.broadcast_to(feq[:, None, None], r.f_post.shape),
                               atol=1e-14)
    assert r.missing[:, 0].any()
    assert abs(r.force[0]) < 1e-13 and abs(r.force[1]) < 1e-13


def test_free_stream_preserved_on_moving_blended_mesh():
    """A uniform state stays uniform to round-off on a mesh that the blending
    function deforms around a plunging and pitching body (Sec. II D)."""
    n = 24
    h = 6.0 / n
    M0 = np.empty((4, n, n))
    M0[0], M0[1], M0[2], M0[3] = 1.05, 0.1, 0.03, 0.3
    body = dict(dof=-1, xc=3.0, yc=3.0, xp=3.0, yp=3.0, r_in=0.75, r_out=2.2)
    s, m, mu = _box_solver(n, n, h, h / 3.0, M0, bodies=[body])
    feq = K.f_eq(1.05, 0.1, 0.03, 0.3)
    for step in range(4):
        s.S_prev = [dict(s.S[0])]
        s.S = [{"h": 0.05 * (step + 1), "alpha": 0.04 * (step + 1), "hdot": 0.0, "adot": 0.0}]
        r = s.step()
    np.testing.assert_allclose(r.f_post, np.broadcast_to(feq[:, None, None], r.f_post.shape),
                               rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("scale", [2.5])
def test_scale_invariance_of_the_step(scale):
    """Scaling the mesh, dt and mu by the same factor leaves every population
    unchanged (reading R14: dt inside the correction Y)."""
    n = 12
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    M0 = np.empty((4, n, n))
    M0[0] = 1 + 0.02 * np.sin(2 * np.pi * i / n)
    M0[1] = 0.08 * np.sin(2 * np.pi * j / n)
    M0[2] = 0.05 * np.cos(2 * np.pi * (i + j) / n)
    M0[3] = 0.25 + 0.01 * np.cos(2 * np.pi * i / n)
    out = []
    for s_ in (1.0, scale):
        h = 0.1 * s_
        sol, m, mu = _box_solver(n, n, h, h / 3.0, M0, tau=0.7, skew=0.3)
        for _ in range(4):
            r = sol.step()
        out.append(r.f_post)
    np.testing.assert_allclose(out[1], out[0], rtol=1e-12, atol=1e-15)
    # and the correction is really active in this state
    dqx, _ = K.delta_q(M0[0], M0[1], M0[2], M0[3])
    assert np.abs(dqx).max() > 1e-3
