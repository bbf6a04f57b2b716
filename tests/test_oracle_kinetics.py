"""Pins of the oracle's kinetic model against what the paper and the
mathematics fix (Sec. II C): closed-form moments of the equilibria, the
textbook D2Q9 equilibrium at T = 1/3, conservation by the collision, the
moments of the correction terms and of Grad's approximation."""
import numpy as np
import pytest

from oracle import kinetics as K

C = K.C


def _rand_state(n=64, seed=1, Tlo=0.2, Thi=0.45):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 1.5, n)
    ux = rng.uniform(-0.2, 0.2, n)
    uy = rng.uniform(-0.2, 0.2, n)
    T = rng.uniform(Tlo, Thi, n)
    return rho, ux, uy, T


def mom(pop, px, py):
    return np.tensordot(C[:, 0] ** px * C[:, 1] ** py, pop, axes=(0, 0))


def test_feq_closed_form_moments():
    rho, ux, uy, T = _rand_state()
    f = K.f_eq(rho, ux, uy, T)
    np.testing.assert_allclose(mom(f, 0, 0), rho, rtol=1e-14)
    np.testing.assert_allclose(mom(f, 1, 0), rho * ux, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(mom(f, 0, 1), rho * uy, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(mom(f, 2, 0), rho * (ux * ux + T), rtol=1e-13)
    np.testing.assert_allclose(mom(f, 0, 2), rho * (uy * uy + T), rtol=1e-13)
    np.testing.assert_allclose(mom(f, 1, 1), rho * ux * uy, rtol=1e-12, atol=1e-15)
    # lattice third moments: c_x^3 = c_x and the mixed one
    np.testing.assert_allclose(mom(f, 3, 0), rho * ux, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(mom(f, 2, 1), rho * uy * (ux * ux + T), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("axis", [0, 1])
def test_feq_is_textbook_d2q9_at_T_one_third(axis):
    """At T = 1/3 and one velocity component zero, the product form equals the
    standard D2Q9 equilibrium rho w_i (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2)."""
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.7, 1.3, 32)
    u = rng.uniform(-0.15, 0.15, 32)
    ux, uy = (u, 0 * u) if axis == 0 else (0 * u, u)
    f = K.f_eq(rho, ux, uy, 1.0 / 3.0)
    w = np.array([4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36])
    cu = C[:, 0:1] * ux + C[:, 1:2] * uy
    usq = ux * ux + uy * uy
    ref = rho * w[:, None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * usq)
    np.testing.assert_allclose(f, ref, rtol=1e-13, atol=1e-16)


def test_geq_closed_form_moments():
    """sum g^eq = 2 rho E, sum g^eq c = 2 rho u H, sum g^eq c c = R^eq, for
    every T (this pins readings R11, R12 and R13 together)."""
    Cv = 2.5
    rho, ux, uy, T = _rand_state()
    g = K.g_eq(rho, ux, uy, T, Cv)
    E = Cv * T + 0.5 * (ux * ux + uy * uy)
    H = (Cv + 1) * T + 0.5 * (ux * ux + uy * uy)
    np.testing.assert_allclose(mom(g, 0, 0), 2 * rho * E, rtol=1e-13)
    np.testing.assert_allclose(mom(g, 1, 0), 2 * rho * ux * H, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(mom(g, 0, 1), 2 * rho * uy * H, rtol=1e-12, atol=1e-14)
    rxx = 2 * rho * E * (T + ux * ux) + 2 * rho * T * (T + 2 * ux * ux)
    ryy = 2 * rho * E * (T + uy * uy) + 2 * rho * T * (T + 2 * uy * uy)
    rxy = 2 * rho * E * ux * uy + 4 * rho * T * ux * uy
    np.testing.assert_allclose(mom(g, 2, 0), rxx, rtol=1e-12)
    np.testing.assert_allclose(mom(g, 0, 2), ryy, rtol=1e-12)
    np.testing.assert_allclose(mom(g, 1, 1), rxy, rtol=1e-11, atol=1e-14)


def test_psi_moments():
    """sum Psi = 0, sum Psi c = 0, sum Psi c_a c_b = -X_a delta_ab, with
    X = rho (1 - 3T)(T^2 + 2 u.u T + E u.u)/T."""
    Cv = 1.0 / 0.4
    rho, ux, uy, T = _rand_state()
    ps = K.psi(rho, ux, uy, T, Cv)
    E = Cv * T + 0.5 * (ux * ux + uy * uy)
    Xx = rho * (1 - 3 * T) * (T * T + 2 * ux * ux * T + E * ux * ux) / T
    Xy = rho * (1 - 3 * T) * (T * T + 2 * uy * uy * T + E * uy * uy) / T
    np.testing.assert_allclose(mom(ps, 0, 0), 0, atol=1e-15)
    np.testing.assert_allclose(mom(ps, 1, 0), 0, atol=1e-15)
    np.testing.assert_allclose(mom(ps, 0, 1), 0, atol=1e-15)
    np.testing.assert_allclose(mom(ps, 2, 0), -Xx, rtol=1e-13)
    np.testing.assert_allclose(mom(ps, 0, 2), -Xy, rtol=1e-13)
    np.testing.assert_allclose(mom(ps, 1, 1), 0, atol=1e-15)
    # T = 1/3 makes the correction vanish
    assert np.abs(K.psi(rho, ux, uy, 0 * T + 1.0 / 3.0, Cv)).max() < 1e-15


def test_weights_moments():
    T = np.linspace(0.1, 0.6, 11)
    W = K.weights(T)
    np.testing.assert_allclose(W.sum(0), 1.0, rtol=1e-15)
    np.testing.assert_allclose(mom(W, 2, 0), T, rtol=1e-14)
    np.testing.assert_allclose(mom(W, 2, 2), T * T, rtol=1e-14)


def test_moments_inverse_of_equilibria():
    Cv = 2.5
    rho, ux, uy, T = _rand_state()
    r2, ux2, uy2, E2, T2 = K.moments(K.f_eq(rho, ux, uy, T), K.g_eq(rho, ux, uy, T, Cv), Cv)
    np.testing.assert_allclose(r2, rho, rtol=1e-14)
    np.testing.assert_allclose(ux2, ux, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(uy2, uy, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(T2, T, rtol=1e-12)


def test_phi_moments():
    rng = np.random.default_rng(4)
    yx, yy = rng.normal(size=(2, 16))
    ph = K.phi_correction(yx, yy)
    np.testing.assert_allclose(mom(ph, 0, 0), 0, atol=1e-15)
    np.testing.assert_allclose(mom(ph, 1, 0), -yx, rtol=1e-15)
    np.testing.assert_allclose(mom(ph, 0, 1), -yy, rtol=1e-15)
    for px, py in ((2, 0), (0, 2), (1, 1)):
        np.testing.assert_allclose(mom(ph, px, py), 0, atol=1e-15)


def _noneq(seed, n=40):
    Cv = 2.5
    rho, ux, uy, T = _rand_state(n, seed)
    f = K.f_eq(rho, ux, uy, T) * (1 + 0.05 * np.random.default_rng(seed + 1).uniform(-1, 1, (9, n)))
    g = K.g_eq(rho, ux, uy, T, Cv) * (1 + 0.05 * np.random.default_rng(seed + 2).uniform(-1, 1, (9, n)))
    return f, g, Cv


def test_collision_conservation():
    """Mass and energy are conserved; momentum changes by dt sum phi c = -dt Y."""
    f, g, Cv = _noneq(7)
    rng = np.random.default_rng(8)
    yx, yy = 1e-3 * rng.normal(size=(2, f.shape[1]))
    dt, mu, Pr = 0.02, 2e-3, 0.71
    fs, gs = K.collide(f, g, yx, yy, mu, dt, Cv, Pr)
    np.testing.assert_allclose(mom(fs, 0, 0), mom(f, 0, 0), rtol=1e-14)
    np.testing.assert_allclose(mom(fs, 1, 0), mom(f, 1, 0) - dt * yx, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(mom(fs, 0, 1), mom(f, 0, 1) - dt * yy, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(mom(gs, 0, 0), mom(g, 0, 0), rtol=1e-14)


def test_collision_relaxation_rates():
    """The stress relaxes at omega and the Fourier part of the heat flux at
    omega_1 (Pr = Cp mu / kappa): check the post-collision moments against the
    relaxation of each moment."""
    f, g, Cv = _noneq(9)
    zero = np.zeros(f.shape[1])
    dt, mu, Pr = 0.05, 3e-3, 0.5
    fs, gs = K.collide(f, g, zero, zero, mu, dt, Cv, Pr)
    rho, ux, uy, E, T = K.moments(f, g, Cv)
    om, om1 = K.relaxation(rho, T, mu, dt, Pr)
    feq = K.f_eq(rho, ux, uy, T)
    # off-diagonal stress: P_xy* - P_xy^eq = (1 - omega)(P_xy - P_xy^eq)
    np.testing.assert_allclose(mom(fs, 1, 1) - mom(feq, 1, 1),
                               (1 - om) * (mom(f, 1, 1) - mom(feq, 1, 1)), rtol=1e-10, atol=1e-15)
    # heat flux: q* - q^eq = (1 - omega_1)(q - q^eq - 2u.P1) + (1 - omega) 2u.P1
    qx_eq, qy_eq = K.heat_flux_eq(rho, ux, uy, T, Cv)
    pxx, pxy, pyy = K.second_moment(f)
    p1xx = pxx - rho * (ux * ux + T)
    p1xy = pxy - rho * ux * uy
    vx = 2 * (ux * p1xx + uy * p1xy)
    qx = mom(g, 1, 0)
    expect = (1 - om1) * (qx - qx_eq - vx) + (1 - om) * vx
    np.testing.assert_allclose(mom(gs, 1, 0) - qx_eq, expect, rtol=1e-9, atol=1e-14)
    # relaxation times from the transport coefficients
    np.testing.assert_allclose((1 / om - 0.5) * rho * T * dt, mu, rtol=1e-14)
    np.testing.assert_allclose((Cv + 1) * mu / ((Cv + 1) * (1 / om1 - 0.5) * rho * T * dt), Pr,
                               rtol=1e-13)


def test_collision_fixed_point_at_equilibrium():
    Cv = 2.5
    rho, ux, uy, T = _rand_state(20, 11)
    f = K.f_eq(rho, ux, uy, T)
    g = K.g_eq(rho, ux, uy, T, Cv)
    zero = np.zeros_like(rho)
    fs, gs = K.collide(f, g, zero, zero, 1e-3, 0.01, Cv, 0.71)
    np.testing.assert_allclose(fs, f, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(gs, g, rtol=1e-13, atol=1e-16)


def test_quasi_equilibrium_heat_flux_at_equilibrium():
    Cv = 2.5
    rho, ux, uy, T = _rand_state(20, 12)
    f = K.f_eq(rho, ux, uy, T)
    qsx, qsy = K.quasi_heat_flux(f, rho, ux, uy, T, Cv)
    qx, qy = K.heat_flux_eq(rho, ux, uy, T, Cv)
    np.testing.assert_allclose(qsx, qx, rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(qsy, qy, rtol=1e-12, atol=1e-16)


def test_grad_nonequilibrium_moments():
    """Moments of dt f^(1), dt g^(1): sum = 0, sum f1 c = 0, sum g1 c = dt q1
    (any T); sum f1 c c = dt P1 and sum g1 c c = dt R1 at T = 1/3 where the
    D2Q9 fourth moments are isotropic."""
    Cv = 2.5
    rng = np.random.default_rng(5)
    n = 16
    rho = rng.uniform(0.8, 1.2, n)
    ux, uy = rng.uniform(-0.1, 0.1, (2, n))
    T = np.full(n, 1.0 / 3.0)
    du = 0.01 * rng.normal(size=(6, n))
    dt, mu, Pr = 0.03, 2e-3, 0.71
    f1, g1 = K.grad_f1(rho, ux, uy, T, Cv, *du, mu, dt, Pr)
    om, om1 = K.relaxation(rho, T, mu, dt, Pr)
    dudx, dudy, dvdx, dvdy, dTdx, dTdy = du
    div = dudx + dvdy
    p1xx = -(1 / om) * rho * T * (2 * dudx - div / Cv)
    p1xy = -(1 / om) * rho * T * (dvdx + dudy)
    p1yy = -(1 / om) * rho * T * (2 * dvdy - div / Cv)
    for pop in (f1, g1):
        np.testing.assert_allclose(mom(pop, 0, 0), 0, atol=1e-15)
    np.testing.assert_allclose(mom(f1, 1, 0), 0, atol=1e-16)
    np.testing.assert_allclose(mom(f1, 2, 0), dt * p1xx, rtol=1e-12, atol=1e-17)
    np.testing.assert_allclose(mom(f1, 1, 1), dt * p1xy, rtol=1e-12, atol=1e-17)
    np.testing.assert_allclose(mom(f1, 0, 2), dt * p1yy, rtol=1e-12, atol=1e-17)
    q1x = -(2 / om1) * rho * (Cv + 1) * T * dTdx + 2 * (ux * p1xx + uy * p1xy)
    np.testing.assert_allclose(mom(g1, 1, 0), dt * q1x, rtol=1e-12, atol=1e-17)
    q1y = -(2 / om1) * rho * (Cv + 1) * T * dTdy + 2 * (ux * p1xy + uy * p1yy)
    np.testing.assert_allclose(mom(g1, 0, 1), dt * q1y, rtol=1e-12, atol=1e-17)
    # R^(1) (Eq. gnoneq): grad E = Cv grad T + (grad u) . u
    E = Cv * T + 0.5 * (ux * ux + uy * uy)
    dEdx = Cv * dTdx + ux * dudx + uy * dvdx
    dEdy = Cv * dTdy + ux * dudy + uy * dvdy
    pre = -(2 / om1) * rho * T
    r1xx = pre * (2 * dudx * (E + 2 * T) + 2 * ux * dEdx)
    r1xy = pre * ((dvdx + dudy) * (E + 2 * T) + ux * dEdy + uy * dEdx)
    r1yy = pre * (2 * dvdy * (E + 2 * T) + 2 * uy * dEdy)
    np.testing.assert_allclose(mom(g1, 2, 0), dt * r1xx, rtol=1e-12, atol=1e-17)
    np.testing.assert_allclose(mom(g1, 1, 1), dt * r1xy, rtol=1e-12, atol=1e-17)
    np.testing.assert_allclose(mom(g1, 0, 2), dt * r1yy, rtol=1e-12, atol=1e-17)


def test_grad_stress_is_the_navier_stokes_stress():
    """Grad's populations f^eq + dt f^(1) (Eq. fnoneq) carry the viscous stress
    of the Navier-Stokes-Fourier equations the model recovers (Sec. II C):
    the wall-force stress -p I - (1 - omega/2) sum (f - f^eq) c c equals
    -p I + mu [grad u + grad u^T - (1/Cv)(div u) I] with
    mu = (1/omega - 1/2) p dt.  This ties P^(1) to a different equation of
    the paper than the one it is printed in: a wrong sign, factor or bulk
    term in P^(1) fails it (T = 1/3, where the D2Q9 fourth moments are
    isotropic)."""
    from oracle import forces
    Cv = 2.5
    rng = np.random.default_rng(8)
    n = 24
    rho = rng.uniform(0.8, 1.2, n)
    ux, uy = rng.uniform(-0.1, 0.1, (2, n))
    T = np.full(n, 1.0 / 3.0)
    dudx, dudy, dvdx, dvdy, dTdx, dTdy = 0.02 * rng.normal(size=(6, n))
    dt, mu, Pr = 0.02, 3e-3, 0.71
    f1, g1 = K.grad_f1(rho, ux, uy, T, Cv, dudx, dudy, dvdx, dvdy, dTdx, dTdy, mu, dt, Pr)
    f = K.f_eq(rho, ux, uy, T) + f1
    g = K.g_eq(rho, ux, uy, T, Cv) + g1
    sxx, sxy, syy = forces.node_stress(f, g, Cv, mu, dt, Pr)
    p = rho * T
    div = dudx + dvdy
    np.testing.assert_allclose(sxx, -p + mu * (2 * dudx - div / Cv), rtol=1e-12)
    np.testing.assert_allclose(syy, -p + mu * (2 * dvdy - div / Cv), rtol=1e-12)
    np.testing.assert_allclose(sxy, mu * (dvdx + dudy), rtol=1e-10, atol=1e-16)


def test_grad_heat_flux_and_energy_moment_at_a_no_slip_wall():
    """At a no-slip wall target (u = 0) Grad's g carries the Fourier heat
    flux of Sec. II C: with kappa = Cp (1/omega_1 - 1/2) p dt, the flux
    sum dt g^(1) c = dt q^(1) is -2 kappa / (1 - omega_1/2) grad T; and
    sum dt g^(1) c c reduces to -(2/omega_1) p (Cv + 2) T dt S, the only
    term of R^(1) left when u = 0 (E = Cv T)."""
    Cv = 2.5
    rng = np.random.default_rng(9)
    n = 12
    rho = rng.uniform(0.8, 1.2, n)
    zero = np.zeros(n)
    T = np.full(n, 1.0 / 3.0)
    dudx, dudy, dvdx, dvdy, dTdx, dTdy = 0.02 * rng.normal(size=(6, n))
    dt, mu, Pr = 0.02, 3e-3, 0.6
    _, g1 = K.grad_f1(rho, zero, zero, T, Cv, dudx, dudy, dvdx, dvdy, dTdx, dTdy, mu, dt, Pr)
    om, om1 = K.relaxation(rho, T, mu, dt, Pr)
    p = rho * T
    kappa = (Cv + 1) * (1 / om1 - 0.5) * p * dt
    fac = -2 * kappa / (1 - 0.5 * om1)
    np.testing.assert_allclose(mom(g1, 1, 0), fac * dTdx, rtol=1e-12)
    np.testing.assert_allclose(mom(g1, 0, 1), fac * dTdy, rtol=1e-12)
    r = -(2 / om1) * p * (Cv + 2) * T * dt
    np.testing.assert_allclose(mom(g1, 2, 0), r * 2 * dudx, rtol=1e-12)
    np.testing.assert_allclose(mom(g1, 1, 1), r * (dvdx + dudy), rtol=1e-12)
    np.testing.assert_allclose(mom(g1, 0, 2), r * 2 * dvdy, rtol=1e-12)
