"""Pins of the oracle's blended mesh and ALE kinematics (Sec. II A, II D),
rigid-body ODEs (Sec. III, IV A) and wall force (Sec. III)."""
import math

import numpy as np

from oracle import ale, forces, kinetics as K, structure
from oracle.solver import zero_state


def _body(dof=1, **kw):
    b = dict(dof=dof, xc=0.0, yc=0.0, xp=0.0, yp=0.0, r_in=0.75, r_out=2.5)
    b.update(kw)
    return b


def test_r5_closed_form():
    assert ale.r5(0.0) == 0.0 and ale.r5(1.0) == 1.0
    assert abs(ale.r5(0.5) - 0.5) < 1e-15
    h = 1e-4
    for s in (0.0, 1.0):
        d1 = (ale.r5(s + h) - ale.r5(s - h)) / (2 * h)
        d2 = (ale.r5(s + h) - 2 * ale.r5(s) + ale.r5(s - h)) / h ** 2
        assert abs(d1) < 1e-6 and abs(d2) < 1e-2
    h = 1e-5
    s = np.linspace(0.05, 0.95, 19)
    np.testing.assert_allclose(ale.dr5(s), (ale.r5(s + h) - ale.r5(s - h)) / (2 * h), rtol=1e-7)


def test_blend_limits_rigid_and_fixed_regions():
    rng = np.random.default_rng(0)
    ang = rng.uniform(0, 2 * np.pi, 200)
    rad = rng.uniform(0.5, 4.0, 200)
    X = np.stack([rad * np.cos(ang), rad * np.sin(ang)], -1)
    b = _body()
    st = {"h": 0.3, "alpha": 0.0, "hdot": 0.0, "adot": 0.0}
    x = ale.mesh_position(X, [b], [st])
    outside = rad > 2.5
    assert np.array_equal(x[outside], X[outside])          # bit-identical
    inside = rad < 0.75
    np.testing.assert_allclose(x[inside] - X[inside], np.broadcast_to([0.0, 0.3], X[inside].shape),
                               atol=1e-15)


def test_deformation_gradient_matches_finite_differences():
    """Analytic F = dx/dX of the blended map (reading R5) against central
    differences of the map itself, with plunge and pitch."""
    rng = np.random.default_rng(1)
    ang = rng.uniform(0, 2 * np.pi, 100)
    rad = rng.uniform(0.8, 2.4, 100)
    X = np.stack([rad * np.cos(ang), rad * np.sin(ang)], -1)
    b = _body(xp=0.2, yp=-0.1)
    st = {"h": 0.2, "alpha": 0.15, "hdot": 0.0, "adot": 0.0}
    F = ale.deformation_gradient(X, [b], [st])
    h = 1e-6
    for k in range(2):
        dX = np.zeros(2)
        dX[k] = h
        fd = (ale.mesh_position(X + dX, [b], [st]) - ale.mesh_position(X - dX, [b], [st])) / (2 * h)
        np.testing.assert_allclose(F[..., :, k], fd, atol=1e-8)
    assert np.all(F[..., 0, 0] * F[..., 1, 1] - F[..., 0, 1] * F[..., 1, 0] > 0)


def test_translation_gives_body_velocity_and_unit_jacobian():
    X = np.array([[0.55, 0.1], [0.0, -0.7], [3.0, 0.0]])
    b = _body()
    s0 = {"h": 0.1, "alpha": 0.0, "hdot": 0.0, "adot": 0.0}
    s1 = {"h": 0.1 + 0.002, "alpha": 0.0, "hdot": 0.0, "adot": 0.0}
    dt = 0.01
    VG = ale.mesh_velocity(X, [b], [s1], [s0], dt)
    np.testing.assert_allclose(VG[:2], [[0.0, 0.2], [0.0, 0.2]], rtol=1e-12)
    assert np.all(VG[2] == 0.0)
    F = ale.deformation_gradient(X[:2], [b], [s1])
    np.testing.assert_allclose(F, np.broadcast_to(np.eye(2), F.shape), atol=1e-15)


def test_rotation_preserves_speed_of_discrete_velocities():
    """In the rigid zone a pitch rotation gives g^{-T} = R(alpha) (reading R2):
    |c_hat_i| = |c_i| and c_hat_i = R c_i."""
    X = np.array([[0.5, 0.2], [-0.3, -0.5]])
    b = _body()
    st = {"h": 0.0, "alpha": 0.3, "hdot": 0.0, "adot": 0.0}
    F = ale.deformation_gradient(X, [b], [st])
    VG = np.zeros_like(X)
    ch = ale.transformed_velocities(F, VG)
    np.testing.assert_allclose(np.linalg.norm(ch, axis=-1),
                               np.broadcast_to(np.linalg.norm(K.C, axis=-1)[:, None], (9, 2)),
                               rtol=1e-14)
    R = ale.rotation(-0.3)     # F = R(alpha) so F^{-1} c = R(-alpha) c
    np.testing.assert_allclose(ch[:, 0], K.C @ R.T, atol=1e-15)


def test_rk4_homogeneous_step_is_taylor_polynomial():
    m, k, c = 2.0, 5.0, 0.3
    A = np.array([[0, 1], [-k / m, -c / m]])
    dt = 0.1
    y0 = np.array([0.4, -0.2])
    P = sum(np.linalg.matrix_power(dt * A, n) / math.factorial(n) for n in range(5))
    h, v = structure.advance_one_dof(y0[0], y0[1], 0.0, m, k, c, dt)
    np.testing.assert_allclose([h, v], P @ y0, rtol=1e-14)


def test_rk4_forced_oscillator_converges_to_analytic_solution():
    m, k, F = 1.5, 9.0, 0.7
    w = math.sqrt(k / m)
    h, v = 0.1, 0.0
    dt = 1e-3
    n = 3000
    for _ in range(n):
        h, v = structure.advance_one_dof(h, v, F, m, k, 0.0, dt)
    t = n * dt
    ref = F / k + (0.1 - F / k) * math.cos(w * t)
    assert abs(h - ref) < 1e-10


def test_one_dof_nondimensional_form():
    """m h'' + k h = F_y in tau = t f_N, h_bar = h/D gives
    h_bar'' + 4 pi^2 h_bar = 2 V_R^2 C_L / (pi m*)  (Eq. 1dofSM_nonDim)."""
    rng = np.random.default_rng(2)
    for _ in range(10):
        m_star, v_r, D, rho, U, Fy = rng.uniform(0.5, 20, 6)
        m, k, c = structure.one_dof_parameters(m_star, v_r, 0.0, D, rho, U)
        f_n = math.sqrt(k / m) / (2 * math.pi)
        assert abs(v_r - U / (f_n * D)) < 1e-12 * v_r
        assert abs(m_star - 4 * m / (rho * math.pi * D * D)) < 1e-12 * m_star
        lhs_k = k / (m * f_n ** 2)
        assert abs(lhs_k - 4 * math.pi ** 2) < 1e-10
        CL = 2 * Fy / (rho * U * U * D)
        assert abs(Fy / (m * f_n ** 2 * D) - 2 * v_r ** 2 * CL / (math.pi * m_star)) < 1e-10 * abs(Fy / (m * f_n ** 2 * D))


def _polygon(n=24, R=0.5, centre=(0.1, -0.2)):
    th = 2 * np.pi * np.arange(n) / n
    P = np.stack([centre[0] + R * np.cos(th), centre[1] + R * np.sin(th)], -1)
    x = np.empty((2 * n, 2))
    x[0::2] = P
    x[1::2] = 0.5 * (P + np.roll(P, -1, 0))
    return x, 0.5 * n * R * R * np.sin(2 * np.pi / n)


def test_force_of_uniform_stress_vanishes():
    x, _ = _polygon()
    p = 0.37
    Fx, Fy, M = forces.wall_force(x, -p + 0 * x[:, 0], 0 * x[:, 0], -p + 0 * x[:, 0], (0.1, -0.2))
    assert abs(Fx) < 1e-15 and abs(Fy) < 1e-15 and abs(M) < 1e-15


def test_force_of_linear_pressure_is_minus_area_times_gradient():
    """sigma = -p I, p = p0 + a.x: F = -A a (divergence theorem), and the moment
    about the centroid vanishes."""
    x, area = _polygon()
    a = np.array([0.3, -0.8])
    p = 1.0 + x @ a
    Fx, Fy, M = forces.wall_force(x, -p, 0 * p, -p, (0.1, -0.2))
    np.testing.assert_allclose([Fx, Fy], -area * a, rtol=1e-12)
    assert abs(M) < 1e-14


def test_stress_at_equilibrium_is_pressure():
    Cv = 2.5
    rho = np.array([0.9, 1.1])
    ux = np.array([0.1, -0.05])
    uy = np.array([0.02, 0.0])
    T = np.array([0.3, 0.35])
    sxx, sxy, syy = forces.node_stress(K.f_eq(rho, ux, uy, T), K.g_eq(rho, ux, uy, T, Cv), Cv,
                                       1e-3, 0.01, 0.71)
    np.testing.assert_allclose(sxx, -rho * T, rtol=1e-12)
    np.testing.assert_allclose(syy, -rho * T, rtol=1e-12)
    np.testing.assert_allclose(sxy, 0, atol=1e-16)


def test_zero_state_helper():
    assert zero_state() == {"h": 0.0, "alpha": 0.0, "hdot": 0.0, "adot": 0.0}


def test_forced_pitch_step_matches_the_driven_oscillator():
    """Prescribed pitch alpha = A sin(w t) (Sec. IV D forcing): with no fluid
    load the plunge row m h'' + k_h h = -S_alpha alpha''(t) is a driven
    oscillator with the closed-form response from rest
    h = C (sin(w t) - (w / w_h) sin(w_h t)),  C = S_alpha A w^2 / (k_h - m w^2);
    RK4 reproduces it to its fourth-order error, and alpha, alpha' are the
    prescribed values at every step end."""
    import math
    from oracle import structure as S
    m, s_a, k_h, A, w = 2.0, 0.3, 5.0, 0.0175, 1.3
    w_h = math.sqrt(k_h / m)
    C = s_a * A * w * w / (k_h - m * w * w)
    errs = []
    for dt in (1e-2, 5e-3):
        h = hd = 0.0
        t = 0.0
        n = int(round(3.0 / dt))
        for k in range(n):
            h, a, hd, ad = S.advance_plunge_forced_pitch(h, hd, 0.0, m, s_a, k_h, A, w, k, dt)
            t = (k + 1) * dt
            assert a == A * math.sin(w * t) and ad == A * w * math.cos(w * t)
        exact = C * (math.sin(w * t) - (w / w_h) * math.sin(w_h * t))
        exact_d = C * w * (math.cos(w * t) - math.cos(w_h * t))
        assert abs(h - exact) < 1e-8 * abs(C) * (dt / 1e-2) ** 4
        assert abs(hd - exact_d) < 1e-8 * abs(C * w) * (dt / 1e-2) ** 4
        errs.append(abs(h - exact))
    assert 12.0 < errs[0] / errs[1] < 20.0        # fourth order
