"""Pins of the oracle's unstructured Q2 building blocks (readings R7-R9 on an
element list, R33 for gradients) against facts that do not come from the
code under test:
- a structured O-grid relabelled into a shuffled element list gives, for
  every node and lattice direction, the departure point and Q2 value of the
  structured oracle (the same elements, a different numbering);
- the nodal gradient is exact for a field linear in X on a curved
  subparametric mesh and for a quadratic on affine elements;
- at an element's centre node it is reading R18's central difference;
- a departure point outside the node's elements is refused even where some
  other element of the mesh contains it (brute force over all elements)."""
import numpy as np

import oracle.mesh as OM
import oracle.unstructured as OU
from paper_2107_01370_gb300 import inputs

C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)


def _ogrid(nr=13, nt=24):
    return inputs.algebraic_ogrid(inputs.ellipse_wall(nt, 0.6, 0.4), nr, 4.0, 0.08)


def _shuffled(X, seed=5):
    rng = np.random.default_rng(seed)
    Ni, Nj = X.shape[:2]
    perm = rng.permutation(Ni * Nj)
    Xl, els = OU.from_ogrid(X, perm)
    els = els[rng.permutation(els.shape[0])]
    return OU.UnstructuredQ2Mesh(Xl, els), perm


def test_relabelled_ogrid_reproduces_structured_departures():
    X = _ogrid()
    Ni, Nj = X.shape[:2]
    um, perm = _shuffled(X)
    sm = OM.Q2Mesh(X, periodic_i=False, periodic_j=True)
    rng = np.random.default_rng(1)
    field = rng.standard_normal((Ni, Nj))
    ufield = np.empty(Ni * Nj)
    ufield[perm] = field.reshape(-1)
    dt = 0.3 * 0.08
    checked = 0
    for i in range(Ni - 1):
        for j in range(Nj):
            for q in range(9):
                P = X[i, j] - dt * C[q]     # wall nodes: some points fall in the body, found by neither
                wa, wb, xi, eta, found = sm.locate(P[None], np.array([i]), np.array([j]))
                got = um.locate(perm[i * Nj + j], P)
                assert (got is not None) == bool(found[0]), (i, j, q)
                if got is None:
                    continue
                v_s = sm.interpolate(field, wa, wb, xi, eta)[0]
                v_u = um.interpolate(ufield, *got)
                assert abs(v_s - v_u) < 1e-12 * (1 + abs(v_s)), (i, j, q)
                checked += 1
    assert checked > 8 * (Ni - 2) * Nj


def test_gradient_exact_for_linear_fields_on_a_curved_mesh():
    X = _ogrid()
    um, perm = _shuffled(X, seed=7)
    f = 0.3 + 1.7 * um.X[:, 0] - 0.9 * um.X[:, 1]
    gx, gy = um.grad_X(f)
    assert np.abs(gx - 1.7).max() < 1e-11 and np.abs(gy + 0.9).max() < 1e-11


def _affine_elements(na=4, nb=3, skew=0.35):
    """A parallelogram patch of na x nb Q2 elements (not periodic)."""
    Ni, Nj = 2 * na + 1, 2 * nb + 1
    i, j = np.meshgrid(np.arange(Ni), np.arange(Nj), indexing="ij")
    X = np.stack([0.5 * i + skew * 0.4 * j, 0.4 * j + 0.1 * i], axis=-1).reshape(-1, 2)
    idx = np.arange(Ni * Nj).reshape(Ni, Nj)
    els = [[[idx[wa + a, wb + b] for b in range(3)] for a in range(3)]
           for wa in range(0, Ni - 2, 2) for wb in range(0, Nj - 2, 2)]
    return OU.UnstructuredQ2Mesh(X, np.array(els))


def test_gradient_exact_for_quadratics_on_affine_elements():
    m = _affine_elements()
    x, y = m.X[:, 0], m.X[:, 1]
    f = 0.7 + 1.3 * x - 0.4 * y + 0.9 * x * x - 1.1 * x * y + 0.6 * y * y
    gx, gy = m.grad_X(f)
    assert np.abs(gx - (1.3 + 1.8 * x - 1.1 * y)).max() < 1e-11
    assert np.abs(gy - (-0.4 - 1.1 * x + 1.2 * y)).max() < 1e-11


def test_gradient_at_element_centres_is_the_structured_stencil():
    X = _ogrid()
    Ni, Nj = X.shape[:2]
    um, perm = _shuffled(X, seed=9)
    sm = OM.Q2Mesh(X, periodic_i=False, periodic_j=True)
    rng = np.random.default_rng(2)
    field = rng.standard_normal((Ni, Nj))
    ufield = np.empty(Ni * Nj)
    ufield[perm] = field.reshape(-1)
    sx, sy = sm.grad_X(field)
    ux, uy = um.grad_X(ufield)
    for i in range(1, Ni - 1, 2):
        for j in range(1, Nj, 2):
            n = perm[i * Nj + j]
            assert abs(ux[n] - sx[i, j]) < 1e-11 * (1 + abs(sx[i, j]))
            assert abs(uy[n] - sy[i, j]) < 1e-11 * (1 + abs(sy[i, j]))
    # elsewhere the two operators are different second-order stencils
    corner = perm[2 * Nj + 2]
    assert abs(ux[corner] - sx[2, 2]) > 1e-6


def test_departure_outside_the_nodes_elements_is_refused():
    X = _ogrid()
    Ni, Nj = X.shape[:2]
    um, perm = _shuffled(X, seed=11)
    i, j = 6, 5
    n = perm[i * Nj + j]
    P = X[i + 3, j]            # two elements away along i
    assert um.locate(n, P) is None
    # brute force: some element of the mesh does contain it
    inside = []
    for e in range(um.E.shape[0]):
        E = um.E[e]
        xi, eta = OM.Q2Mesh.bilinear_inverse(um.X[E[0, 0]], um.X[E[2, 0]], um.X[E[0, 2]], um.X[E[2, 2]], P)
        inside.append(abs(xi) <= 1 + 1e-12 and abs(eta) <= 1 + 1e-12)
    assert any(inside)
    assert um.locate(perm[(i + 3) * Nj + j], P) is not None


# ----- the whole step on an unstructured periodic mesh ----------------------
import oracle.solver as OS   # noqa: E402


def _box_pair(n_i, n_j, h, skew, seed):
    sm = OM.periodic_box_mesh(n_i, n_j, n_i * h, n_j * h, skew=skew)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n_i * n_j)
    um = OU.from_box(sm, perm, rng.permutation((n_i // 2) * (n_j // 2)))
    return sm, um, perm


def _to_u(A, perm):
    """[..., Ni, Nj] grid field -> [..., N, 1] in the unstructured numbering."""
    flat = A.reshape(A.shape[:-2] + (-1,))
    out = np.empty_like(flat)
    out[..., perm] = flat
    return out[..., None]


def _solver(mesh, M0, dt, tau=0.6):
    mu = (tau - 0.5) * float(np.mean(M0[0])) * float(np.mean(M0[3])) * dt
    return OS.Solver(mesh, gamma=1.4, Pr=0.71, mu=mu, dt=dt, rho_inf=1.0, u_inf=(0.0, 0.0),
                     T_inf=float(np.mean(M0[3])), bodies=[], M0=M0, walls=False), mu


def test_unstructured_box_step_equals_structured_step_with_its_stencil():
    """With the structured stencil (R18) as its gradient, the oracle's step
    on the shuffled element list of a skewed periodic box is the structured
    step: departures across the periods, interpolation and the adapter to the
    solver agree to round-off over several steps."""
    n_i, n_j = 12, 8
    sm, um, perm = _box_pair(n_i, n_j, 1.0, 0.3, 3)
    rng = np.random.default_rng(4)
    M0 = np.empty((4, n_i, n_j))
    M0[0] = 1.0 + 0.01 * rng.uniform(-1, 1, (n_i, n_j))
    M0[1] = 0.03 * rng.uniform(-1, 1, (n_i, n_j))
    M0[2] = 0.03 * rng.uniform(-1, 1, (n_i, n_j))
    M0[3] = 1.0 / 3.0 + 0.005 * rng.uniform(-1, 1, (n_i, n_j))

    def r18(F):
        grid = F[..., perm].reshape(F.shape[:-1] + (n_i, n_j))
        gx, gy = sm.grad_X(grid)
        ox = np.empty_like(F)
        oy = np.empty_like(F)
        ox[..., perm] = gx.reshape(F.shape)
        oy[..., perm] = gy.reshape(F.shape)
        return ox, oy

    s_s, _ = _solver(sm, M0, 0.5, tau=0.8)
    s_u, _ = _solver(OU.AsGrid(um, grad=r18), _to_u(M0, perm), 0.5, tau=0.8)
    for _ in range(5):
        a = s_s.step()
        b = s_u.step()
    assert np.abs(_to_u(a.f_post, perm) - b.f_post).max() < 1e-13
    assert np.abs(_to_u(a.M, perm) - b.M).max() < 1e-13


def test_taylor_green_decay_on_an_unstructured_box():
    """The genuine unstructured step (gradients by reading R33) on the
    shuffled element list of a periodic box: u = U (sin kx cos ky,
    -cos kx sin ky) decays as exp(-2 nu k^2 t) (Sec. II C)."""
    n = 32
    sm, um, perm = _box_pair(n, n, 1.0, 0.0, 6)
    x = np.arange(n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    k = 2 * np.pi / n
    U = 0.02
    M0 = np.empty((4, n, n))
    M0[0] = 1.0
    M0[1] = U * np.sin(k * X) * np.cos(k * Y)
    M0[2] = -U * np.cos(k * X) * np.sin(k * Y)
    M0[3] = 1.0 / 3.0
    s, mu = _solver(OU.AsGrid(um), _to_u(M0, perm), 1.0, tau=0.6)
    basis = _to_u(np.sin(k * X) * np.cos(k * Y), perm)
    amps, ts = [], []
    for step in range(1, 161):
        r = s.step()
        if step >= 20:
            amps.append((r.M[1] * basis).sum())
            ts.append(step)
    rate = -np.polyfit(ts, np.log(np.abs(amps)), 1)[0]
    assert abs(rate / (2 * mu * k * k) - 1) < 0.02


# ----- the coupled step on an element list with a wall and a far field --------
def _cyl_pair(nr=13, nt=32, seed=7, body=None):
    """A separable cylinder O-grid (odd nr, so the elements tile it), its
    shuffled element list, chains and the R18 stencil mapped through the
    numbering."""
    case = inputs.cylinder_case(nr, nt, r_far=6.0, body=body)
    sm = OM.ogrid_mesh(case.r, case.e)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(nr * nt)
    Xl, els = OU.from_ogrid(sm.X, perm)
    els = els[rng.permutation(els.shape[0])]
    um = OU.UnstructuredQ2Mesh(Xl, els)
    wall, far = OU.ogrid_chains(nr, nt, perm)

    def r18(F):
        grid = F[..., perm].reshape(F.shape[:-1] + (nr, nt))
        gx, gy = sm.grad_X(grid)
        ox = np.empty_like(F)
        oy = np.empty_like(F)
        ox[..., perm] = gx.reshape(F.shape)
        oy[..., perm] = gy.reshape(F.shape)
        return ox, oy

    return case, sm, um, perm, wall, far, r18


def _flat(A, perm):
    flat = A.reshape(A.shape[:-2] + (-1,))
    out = np.empty_like(flat)
    out[..., perm] = flat
    return out


def test_chain_normals_of_a_circle_are_radial():
    """Reading R34: the wall chain's normals point out of the body and the
    far chain's out of the domain, both along the node's polar angle on a
    circle (so the far polygon's normal is the O-grid's grid-line direction
    of reading R20)."""
    case, sm, um, perm, wall, far, _ = _cyl_pair()
    th = 2 * np.pi * np.arange(case.ntheta) / case.ntheta
    radial = np.stack([np.cos(th), np.sin(th)], axis=1)
    np.testing.assert_allclose(OU.chain_normals(um.X[wall]), radial, atol=1e-14)
    np.testing.assert_allclose(OU.chain_normals(um.X[far]), radial, atol=1e-14)


def test_element_list_step_with_wall_and_far_field_equals_structured_step():
    """With the structured stencil (R18) as its gradient, the coupled step on
    the shuffled element list of a cylinder O-grid (wall chain, far-field
    chain, a plunging 1-DOF body whose blend moves the mesh, flow from the
    left) is the structured oracle's step: departures and boundary targets
    searched in holding elements, wall and far-field sets of reading R34,
    load and RK4 agree to round-off over several steps."""
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=2.0, v_r=4.0)
    case, sm, um, perm, wall, far, r18 = _cyl_pair(body=body)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=2, noise=2e-2)
    st = {"h": 0.02, "alpha": 0.0, "hdot": 0.004, "adot": 0.0}
    pv = {"h": 0.0199, "alpha": 0.0, "hdot": 0.004, "adot": 0.0}
    s_s = OS.Solver.from_case(sm, case, M0)
    s_u = OU.UnstructuredSolver.from_case(um, wall, far, case, _flat(M0, perm), grad=r18)
    for s in (s_s, s_u):
        s.S, s.S_prev = [dict(st)], [dict(pv)]
    for _ in range(5):
        a = s_s.step()
        b = s_u.step()
        assert max(abs(x - y) for x, y in zip(a.force, b.force)) < 1e-13
    for x, y in ((a.f_post, b.f_post), (a.g_post, b.g_post), (a.M, b.M)):
        assert np.abs(_flat(x, perm) - y).max() < 1e-13 * np.abs(y).max()
    assert np.array_equal(_flat(a.missing, perm), b.missing)
    for k in ("h", "hdot"):
        assert abs(s_s.S[0][k] - s_u.S[0][k]) < 1e-15


def test_element_list_rest_state_around_wall_is_fixed_point():
    """The genuine element-list step (gradients by reading R33): gas at rest
    around a fixed cylinder stays at its equilibrium (wall by Grad's
    approximation at zero gradients, far field, collision)."""
    case, sm, um, perm, wall, far, _ = _cyl_pair(nr=9, nt=16)
    N = um.N
    M0 = np.empty((4, N))
    M0[0], M0[1], M0[2], M0[3] = 1.0, 0.0, 0.0, 1.0 / 3.0
    s = OU.UnstructuredSolver(um, wall, far, gamma=1.4, Pr=0.71, mu=1e-3, dt=case.flow.dt,
                              rho_inf=1.0, u_inf=(0.0, 0.0), T_inf=1.0 / 3.0,
                              bodies=[OS.body_dict(case.bodies[0], 1.0, 0.1)], M0=M0)
    from oracle import kinetics as K
    feq = K.f_eq(1.0, 0.0, 0.0, 1.0 / 3.0)
    for _ in range(4):
        r = s.step()
    np.testing.assert_allclose(r.f_post, np.broadcast_to(feq[:, None], r.f_post.shape), atol=1e-14)
    assert r.missing[:, wall].any() and abs(r.force[0]) < 1e-13 and abs(r.force[1]) < 1e-13


def test_element_list_step_with_its_own_gradient_stays_close_to_structured():
    """The two gradient readings (R18 on the structured grid, R33 on the
    element list) are different second-order stencils: on a smooth start the
    steps differ at the level of the discretisation, not more."""
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=2.0, v_r=4.0)
    case, sm, um, perm, wall, far, _ = _cyl_pair(body=body)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=2)
    s_s = OS.Solver.from_case(sm, case, M0)
    s_u = OU.UnstructuredSolver.from_case(um, wall, far, case, _flat(M0, perm))
    for _ in range(3):
        a = s_s.step()
        b = s_u.step()
    d = np.abs(_flat(a.M, perm) - b.M).max(axis=1)
    assert d.max() < 1e-3 and d.max() > 1e-12


def test_cgrid_element_list_keeps_a_symmetric_flow_symmetric():
    """A C-grid as an element list with its wake cut merged (the two sides
    share the cut's nodes; no mirrored rows): uniform flow along the axis of
    a symmetric section stays mirror-symmetric, rho, u_x and T even and u_y
    odd in y, to round-off over several steps of the element-list step (R33
    gradients, R34 chains) -- the cut is an ordinary interior line."""
    case = inputs.cgrid_case(33, 8, 13, 0.5, 0.25, r_far=5.0, wake=4.0)
    el = inputs.cgrid_element_list(case.X, case.n_cut, seed=3)
    um = OU.UnstructuredQ2Mesh(el.X, el.elements)
    N = um.N
    nr, nt = el.nr, el.nt
    canon = np.arange(nr * nt).reshape(nr, nt)
    for j in range(case.n_cut + 1):
        canon[0, nt - 1 - j] = canon[0, j]
    mirror = np.empty(N, dtype=np.int64)
    for i in range(nr):
        for j in range(nt):
            mirror[el.perm[canon[i, j]]] = el.perm[canon[i, nt - 1 - j]]
    np.testing.assert_allclose(el.X[mirror, 0], el.X[:, 0], atol=1e-14)
    np.testing.assert_allclose(el.X[mirror, 1], -el.X[:, 1], atol=1e-14)
    M0 = np.empty((4, N))
    M0[0], M0[1], M0[2], M0[3] = 1.0, case.flow.u_inf, 0.0, case.flow.t_inf
    s = OU.UnstructuredSolver.from_case(um, el.wall, el.far, case, M0)
    for _ in range(4):
        r = s.step()
    M = r.M
    assert np.abs(M[2]).max() > 1e-6                    # the flow is not trivial
    for c, sign in ((0, 1), (1, 1), (2, -1), (3, 1)):
        np.testing.assert_allclose(M[c][mirror], sign * M[c], rtol=0, atol=1e-13 * np.abs(M[c]).max() + 1e-16)
