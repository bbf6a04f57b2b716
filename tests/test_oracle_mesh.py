"""Pins of the oracle's departure-point solve, Q2 interpolation and FE
gradient (Sec. II B): brute-force element search on tiny meshes, polynomial
exactness, partition of unity and textbook streaming on a lattice-matched
mesh."""
import numpy as np

from oracle import mesh as OM
from paper_2107_01370_gb300 import inputs


def _tiny_ogrid(nr=7, nt=8):
    r = inputs.ogrid_radii(nr, 0.5, 3.0, 2 * np.pi * 0.5 / nt)
    e = inputs.ogrid_directions(nt)
    return OM.ogrid_mesh(r, e)


def _brute_force_cell(m, P):
    """Search every cell of the mesh with an independent containment test
    (point in the quadrilateral of the cell's four corner nodes, via cross
    products); return (a, b) of the first match or None."""
    for a in range(m.Ni - 1):
        for b in range(m.Nj):
            q = [m.coords(np.array(a), np.array(b)), m.coords(np.array(a + 1), np.array(b)),
                 m.coords(np.array(a + 1), np.array(b + 1)), m.coords(np.array(a), np.array(b + 1))]
            s = []
            for k in range(4):
                e = q[(k + 1) % 4] - q[k]
                d = P - q[k]
                s.append(e[0] * d[1] - e[1] * d[0])
            s = np.array(s)
            if np.all(s >= -1e-13) or np.all(s <= 1e-13):
                return a, b
    return None


def test_locate_agrees_with_brute_force_search():
    m = _tiny_ogrid()
    rng = np.random.default_rng(0)
    dt = 0.6 * (m.X[1, 0, 0] - m.X[0, 0, 0])
    for _ in range(200):
        i = rng.integers(1, m.Ni - 1)
        j = rng.integers(0, m.Nj)
        d = rng.uniform(-1, 1, 2)
        d = d / np.hypot(*d) * rng.uniform(0, dt)
        P = m.X[i, j] + d
        wa, wb, xi, eta, found = m.locate(P[None], np.array([i]), np.array([j]))
        bf = _brute_force_cell(m, P)
        assert found[0] and bf is not None
        # the located window contains the brute-force cell and the bilinear
        # map sends (xi, eta) back to P
        la, lb = bf[0] - wa[0], (bf[1] - wb[0]) % m.Nj
        assert la in (0, 1) and lb in (0, 1)
        c = [m.coords(wa + 0, wb + 0)[0], m.coords(wa + 2, wb)[0], m.coords(wa, wb + 2)[0],
             m.coords(wa + 2, wb + 2)[0]]
        x, y = xi[0], eta[0]
        Q = (c[0] * (1 - x) * (1 - y) + c[1] * (1 + x) * (1 - y) + c[2] * (1 - x) * (1 + y)
             + c[3] * (1 + x) * (1 + y)) / 4
        np.testing.assert_allclose(Q, P, atol=1e-13)


def test_interpolation_dense_operator_partition_of_unity():
    """Every row of the interpolation operator sums to one (constants are
    reproduced) and the operator evaluated on the coordinate fields returns the
    departure point itself (the subparametric geometry is reproduced)."""
    m = _tiny_ogrid(9, 12)
    rng = np.random.default_rng(1)
    ii, jj = np.meshgrid(np.arange(m.Ni - 1), np.arange(m.Nj), indexing="ij")
    dt = 0.4 * (m.X[1, 0, 0] - m.X[0, 0, 0])
    d = rng.uniform(-1, 1, ii.shape + (2,)) * dt
    d[0] = np.abs(d[0]) * np.array([1, 0]) + 0.0  # wall row: move outward
    P = m.X[:m.Ni - 1] + d
    P[0] = m.X[0] * (1 + rng.uniform(0, dt, (m.Nj, 1)) / 0.5)
    wa, wb, xi, eta, found = m.locate(P, ii, jj)
    assert found.all()
    one = m.interpolate(np.ones((m.Ni, m.Nj)), wa, wb, xi, eta)
    np.testing.assert_allclose(one, 1.0, atol=1e-14)
    for comp in range(2):
        v = m.interpolate(m.X[..., comp], wa, wb, xi, eta)
        np.testing.assert_allclose(v, P[..., comp], atol=1e-13)


def _affine_mesh(ni=9, nj=11):
    A = np.array([[0.7, 0.25], [-0.1, 0.9]])
    i, j = np.meshgrid(np.arange(ni), np.arange(nj), indexing="ij")
    X = np.stack([A[0, 0] * i + A[0, 1] * j + 0.3, A[1, 0] * i + A[1, 1] * j - 0.2], -1)
    return OM.Q2Mesh(X, periodic_i=False, periodic_j=False)


def test_interpolation_exact_for_quadratics_on_affine_mesh():
    m = _affine_mesh()
    rng = np.random.default_rng(2)
    co = rng.normal(size=6)

    def q(X):
        x, y = X[..., 0], X[..., 1]
        return co[0] + co[1] * x + co[2] * y + co[3] * x * x + co[4] * x * y + co[5] * y * y
    field = q(m.X)
    for _ in range(100):
        i = rng.integers(1, m.Ni - 1)
        j = rng.integers(1, m.Nj - 1)
        P = m.X[i, j] + rng.uniform(-0.3, 0.3, 2)
        wa, wb, xi, eta, found = m.locate(P[None], np.array([i]), np.array([j]))
        assert found[0]
        np.testing.assert_allclose(m.interpolate(field, wa, wb, xi, eta)[0], q(P), rtol=1e-12,
                                   atol=1e-12)


def test_fe_gradient_exact_for_quadratics_on_affine_mesh():
    m = _affine_mesh()
    co = np.array([0.3, -1.2, 0.7, 0.9, -0.4, 0.25])
    x, y = m.X[..., 0], m.X[..., 1]
    field = co[0] + co[1] * x + co[2] * y + co[3] * x * x + co[4] * x * y + co[5] * y * y
    dX, dY = m.grad_X(field)
    np.testing.assert_allclose(dX, co[1] + 2 * co[3] * x + co[4] * y, atol=1e-11)
    np.testing.assert_allclose(dY, co[2] + co[4] * x + 2 * co[5] * y, atol=1e-11)


def test_lattice_matched_mesh_reduces_to_textbook_streaming():
    """Cartesian mesh with spacing h = dt and c_hat = c: every departure point
    is a node, the Q2 weights are Kronecker deltas and propagation is the
    textbook shift f_i(x - c_i dt)."""
    from oracle import kinetics as K
    n = 8
    m = OM.periodic_box_mesh(n, n, 1.0, 1.0)
    h = 1.0 / n
    rng = np.random.default_rng(3)
    f = rng.uniform(size=(n, n))
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for k, (cx, cy) in enumerate(K.C):
        P = m.X - h * np.array([cx, cy])
        wa, wb, xi, eta, found = m.locate(P, ii, jj)
        assert found.all()
        got = m.interpolate(f, wa, wb, xi, eta)
        ref = np.roll(np.roll(f, int(cx), axis=0), int(cy), axis=1)
        np.testing.assert_allclose(got, ref, atol=1e-14)


def test_departure_beyond_adjacent_cells_is_not_found():
    m = _tiny_ogrid()
    i, j = 3, 2
    P = m.X[i + 2, j]          # two cells away
    _, _, _, _, found = m.locate(P[None], np.array([i]), np.array([j]))
    assert not found[0]


def test_ogrid_tables_are_subparametric():
    r = inputs.ogrid_radii(12, 0.5, 5.0, 0.05)
    assert abs(r[-1] - 5.0) < 1e-9
    np.testing.assert_allclose(r[1:-2:2], 0.5 * (r[0:-3:2] + r[2:-1:2]), rtol=1e-15)
    np.testing.assert_allclose(r[-1] - r[-2], r[-2] - r[-3], rtol=1e-12)
    e = inputs.ogrid_directions(10)
    np.testing.assert_allclose(e[1::2], 0.5 * (e[0::2] + np.roll(e[0::2], -1, 0)), rtol=1e-15)
