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
