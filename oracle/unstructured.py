"""Unstructured Q2 meshes: the building blocks of the step on a mesh given
as quadrilateral Q2 elements over a node list (the paper's own meshes are
of this kind, Sec. II C and Sec. IV).  TEST INFRASTRUCTURE ONLY (see the
package docstring).

An element is 3 x 3 node indices [a][b] (a along its first reference
coordinate xi, b along eta; entry (a, b) sits at (xi, eta) = (a - 1, b - 1)).
Its geometry is the bilinear map of its four corners (subparametric, reading
R7), its fields are interpolated with the nine Q2 Lagrange products (Eq.
SemiLagrProp).  An element may carry its own node coordinates (a periodic
mesh: the element that wraps sees its nodes across the period); a point
given in a node's frame is moved into a holding element's frame by the
difference of that node's two positions.  The departure point of a node
(Eq. depPnt) is searched in the elements that hold the node, in increasing
element index (reading R9, with the two containment passes of reading R8).

Gradients (reading R33, the unstructured counterpart of R18): at a node, the
derivative of each holding element's Q2 interpolant at the node's reference
position, mapped to X by that element's Q2 metric there (Eq. ddx+fem), then
the mean over the holding elements.  This is exact for fields linear in X on
any subparametric mesh and for quadratics on affine elements; at an
element's centre node (one holding element) it is the central difference of
reading R18.

``AsGrid`` presents such a mesh as an [N, 1] grid to ``solver.Solver`` (no
walls: a periodic mesh), so the step of the structured oracle runs on it
unchanged."""
from __future__ import annotations

import numpy as np

from .mesh import XI_TOL, XI_TOL_THIN, Q2Mesh


def _lagrange(t):
    """1-D Q2 Lagrange basis on -1, 0, 1 (values at t)."""
    return 0.5 * t * (t - 1.0), 1.0 - t * t, 0.5 * t * (t + 1.0)


def _lagrange_d(t):
    """Derivatives of the 1-D Q2 Lagrange basis at t."""
    return t - 0.5, -2.0 * t, t + 0.5


class UnstructuredQ2Mesh:
    def __init__(self, X, elements, elem_coords=None):
        self.X = np.asarray(X, dtype=np.float64)            # [N, 2]
        self.E = np.asarray(elements, dtype=np.int64)       # [Ne, 3, 3]
        if self.E.ndim != 3 or self.E.shape[1:] != (3, 3):
            raise ValueError("elements must be [Ne][3][3] node indices")
        self.N = self.X.shape[0]
        # per-element node coordinates [Ne, 3, 3, 2]
        self.XE = self.X[self.E] if elem_coords is None else np.asarray(elem_coords, dtype=np.float64)
        # node -> holding elements, in increasing element index, with the
        # node's entry (a, b) in each
        hold = [[] for _ in range(self.N)]
        for e in range(self.E.shape[0]):
            for a in range(3):
                for b in range(3):
                    hold[self.E[e, a, b]].append((e, a, b))
        if any(len(h) == 0 for h in hold):
            raise ValueError("every node must belong to an element")
        self.hold = hold
        K = max(len(h) for h in hold)
        self.cand = -np.ones((self.N, K), dtype=np.int64)        # holding elements, padded
        self.shift = np.zeros((self.N, K, 2))                     # element frame - node frame
        for n, h in enumerate(hold):
            for k, (e, a, b) in enumerate(h):
                self.cand[n, k] = e
                self.shift[n, k] = self.XE[e, a, b] - self.X[n]
        # gradient entries: one per (node, holding element)
        ent = [(n, e, a, b) for n, h in enumerate(hold) for (e, a, b) in h]
        self.g_n = np.array([t[0] for t in ent])
        self.g_e = np.array([t[1] for t in ent])
        self.g_a = np.array([t[2] for t in ent])
        self.g_b = np.array([t[3] for t in ent])
        self.g_w = 1.0 / np.array([len(hold[t[0]]) for t in ent], dtype=np.float64)

    # ----- Eq. depPnt ----------------------------------------------------
    def locate_all(self, P, nodes=None):
        """For every node n (or the given nodes), the first holding element
        (increasing index) that contains P[n] (given in the node's frame)
        within reading R8's tolerance, else within its second pass, and P's
        reference coordinates there.  Returns (element, xi, eta, found)."""
        P = np.asarray(P, dtype=np.float64)
        nodes = np.arange(self.N) if nodes is None else np.asarray(nodes)
        cand, shift = self.cand[nodes], self.shift[nodes]
        K = cand.shape[1]
        valid = cand >= 0
        e_s = np.where(valid, cand, 0)
        C = self.XE[e_s]                                          # [n, K, 3, 3, 2]
        Pk = P[:, None, :] + shift                                # [n, K, 2]
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            xi, eta = Q2Mesh.bilinear_inverse(C[:, :, 0, 0], C[:, :, 2, 0], C[:, :, 0, 2], C[:, :, 2, 2], Pk)
        fin = valid & np.isfinite(xi) & np.isfinite(eta)
        e_o = np.zeros(len(nodes), dtype=np.int64)
        xi_o = np.zeros(len(nodes))
        eta_o = np.zeros(len(nodes))
        found = np.zeros(len(nodes), dtype=bool)
        for tol in (XI_TOL, XI_TOL_THIN):
            ins = fin & (np.abs(xi) <= 1 + tol) & (np.abs(eta) <= 1 + tol)
            for k in range(K):
                take = ins[:, k] & ~found
                e_o = np.where(take, e_s[:, k], e_o)
                xi_o = np.where(take, xi[:, k], xi_o)
                eta_o = np.where(take, eta[:, k], eta_o)
                found |= take
        return e_o, xi_o, eta_o, found

    def locate(self, n, P):
        """locate_all for one node: (element, xi, eta) or None."""
        e, xi, eta, found = self.locate_all(np.asarray(P, dtype=np.float64)[None], np.array([n]))
        return (int(e[0]), float(xi[0]), float(eta[0])) if found[0] else None

    # ----- Eq. SemiLagrProp ----------------------------------------------
    def interpolate(self, field, e, xi, eta):
        """sum over the element's nine nodes of field(node) L_a(xi) L_b(eta);
        field has shape [..., N]; e, xi, eta broadcast together."""
        lx = _lagrange(np.asarray(xi, dtype=np.float64))
        ly = _lagrange(np.asarray(eta, dtype=np.float64))
        E = self.E[np.asarray(e)]
        out = 0.0
        for a in range(3):
            for b in range(3):
                out = out + lx[a] * ly[b] * field[..., E[..., a, b]]
        return out

    # ----- reading R33: nodal gradient -----------------------------------
    def grad_X(self, F):
        """(dF/dX, dF/dY) at every node; F has shape [..., N]."""
        F = np.asarray(F, dtype=np.float64)
        shape = F.shape
        F = F.reshape(-1, self.N)
        E, XE = self.E[self.g_e], self.XE[self.g_e]        # [M, 3, 3], [M, 3, 3, 2]
        a, b = self.g_a, self.g_b
        m = np.arange(len(a))
        dxi = _lagrange_d(a - 1.0)
        deta = _lagrange_d(b - 1.0)
        f_xi = sum(dxi[k] * F[..., E[m, k, b]] for k in range(3))
        f_eta = sum(deta[k] * F[..., E[m, a, k]] for k in range(3))
        x_xi = sum(dxi[k][:, None] * XE[m, k, b] for k in range(3))
        x_eta = sum(deta[k][:, None] * XE[m, a, k] for k in range(3))
        det = x_xi[:, 0] * x_eta[:, 1] - x_xi[:, 1] * x_eta[:, 0]
        gx_e = self.g_w * (x_eta[:, 1] * f_xi - x_xi[:, 1] * f_eta) / det      # [B, M]
        gy_e = self.g_w * (-x_eta[:, 0] * f_xi + x_xi[:, 0] * f_eta) / det
        # the mean over the holding elements, summed in their order
        gx = np.zeros((self.N, F.shape[0]))
        gy = np.zeros((self.N, F.shape[0]))
        np.add.at(gx, self.g_n, gx_e.T)
        np.add.at(gy, self.g_n, gy_e.T)
        return gx.T.reshape(shape), gy.T.reshape(shape)


class AsGrid:
    """An unstructured mesh seen as an [N, 1] grid by ``solver.Solver``
    (walls=False).  grad: an optional replacement of the gradient operator
    (a function of [..., N] fields), e.g. a structured mesh's R18 stencil
    mapped through a renumbering."""

    def __init__(self, um, grad=None):
        self.um = um
        self.X = um.X[:, None, :]
        self.Ni, self.Nj = um.N, 1
        self._grad = grad

    def locate(self, P, ii, jj):
        e, xi, eta, found = self.um.locate_all(P[:, 0, :])
        z = np.zeros_like(e)
        return e[:, None], z[:, None], xi[:, None], eta[:, None], found[:, None]

    def interpolate(self, field, wa, wb, xi, eta):
        return self.um.interpolate(field[..., 0], wa[:, 0], xi[:, 0], eta[:, 0])[:, None]

    def grad_X(self, F):
        gx, gy = (self._grad or self.um.grad_X)(F[..., 0])
        return gx[..., None], gy[..., None]


def from_ogrid(X, perm_nodes=None, perm_elements=None):
    """The elements of a structured O-grid X [Ni][Nj][2] (Ni odd: the windows
    of reading R7 then tile it; Nj even, periodic in j): element (wa, wb) =
    nodes (wa .. wa+2, wb .. wb+2) for even wa, wb.  Nodes are numbered
    i Nj + j, then relabelled by perm_nodes (new index of each old node) and
    the elements reordered by perm_elements.  Returns (X_list, elements)."""
    X = np.asarray(X, dtype=np.float64)
    Ni, Nj = X.shape[:2]
    if Ni % 2 == 0 or Nj % 2:
        raise ValueError("an O-grid of odd Ni and even Nj")
    old = np.arange(Ni * Nj).reshape(Ni, Nj)
    els = []
    for wa in range(0, Ni - 2, 2):
        for wb in range(0, Nj, 2):
            els.append([[old[wa + a, (wb + b) % Nj] for b in range(3)] for a in range(3)])
    els = np.array(els, dtype=np.int64)
    Xl = X.reshape(-1, 2)
    if perm_nodes is not None:
        perm_nodes = np.asarray(perm_nodes)
        Xn = np.empty_like(Xl)
        Xn[perm_nodes] = Xl
        Xl = Xn
        els = perm_nodes[els]
    if perm_elements is not None:
        els = els[np.asarray(perm_elements)]
    return Xl, els


def from_box(mesh, perm_nodes=None, perm_elements=None):
    """The elements of a doubly periodic structured box (``mesh.Q2Mesh`` with
    both directions periodic, even node counts): element (wa, wb) for even
    wa, wb, its nodes' coordinates unwrapped across the periods.  Returns an
    UnstructuredQ2Mesh (nodes relabelled by perm_nodes, elements reordered by
    perm_elements)."""
    Ni, Nj = mesh.Ni, mesh.Nj
    old = np.arange(Ni * Nj).reshape(Ni, Nj)
    els, xe = [], []
    for wa in range(0, Ni, 2):
        for wb in range(0, Nj, 2):
            els.append([[old[(wa + a) % Ni, (wb + b) % Nj] for b in range(3)] for a in range(3)])
            xe.append([[mesh.coords(np.array(wa + a), np.array(wb + b)) for b in range(3)] for a in range(3)])
    els = np.array(els, dtype=np.int64)
    xe = np.array(xe, dtype=np.float64)
    Xl = mesh.X.reshape(-1, 2)
    if perm_nodes is not None:
        perm_nodes = np.asarray(perm_nodes)
        Xn = np.empty_like(Xl)
        Xn[perm_nodes] = Xl
        Xl = Xn
        els = perm_nodes[els]
    if perm_elements is not None:
        els = els[np.asarray(perm_elements)]
        xe = xe[np.asarray(perm_elements)]
    return UnstructuredQ2Mesh(Xl, els, xe)
