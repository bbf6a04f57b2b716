"""Unstructured Q2 meshes: the building blocks of the step on a mesh given
as quadrilateral Q2 elements over a node list (the paper's own meshes are
of this kind, Sec. II C and Sec. IV).  TEST INFRASTRUCTURE ONLY (see the
package docstring).

An element is 3 x 3 node indices [a][b] (a along its first reference
coordinate xi, b along eta; entry (a, b) sits at (xi, eta) = (a - 1, b - 1)).
Its geometry is the bilinear map of its four corners (subparametric, reading
R7), its fields are interpolated with the nine Q2 Lagrange products (Eq.
SemiLagrProp).  The departure point of a node (Eq. depPnt) is searched in the
elements that hold the node, in increasing element index (reading R9, with
the two containment passes of reading R8).

Gradients (reading R33, the unstructured counterpart of R18): at a node, the
derivative of each holding element's Q2 interpolant at the node's reference
position, mapped to X by that element's Q2 metric there (Eq. ddx+fem), then
the mean over the holding elements.  This is exact for fields linear in X on
any subparametric mesh and for quadratics on affine elements; at an
element's centre node (one holding element) it is the central difference of
reading R18."""
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
    def __init__(self, X, elements):
        self.X = np.asarray(X, dtype=np.float64)            # [N, 2]
        self.E = np.asarray(elements, dtype=np.int64)       # [Ne, 3, 3]
        if self.E.ndim != 3 or self.E.shape[1:] != (3, 3):
            raise ValueError("elements must be [Ne][3][3] node indices")
        self.N = self.X.shape[0]
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

    # ----- Eq. depPnt ----------------------------------------------------
    def locate(self, n, P):
        """Element holding node n that contains P, and P's reference
        coordinates there: the first element (increasing index) within the
        containment tolerance of reading R8, else the first within its second
        pass.  Returns (element, xi, eta) or None."""
        cand = []
        for e, _, _ in self.hold[n]:
            E = self.E[e]
            xi, eta = Q2Mesh.bilinear_inverse(self.X[E[0, 0]], self.X[E[2, 0]], self.X[E[0, 2]],
                                              self.X[E[2, 2]], np.asarray(P, dtype=np.float64))
            cand.append((e, float(xi), float(eta)))
        for tol in (XI_TOL, XI_TOL_THIN):
            for e, xi, eta in cand:
                if np.isfinite(xi) and np.isfinite(eta) and abs(xi) <= 1 + tol and abs(eta) <= 1 + tol:
                    return e, xi, eta
        return None

    # ----- Eq. SemiLagrProp ----------------------------------------------
    def interpolate(self, field, e, xi, eta):
        """sum over the element's nine nodes of field(node) L_a(xi) L_b(eta);
        field has shape [..., N]."""
        lx = _lagrange(xi)
        ly = _lagrange(eta)
        out = 0.0
        for a in range(3):
            for b in range(3):
                out = out + lx[a] * ly[b] * field[..., self.E[e, a, b]]
        return out

    # ----- reading R33: nodal gradient -----------------------------------
    def grad_X(self, F):
        """(dF/dX, dF/dY) at every node; F has shape [..., N]."""
        F = np.asarray(F, dtype=np.float64)
        gx = np.zeros(F.shape)
        gy = np.zeros(F.shape)
        for n in range(self.N):
            sx = 0.0
            sy = 0.0
            for e, a, b in self.hold[n]:
                E = self.E[e]
                dxi = _lagrange_d(float(a - 1))    # d/dxi of L_a' at the node (L_b'(eta_b) = delta)
                deta = _lagrange_d(float(b - 1))
                f_xi = sum(dxi[k] * F[..., E[k, b]] for k in range(3))
                f_eta = sum(deta[k] * F[..., E[a, k]] for k in range(3))
                x_xi = sum(dxi[k] * self.X[E[k, b]] for k in range(3))
                x_eta = sum(deta[k] * self.X[E[a, k]] for k in range(3))
                det = x_xi[0] * x_eta[1] - x_xi[1] * x_eta[0]
                sx = sx + (x_eta[1] * f_xi - x_xi[1] * f_eta) / det
                sy = sy + (-x_eta[0] * f_xi + x_xi[0] * f_eta) / det
            m = len(self.hold[n])
            gx[..., n] = sx / m
            gy[..., n] = sy / m
        return gx, gy


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
