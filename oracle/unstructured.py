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
unchanged.  ``UnstructuredSolver`` is the coupled step on an element list
with a body: a closed wall chain and a closed far-field chain of nodes.

Boundaries on an element list (reading R34, the unstructured counterpart of
R10, R19 and R20): the wall chain and the far-field chain are node lists in
counterclockwise order (even entries the vertices of the straight element
edges); the wall normal n0 and the far field's outward direction n_out are
the normals of those polygons, as on a structured mesh's wall row (on an
O-grid whose grid lines meet the far circle radially the far polygon's
normal is the grid-line direction of R20).  The targets' points B are
searched in the node's holding elements like a departure point."""
from __future__ import annotations

import types

import numpy as np

from . import ale, boundary, forces
from . import kinetics as K
from .mesh import XI_TOL, XI_TOL_THIN, DepartureError, Q2Mesh
from .solver import Solver


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


def chain_normals(P):
    """Unit normals at the nodes of a closed chain P[n, 2] (counterclockwise
    around what it bounds; even entries the vertices of its straight edges):
    the wall normals of boundary.wall_normals applied to the chain, out of
    the enclosed region for a counterclockwise chain around a body, out of
    the domain for a counterclockwise chain around the domain."""
    return boundary.wall_normals(types.SimpleNamespace(Nj=len(P), X=np.asarray(P)[None]))


class UnstructuredSolver(Solver):
    """The coupled step (Sec. III: fluid step, loads, RK4) on an element list
    with one body: wall = closed chain of node indices around the body,
    far = closed chain around the domain (both counterclockwise), grad = the
    nodal gradient operator ([..., N] -> (d/dX, d/dY); reading R33 by
    default).  The step follows the structured oracle's order (solver.py)
    with the node sets of reading R34: far-field nodes take equilibria at
    their targets, every other node streams, wall nodes replace their
    missing populations by Grad's approximation."""

    def __init__(self, um, wall, far, *, gamma, Pr, mu, dt, rho_inf, u_inf, T_inf, bodies, M0,
                 grad=None):
        super().__init__(um, gamma=gamma, Pr=Pr, mu=mu, dt=dt, rho_inf=rho_inf, u_inf=u_inf,
                         T_inf=T_inf, bodies=bodies, M0=M0, walls=False)
        self.um = um
        self.wall = np.asarray(wall, dtype=np.int64)
        self.far = np.asarray(far, dtype=np.int64)
        self.grad = grad or um.grad_X
        self.n0 = chain_normals(um.X[self.wall])
        self.n_far = chain_normals(um.X[self.far])
        self.is_far = np.zeros(um.N, dtype=bool)
        self.is_far[self.far] = True

    @classmethod
    def from_case(cls, um, wall, far, case, M0, grad=None):
        import math
        from .solver import body_dict
        fl = case.flow
        u_inf = fl.ma * math.sqrt(fl.gamma * fl.t_inf)
        bodies = [body_dict(b, fl.rho_inf, u_inf) for b in case.bodies]
        mu = fl.rho_inf * u_inf * fl.length / fl.re
        return cls(um, wall, far, gamma=fl.gamma, Pr=fl.pr, mu=mu, dt=fl.dt, rho_inf=fl.rho_inf,
                   u_inf=(u_inf, 0.0), T_inf=fl.t_inf, bodies=bodies, M0=M0, grad=grad)

    def _locate(self, P, nodes):
        e, xi, eta, found = self.um.locate_all(P, nodes)
        return e, xi, eta, found

    def _pgrad(self, F, field):
        dX, dY = self.grad(field)
        return ale.physical_gradient(F, dX, dY)

    def step(self):
        um, dt, Cv = self.um, self.dt, self.Cv
        X, N = um.X, um.N
        wall, far = self.wall, self.far
        inner = np.nonzero(~self.is_far)[0]
        # 1. kinematics
        F = ale.deformation_gradient(X, self.bodies, self.S)
        VG = ale.mesh_velocity(X, self.bodies, self.S, self.S_prev, dt)
        chat = ale.transformed_velocities(F, VG)
        # 2. departure points in the holding elements and Q2 interpolation
        f_pre = np.zeros((9, N))
        g_pre = np.zeros((9, N))
        missing = np.zeros((9, N), dtype=bool)
        missing[:, wall] = boundary.missing_mask(chat[:, wall], self.n0)
        for k in range(9):
            e, xi, eta, found = self._locate(X[inner] - dt * chat[k, inner], inner)
            need = ~missing[k, inner]
            if np.any(need & ~found):
                bad = inner[np.argmax(need & ~found)]
                raise DepartureError(f"departure point of direction {k} at node {bad} is not in "
                                     f"an element holding the node")
            e = np.where(need, e, 0)
            f_pre[k, inner] = np.where(need, um.interpolate(self.f[k], e, xi, eta), 0.0)
            g_pre[k, inner] = np.where(need, um.interpolate(self.g[k], e, xi, eta), 0.0)
        # 3. wall: Grad's approximation at the targets (B = A + dt n0)
        e, xi, eta, found = self._locate(X[wall] + dt * self.n0, wall)
        if not np.all(found):
            raise RuntimeError("wall target point B outside the elements holding its node")
        rho_b = um.interpolate(self.M_prev[0], e, xi, eta)
        T_b = um.interpolate(self.M_prev[3], e, xi, eta)
        grads = []
        for comp in (1, 2, 3):
            gx, gy = self._pgrad(F, self.M_prev[comp])
            grads.append((gx[wall], gy[wall]))
        fm, gm = boundary.grad_populations(rho_b, VG[wall, 0], VG[wall, 1], T_b, grads, Cv,
                                           self.mu, dt, self.Pr)
        f_pre[:, wall] = np.where(missing[:, wall], fm, f_pre[:, wall])
        g_pre[:, wall] = np.where(missing[:, wall], gm, g_pre[:, wall])
        # 4. moments; far-field targets at B = A - dt n_out (reading R20 on
        # the far polygon's normal)
        M = np.empty((4, N))
        rho, ux, uy, E, T = K.moments(f_pre[:, inner], g_pre[:, inner], Cv)
        M[0, inner], M[1, inner], M[2, inner], M[3, inner] = rho, ux, uy, T
        e, xi, eta, found = self._locate(X[far] - dt * self.n_far, far)
        if not np.all(found):
            raise RuntimeError("far-field point B outside the elements holding its node")
        ob = [um.interpolate(self.M_prev[c], e, xi, eta) for c in range(4)]
        inlet = (self.u_inf[0] * self.n_far[:, 0] + self.u_inf[1] * self.n_far[:, 1]) < 0.0
        M[0, far] = ob[0]
        M[1, far] = np.where(inlet, self.u_inf[0], ob[1])
        M[2, far] = np.where(inlet, self.u_inf[1], ob[2])
        M[3, far] = np.where(inlet, self.T_inf, ob[3])
        # 5. correction fields
        dqx, dqy = K.delta_q(M[0], M[1], M[2], M[3])
        mu_p = self.mu / (M[0] * M[3])
        ddx, _ = self._pgrad(F, dqx)
        _, ddy = self._pgrad(F, dqy)
        Yx, _ = self._pgrad(F, mu_p * ddx)
        _, Yy = self._pgrad(F, mu_p * ddy)
        # 6. collision; the far field takes the equilibria at its targets
        f_post = np.empty_like(f_pre)
        g_post = np.empty_like(g_pre)
        f_post[:, inner], g_post[:, inner] = K.collide(f_pre[:, inner], g_pre[:, inner], Yx[inner],
                                                       Yy[inner], self.mu, dt, Cv, self.Pr)
        f_post[:, far] = K.f_eq(M[0, far], M[1, far], M[2, far], M[3, far])
        g_post[:, far] = K.g_eq(M[0, far], M[1, far], M[2, far], M[3, far], Cv)
        # 7. load on the body from the wall chain
        force = (0.0, 0.0, 0.0)
        if self.bodies:
            b, st = self.bodies[0], self.S[0]
            sxx, sxy, syy = forces.node_stress(f_pre[:, wall], g_pre[:, wall], Cv, self.mu, dt,
                                               self.Pr)
            x_wall = ale.mesh_position(X[wall], self.bodies, self.S)
            x_ref = np.array([b["xp"], b["yp"] + st["h"]])
            force = (self.load_reduction or forces.wall_force)(x_wall, sxx, sxy, syy, x_ref)
        # 8. structural update
        new_S = self._advance_bodies([force] * len(self.bodies))
        self.S_prev = [dict(s) for s in self.S]
        self.S = new_S
        self.f, self.g = f_post, g_post
        self.M_prev = M
        self.n += 1
        from .solver import StepResult
        return StepResult(f_pre, g_pre, f_post, g_post, M, force, missing)


def ogrid_chains(Ni, Nj, perm_nodes=None):
    """Wall chain (row 0) and far-field chain (row Ni - 1) of a structured
    O-grid numbered i Nj + j (relabelled by perm_nodes): both in increasing
    j, i.e. counterclockwise for a grid whose angular index runs
    counterclockwise."""
    wall = np.arange(Nj)
    far = (Ni - 1) * Nj + np.arange(Nj)
    if perm_nodes is not None:
        perm_nodes = np.asarray(perm_nodes)
        wall, far = perm_nodes[wall], perm_nodes[far]
    return wall, far
