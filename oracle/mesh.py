"""Mesh side of the oracle: second-order (Q2) elements on a structured
body-fitted mesh, the departure-point solve and the finite-element
interpolation and gradient (Sec. II B, Eqs. SemiLagrProp, depPnt, ddx+fem).

Test infrastructure only (see the package docstring).

A mesh is an array X[Ni, Nj, 2] of node coordinates in the undeformed domain.
Either index direction may be periodic; a periodic direction carries a shift
vector added per wrap (zero for the angular direction of an O-grid, the
period for a doubly periodic box).  Elements are 3x3-node windows whose
first node has even indices; a cell (a, b) = [a, a+1] x [b, b+1] in index
space belongs to the window starting at 2*floor(a/2) (clamped to Ni-3 in a
non-periodic direction).  Reading R7: meshes are subparametric (mid nodes on
the bilinear positions), so the first-order departure-point solve of Eq.
depPnt is exact for the Q2 geometry.
"""
from __future__ import annotations

import numpy as np

XI_TOL = 1e-12       # reading R8: a cell contains a point if its local coords are within 1e-12
# reading R8, second pass: when no adjacent cell holds the point within XI_TOL,
# the first (in the fixed order) within XI_TOL_THIN.  The bilinear inverse in
# absolute coordinates rounds at |X| eps / h in reference units, which passes
# 1e-12 on cells thousands of times longer than wide far from the origin (the
# wake of a C-grid behind a sharp trailing edge); such points lie on the edge
# two elements share, where their Q2 interpolants agree.
XI_TOL_THIN = 1e-9
NEWTON_TOL = 1e-13
NEWTON_MAX = 50


class DepartureError(RuntimeError):
    """Departure point outside the cells adjacent to its node (CFL violated)."""


class Q2Mesh:
    def __init__(self, X, periodic_i=False, periodic_j=True, shift_i=(0.0, 0.0),
                 shift_j=(0.0, 0.0)):
        self.X = np.asarray(X, dtype=np.float64)
        self.Ni, self.Nj = self.X.shape[:2]
        self.periodic_i = periodic_i
        self.periodic_j = periodic_j
        self.shift_i = np.asarray(shift_i, dtype=np.float64)
        self.shift_j = np.asarray(shift_j, dtype=np.float64)
        if periodic_i and self.Ni % 2:
            raise ValueError("periodic direction needs an even node count")
        if periodic_j and self.Nj % 2:
            raise ValueError("periodic direction needs an even node count")

    # ----- node access with periodic wrap -------------------------------
    def wrap(self, a, b):
        a = np.asarray(a)
        b = np.asarray(b)
        ka = np.floor_divide(a, self.Ni) if self.periodic_i else np.zeros_like(a)
        kb = np.floor_divide(b, self.Nj) if self.periodic_j else np.zeros_like(b)
        return a - ka * self.Ni, b - kb * self.Nj, ka, kb

    def coords(self, a, b):
        """Unwrapped coordinates of node (a, b): X of the wrapped node plus the
        period shifts."""
        aw, bw, ka, kb = self.wrap(a, b)
        x = self.X[aw, bw]
        return x + ka[..., None] * self.shift_i + kb[..., None] * self.shift_j

    def valid_cell(self, a, b):
        ok = np.ones(np.broadcast(a, b).shape, dtype=bool)
        if not self.periodic_i:
            ok &= (a >= 0) & (a <= self.Ni - 2)
        if not self.periodic_j:
            ok &= (b >= 0) & (b <= self.Nj - 2)
        return ok

    def window_of_cell(self, a, b):
        wa = 2 * np.floor_divide(a, 2)
        wb = 2 * np.floor_divide(b, 2)
        if not self.periodic_i:
            wa = np.minimum(wa, self.Ni - 3)
        if not self.periodic_j:
            wb = np.minimum(wb, self.Nj - 3)
        return wa, wb

    # ----- Eq. depPnt: bilinear inverse over the element's four corners --
    @staticmethod
    def bilinear_inverse(c00, c10, c01, c11, P):
        """Solve P = sum_{s=1..4} X_s N'_s(xi, eta) for (xi, eta) by Newton's
        method from (0, 0) (Eq. depPnt; reading R8: stop when the update is
        below 1e-13).  Corner s has reference position (-+1, -+1):
        c00 = (-1,-1), c10 = (+1,-1), c01 = (-1,+1), c11 = (+1,+1)."""
        # work relative to the first corner so that round-off scales with the
        # element size, not with the distance from the origin
        c10 = c10 - c00
        c01 = c01 - c00
        c11 = c11 - c00
        P = P - c00
        c00 = np.zeros_like(c00)
        xi = np.zeros(P.shape[:-1])
        eta = np.zeros(P.shape[:-1])
        for _ in range(NEWTON_MAX):
            n00 = 0.25 * (1 - xi) * (1 - eta)
            n10 = 0.25 * (1 + xi) * (1 - eta)
            n01 = 0.25 * (1 - xi) * (1 + eta)
            n11 = 0.25 * (1 + xi) * (1 + eta)
            r = (n00[..., None] * c00 + n10[..., None] * c10 + n01[..., None] * c01
                 + n11[..., None] * c11 - P)
            dxi = 0.25 * ((c10 - c00)[..., :] * (1 - eta)[..., None]
                          + (c11 - c01) * (1 + eta)[..., None])
            deta = 0.25 * ((c01 - c00) * (1 - xi)[..., None]
                           + (c11 - c10) * (1 + xi)[..., None])
            det = dxi[..., 0] * deta[..., 1] - dxi[..., 1] * deta[..., 0]
            s_xi = -(deta[..., 1] * r[..., 0] - deta[..., 0] * r[..., 1]) / det
            s_eta = -(-dxi[..., 1] * r[..., 0] + dxi[..., 0] * r[..., 1]) / det
            xi = xi + s_xi
            eta = eta + s_eta
            # keep iterating while some point that may still be inside the
            # element has not converged
            live = (np.maximum(np.abs(s_xi), np.abs(s_eta)) >= NEWTON_TOL)
            live &= np.isfinite(xi) & np.isfinite(eta)
            live &= (np.abs(xi) < 4.0) & (np.abs(eta) < 4.0)
            if not np.any(live):
                break
        return xi, eta

    def locate_in_cell(self, a, b, P, tol=XI_TOL):
        """Reference coordinates of P in the window of cell (a, b) and whether
        P lies in that cell (with the R8 tolerance)."""
        wa, wb = self.window_of_cell(a, b)
        c00 = self.coords(wa, wb)
        c10 = self.coords(wa + 2, wb)
        c01 = self.coords(wa, wb + 2)
        c11 = self.coords(wa + 2, wb + 2)
        xi, eta = self.bilinear_inverse(c00, c10, c01, c11, P)
        la = a - wa
        lb = b - wb
        inside = ((xi >= la - 1 - tol) & (xi <= la + tol)
                  & (eta >= lb - 1 - tol) & (eta <= lb + tol))
        inside &= np.isfinite(xi) & np.isfinite(eta)
        return wa, wb, xi, eta, inside

    def locate(self, P, i, j, candidates=None):
        """Find the cell adjacent to node (i, j) that contains P (unwrapped,
        i.e. expressed in the node's own periodic image).  The candidates are
        the four cells sharing the node, tried in the fixed order
        (i-1, j-1), (i-1, j), (i, j-1), (i, j); the first that contains P wins
        (reading R9); the points no candidate holds within XI_TOL go through
        the second pass of reading R8.  Returns wa, wb, xi, eta, found."""
        i = np.asarray(i)
        j = np.asarray(j)
        if candidates is None:
            candidates = [(-1, -1), (-1, 0), (0, -1), (0, 0)]
        out = self._locate_pass(P, i, j, candidates, XI_TOL)
        found = out[4]
        if not found.all():
            shape = found.shape
            miss = np.nonzero(~found.ravel())[0]
            Pf = np.broadcast_to(P, shape + (2,)).reshape(-1, 2)[miss]
            i_f = np.broadcast_to(i, shape).ravel()[miss]
            j_f = np.broadcast_to(j, shape).ravel()[miss]
            second = self._locate_pass(Pf, i_f, j_f, candidates, XI_TOL_THIN)
            out = [o.ravel().copy() for o in out]
            for o_all, o_sub in zip(out, second):
                o_all[miss] = o_sub
            out = [o.reshape(shape) for o in out]
        return tuple(out)

    def _locate_pass(self, P, i, j, candidates, tol):
        shape = np.broadcast(i, j).shape
        wa_o = np.zeros(shape, dtype=np.int64)
        wb_o = np.zeros(shape, dtype=np.int64)
        xi_o = np.zeros(shape)
        eta_o = np.zeros(shape)
        found = np.zeros(shape, dtype=bool)
        for da, db in candidates:
            a = i + da
            b = j + db
            ok = self.valid_cell(a, b)
            if not np.any(ok & ~found):
                continue
            a_s = np.where(ok, a, 0)
            b_s = np.where(ok, b, 0)
            with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
                wa, wb, xi, eta, inside = self.locate_in_cell(a_s, b_s, P, tol)
            take = ok & inside & ~found
            wa_o = np.where(take, wa, wa_o)
            wb_o = np.where(take, wb, wb_o)
            xi_o = np.where(take, xi, xi_o)
            eta_o = np.where(take, eta, eta_o)
            found |= take
        return wa_o, wb_o, xi_o, eta_o, found

    # ----- Eq. SemiLagrProp: Q2 Lagrange interpolation -------------------
    @staticmethod
    def lagrange_q2(t):
        """1-D second-order Lagrange basis on nodes -1, 0, 1."""
        return 0.5 * t * (t - 1.0), 1.0 - t * t, 0.5 * t * (t + 1.0)

    def q2_weights(self, xi, eta):
        """N_s(xi, eta) = L_a(xi) L_b(eta), s = (a, b), a, b in {0, 1, 2}."""
        lx = self.lagrange_q2(xi)
        ly = self.lagrange_q2(eta)
        return [[lx[a] * ly[b] for b in range(3)] for a in range(3)]

    def interpolate(self, field, wa, wb, xi, eta):
        """sum_{s=1..9} field(node s) N_s(xi, eta) over the window at (wa, wb)
        (Eq. SemiLagrProp).  field has shape [..., Ni, Nj]."""
        N = self.q2_weights(xi, eta)
        out = 0.0
        for a in range(3):
            for b in range(3):
                aw, bw, _, _ = self.wrap(wa + a, wb + b)
                out = out + N[a][b] * field[..., aw, bw]
        return out

    # ----- Eq. ddx+fem: finite-element gradient at the nodes -------------
    def _d_index(self, F, axis, periodic, shift):
        """Derivative of the 1-D Q2 Lagrange interpolant through a node and its
        two neighbours along one index direction, at the node (reading R18):
        (F[+1] - F[-1]) / 2 inside, (-3 F0 + 4 F1 - F2)/2 and
        (3 F[N-1] - 4 F[N-2] + F[N-3])/2 on non-periodic ends."""
        n = F.shape[axis]
        Fm = np.moveaxis(F, axis, 0)
        d = np.empty_like(Fm)
        if periodic:
            up = np.roll(Fm, -1, axis=0)
            dn = np.roll(Fm, 1, axis=0)
            if shift is not None:
                up = up.copy()
                dn = dn.copy()
                up[n - 1] = up[n - 1] + shift
                dn[0] = dn[0] - shift
            d = 0.5 * (up - dn)
        else:
            d[1:n - 1] = 0.5 * (Fm[2:] - Fm[:n - 2])
            d[0] = 0.5 * (-3.0 * Fm[0] + 4.0 * Fm[1] - Fm[2])
            d[n - 1] = 0.5 * (3.0 * Fm[n - 1] - 4.0 * Fm[n - 2] + Fm[n - 3])
        return np.moveaxis(d, 0, axis)

    def metrics(self):
        """x_xi, y_xi, x_eta, y_eta at every node (same stencil as the field)."""
        Xx = self.X[..., 0]
        Xy = self.X[..., 1]
        x_xi = self._d_index(Xx, 0, self.periodic_i, self.shift_i[0])
        y_xi = self._d_index(Xy, 0, self.periodic_i, self.shift_i[1])
        x_eta = self._d_index(Xx, 1, self.periodic_j, self.shift_j[0])
        y_eta = self._d_index(Xy, 1, self.periodic_j, self.shift_j[1])
        return x_xi, y_xi, x_eta, y_eta

    def grad_X(self, F):
        """d_X F = J^{-1} sum_s F_s d_xi N_s with
        J^{-1} = (1/det J) [[y_eta, -y_xi], [-x_eta, x_xi]] (Eq. ddx+fem).
        F has shape [..., Ni, Nj]; returns (dF/dX, dF/dY)."""
        x_xi, y_xi, x_eta, y_eta = self.metrics()
        F_xi = self._d_index(F, F.ndim - 2, self.periodic_i, None)
        F_eta = self._d_index(F, F.ndim - 1, self.periodic_j, None)
        det = x_xi * y_eta - y_xi * x_eta
        dX = (y_eta * F_xi - y_xi * F_eta) / det
        dY = (-x_eta * F_xi + x_xi * F_eta) / det
        return dX, dY


def ogrid_mesh(r, e, centre=(0.0, 0.0)):
    """Node coordinates X[i, j] = centre + r[i] e[j]; periodic in j."""
    r = np.asarray(r, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    X = np.empty((r.size, e.shape[0], 2))
    X[..., 0] = centre[0] + r[:, None] * e[None, :, 0]
    X[..., 1] = centre[1] + r[:, None] * e[None, :, 1]
    return Q2Mesh(X, periodic_i=False, periodic_j=True)


def periodic_box_mesh(ni, nj, lx, ly, skew=0.0):
    """Doubly periodic box: X[i, j] = (i lx/ni + skew j ly/nj, j ly/nj), an
    affine mesh (parallelograms when skew != 0)."""
    hx = lx / ni
    hy = ly / nj
    i = np.arange(ni)[:, None]
    j = np.arange(nj)[None, :]
    X = np.empty((ni, nj, 2))
    X[..., 0] = i * hx + skew * j * hy
    X[..., 1] = j * hy + 0.0 * i
    return Q2Mesh(X, periodic_i=True, periodic_j=True, shift_i=(lx, 0.0),
                  shift_j=(skew * ly, ly))


class CGridMesh(Q2Mesh):
    """C-grid with a wake cut (the airfoil topology of Sec. IV D; readings
    R28-R31).  Row 0 runs counterclockwise around the bodies: cut segments
    (parts of row 0 that lie on cut lines in the fluid) and wall chains.  With
    one wall (n_cut given) row 0 is the upper side of the cut from the outlet
    to the body (j < jc), the wall from its rear point over the upper surface
    and the front back to the rear point (jc <= j <= Nj-1-jc), then the lower
    side of the cut; with several bodies in tandem (walls given: inclusive
    column ranges of the wall chains) the cut also runs along the gaps
    between the bodies, and a downstream body's wall is split into an upper
    and a lower chain.  Row 0 is palindromic: its cut nodes j and Nj-1-j are
    one point, and so are the ends of the wall chains that border the cut
    (the junctions).  Rows grow away from row 0; columns 0 and Nj-1 are
    outlet boundaries (not periodic).  Across the cut the mesh continues below
    row 0 as its mirror: node (-k, c) is node (k, Nj-1-c).  A cell below row 0
    is the mirror of a cell of the other side, and so is its element: all
    nine nodes of a window that starts below row 0, its row 0 included, are
    the mirrored ones."""

    def __init__(self, X, n_cut=None, walls=None, wall_body=None):
        super().__init__(X, periodic_i=False, periodic_j=False)
        Nj = self.Nj
        if Nj % 2 == 0:
            raise ValueError("a C-grid needs an odd node count along the C")
        if walls is None:
            if n_cut is None or n_cut < 2 or n_cut % 2 or 2 * n_cut >= Nj - 1:
                raise ValueError("n_cut must be even, >= 2 and leave a wall of at least 3 nodes")
            walls = [(n_cut, Nj - 1 - n_cut)]
        self.walls = [(int(a), int(b)) for a, b in walls]
        # the body each chain belongs to (reading R32: independent bodies)
        self.wall_body = [0] * len(self.walls) if wall_body is None else [int(b) for b in wall_body]
        if len(self.wall_body) != len(self.walls):
            raise ValueError("one body index per wall chain")
        wall = np.zeros(Nj, dtype=bool)
        for a, b in self.walls:
            if a < 1 or b > Nj - 2 or a % 2 or b % 2 or b - a < 2:
                raise ValueError("wall chains must run between even columns inside the outlets")
            if np.any(wall[a:b + 1]):
                raise ValueError("wall chains overlap")
            wall[a:b + 1] = True
        if not np.array_equal(wall, wall[::-1]):
            raise ValueError("the cut and the wall chains must be symmetric in j -> Nj-1-j")
        self.wall_mask = wall
        cut = ~wall
        jj = np.arange(Nj)
        nb_cut = np.zeros(Nj, dtype=bool)
        nb_cut[1:] |= cut[:-1]
        nb_cut[:-1] |= cut[1:]
        self.junction = wall & nb_cut
        # one wall: jc is the first copy of the rear point
        self.jc = self.walls[0][0] if len(self.walls) == 1 else None
        scale = float(np.max(np.abs(self.X)))
        for j in np.nonzero(cut | self.junction)[0]:
            if np.max(np.abs(self.X[0, j] - self.X[0, Nj - 1 - j])) > 1e-12 * scale:
                raise ValueError("row-0 nodes j and Nj-1-j must coincide along the cut")
        # a junction's one-sided derivative along j points to its cut neighbour
        self.junction_dir = np.zeros(Nj, dtype=np.int64)
        for j in np.nonzero(self.junction)[0]:
            self.junction_dir[j] = -1 if (j > 0 and cut[j - 1]) else 1

    # ----- node sets ------------------------------------------------------
    def cut_columns(self):
        return ~self.wall_mask

    def wall_columns(self):
        return self.wall_mask.copy()

    def duplicate_columns(self):
        """Row-0 columns whose node is a second copy of node (0, Nj-1-j): the
        cut and junction columns past the middle of row 0."""
        return (self.cut_columns() | self.junction) & (np.arange(self.Nj) > (self.Nj - 1) // 2)

    # ----- window nodes through the cut ------------------------------------
    def window_node(self, wa, wb, a, b):
        """Physical node of entry (a, b) of the window that starts at (wa, wb)."""
        i = np.asarray(wa) + a
        j = np.asarray(wb) + b
        ghost = np.asarray(wa) < 0
        return np.where(ghost, -i, i), np.where(ghost, self.Nj - 1 - j, j)

    def valid_cell(self, a, b):
        return (a >= -1) & (a <= self.Ni - 2) & (b >= 0) & (b <= self.Nj - 2)

    def locate_in_cell(self, a, b, P, tol=XI_TOL):
        wa, wb = self.window_of_cell(a, b)
        corner = {}
        for ca, cb in ((0, 0), (2, 0), (0, 2), (2, 2)):
            ii, jj = self.window_node(wa, wb, ca, cb)
            corner[ca, cb] = self.X[ii, jj]
        xi, eta = self.bilinear_inverse(corner[0, 0], corner[2, 0], corner[0, 2], corner[2, 2], P)
        la = a - wa
        lb = b - wb
        inside = ((xi >= la - 1 - tol) & (xi <= la + tol)
                  & (eta >= lb - 1 - tol) & (eta <= lb + tol))
        inside &= np.isfinite(xi) & np.isfinite(eta)
        return wa, wb, xi, eta, inside

    def interpolate(self, field, wa, wb, xi, eta):
        N = self.q2_weights(xi, eta)
        out = 0.0
        for a in range(3):
            for b in range(3):
                ii, jj = self.window_node(wa, wb, a, b)
                out = out + N[a][b] * field[..., ii, jj]
        return out

    # ----- gradients: central across the cut --------------------------------
    def _d_rows(self, F):
        """Derivative along i (reading R18) with the cut: at the row-0 cut
        nodes and at the junctions (both copies), the central difference with
        the mirrored row below, (F(1, j) - F(1, Nj-1-j)) / 2; one-sided on the
        rest of the wall (reading R30)."""
        d = self._d_index(F, F.ndim - 2, False, None)
        Nj = self.Nj
        c = np.nonzero(self.cut_columns() | self.junction)[0]
        d[..., 0, c] = 0.5 * (F[..., 1, c] - F[..., 1, Nj - 1 - c])
        return d

    def _d_cols(self, F):
        """Derivative along j: central, one-sided on the outlet columns; at a
        junction (reading R30) one-sided along the cut, the nodes both copies
        share: backward where the cut lies before it, forward where after."""
        d = self._d_index(F, F.ndim - 1, False, None)
        for k in np.nonzero(self.junction)[0]:
            if self.junction_dir[k] < 0:
                d[..., 0, k] = 0.5 * (3.0 * F[..., 0, k] - 4.0 * F[..., 0, k - 1] + F[..., 0, k - 2])
            else:
                d[..., 0, k] = 0.5 * (-3.0 * F[..., 0, k] + 4.0 * F[..., 0, k + 1] - F[..., 0, k + 2])
        return d

    def metrics(self):
        Xx = self.X[..., 0]
        Xy = self.X[..., 1]
        return self._d_rows(Xx), self._d_rows(Xy), self._d_cols(Xx), self._d_cols(Xy)

    def grad_X(self, F):
        x_xi, y_xi, x_eta, y_eta = self.metrics()
        F_xi = self._d_rows(F)
        F_eta = self._d_cols(F)
        det = x_xi * y_eta - y_xi * x_eta
        dX = (y_eta * F_xi - y_xi * F_eta) / det
        dY = (-x_eta * F_xi + x_xi * F_eta) / det
        return dX, dY
