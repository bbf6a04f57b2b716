"""The oracle's coupled time step (Sec. III: weak, staggered coupling; Sec.
II: ALE semi-Lagrangian two-population LBM).

Test infrastructure only (see the package docstring).

One step n, in the order of Sec. III (fluid step, then forces, then the
structural solver, whose displacement the next fluid step uses):
  1. mesh kinematics from the current body states S and those of the previous
     step S_prev: F = dx/dX (so g = F^T), V_G = (x(S) - x(S_prev)) / dt,
     c_hat_i = F^{-1} c_i - V_G                       (Sec. II A, II D)
  2. departure points X - c_hat_i dt, their cells and reference coordinates
     (Eq. depPnt), Q2 interpolation of the post-collision populations of the
     previous step (Eq. SemiLagrProp)
  3. wall nodes: populations whose departure point lies in the body are
     replaced by Grad's approximation at the wall targets (Sec. III A)
  4. moments rho, u, T of the post-propagation state; far-field targets
  5. correction fields Y_a = d_a[(mu/p) d_a dQ_a] from the moment field
     (mu/p = (1/omega - 1/2) dt)
  6. collision (Eq. f_boltz) at every node but the far field, whose
     post-collision populations are the equilibria at its targets
  7. force and moment on the body from the wall nodes' post-propagation
     populations (Sec. III)
  8. RK4 of the body ODEs with that load held constant (Sec. III B)
At the first step S_prev = S (reading R4: x^{-1} = x^0).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import kinetics as K
from . import ale, boundary, forces, structure
from .mesh import CGridMesh, DepartureError


def body_dict(spec, flow_rho, u_inf):
    """Plain dict of a body description (any object with the BodySpec
    attribute names) plus the dimensional ODE parameters."""
    b = {k: float(getattr(spec, k)) for k in
         ("xc", "yc", "xp", "yp", "r_in", "r_out", "length", "m_star", "v_r", "zeta",
          "x_alpha", "r_alpha", "wh_wa")}
    b["dof"] = int(spec.dof)
    b["pitch_amp"] = float(getattr(spec, "pitch_amp", 0.0))
    b["forced_periods"] = float(getattr(spec, "forced_periods", 0.0))
    if b["dof"] == 1:
        b["m"], b["k"], b["c"] = structure.one_dof_parameters(
            b["m_star"], b["v_r"], b["zeta"], b["length"], flow_rho, u_inf)
    elif b["dof"] == 2:
        (b["m"], b["s_a"], b["i_a"], b["k_h"], b["k_a"]) = structure.two_dof_parameters(
            b["m_star"], b["v_r"], b["x_alpha"], b["r_alpha"], b["wh_wa"],
            0.5 * b["length"], flow_rho, u_inf)
        # forced pitching (Sec. IV D): alpha = pitch_amp sin(w_alpha t) for
        # forced_periods periods of the uncoupled pitch frequency, then free
        half = 0.5 * b["length"]
        b["w_a"] = u_inf / (b["v_r"] * half * math.sqrt(b["m_star"]))
        b["t_forced"] = b["forced_periods"] * 2.0 * math.pi / b["w_a"]
    return b


def zero_state():
    return {"h": 0.0, "alpha": 0.0, "hdot": 0.0, "adot": 0.0}


@dataclass
class StepResult:
    f_pre: np.ndarray
    g_pre: np.ndarray
    f_post: np.ndarray
    g_post: np.ndarray
    M: np.ndarray
    force: tuple
    missing: np.ndarray
    forces: list = None      # per body (C-grids with several bodies)


class Solver:
    """Coupled solver on one mesh.  walls=True: O-grid with the body wall on
    row 0 and the far field on the last row, or a C-grid (CGridMesh: the wall
    on part of row 0, the wake cut on the rest, the far field on the last row
    and the outlet columns); walls=False: no boundary rows (doubly periodic
    box)."""

    def __init__(self, mesh, *, gamma, Pr, mu, dt, rho_inf, u_inf, T_inf, bodies, M0,
                 walls=True):
        self.mesh = mesh
        self.gamma = float(gamma)
        self.Cv = 1.0 / (self.gamma - 1.0)
        self.Pr = float(Pr)
        self.mu = float(mu)
        self.dt = float(dt)
        self.rho_inf = float(rho_inf)
        self.u_inf = np.asarray(u_inf, dtype=np.float64)
        self.T_inf = float(T_inf)
        self.bodies = list(bodies)
        self.walls = walls
        M0 = np.asarray(M0, dtype=np.float64)
        if isinstance(mesh, CGridMesh):
            # reading R28: the two copies of a cut node start from the first
            # copy's values
            M0 = M0.copy()
            dup = np.nonzero(mesh.duplicate_columns())[0]
            M0[:, 0, dup] = M0[:, 0, mesh.Nj - 1 - dup]
        self.f = K.f_eq(M0[0], M0[1], M0[2], M0[3])
        self.g = K.g_eq(M0[0], M0[1], M0[2], M0[3], self.Cv)
        self.M_prev = M0.copy()
        self.S = [zero_state() for _ in self.bodies]
        self.S_prev = [dict(s) for s in self.S]
        self.n = 0
        self.cgrid = isinstance(mesh, CGridMesh)
        if walls:
            self.n0 = boundary.wall_normals_cgrid(mesh) if self.cgrid else boundary.wall_normals(mesh)
        # the O-grid step's wall-load sum (step 7): forces.wall_force unless a
        # caller that holds only part of the wall (a rank of a split mesh)
        # supplies the same sum assembled from every part
        self.load_reduction = None

    @classmethod
    def from_case(cls, mesh, case, M0):
        """Build from a case object (CylinderCase-like: flow, bodies)."""
        fl = case.flow
        u_inf = fl.ma * math.sqrt(fl.gamma * fl.t_inf)
        bodies = [body_dict(b, fl.rho_inf, u_inf) for b in case.bodies]
        mu = fl.rho_inf * u_inf * fl.length / fl.re
        return cls(mesh, gamma=fl.gamma, Pr=fl.pr, mu=mu, dt=fl.dt, rho_inf=fl.rho_inf,
                   u_inf=(u_inf, 0.0), T_inf=fl.t_inf, bodies=bodies, M0=M0)

    # ------------------------------------------------------------------
    def _physical_grad(self, F, field):
        dX, dY = self.mesh.grad_X(field)
        return ale.physical_gradient(F, dX, dY)

    def step(self) -> StepResult:
        if self.cgrid:
            return self._step_cgrid()
        mesh, dt, Cv = self.mesh, self.dt, self.Cv
        X = mesh.X
        Ni, Nj = mesh.Ni, mesh.Nj
        last = Ni - 1
        # 1. kinematics
        F = ale.deformation_gradient(X, self.bodies, self.S)
        VG = ale.mesh_velocity(X, self.bodies, self.S, self.S_prev, dt)
        chat = ale.transformed_velocities(F, VG)
        # 2. departure points and interpolation
        nrows = last if self.walls else Ni
        ii, jj = np.meshgrid(np.arange(nrows), np.arange(Nj), indexing="ij")
        f_pre = np.zeros((9, Ni, Nj))
        g_pre = np.zeros((9, Ni, Nj))
        missing = np.zeros((9, Ni, Nj), dtype=bool)
        if self.walls:
            missing[:, 0, :] = boundary.missing_mask(chat[:, 0], self.n0)
        for k in range(9):
            P = X[:nrows] - dt * chat[k, :nrows]
            wa, wb, xi, eta, found = mesh.locate(P, ii, jj)
            need = ~missing[k, :nrows]
            if np.any(need & ~found):
                bad = np.argwhere(need & ~found)[0]
                raise DepartureError(f"departure point of direction {k} at node "
                                     f"{tuple(bad)} is not in an adjacent cell")
            f_pre[k, :nrows] = np.where(need, mesh.interpolate(self.f[k], wa, wb, xi, eta), 0.0)
            g_pre[k, :nrows] = np.where(need, mesh.interpolate(self.g[k], wa, wb, xi, eta), 0.0)
        # 3. wall: Grad's approximation at the targets
        if self.walls:
            rho_b, T_b, grads = boundary.wall_targets(mesh, self.M_prev, self.n0, dt, F[0])
            uw = VG[0]
            fm, gm = boundary.grad_populations(rho_b, uw[:, 0], uw[:, 1], T_b, grads, Cv,
                                               self.mu, dt, self.Pr)
            f_pre[:, 0] = np.where(missing[:, 0], fm, f_pre[:, 0])
            g_pre[:, 0] = np.where(missing[:, 0], gm, g_pre[:, 0])
        # 4. moments and far-field targets
        M = np.empty((4, Ni, Nj))
        rho, ux, uy, E, T = K.moments(f_pre[:, :nrows], g_pre[:, :nrows], Cv)
        M[0, :nrows], M[1, :nrows], M[2, :nrows], M[3, :nrows] = rho, ux, uy, T
        if self.walls:
            tr, tux, tuy, tT, _ = boundary.far_field_targets(mesh, self.M_prev, self.u_inf,
                                                             self.T_inf, dt)
            M[0, last], M[1, last], M[2, last], M[3, last] = tr, tux, tuy, tT
        # 5. correction fields
        dqx, dqy = K.delta_q(M[0], M[1], M[2], M[3])
        mu_p = self.mu / (M[0] * M[3])
        ddx, _ = self._physical_grad(F, dqx)
        _, ddy = self._physical_grad(F, dqy)
        Dx = mu_p * ddx
        Dy = mu_p * ddy
        Yx, _ = self._physical_grad(F, Dx)
        _, Yy = self._physical_grad(F, Dy)
        # 6. collision
        f_post = np.empty_like(f_pre)
        g_post = np.empty_like(g_pre)
        f_post[:, :nrows], g_post[:, :nrows] = K.collide(
            f_pre[:, :nrows], g_pre[:, :nrows], Yx[:nrows], Yy[:nrows], self.mu, dt, Cv,
            self.Pr)
        if self.walls:
            f_post[:, last] = K.f_eq(M[0, last], M[1, last], M[2, last], M[3, last])
            g_post[:, last] = K.g_eq(M[0, last], M[1, last], M[2, last], M[3, last], Cv)
        # 7. force and moment on body 0 (the wall of the O-grid)
        force = (0.0, 0.0, 0.0)
        if self.walls and self.bodies:
            b, st = self.bodies[0], self.S[0]
            sxx, sxy, syy = forces.node_stress(f_pre[:, 0], g_pre[:, 0], Cv, self.mu, dt,
                                               self.Pr)
            x_wall = ale.mesh_position(X[0], self.bodies, self.S)
            x_ref = np.array([b["xp"], b["yp"] + st["h"]])
            force = (self.load_reduction or forces.wall_force)(x_wall, sxx, sxy, syy, x_ref)
        # 8. structural update
        new_S = []
        for b, st in zip(self.bodies, self.S):
            s = dict(st)
            if b["dof"] == 1:
                s["h"], s["hdot"] = structure.advance_one_dof(
                    st["h"], st["hdot"], force[1], b["m"], b["k"], b["c"], dt)
            elif b["dof"] == 2 and (self.n + 1) * dt <= b["t_forced"]:
                # a step that ends within the forcing interval: pitch prescribed
                s["h"], s["alpha"], s["hdot"], s["adot"] = structure.advance_plunge_forced_pitch(
                    st["h"], st["hdot"], force[1], b["m"], b["s_a"], b["k_h"], b["pitch_amp"],
                    b["w_a"], self.n, dt)
            elif b["dof"] == 2:
                s["h"], s["alpha"], s["hdot"], s["adot"] = structure.advance_two_dof(
                    st["h"], st["alpha"], st["hdot"], st["adot"], force[1], force[2],
                    b["m"], b["s_a"], b["i_a"], b["k_h"], b["k_a"], dt)
            new_S.append(s)
        self.S_prev = [dict(s) for s in self.S]
        self.S = new_S
        self.f, self.g = f_post, g_post
        self.M_prev = M
        self.n += 1
        return StepResult(f_pre, g_pre, f_post, g_post, M, force, missing)

    def _advance_bodies(self, forces):
        """Step 8 (RK4 of every body with its load held, Sec. III B)."""
        dt = self.dt
        new_S = []
        for b, st, force in zip(self.bodies, self.S, forces):
            s = dict(st)
            if b["dof"] == 1:
                s["h"], s["hdot"] = structure.advance_one_dof(
                    st["h"], st["hdot"], force[1], b["m"], b["k"], b["c"], dt)
            elif b["dof"] == 2 and (self.n + 1) * dt <= b["t_forced"]:
                s["h"], s["alpha"], s["hdot"], s["adot"] = structure.advance_plunge_forced_pitch(
                    st["h"], st["hdot"], force[1], b["m"], b["s_a"], b["k_h"], b["pitch_amp"],
                    b["w_a"], self.n, dt)
            elif b["dof"] == 2:
                s["h"], s["alpha"], s["hdot"], s["adot"] = structure.advance_two_dof(
                    st["h"], st["alpha"], st["hdot"], st["adot"], force[1], force[2],
                    b["m"], b["s_a"], b["i_a"], b["k_h"], b["k_a"], dt)
            new_S.append(s)
        return new_S

    def _step_cgrid(self) -> StepResult:
        """One step on a C-grid: the O-grid step with the C-grid's node sets
        (readings R28-R30).  Every node but the far field is streamed, the
        row-0 cut nodes like interior nodes (their departure points may lie
        across the cut); the wall columns of row 0 take the wall treatment;
        the far field is the last row and the outlet columns.  The second
        copies of the row-0 nodes along the cut take the values of the first
        copies (j <= jc) after the propagation and after the collision."""
        mesh, dt, Cv = self.mesh, self.dt, self.Cv
        X = mesh.X
        Ni, Nj = mesh.Ni, mesh.Nj
        far = boundary.far_field_mask_cgrid(mesh)
        wall = np.zeros((Ni, Nj), dtype=bool)
        wall[0] = mesh.wall_columns()
        dup = np.nonzero(mesh.duplicate_columns())[0]
        own = Nj - 1 - dup
        # 1. kinematics
        F = ale.deformation_gradient(X, self.bodies, self.S)
        VG = ale.mesh_velocity(X, self.bodies, self.S, self.S_prev, dt)
        chat = ale.transformed_velocities(F, VG)
        # 2. departure points and interpolation at every node off the far field
        ii, jj = np.meshgrid(np.arange(Ni), np.arange(Nj), indexing="ij")
        f_pre = np.zeros((9, Ni, Nj))
        g_pre = np.zeros((9, Ni, Nj))
        missing = np.zeros((9, Ni, Nj), dtype=bool)
        missing[:, 0, :] = boundary.missing_mask(chat[:, 0], self.n0) & wall[0][None, :]
        for k in range(9):
            P = X - dt * chat[k]
            wa, wb, xi, eta, found = mesh.locate(P, ii, jj)
            need = ~far & ~missing[k]
            if np.any(need & ~found):
                bad = np.argwhere(need & ~found)[0]
                raise DepartureError(f"departure point of direction {k} at node "
                                     f"{tuple(bad)} is not in an adjacent cell")
            wa = np.where(need, wa, 0)
            wb = np.where(need, wb, 0)
            f_pre[k] = np.where(need, mesh.interpolate(self.f[k], wa, wb, xi, eta), 0.0)
            g_pre[k] = np.where(need, mesh.interpolate(self.g[k], wa, wb, xi, eta), 0.0)
        # 3. wall nodes: Grad's approximation at the targets
        rho_b, T_b, grads = boundary.wall_targets(mesh, self.M_prev, self.n0, dt, F[0])
        uw = VG[0]
        fm, gm = boundary.grad_populations(rho_b, uw[:, 0], uw[:, 1], T_b, grads, Cv,
                                           self.mu, dt, self.Pr)
        f_pre[:, 0] = np.where(missing[:, 0], fm, f_pre[:, 0])
        g_pre[:, 0] = np.where(missing[:, 0], gm, g_pre[:, 0])
        # 4. moments; far-field targets (the far-field entries of f_pre are
        # zero: their moments are replaced by the targets)
        with np.errstate(divide="ignore", invalid="ignore"):
            rho, ux, uy, E, T = K.moments(f_pre, g_pre, Cv)
        M = np.stack([rho, ux, uy, T])
        tr, tux, tuy, tT, _ = boundary.far_field_targets_cgrid(mesh, self.M_prev, self.u_inf,
                                                               self.T_inf, dt)
        for c, t in enumerate((tr, tux, tuy, tT)):
            M[c] = np.where(far, t, M[c])
        f_pre[:, 0, dup] = f_pre[:, 0, own]
        g_pre[:, 0, dup] = g_pre[:, 0, own]
        missing[:, 0, dup] = missing[:, 0, own]
        M[:, 0, dup] = M[:, 0, own]
        # 5. correction fields
        dqx, dqy = K.delta_q(M[0], M[1], M[2], M[3])
        mu_p = self.mu / (M[0] * M[3])
        ddx, _ = self._physical_grad(F, dqx)
        _, ddy = self._physical_grad(F, dqy)
        Yx, _ = self._physical_grad(F, mu_p * ddx)
        _, Yy = self._physical_grad(F, mu_p * ddy)
        # 6. collision; the far field takes the equilibria at its targets
        with np.errstate(divide="ignore", invalid="ignore"):
            f_post, g_post = K.collide(f_pre, g_pre, Yx, Yy, self.mu, dt, Cv, self.Pr)
        f_far = K.f_eq(M[0], M[1], M[2], M[3])
        g_far = K.g_eq(M[0], M[1], M[2], M[3], Cv)
        f_post = np.where(far[None], f_far, f_post)
        g_post = np.where(far[None], g_far, g_post)
        f_post[:, 0, dup] = f_post[:, 0, own]
        g_post[:, 0, dup] = g_post[:, 0, own]
        # 7. force and moment on each body: the sum over its wall chains
        # (one body holding several chains: rigidly linked bodies, reading
        # R31; several bodies: reading R32), the moment about its own
        # reference point
        per_body = []
        for k, (b, st) in enumerate(zip(self.bodies, self.S)):
            x_ref = np.array([b["xp"], b["yp"] + st["h"]])
            tot = np.zeros(3)
            for (a_, b_), owner in zip(mesh.walls, mesh.wall_body):
                if owner != k:
                    continue
                cols = np.arange(a_, b_ + 1)
                sxx, sxy, syy = forces.node_stress(f_pre[:, 0, cols], g_pre[:, 0, cols], Cv,
                                                   self.mu, dt, self.Pr)
                x_wall = ale.mesh_position(X[0, cols], self.bodies, self.S)
                tot += np.array(forces.wall_force(x_wall, sxx, sxy, syy, x_ref, closed=False))
            per_body.append(tuple(float(v) for v in tot))
        force = per_body[0] if per_body else (0.0, 0.0, 0.0)
        # 8. structural update
        new_S = self._advance_bodies(per_body)
        self.S_prev = [dict(s) for s in self.S]
        self.S = new_S
        self.f, self.g = f_post, g_post
        self.M_prev = M
        self.n += 1
        return StepResult(f_pre, g_pre, f_post, g_post, M, force, missing, per_body)

    def run(self, nsteps):
        res = None
        hist = []
        for _ in range(nsteps):
            res = self.step()
            hist.append(res.force)
        return res, np.array(hist)
