"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the method. It only produces the geometry of
the body-fitted meshes (node coordinates as 1-D tables) and the seeded initial
macroscopic fields. Both implementations receive these arrays as inputs.

Mesh shape (stand-in for the paper's unstructured second-order FE meshes,
Sec. IV A, Sec. IV C): a structured O-grid around a circular cylinder.
Node (i, j) sits at  X = centre + r[i] * e[j],  i radial (i = 0 on the wall),
j angular (periodic).  Second-order elements are the 3x3-node windows whose
corners have even indices.  The mesh is subparametric: odd-index radii are
the midpoints of their even neighbours and odd-index direction vectors are the
averages of their even neighbours, so every element is the bilinear image of
the reference square and its 9 nodes sit at the bilinear positions of
xi, eta in {-1, 0, 1}.  With an even number of radial nodes the last three
radial spacings are equal (the last window overlaps its neighbour by one row).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def ogrid_radii(nr: int, radius: float, r_far: float, dr0: float) -> np.ndarray:
    """Radial node table: element widths grow geometrically from 2*dr0 at the
    wall so that the last node lands on r_far."""
    if nr < 5:
        raise ValueError("nr must be >= 5")
    n_even = (nr - 1) // 2 + 1 if nr % 2 == 1 else (nr - 2) // 2 + 1
    n_elem = n_even - 1

    def last_radius(q: float) -> float:
        with np.errstate(over="ignore"):   # trial growth factors of the bisection may overflow
            w = 2.0 * dr0 * q ** np.arange(n_elem)
        r_even = radius + np.concatenate([[0.0], np.cumsum(w)])
        if nr % 2 == 1:
            return r_even[-1]
        return r_even[-1] + 0.5 * w[-1]

    lo, hi = 1.0, 2.0
    if last_radius(lo) > r_far:
        raise ValueError("r_far too small for dr0 and nr")
    while last_radius(hi) < r_far:
        hi *= 1.5
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if last_radius(mid) < r_far:
            lo = mid
        else:
            hi = mid
    q = 0.5 * (lo + hi)
    w = 2.0 * dr0 * q ** np.arange(n_elem)
    r_even = radius + np.concatenate([[0.0], np.cumsum(w)])
    r = np.empty(nr)
    r[0:2 * n_even - 1:2] = r_even
    r[1:2 * n_even - 2:2] = 0.5 * (r_even[:-1] + r_even[1:])
    if nr % 2 == 0:
        r[nr - 1] = r[nr - 2] + (r[nr - 2] - r[nr - 3])
    return r


def ogrid_directions(ntheta: int, theta0: float = 0.0) -> np.ndarray:
    """Angular node table e[j] (shape [ntheta, 2]); even j on the unit circle,
    odd j the average of the two even neighbours (chord midpoints)."""
    if ntheta % 2 or ntheta < 4:
        raise ValueError("ntheta must be even and >= 4")
    e = np.empty((ntheta, 2))
    th = theta0 + 2.0 * np.pi * np.arange(0, ntheta, 2) / ntheta
    e[0::2, 0] = np.cos(th)
    e[0::2, 1] = np.sin(th)
    nxt = np.roll(e[0::2], -1, axis=0)
    e[1::2] = 0.5 * (e[0::2] + nxt)
    return e


@dataclass
class BodySpec:
    """Rigid body on a spring (Sec. III, Sec. IV).  dof: 0 fixed,
    1 transverse spring-mass(-damper), 2 pitch-plunge."""
    dof: int = 0
    xc: float = 0.0          # centre of the blend region (undeformed)
    yc: float = 0.0
    xp: float = 0.0          # reference point: cylinder centre / elastic axis
    yp: float = 0.0
    r_in: float = 0.75       # rigid-zone radius, measured from (xc, yc)
    r_out: float = 2.5       # outer radius of the blended zone
    length: float = 1.0      # D for cylinders, chord 2b for airfoils
    m_star: float = 10.0
    v_r: float = 5.0
    zeta: float = 0.0
    x_alpha: float = 0.0
    r_alpha: float = 1.0
    wh_wa: float = 1.0
    pitch_amp: float = 0.0       # forced pitching amplitude [rad] (pitch-plunge)
    forced_periods: float = 0.0  # duration of the forcing in uncoupled pitch periods


@dataclass
class FlowSpec:
    ma: float = 0.2
    re: float = 100.0
    t_inf: float = 1.0 / 3.0
    gamma: float = 1.4
    pr: float = 0.71
    rho_inf: float = 1.0
    dt: float = 0.0
    length: float = 1.0

    @property
    def u_inf(self) -> float:
        return self.ma * math.sqrt(self.gamma * self.t_inf)

    @property
    def mu(self) -> float:
        return self.rho_inf * self.u_inf * self.length / self.re


@dataclass
class CylinderCase:
    nr: int
    ntheta: int
    r: np.ndarray
    e: np.ndarray
    centre: tuple
    flow: FlowSpec
    bodies: list = field(default_factory=list)
    steps: int = 0
    name: str = ""

    @property
    def nodes(self) -> int:
        return self.nr * self.ntheta


def cylinder_case(nr: int, ntheta: int, *, radius: float = 0.5, r_far: float = 20.0,
                  ma: float = 0.2, re: float = 100.0, t_inf: float = 1.0 / 3.0,
                  gamma: float = 1.4, pr: float = 0.71, body: BodySpec | None = None,
                  steps: int = 0, name: str = "") -> CylinderCase:
    """O-grid around a cylinder of diameter 2*radius.  First radial spacing
    equals the wall arc spacing; the time step is a third of it (the constant
    near-wall CFL of the paper's cases, Sec. IV)."""
    dr0 = 2.0 * np.pi * radius / ntheta
    r = ogrid_radii(nr, radius, r_far, dr0)
    e = ogrid_directions(ntheta)
    flow = FlowSpec(ma=ma, re=re, t_inf=t_inf, gamma=gamma, pr=pr,
                    dt=dr0 / 3.0, length=2.0 * radius)
    b = body if body is not None else BodySpec(dof=0)
    return CylinderCase(nr=nr, ntheta=ntheta, r=r, e=e, centre=(0.0, 0.0), flow=flow,
                        bodies=[b], steps=steps, name=name)


# ----- general (non-separable) O-grids given by node coordinates ----------

def radial_fractions(nr: int, first: float) -> np.ndarray:
    """Radial parameter t_i in [0, 1] of an O-grid ring (t_0 = 0 at the
    wall, t_{nr-1} = 1 at the far field): element widths grow geometrically
    from 2*first, odd rows at the midpoints (subparametric; for even nr the
    last three spacings equal)."""
    return ogrid_radii(nr, 0.0, 1.0, first)


def closed_curve_midpoints(P: np.ndarray) -> np.ndarray:
    """Points of a closed curve at the even indices; odd indices replaced by
    the midpoints of their even neighbours (the straight element edges of
    the subparametric mesh)."""
    Q = np.array(P, dtype=np.float64)
    Q[1::2] = 0.5 * (Q[0::2] + np.roll(Q[0::2], -1, axis=0))
    return Q


def algebraic_ogrid(wall: np.ndarray, nr: int, r_far: float, first: float,
                    centre=(0.0, 0.0)) -> np.ndarray:
    """O-grid between a closed wall curve (wall[ntheta, 2], counter-
    clockwise, even points on the body at the curve parameter 2 pi j /
    ntheta, odd points midpoints) and the circle of radius r_far about
    'centre': X[i, j] = W_j + t_i (C_j - W_j) along straight lines, C_j the
    circle point at the same parameter angle (midpoints likewise), so the
    lines leave a smooth convex wall close to its normal.  Each 3x3 window is
    then the bilinear image of its corners.  A circular wall about 'centre'
    gives the separable O-grid."""
    W = np.asarray(wall, dtype=np.float64)
    nt = W.shape[0]
    ang = 2.0 * np.pi * np.arange(0, nt, 2) / nt
    C = np.empty_like(W)
    C[0::2, 0] = centre[0] + r_far * np.cos(ang)
    C[0::2, 1] = centre[1] + r_far * np.sin(ang)
    C = closed_curve_midpoints(C)
    t = radial_fractions(nr, first)
    X = W[None, :, :] + t[:, None, None] * (C - W)[None, :, :]
    return X


def ellipse_wall(ntheta: int, a: float, b: float, centre=(0.0, 0.0)) -> np.ndarray:
    """Elliptic body of semi-axes a (x) and b (y), wall nodes at equal
    parameter angles (odd nodes: chord midpoints)."""
    th = 2.0 * np.pi * np.arange(ntheta) / ntheta
    P = np.stack([centre[0] + a * np.cos(th), centre[1] + b * np.sin(th)], axis=1)
    return closed_curve_midpoints(P)


@dataclass
class XYCase:
    """A case on a general O-grid: node coordinates X[nr, ntheta, 2]."""
    nr: int
    ntheta: int
    X: np.ndarray
    centre: tuple
    flow: FlowSpec
    bodies: list = field(default_factory=list)
    steps: int = 0
    name: str = ""

    @property
    def nodes(self) -> int:
        return self.nr * self.ntheta


def xy_case(wall: np.ndarray, nr: int, *, r_far: float = 8.0, centre=(0.0, 0.0),
            length: float = 1.0, ma: float = 0.2, re: float = 100.0, t_inf: float = 1.0 / 3.0,
            gamma: float = 1.4, pr: float = 0.71, body: BodySpec | None = None, steps: int = 0,
            name: str = "") -> XYCase:
    """General O-grid case: first radial spacing equal to the smallest wall
    edge spacing, time step a third of it (the constant near-wall CFL of the
    cylinder cases)."""
    W = np.asarray(wall, dtype=np.float64)
    d = np.hypot(*(np.roll(W, -1, axis=0) - W).T)
    first = float(d.min())
    span = float(np.min(np.hypot(W[:, 0] - centre[0], W[:, 1] - centre[1])))
    X = algebraic_ogrid(W, nr, r_far, first / max(r_far - span, 1e-12), centre)
    flow = FlowSpec(ma=ma, re=re, t_inf=t_inf, gamma=gamma, pr=pr, dt=first / 3.0, length=length)
    b = body if body is not None else BodySpec(dof=0)
    return XYCase(nr=nr, ntheta=W.shape[0], X=X, centre=tuple(centre), flow=flow, bodies=[b],
                  steps=steps, name=name)


@dataclass
class CGridCase:
    """A case on a C-grid: node coordinates X[nr, nt, 2] (nt odd), the first
    n_cut row-0 nodes on each side of the wall lying on the wake cut."""
    nr: int
    ntheta: int
    n_cut: int
    X: np.ndarray
    centre: tuple
    flow: FlowSpec
    bodies: list = field(default_factory=list)
    steps: int = 0
    name: str = ""

    @property
    def nodes(self) -> int:
        return self.nr * self.ntheta


def naca4_thickness(x: np.ndarray, t: float) -> np.ndarray:
    """Half thickness of a symmetric NACA 4-digit section of chord 1 and
    thickness ratio t at chord fraction x (the public formula, closed
    trailing edge: last coefficient -0.1036)."""
    return 5.0 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2 + 0.2843 * x ** 3 - 0.1036 * x ** 4)


def naca_wall_chain(n_wall: int, t: float = 0.12) -> np.ndarray:
    """Open wall chain of a symmetric NACA section of chord 1 centred at the
    origin, counterclockwise from the trailing edge (0.5, 0) over the upper
    surface and the leading edge back to the trailing edge: even nodes at
    chord fractions x = (1 + cos theta)/2, theta = 2 pi m / (n_wall - 1)
    (clustered at both edges), odd nodes chord midpoints."""
    th = 2.0 * np.pi * np.arange(n_wall) / (n_wall - 1)
    xc = 0.5 * (1.0 + np.cos(th))
    y = naca4_thickness(xc, t) * np.where(th <= np.pi, 1.0, -1.0)
    W = np.stack([xc - 0.5, y], axis=1)
    W[1::2] = 0.5 * (W[0:-1:2] + W[2::2])
    W[0] = (0.5, 0.0)
    W[-1] = (0.5, 0.0)
    return W


def cgrid_ellipse(n_wall: int, n_cut: int, nr: int, a: float, b: float, *, r_far: float = 8.0,
                  wake: float = 6.0, wall: np.ndarray | None = None):
    """C-grid around an elliptic section (semi-axes a along x, b along y,
    centred at the origin) with a straight wake cut along y = 0 from the rear
    point (a, 0) to x = a + wake.  Row 0, counterclockwise: the upper side of
    the cut from the outlet to the rear point (j < n_cut), the wall (n_wall
    nodes, odd, both ends at the rear point; even nodes on the ellipse at
    equal parameter steps, odd nodes chord midpoints), the lower side of the
    cut back to the outlet.  The cut's element lengths grow geometrically from
    the wall's first edge.  Grid lines leave the cut at 45 degrees towards
    the outlet (to the lines y = +-r_far), so that those leaving the wall near
    the rear point are not tangent to it; the wall's lines end on the arc of
    radius sqrt(2) r_far about (a, 0) at the angle pi/4 + 3 theta/4 for the
    wall point of parameter angle theta.  X = W + t_i (C - W) along straight
    lines (subparametric)."""
    if n_wall % 2 == 0 or n_wall < 5:
        raise ValueError("n_wall must be odd and >= 5")
    if n_cut % 2 or n_cut < 4:
        raise ValueError("n_cut must be even and >= 4")
    nt = n_wall + 2 * n_cut
    th = 2.0 * np.pi * np.arange(n_wall) / (n_wall - 1)
    if wall is None:
        wall = np.stack([a * np.cos(th), b * np.sin(th)], axis=1)
        wall[1::2] = 0.5 * (wall[0:-1:2] + wall[2::2])
        wall[0] = (a, 0.0)
        wall[-1] = (a, 0.0)
    else:
        # another section with its rear point at (a, 0), given as its chain
        wall = np.asarray(wall, dtype=np.float64)
    first = float(np.hypot(*(wall[2] - wall[0])))
    s = ogrid_radii(n_cut + 1, 0.0, wake, 0.5 * first)       # s[0] = 0 at the rear point
    W = np.empty((nt, 2))
    C = np.empty((nt, 2))
    for k in range(1, n_cut + 1):
        for j, sgn in ((n_cut - k, 1.0), (nt - 1 - n_cut + k, -1.0)):
            W[j] = (a + s[k], 0.0)
            C[j] = (a + s[k] + r_far, sgn * r_far)
    W[n_cut:n_cut + n_wall] = wall
    psi = 0.25 * np.pi + 0.75 * th
    C[n_cut:n_cut + n_wall, 0] = a + np.sqrt(2.0) * r_far * np.cos(psi)
    C[n_cut:n_cut + n_wall, 1] = np.sqrt(2.0) * r_far * np.sin(psi)
    C[n_cut] = (a + r_far, r_far)
    C[n_cut + n_wall - 1] = (a + r_far, -r_far)
    cw = C[n_cut:n_cut + n_wall]
    cw[1::2] = 0.5 * (cw[0:-1:2] + cw[2::2])
    t = radial_fractions(nr, first / r_far)
    return W[None, :, :] + t[:, None, None] * (C - W)[None, :, :]


def tandem_cgrid(n_front: int, n_rear: int, n_gap: int, n_wake: int, nr: int, *, spacing: float = 4.0,
                 radius: float = 0.5, envelope: float = 1.0, r_far: float = 6.0, wake: float = 6.0,
                 n_inner: int = 8):
    """C-grid around two circular cylinders in tandem (centres (0, 0) and
    (spacing, 0)), the cut along y = 0 through the gap and the wake.  Row 0,
    upper half (then mirrored): the wake from the outlet to the rear body's
    rear point (n_wake nodes), the rear body's upper half from its rear to its
    front point (n_rear nodes, odd), the gap (n_gap nodes strictly between the
    bodies), the front body from its rear point to its front (n_front nodes;
    the middle column of row 0 is its front).  Returns X [nr, nt, 2] and the
    wall chains as inclusive column ranges: the rear body's upper and lower
    halves and the front body.  Grid lines are straight in two stages, kinked
    at row n_inner on an envelope y = +-envelope (around the front body an arc
    about its rear point): from the gap they fan from 45 degrees towards the
    rear body's front to 45 degrees away from the front body's rear (so they
    do not cross below the envelope), from the rear body's surface they reach
    the envelope above the same angle, beyond it they continue at 45 degrees
    (radially around the front), so no two lines cross and none leaves a
    wall tangentially.  Subparametric: odd rows and columns at midpoints."""
    r, L, h = radius, spacing, envelope
    if n_rear % 2 == 0 or n_wake % 2 or n_gap % 2 == 0 or n_inner % 2:
        raise ValueError("n_rear and n_gap odd, n_wake and n_inner even")
    th_f = np.pi * np.arange(n_front) / (n_front - 1)
    th_r = np.pi * np.arange(n_rear) / (n_rear - 1)
    first = r * (th_f[2] - th_f[0])
    s = ogrid_radii(n_wake + 1, 0.0, wake, min(2.0 * first, 0.45 * wake / n_wake))
    W, E = [], []
    for x in (L + r + s[1:])[::-1]:
        W.append((x, 0.0))
        E.append((x + h, h))
    for t in th_r:
        W.append((L + r * np.cos(t), r * np.sin(t)))
        E.append((L + (r + h) * np.cos(t), h))
    for x in np.linspace(L - r, r, n_gap + 2)[1:-1]:
        f = (x - r) / (L - 2.0 * r)
        W.append((x, 0.0))
        E.append((x + h * (1.0 - 2.0 * f), h))
    for t in th_f:
        W.append((r * np.cos(t), r * np.sin(t)))
        psi = 0.25 * np.pi + 0.75 * t
        E.append((r + np.sqrt(2.0) * h * np.cos(psi), np.sqrt(2.0) * h * np.sin(psi)))
    W = np.array(W)
    E = np.array(E)
    up = W.shape[0]
    nt = 2 * up - 1
    flip = np.array([1.0, -1.0])
    Wf = np.concatenate([W, (W[:-1] * flip)[::-1]])
    Ef = np.concatenate([E, (E[:-1] * flip)[::-1]])
    C = np.empty((nt, 2))
    for j in range(nt):
        e = Ef[j]
        if abs(e[1]) >= h - 1e-12 and e[0] >= r + h - 1e-12:
            C[j] = (e[0] + (r_far - h), np.sign(e[1]) * r_far)
        else:
            d = e - np.array([r, 0.0])
            C[j] = np.array([r, 0.0]) + d / np.hypot(d[0], d[1]) * np.sqrt(2.0) * r_far
    for A in (Wf, Ef, C):
        A[1::2] = 0.5 * (A[0:-1:2] + A[2::2])
    t1 = radial_fractions(n_inner + 1, min(0.05, 0.4 / n_inner))
    t2 = radial_fractions(nr - n_inner, min(0.02, 0.4 / (nr - n_inner)))
    X = np.empty((nr, nt, 2))
    for i in range(n_inner + 1):
        X[i] = Wf + t1[i] * (Ef - Wf)
    for i in range(n_inner, nr):
        X[i] = Ef + t2[i - n_inner] * (C - Ef)
    a_r = n_wake
    b_r = n_wake + n_rear - 1
    a_f = b_r + n_gap + 1
    walls = [(a_r, b_r), (a_f, nt - 1 - a_f), (nt - 1 - b_r, nt - 1 - a_r)]
    return X, walls


def tandem_case(n_front: int, n_rear: int, n_gap: int, n_wake: int, nr: int, *, spacing: float = 4.0,
                ma: float = 0.2, re: float = 100.0, t_inf: float = 1.0 / 3.0, gamma: float = 1.4,
                pr: float = 0.71, body: BodySpec | None = None, steps: int = 0, name: str = "") -> CGridCase:
    """Two cylinders of diameter 1 in tandem on a C-grid (tandem_cgrid); the
    time step a third of the smallest row-0 spacing.  The case's n_cut is
    None; its walls give the chains."""
    X, walls = tandem_cgrid(n_front, n_rear, n_gap, n_wake, nr, spacing=spacing,
                            n_inner=min(16, max(8, 2 * (nr // 16))))
    # the smallest edge of the whole mesh (the layer between the wall and
    # the envelope can be thinner than the wall spacing)
    di = np.hypot(*(X[1:] - X[:-1]).reshape(-1, 2).T)
    dj = np.hypot(*(X[:, 1:] - X[:, :-1]).reshape(-1, 2).T)
    first = float(min(di[di > 0].min(), dj[dj > 0].min()))
    flow = FlowSpec(ma=ma, re=re, t_inf=t_inf, gamma=gamma, pr=pr, dt=first / 3.0, length=1.0)
    bd = body if body is not None else BodySpec(dof=0)
    c = CGridCase(nr=nr, ntheta=X.shape[1], n_cut=None, X=X, centre=(0.0, 0.0), flow=flow, bodies=[bd],
                  steps=steps, name=name)
    c.walls = walls
    return c


# reduced velocities of the tandem sweep (one solve each)
TANDEM_VR_SWEEP = (3.0, 4.0, 5.0, 6.0, 7.0, 8.0)
# chains of tandem_cgrid: rear body's lower half, front body, rear body's upper half
TANDEM_WALL_BODY = (1, 0, 1)


def tandem_independent_pair(v_r: float, m_star: float = 10.0) -> list:
    """The front (x = 0) and rear (x = 4) cylinders as independent 1-DOF
    transverse bodies, each with its own blended region (r_in 0.75, r_out
    1.9 about its centre: the regions of the two stay apart)."""
    return [BodySpec(dof=1, xc=x, yc=0.0, xp=x, yp=0.0, r_in=0.75, r_out=1.9, m_star=m_star, v_r=v_r,
                     zeta=0.0, length=1.0) for x in (0.0, 4.0)]


def tandem_1m_independent(v_r: float = 5.0, steps: int = 0) -> CGridCase:
    """Two cylinders 4 D apart as independent 1-DOF bodies on a 512 x 2049
    C-grid (1,049,088 nodes, three wall chains), Re 100, Ma 0.2, m* 10,
    zeta 0: the tandem workload at its full size (a sweep over
    TANDEM_VR_SWEEP runs one solve per reduced velocity)."""
    c = tandem_case(257, 257, 255, 256, 512, steps=steps,
                    name="two cylinders in tandem 4 D apart, independent 1-DOF bodies (m* 10), "
                         "C-grid 512x2049 with three wall chains, Re 100, Ma 0.2")
    c.bodies = tandem_independent_pair(v_r)
    c.wall_body = list(TANDEM_WALL_BODY)
    return c


def naca0012_flutter_case(steps: int = 0) -> CGridCase:
    """The transonic flutter workload: a NACA 0012 section (chord 1) on a
    192 x 769 C-grid (147,648 nodes, wake cut 128 nodes per side), 2-DOF
    pitch-plunge (m* 100, w_h/w_a 0.3, x_a 1.8, r_a 1.87, V_R 0.5025, elastic
    axis half a chord ahead of the leading edge), Ma 0.8, T_inf 0.2, Re 1e5,
    1 degree forced pitching for two periods then free."""
    body = BodySpec(dof=2, xp=-1.0, yp=0.0, r_in=0.6, r_out=2.0, m_star=100.0, v_r=0.5025,
                    x_alpha=1.8, r_alpha=1.87, wh_wa=0.3, length=1.0,
                    pitch_amp=math.pi / 180.0, forced_periods=2.0)
    return cgrid_case(513, 128, 192, 0.5, 0.06, r_far=10.0, wake=10.0, length=1.0, ma=0.8,
                      t_inf=0.2, re=1e5, body=body, naca=0.12, steps=steps,
                      name="NACA 0012 C-grid 192x769 (cut 128), 2-DOF, Ma 0.8, forced pitch")


def cgrid_case(n_wall: int, n_cut: int, nr: int, a: float, b: float, *, r_far: float = 8.0,
               wake: float = 6.0, length: float = 1.0, ma: float = 0.2, re: float = 100.0,
               t_inf: float = 1.0 / 3.0, gamma: float = 1.4, pr: float = 0.71,
               body: BodySpec | None = None, steps: int = 0, name: str = "",
               naca: float | None = None) -> CGridCase:
    """Elliptic section (or, with naca = t, the symmetric NACA 4-digit
    section of thickness t and chord 2a) on a C-grid (cgrid_ellipse); time
    step a third of the smallest row-0 spacing, as for the O-grid cases."""
    wall = None
    if naca is not None:
        wall = naca_wall_chain(n_wall, naca) * (2.0 * a)
    X = cgrid_ellipse(n_wall, n_cut, nr, a, b, r_far=r_far, wake=wake, wall=wall)
    d = np.hypot(*(X[0, 1:] - X[0, :-1]).T)
    first = float(d[d > 0].min())
    flow = FlowSpec(ma=ma, re=re, t_inf=t_inf, gamma=gamma, pr=pr, dt=first / 3.0, length=length)
    bd = body if body is not None else BodySpec(dof=0)
    return CGridCase(nr=nr, ntheta=X.shape[1], n_cut=n_cut, X=X, centre=(0.0, 0.0), flow=flow,
                     bodies=[bd], steps=steps, name=name)


def box_mesh(ni: int, nj: int, lx: float, ly: float, skew: float = 0.0):
    """One period of a doubly periodic box: X[i, j] = (i lx/ni + skew j ly/nj,
    j ly/nj) (a parallelogram box when skew != 0) and its period vectors
    shift_i = (lx, 0), shift_j = (skew ly, ly)."""
    i = np.arange(ni)[:, None]
    j = np.arange(nj)[None, :]
    X = np.empty((ni, nj, 2))
    X[..., 0] = i * (lx / ni) + skew * j * (ly / nj)
    X[..., 1] = j * (ly / nj) + 0.0 * i
    return X, (lx, 0.0), (skew * ly, ly)


@dataclass
class ElementList:
    """An O-grid renumbered into an unstructured element list: node
    coordinates X [N, 2], elements [Ne, 3, 3] node indices (entry (a, b) at
    reference (a - 1, b - 1)), the wall chain and the far-field chain (node
    indices in increasing angular index, counterclockwise), each node's (i,
    j) on the original grid, and perm (new index of old node i Nj + j)."""
    X: np.ndarray
    elements: np.ndarray
    wall: np.ndarray
    far: np.ndarray
    grid_ij: np.ndarray
    perm: np.ndarray
    nr: int
    nt: int

    def to_list(self, field):
        """[..., nr, nt] grid field -> [..., N] in the element list's numbering."""
        flat = np.asarray(field).reshape(np.shape(field)[:-2] + (-1,))
        out = np.empty_like(flat)
        out[..., self.perm] = flat
        return out

    def to_grid(self, field):
        """[..., N] -> [..., nr, nt]."""
        f = np.asarray(field)
        return f[..., self.perm].reshape(f.shape[:-1] + (self.nr, self.nt))


def ogrid_element_list(X, seed: int = 0, shuffle: bool = True) -> ElementList:
    """The Q2 elements of a structured O-grid X [nr, nt, 2] (nr odd, so the
    3 x 3 windows at even indices tile it; nt even, periodic), nodes and
    elements shuffled by a seeded permutation (shuffle=False keeps the grid
    order i nt + j)."""
    X = np.asarray(X, dtype=np.float64)
    nr, nt = X.shape[:2]
    if nr % 2 == 0 or nt % 2:
        raise ValueError("an O-grid of odd nr and even nt")
    rng = np.random.default_rng(seed)
    perm = rng.permutation(nr * nt) if shuffle else np.arange(nr * nt)
    old = np.arange(nr * nt).reshape(nr, nt)
    els = np.array([[[old[wa + a, (wb + b) % nt] for b in range(3)] for a in range(3)]
                    for wa in range(0, nr - 2, 2) for wb in range(0, nt, 2)], dtype=np.int64)
    if shuffle:
        els = els[rng.permutation(els.shape[0])]
    Xl = np.empty((nr * nt, 2))
    Xl[perm] = X.reshape(-1, 2)
    ij = np.empty((nr * nt, 2), dtype=np.int64)
    ii, jj = np.meshgrid(np.arange(nr), np.arange(nt), indexing="ij")
    ij[perm, 0] = ii.reshape(-1)
    ij[perm, 1] = jj.reshape(-1)
    return ElementList(X=Xl, elements=perm[els], wall=perm[old[0]], far=perm[old[nr - 1]],
                       grid_ij=ij, perm=perm, nr=nr, nt=nt)


def cgrid_element_list(X, n_cut: int, seed: int = 0, shuffle: bool = True) -> ElementList:
    """The Q2 elements of a C-grid X [nr, nt, 2] (nr and nt odd) as an
    element list with the wake cut merged: row-0 nodes j and nt-1-j are one
    node for j <= n_cut (the cut and the two ends of the wall), so the cells
    on both sides of the cut share its nodes and no mirrored rows are
    needed.  Wall chain: row 0 from n_cut around the body to nt-2-n_cut
    (counterclockwise; its end meets its start at the rear point).
    Far-field chain, counterclockwise around the domain: up the outlet column
    j = 0, along the last row, down the outlet column j = nt-1.  grid_ij is
    the first copy's (i, j) (no one-to-one grid map: R33 gradients only)."""
    X = np.asarray(X, dtype=np.float64)
    nr, nt = X.shape[:2]
    if nr % 2 == 0 or nt % 2 == 0:
        raise ValueError("a C-grid of odd nr and odd nt")
    canon = np.arange(nr * nt).reshape(nr, nt)
    for j in range(n_cut + 1):
        canon[0, nt - 1 - j] = canon[0, j]
    keep = np.unique(canon)
    rng = np.random.default_rng(seed)
    newid = np.full(nr * nt, -1, dtype=np.int64)
    newid[keep] = rng.permutation(len(keep)) if shuffle else np.arange(len(keep))
    node = newid[canon]
    els = np.array([[[node[wa + a, wb + b] for b in range(3)] for a in range(3)]
                    for wa in range(0, nr - 2, 2) for wb in range(0, nt - 2, 2)], dtype=np.int64)
    if shuffle:
        els = els[rng.permutation(els.shape[0])]
    N = len(keep)
    Xl = np.empty((N, 2))
    ij = np.empty((N, 2), dtype=np.int64)
    flat = X.reshape(-1, 2)
    for old in keep:
        Xl[newid[old]] = flat[old]
        ij[newid[old]] = divmod(int(old), nt)
    wall = node[0, n_cut:nt - 1 - n_cut]
    far = np.concatenate([node[:nr - 1, 0], node[nr - 1, :nt - 1], node[nr - 1:0:-1, nt - 1]])
    return ElementList(X=Xl, elements=els, wall=wall, far=far, grid_ij=ij, perm=newid, nr=nr, nt=nt)


def fixed_cylinder_128x64(steps: int = 1000) -> CylinderCase:
    """Fixed cylinder, 128 radial x 64 angular nodes, far field at 20 D,
    Re 100, Ma 0.2 (FP64 parity workload)."""
    return cylinder_case(128, 64, body=BodySpec(dof=0), steps=steps,
                         name="fixed cylinder O-grid 128x64, Re 100, Ma 0.2")


def viv_cylinder_512x256(steps: int = 20000, v_r: float = 5.0, m_star: float = 10.0) -> CylinderCase:
    """1-DOF transverse VIV of a cylinder (m* 10, zeta 0, V_R 5) on a
    512 x 256 O-grid deformed by the blending polynomial; Re 100, Ma 0.2."""
    b = BodySpec(dof=1, r_in=0.75, r_out=2.5, m_star=m_star, v_r=v_r, zeta=0.0)
    return cylinder_case(512, 256, body=b, steps=steps,
                         name="1-DOF VIV cylinder O-grid 512x256, m* 10, V_R 5, Re 100, Ma 0.2")


def initial_field(nr: int, ntheta: int, flow: FlowSpec, noise: float = 1e-3,
                  seed: int = 0) -> np.ndarray:
    """Uniform free stream (rho_inf, U_inf along +x, T_inf) plus seeded
    uniform velocity noise of amplitude noise*U_inf.  Shape [4, nr, ntheta]:
    rho, u_x, u_y, T."""
    rng = np.random.default_rng(seed)
    m = np.empty((4, nr, ntheta))
    m[0] = flow.rho_inf
    xi = rng.uniform(-1.0, 1.0, size=(2, nr, ntheta))
    m[1] = flow.u_inf + noise * flow.u_inf * xi[0]
    m[2] = noise * flow.u_inf * xi[1]
    m[3] = flow.t_inf
    return m


def random_populations_like(shape, seed: int, scale: float = 0.02) -> np.ndarray:
    """Seeded perturbation array used by tests to move populations off
    equilibrium."""
    rng = np.random.default_rng(seed)
    return scale * rng.uniform(-1.0, 1.0, size=shape)
