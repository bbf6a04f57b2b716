// Host-side helpers: mesh validation and derived geometry, body and flow
// parameters, device allocation of a mesh's geometry.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lbfsi_device.cuh"
#include "lbfsi_host.h"

namespace lbfsi {

namespace {

// Wall polygon of the O-grid (Sec. III): the wall edges are the straight
// element edges between even-indexed wall nodes.  For every wall node: the unit
// normal n0 out of the body (odd node: its edge's normal; even node: the
// normalised sum of its two edges' normals) and its Simpson share of the
// adjacent edges (weight*length and edge normal, up to two edges).
void wall_geometry(HostMesh& m) {
    const int nt = m.nt, ne = nt / 2;
    const std::vector<double>& X = m.xw;
    std::vector<double> en(2 * ne), ds(ne);
    for (int k = 0; k < ne; ++k) {
        const int a = 2 * k, c = (2 * k + 2) % nt;
        const double tx = X[2 * c] - X[2 * a], ty = X[2 * c + 1] - X[2 * a + 1];
        const double L = std::sqrt(tx * tx + ty * ty);
        ds[k] = L;
        en[2 * k] = ty / L;
        en[2 * k + 1] = -tx / L;
    }
    m.n0.assign(2 * nt, 0.0);
    m.wall_geo.assign(6 * nt, 0.0);
    for (int j = 0; j < nt; ++j) {
        double* g = &m.wall_geo[6 * j];
        if (j % 2) {
            const int k = j / 2;
            m.n0[2 * j] = en[2 * k];
            m.n0[2 * j + 1] = en[2 * k + 1];
            g[0] = 4.0 / 6.0 * ds[k];
            g[1] = en[2 * k];
            g[2] = en[2 * k + 1];
        } else {
            const int k2 = j / 2, k1 = (j / 2 - 1 + ne) % ne;
            const double vx = en[2 * k1] + en[2 * k2], vy = en[2 * k1 + 1] + en[2 * k2 + 1];
            const double L = std::sqrt(vx * vx + vy * vy);
            m.n0[2 * j] = vx / L;
            m.n0[2 * j + 1] = vy / L;
            g[0] = ds[k2] / 6.0;
            g[1] = en[2 * k2];
            g[2] = en[2 * k2 + 1];
            g[3] = ds[k1] / 6.0;
            g[4] = en[2 * k1];
            g[5] = en[2 * k1 + 1];
        }
    }
}

// Per-row and per-column geometry of the O-grid X = centre + r_i e_j used by
// the step kernel:
//   row i: [0] r_i, [1] 1/r'_i and [2] 1/r_i (r'_i the derivative along the
//          radial index of the quadratic through the node and its neighbours,
//          one-sided on the first and last rows, Eq. ddx+fem), then for the two
//          candidate radial cells a = i-1, a = i: [3|5] the node's xi in the
//          cell's element, [4|6] 1 / (dR/dxi) of that element.
//   col j: [0,1] e_j, [2..5] the angular factors of the inverse metric
//          (de_y, e_y, de_x, e_x) / (e x de) with de = (e_{j+1} - e_{j-1})/2, then
//          for the two candidate angular cells b = j-1, b = j: [6|10] the node's
//          eta in the element, [7,8|11,12] dE/deta of the element,
//          [9|13] (dE/deta) x e_j.
void geometry_tables(HostMesh& m) {
    const int nr = m.nr, nt = m.nt;
    const double* r = m.r.data();
    const double* e = m.e.data();
    m.rowtab.assign((size_t)nr * ROWTAB, 0.0);
    for (int i = 0; i < nr; ++i) {
        double drc;
        if (i == 0)
            drc = 0.5 * (-3.0 * r[0] + 4.0 * r[1] - r[2]);
        else if (i == nr - 1)
            drc = 0.5 * (3.0 * r[nr - 1] - 4.0 * r[nr - 2] + r[nr - 3]);
        else
            drc = 0.5 * (r[i + 1] - r[i - 1]);
        double* t = &m.rowtab[(size_t)i * ROWTAB];
        t[RT_R] = r[i];
        t[RT_IDRC] = 1.0 / drc;
        t[RT_IR] = 1.0 / r[i];
        for (int c = 0; c < 2; ++c) {
            const int a = i - 1 + c;
            if (a < 0 || a > nr - 2) continue;
            const int wa = std::min(2 * (a / 2), nr - 3);
            t[RT_XIN0 + 2 * c] = (double)(i - wa - 1);
            t[RT_IDR0 + 2 * c] = 2.0 / (r[wa + 2] - r[wa]);
        }
    }
    m.coltab.assign((size_t)nt * COLTAB, 0.0);
    auto wr = [nt](int j) { return ((j % nt) + nt) % nt; };
    for (int j = 0; j < nt; ++j) {
        const double ex = e[2 * j], ey = e[2 * j + 1];
        const int jp = wr(j + 1), jm = wr(j - 1);
        const double dex = 0.5 * (e[2 * jp] - e[2 * jm]), dey = 0.5 * (e[2 * jp + 1] - e[2 * jm + 1]);
        const double cr = ex * dey - ey * dex;
        double* t = &m.coltab[(size_t)j * COLTAB];
        t[CT_E] = ex;
        t[CT_E + 1] = ey;
        t[CT_G] = dey / cr;
        t[CT_G + 1] = ey / cr;
        t[CT_G + 2] = dex / cr;
        t[CT_G + 3] = ex / cr;
        for (int c = 0; c < 2; ++c) {
            const int b = j - 1 + c;
            const int wb = (b >= 0) ? 2 * (b / 2) : -2 * ((-b + 1) / 2);
            const int w0 = wr(wb), w2 = wr(wb + 2);
            const double dEx = 0.5 * (e[2 * w2] - e[2 * w0]), dEy = 0.5 * (e[2 * w2 + 1] - e[2 * w0 + 1]);
            double* tc = t + CT_C0 + 4 * c;
            tc[0] = (double)(j - wb - 1);
            tc[1] = dEx;
            tc[2] = dEy;
            tc[3] = dEx * ey - dEy * ex;
        }
    }
}

// Scale every (x, y) pair of v to unit length: the outward directions of
// the far field, whose outlet targets sit one time step inside along them.
void normalise_pairs(std::vector<double>& v) {
    for (size_t k = 0; k + 1 < v.size(); k += 2) {
        const double l = std::hypot(v[k], v[k + 1]);
        if (l > 0.0) {
            v[k] /= l;
            v[k + 1] /= l;
        }
    }
}

}  // namespace

void chain_geometry(const std::vector<double>& P, std::vector<double>& n0, std::vector<double>& wgeo) {
    HostMesh t;
    t.nt = (int)(P.size() / 2);
    t.xw = P;
    wall_geometry(t);
    n0 = t.n0;
    wgeo = t.wall_geo;
}

int build_host_mesh(int nr, int nt, const double* r, const double* e, double xc, double yc,
                    HostMesh& m) {
    if (nr < 5) return set_error(LBFSI_EINVAL, "nr must be >= 5");
    if (nt < 4 || nt % 2) return set_error(LBFSI_EINVAL, "ntheta must be even and >= 4");
    if (!r || !e) return set_error(LBFSI_EINVAL, "null table pointer");
    m.nr = nr;
    m.nt = nt;
    m.N = nr * nt;
    m.Nx = m.N;
    m.ntj = tiles_j(nt);
    m.xm = xc;
    m.ym = yc;
    m.r.assign(r, r + nr);
    m.e.assign(e, e + 2 * nt);
    for (int i = 1; i < nr; ++i)
        if (!(m.r[i] > m.r[i - 1])) return set_error(LBFSI_EINVAL, "radial table must increase");
    // subparametric tables: odd entries are the averages of their even
    // neighbours (and, for even nr, the clamped last window is uniform), so
    // every window is the bilinear image of the reference square
    auto near = [](double a, double b, double scale) { return std::fabs(a - b) <= 1e-12 * scale; };
    bool sub = true;
    for (int i = 1; i + 1 < nr; i += 2)
        sub = sub && near(m.r[i], 0.5 * (m.r[i - 1] + m.r[i + 1]), std::fabs(m.r[i + 1]));
    if (nr % 2 == 0)
        sub = sub && near(m.r[nr - 2], 0.5 * (m.r[nr - 3] + m.r[nr - 1]), std::fabs(m.r[nr - 1]));
    for (int j = 1; j < nt; j += 2)
        for (int c = 0; c < 2; ++c)
            sub = sub && near(m.e[2 * j + c], 0.5 * (m.e[2 * (j - 1) + c] + m.e[2 * ((j + 1) % nt) + c]), 1.0);
    if (!sub)
        return set_error(LBFSI_EINVAL,
                         "r and e tables must be subparametric (odd entries = mean of even neighbours)");
    m.xw.assign(2 * (size_t)nt, 0.0);
    m.fardir.assign(2 * (size_t)nt, 0.0);
    for (int j = 0; j < nt; ++j)
        for (int c = 0; c < 2; ++c) {
            m.xw[2 * j + c] = (c ? m.ym : m.xm) + m.r[0] * m.e[2 * j + c];
            m.fardir[2 * j + c] = (m.r[nr - 1] - m.r[nr - 2]) * m.e[2 * j + c];
        }
    normalise_pairs(m.fardir);
    wall_geometry(m);
    geometry_tables(m);
    return LBFSI_OK;
}

int build_host_mesh_xy(int nr, int nt, const double* X, double xc, double yc, HostMesh& m) {
    if (nr < 5) return set_error(LBFSI_EINVAL, "nr must be >= 5");
    if (nt < 4 || nt % 2) return set_error(LBFSI_EINVAL, "ntheta must be even and >= 4");
    if (!X) return set_error(LBFSI_EINVAL, "null coordinate pointer");
    m.general = true;
    m.nr = nr;
    m.nt = nt;
    m.N = nr * nt;
    m.Nx = m.N;
    m.ntj = tiles_j(nt);
    m.xm = xc;
    m.ym = yc;
    m.X.assign(X, X + 2 * (size_t)m.N);
    double scale = 0.0;
    for (double v : m.X) {
        if (!std::isfinite(v)) return set_error(LBFSI_EINVAL, "node coordinates must be finite");
        scale = std::max(scale, std::fabs(v));
    }
    auto P = [&](int i, int j, int c) { return m.X[2 * ((size_t)i * nt + ((j % nt) + nt) % nt) + c]; };
    // subparametric: every window is the bilinear image of its corner nodes
    auto check_window = [&](int wa, int wb) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const double xi = a - 1.0, et = b - 1.0;
                for (int c = 0; c < 2; ++c) {
                    const double v = 0.25 * ((1 - xi) * (1 - et) * P(wa, wb, c) + (1 + xi) * (1 - et) * P(wa + 2, wb, c) +
                                             (1 - xi) * (1 + et) * P(wa, wb + 2, c) + (1 + xi) * (1 + et) * P(wa + 2, wb + 2, c));
                    if (std::fabs(v - P(wa + a, wb + b, c)) > 1e-12 * scale) return false;
                }
            }
        return true;
    };
    for (int wa = 0; wa + 2 < nr; wa += 2)
        for (int wb = 0; wb < nt; wb += 2)
            if (!check_window(wa, wb) || (nr % 2 == 0 && !check_window(nr - 3, wb)))
                return set_error(LBFSI_EINVAL, "node coordinates must be subparametric "
                                               "(every window the bilinear image of its corners)");
    m.xw.assign(2 * (size_t)nt, 0.0);
    m.fardir.assign(2 * (size_t)nt, 0.0);
    for (int j = 0; j < nt; ++j)
        for (int c = 0; c < 2; ++c) {
            m.xw[2 * j + c] = P(0, j, c);
            m.fardir[2 * j + c] = P(nr - 1, j, c) - P(nr - 2, j, c);
        }
    normalise_pairs(m.fardir);
    wall_geometry(m);
    // inverse metric at the nodes: derivatives of X along the index
    // directions with the field's stencil (central; one-sided on the wall
    // and far-field rows; periodic in j), then (y_j, -y_i, -x_j, x_i) / det
    m.jinv.assign(4 * (size_t)m.N, 0.0);
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nt; ++j) {
            double di[2], dj[2];
            for (int c = 0; c < 2; ++c) {
                if (i == 0)
                    di[c] = 0.5 * (-3.0 * P(0, j, c) + 4.0 * P(1, j, c) - P(2, j, c));
                else if (i == nr - 1)
                    di[c] = 0.5 * (3.0 * P(nr - 1, j, c) - 4.0 * P(nr - 2, j, c) + P(nr - 3, j, c));
                else
                    di[c] = 0.5 * (P(i + 1, j, c) - P(i - 1, j, c));
                dj[c] = 0.5 * (P(i, j + 1, c) - P(i, j - 1, c));
            }
            const double det = di[0] * dj[1] - di[1] * dj[0];
            if (!(det > 0.0))
                return set_error(LBFSI_EINVAL, "mesh not positively oriented (index-to-space Jacobian <= 0)");
            double* t = &m.jinv[4 * ((size_t)i * nt + j)];
            t[0] = dj[1] / det;
            t[1] = -di[1] / det;
            t[2] = -dj[0] / det;
            t[3] = di[0] / det;
        }
    // element coefficients per cell
    m.cellc.assign((size_t)(nr - 1) * nt * CELLC, 0.0);
    for (int a = 0; a < nr - 1; ++a)
        for (int b = 0; b < nt; ++b) {
            const int wa = std::min(2 * (a / 2), nr - 3), wb = 2 * (b / 2);
            double* t = &m.cellc[((size_t)a * nt + b) * CELLC];
            for (int c = 0; c < 2; ++c) {
                const double c00 = P(wa, wb, c), c10 = P(wa + 2, wb, c), c01 = P(wa, wb + 2, c), c11 = P(wa + 2, wb + 2, c);
                t[0 + c] = 0.25 * (-c00 + c10 - c01 + c11);
                t[2 + c] = 0.25 * (-c00 - c10 + c01 + c11);
                t[4 + c] = 0.25 * (c00 - c10 - c01 + c11);
            }
        }
    return LBFSI_OK;
}

// Wall geometry of a C-grid: open chains of straight edges between their
// even-offset nodes, counterclockwise around each body.  Interior nodes as
// on a closed wall; a chain's end is a junction, one point with the mirrored
// column's node, which ends the mirrored chain (the same chain for a body
// that row 0 wraps around): its normal is the normalised sum of the normals
// of the two edges that meet there, and the first copy carries the Simpson
// shares of both edges (the second copy none: its values are the first's).
static void wall_geometry_chains(HostMesh& m) {
    const int nt = m.nt;
    const std::vector<double>& X = m.xw;
    auto edge = [&](int a, int c, double& L, double& nx, double& ny) {
        const double tx = X[2 * c] - X[2 * a], ty = X[2 * c + 1] - X[2 * a + 1];
        L = std::sqrt(tx * tx + ty * ty);
        nx = ty / L;
        ny = -tx / L;
    };
    m.n0.assign(2 * nt, 0.0);
    m.wall_geo.assign(6 * nt, 0.0);
    for (size_t w = 0; w + 1 < m.walls.size(); w += 2) {
        const int a = m.walls[w], b = m.walls[w + 1];
        for (int j = a; j <= b; ++j) {
            double* g = &m.wall_geo[6 * j];
            double L1, x1, y1, L2, x2, y2;
            if ((j - a) % 2) {
                edge(j - 1, j + 1, L1, x1, y1);
                m.n0[2 * j] = x1;
                m.n0[2 * j + 1] = y1;
                g[0] = 4.0 / 6.0 * L1;
                g[1] = x1;
                g[2] = y1;
                continue;
            }
            if (a < j && j < b) {
                edge(j, j + 2, L1, x1, y1);
                edge(j - 2, j, L2, x2, y2);
            } else {
                const int k = nt - 1 - j;   // the mirrored copy of this junction
                if (j == a) {
                    edge(j, j + 2, L1, x1, y1);
                    edge(k - 2, k, L2, x2, y2);
                } else {
                    edge(j - 2, j, L1, x1, y1);
                    edge(k, k + 2, L2, x2, y2);
                }
            }
            const double vx = x1 + x2, vy = y1 + y2, L = std::sqrt(vx * vx + vy * vy);
            m.n0[2 * j] = vx / L;
            m.n0[2 * j + 1] = vy / L;
            if (m.coltype[j] & CT_DUP) continue;
            g[0] = L1 / 6.0;
            g[1] = x1;
            g[2] = y1;
            g[3] = L2 / 6.0;
            g[4] = x2;
            g[5] = y2;
        }
    }
}

int build_host_mesh_c(int nr, int nt, int nwalls, const int* walls, const double* X, double xc, double yc,
                      HostMesh& m, int nbody, const int* wall_body) {
    if (nr < 5) return set_error(LBFSI_EINVAL, "nr must be >= 5");
    if (nt < 7 || nt % 2 == 0) return set_error(LBFSI_EINVAL, "a C-grid needs an odd node count (>= 7) along the C");
    if (!X || !walls) return set_error(LBFSI_EINVAL, "null coordinate or wall pointer");
    if (nwalls < 1) return set_error(LBFSI_EINVAL, "a C-grid needs at least one wall chain");
    if (nbody < 1 || nbody > MAX_BODIES) return set_error(LBFSI_EINVAL, "nbody must be in 1 .. 4");
    if (nbody > 1 && !wall_body) return set_error(LBFSI_EINVAL, "several bodies need the body of each wall chain");
    std::vector<int> owned(nbody, 0);
    for (int w = 0; w < nwalls && wall_body; ++w) {
        if (wall_body[w] < 0 || wall_body[w] >= nbody) return set_error(LBFSI_EINVAL, "wall_body out of range");
        owned[wall_body[w]] = 1;
    }
    for (int k = 0; k < nbody; ++k)
        if (!owned[k] && wall_body) return set_error(LBFSI_EINVAL, "every body needs a wall chain");
    m.nbody = nbody;
    const int G = CGRID_GHOST_ROWS;
    if (nr < G + 1) return set_error(LBFSI_EINVAL, "a C-grid needs nr > 4");
    // column classes: wall chains (even ends inside the outlets, no overlap),
    // cut elsewhere, symmetric in j -> nt-1-j
    m.coltype.assign(nt, CT_CUT);
    m.walls.assign(walls, walls + 2 * (size_t)nwalls);
    for (int w = 0; w < nwalls; ++w) {
        const int a = walls[2 * w], b = walls[2 * w + 1];
        if (a < 1 || b > nt - 2 || a % 2 || b % 2 || b - a < 2)
            return set_error(LBFSI_EINVAL, "wall chains must run between even columns inside the outlets");
        for (int j = a; j <= b; ++j) {
            if (m.coltype[j] & CT_WALL) return set_error(LBFSI_EINVAL, "wall chains overlap");
            m.coltype[j] = CT_WALL | ((wall_body ? wall_body[w] : 0) << CT_BODY_SHIFT);
        }
    }
    for (int j = 0; j < nt; ++j)
        if (m.coltype[j] != m.coltype[nt - 1 - j])
            return set_error(LBFSI_EINVAL, "the cut and the wall chains (and their bodies) must be symmetric "
                                           "in j -> ntheta-1-j");
    for (int j = 0; j < nt; ++j) {
        if (!(m.coltype[j] & CT_WALL)) continue;
        const bool before = j > 0 && (m.coltype[j - 1] & CT_CUT), after = j < nt - 1 && (m.coltype[j + 1] & CT_CUT);
        if (before || after) m.coltype[j] |= CT_JUNC | (before ? 0 : CT_JFWD);
    }
    for (int j = (nt - 1) / 2 + 1; j < nt; ++j)
        if (m.coltype[j] & (CT_CUT | CT_JUNC)) m.coltype[j] |= CT_DUP;
    m.general = true;
    m.cgrid = true;
    m.G = G;
    m.nr = nr;
    m.nt = nt;
    m.N = nr * nt;
    m.Nx = (nr + G) * nt;
    m.ntj = tiles_j(nt);
    m.xm = xc;
    m.ym = yc;
    std::vector<double> Xu(X, X + 2 * (size_t)m.N);
    double scale = 0.0;
    for (double v : Xu) {
        if (!std::isfinite(v)) return set_error(LBFSI_EINVAL, "node coordinates must be finite");
        scale = std::max(scale, std::fabs(v));
    }
    auto P = [&](int i, int j, int c) { return Xu[2 * ((size_t)i * nt + j) + c]; };
    for (int j = 0; j < nt; ++j)
        if (m.coltype[j] & (CT_CUT | CT_JUNC))
            for (int c = 0; c < 2; ++c)
                if (std::fabs(P(0, j, c) - P(0, nt - 1 - j, c)) > 1e-12 * scale)
                    return set_error(LBFSI_EINVAL, "row-0 nodes j and ntheta-1-j must coincide along the cut "
                                                   "(and at the chains' ends)");
    auto check_window = [&](int wa, int wb) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const double xi = a - 1.0, et = b - 1.0;
                for (int c = 0; c < 2; ++c) {
                    const double v = 0.25 * ((1 - xi) * (1 - et) * P(wa, wb, c) + (1 + xi) * (1 - et) * P(wa + 2, wb, c) +
                                             (1 - xi) * (1 + et) * P(wa, wb + 2, c) + (1 + xi) * (1 + et) * P(wa + 2, wb + 2, c));
                    if (std::fabs(v - P(wa + a, wb + b, c)) > 1e-12 * scale) return false;
                }
            }
        return true;
    };
    for (int wa = 0; wa + 2 < nr; wa += 2)
        for (int wb = 0; wb + 2 < nt; wb += 2)
            if (!check_window(wa, wb) || (nr % 2 == 0 && !check_window(nr - 3, wb)))
                return set_error(LBFSI_EINVAL, "node coordinates must be subparametric "
                                               "(every window the bilinear image of its corners)");
    m.xw.assign(2 * (size_t)nt, 0.0);
    m.fardir.assign(2 * (size_t)nt, 0.0);
    m.fardirj.assign(4 * (size_t)nr, 0.0);
    for (int j = 0; j < nt; ++j)
        for (int c = 0; c < 2; ++c) {
            m.xw[2 * j + c] = P(0, j, c);
            m.fardir[2 * j + c] = P(nr - 1, j, c) - P(nr - 2, j, c);
        }
    for (int i = 0; i < nr; ++i)
        for (int c = 0; c < 2; ++c) {
            m.fardirj[4 * i + c] = P(i, 0, c) - P(i, 1, c);
            m.fardirj[4 * i + 2 + c] = P(i, nt - 1, c) - P(i, nt - 2, c);
        }
    normalise_pairs(m.fardir);
    normalise_pairs(m.fardirj);
    wall_geometry_chains(m);
    // node coordinates with the mirrored rows: X(-k, j) = X(k, nt-1-j)
    const size_t g0 = (size_t)G * nt;
    m.X.assign(2 * (size_t)m.Nx, 0.0);
    for (int i = -G; i < nr; ++i)
        for (int j = 0; j < nt; ++j)
            for (int c = 0; c < 2; ++c)
                m.X[2 * (g0 + (size_t)i * nt + j) + c] = i < 0 ? P(-i, nt - 1 - j, c) : P(i, j, c);
    // inverse metric with the C-grid stencils (central across the cut on row
    // 0 of the cut and at both copies of the rear point; one-sided along the
    // cut at the rear point, along i on the rest of the wall and the far
    // field, along j at the outlet columns); the mirrored rows carry the
    // negated inverse metric of their node (both index directions reversed)
    m.jinv.assign(4 * (size_t)m.Nx, 0.0);
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nt; ++j) {
            const int ct = m.coltype[j];
            const bool across = i == 0 && (ct & (CT_CUT | CT_JUNC));
            const bool jfwd = i == 0 && (ct & CT_JUNC) && (ct & CT_JFWD);
            const bool jbwd = i == 0 && (ct & CT_JUNC) && !(ct & CT_JFWD);
            double di[2], dj[2];
            for (int c = 0; c < 2; ++c) {
                if (across)
                    di[c] = 0.5 * (P(1, j, c) - P(1, nt - 1 - j, c));
                else if (i == 0)
                    di[c] = 0.5 * (-3.0 * P(0, j, c) + 4.0 * P(1, j, c) - P(2, j, c));
                else if (i == nr - 1)
                    di[c] = 0.5 * (3.0 * P(nr - 1, j, c) - 4.0 * P(nr - 2, j, c) + P(nr - 3, j, c));
                else
                    di[c] = 0.5 * (P(i + 1, j, c) - P(i - 1, j, c));
                if (j == 0 || jfwd)
                    dj[c] = 0.5 * (-3.0 * P(i, j, c) + 4.0 * P(i, j + 1, c) - P(i, j + 2, c));
                else if (j == nt - 1 || jbwd)
                    dj[c] = 0.5 * (3.0 * P(i, j, c) - 4.0 * P(i, j - 1, c) + P(i, j - 2, c));
                else
                    dj[c] = 0.5 * (P(i, j + 1, c) - P(i, j - 1, c));
            }
            const double det = di[0] * dj[1] - di[1] * dj[0];
            if (!(det > 0.0))
                return set_error(LBFSI_EINVAL, "mesh not positively oriented (index-to-space Jacobian <= 0)");
            double* t = &m.jinv[4 * (g0 + (size_t)i * nt + j)];
            t[0] = dj[1] / det;
            t[1] = -di[1] / det;
            t[2] = -dj[0] / det;
            t[3] = di[0] / det;
        }
    for (int k = 1; k <= G; ++k)
        for (int j = 0; j < nt; ++j)
            for (int c = 0; c < 4; ++c)
                m.jinv[4 * (g0 - (size_t)k * nt + j) + c] = -m.jinv[4 * (g0 + (size_t)k * nt + (nt - 1 - j)) + c];
    // element coefficients per cell (a, b), a in [-G, nr-2], b in [0, nt-2];
    // a mirrored cell is the cell (-a-1, nt-2-b) with both local coordinates
    // reversed: (b, c, d) -> (-b, -c, d)
    m.cellc.assign((size_t)(nr - 1 + G) * nt * CELLC, 0.0);
    auto cell = [&](int a, int b) { return &m.cellc[(g0 + (size_t)a * nt + b) * CELLC]; };
    for (int a = 0; a < nr - 1; ++a)
        for (int b = 0; b < nt - 1; ++b) {
            const int wa = std::min(2 * (a / 2), nr - 3), wb = std::min(2 * (b / 2), nt - 3);
            double* t = cell(a, b);
            for (int c = 0; c < 2; ++c) {
                const double c00 = P(wa, wb, c), c10 = P(wa + 2, wb, c), c01 = P(wa, wb + 2, c), c11 = P(wa + 2, wb + 2, c);
                t[0 + c] = 0.25 * (-c00 + c10 - c01 + c11);
                t[2 + c] = 0.25 * (-c00 - c10 + c01 + c11);
                t[4 + c] = 0.25 * (c00 - c10 - c01 + c11);
            }
        }
    for (int k = 1; k <= G; ++k)
        for (int b = 0; b < nt - 1; ++b) {
            const double* src = cell(k - 1, nt - 2 - b);
            double* t = cell(-k, b);
            for (int c = 0; c < 4; ++c) t[c] = -src[c];
            t[4] = src[4];
            t[5] = src[5];
        }
    return LBFSI_OK;
}

int build_host_mesh_box(int ni, int nj, const double* X, const double* shift_i, const double* shift_j,
                        HostMesh& m) {
    if (ni < 4 || nj < 4 || ni % 2 || nj % 2) return set_error(LBFSI_EINVAL, "a periodic box needs even ni, nj >= 4");
    if (!X || !shift_i || !shift_j) return set_error(LBFSI_EINVAL, "null argument");
    m.general = true;
    m.box = true;
    m.nr = ni;
    m.nt = nj;
    m.N = ni * nj;
    m.Nx = m.N;
    m.ntj = tiles_j(nj);
    m.X.assign(X, X + 2 * (size_t)m.N);
    double scale = 0.0;
    for (double v : m.X) {
        if (!std::isfinite(v)) return set_error(LBFSI_EINVAL, "node coordinates must be finite");
        scale = std::max(scale, std::fabs(v));
    }
    for (int c = 0; c < 2; ++c) {
        if (!std::isfinite(shift_i[c]) || !std::isfinite(shift_j[c]))
            return set_error(LBFSI_EINVAL, "period vectors must be finite");
        scale = std::max(scale, std::max(std::fabs(shift_i[c]), std::fabs(shift_j[c])));
    }
    // coordinates of any index pair: the node of the period plus the shifts
    auto P = [&](int i, int j, int c) {
        const int ki = (int)std::floor((double)i / ni), kj = (int)std::floor((double)j / nj);
        return m.X[2 * ((size_t)(i - ki * ni) * nj + (j - kj * nj)) + c] + ki * shift_i[c] + kj * shift_j[c];
    };
    for (int wa = 0; wa < ni; wa += 2)
        for (int wb = 0; wb < nj; wb += 2)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    for (int c = 0; c < 2; ++c) {
                        const double xi = a - 1.0, et = b - 1.0;
                        const double v = 0.25 * ((1 - xi) * (1 - et) * P(wa, wb, c) + (1 + xi) * (1 - et) * P(wa + 2, wb, c) +
                                                 (1 - xi) * (1 + et) * P(wa, wb + 2, c) +
                                                 (1 + xi) * (1 + et) * P(wa + 2, wb + 2, c));
                        if (std::fabs(v - P(wa + a, wb + b, c)) > 1e-12 * scale)
                            return set_error(LBFSI_EINVAL, "node coordinates must be subparametric "
                                                           "(every window the bilinear image of its corners)");
                    }
    // no wall and no far field: empty per-column tables
    m.xw.assign(2 * (size_t)nj, 0.0);
    m.fardir.assign(2 * (size_t)nj, 0.0);
    m.n0.assign(2 * (size_t)nj, 0.0);
    m.wall_geo.assign(6 * (size_t)nj, 0.0);
    // inverse metric with central differences in both (periodic) directions
    m.jinv.assign(4 * (size_t)m.N, 0.0);
    for (int i = 0; i < ni; ++i)
        for (int j = 0; j < nj; ++j) {
            double di[2], dj[2];
            for (int c = 0; c < 2; ++c) {
                di[c] = 0.5 * (P(i + 1, j, c) - P(i - 1, j, c));
                dj[c] = 0.5 * (P(i, j + 1, c) - P(i, j - 1, c));
            }
            const double det = di[0] * dj[1] - di[1] * dj[0];
            if (!(det > 0.0))
                return set_error(LBFSI_EINVAL, "mesh not positively oriented (index-to-space Jacobian <= 0)");
            double* t = &m.jinv[4 * ((size_t)i * nj + j)];
            t[0] = dj[1] / det;
            t[1] = -di[1] / det;
            t[2] = -dj[0] / det;
            t[3] = di[0] / det;
        }
    // element coefficients of every cell (windows wrap, corners shifted)
    m.cellc.assign((size_t)ni * nj * CELLC, 0.0);
    for (int a = 0; a < ni; ++a)
        for (int b = 0; b < nj; ++b) {
            const int wa = 2 * (a / 2), wb = 2 * (b / 2);
            double* t = &m.cellc[((size_t)a * nj + b) * CELLC];
            for (int c = 0; c < 2; ++c) {
                const double c00 = P(wa, wb, c), c10 = P(wa + 2, wb, c), c01 = P(wa, wb + 2, c), c11 = P(wa + 2, wb + 2, c);
                t[0 + c] = 0.25 * (-c00 + c10 - c01 + c11);
                t[2 + c] = 0.25 * (-c00 - c10 + c01 + c11);
                t[4 + c] = 0.25 * (c00 - c10 - c01 + c11);
            }
        }
    return LBFSI_OK;
}

int validate_bodies(const HostMesh& m, const lbfsi_body_desc* bodies, int n) {
    if (!bodies) return set_error(LBFSI_EINVAL, "null body pointer");
    const int nbody = m.nbody;
    for (int k = 0; k < n * nbody; ++k) {
        const lbfsi_body_desc& b = bodies[k];
        const int own = k % nbody;
        if (b.dof < 0 || b.dof > 2) return set_error(LBFSI_EINVAL, "body dof must be 0, 1 or 2");
        if (b.dof == 0) continue;
        if (m.box) return set_error(LBFSI_EINVAL, "a periodic box has no wall: bodies must be fixed (dof 0)");
        if (!(b.r_out > b.r_in) || !(b.length > 0) || !(b.m_star > 0) || !(b.v_r > 0))
            return set_error(LBFSI_EINVAL, "moving body needs r_out > r_in, length, m_star, v_r > 0");
        if (!(b.forced_periods >= 0.0) || !std::isfinite(b.pitch_amp) || !std::isfinite(b.forced_periods))
            return set_error(LBFSI_EINVAL, "forced pitching needs a finite amplitude and forced_periods >= 0");
        for (int j = 0; j < m.nt; ++j) {
            if (m.cgrid && !(m.coltype[j] & CT_WALL)) continue;   // the cut
            const int owner = m.cgrid ? (m.coltype[j] >> CT_BODY_SHIFT) & (MAX_BODIES - 1) : 0;
            const double x = m.xw[2 * j] - b.xc;
            const double y = m.xw[2 * j + 1] - b.yc;
            const double dist = std::sqrt(x * x + y * y);
            if (owner == own && dist >= b.r_in)
                return set_error(LBFSI_EINVAL, "the wall must lie inside the rigid zone (r_in)");
            if (owner != own && dist <= b.r_out)
                return set_error(LBFSI_EINVAL, "another body's wall lies inside this body's blended region (r_out)");
        }
        for (int o = k - own; o < k; ++o) {
            const lbfsi_body_desc& c = bodies[o];
            if (c.dof == 0) continue;
            if (std::hypot(b.xc - c.xc, b.yc - c.yc) < b.r_out + c.r_out)
                return set_error(LBFSI_EINVAL, "the blended regions of two moving bodies overlap");
        }
    }
    return LBFSI_OK;
}

// Dimensional ODE coefficients from the paper's nondimensional groups
// (Sec. IV A for the transverse model, Sec. IV D for pitch-plunge).
BodyDev body_dev(const lbfsi_body_desc& d, double rho, double U) {
    BodyDev b{};
    b.dof = d.dof;
    b.xc = d.xc; b.yc = d.yc; b.xp = d.xp; b.yp = d.yp;
    b.r_in = d.r_in; b.r_out = d.r_out;
    b.inv_w = 1.0 / (d.r_out - d.r_in);
    const double pi = 3.14159265358979323846;
    if (d.dof == LBFSI_BODY_TRANSVERSE) {
        const double D = d.length;
        b.m = d.m_star * rho * pi * D * D / 4.0;
        const double wn = 2.0 * pi * U / (d.v_r * D);
        b.k = b.m * wn * wn;
        b.c = 2.0 * d.zeta * b.m * wn;
    } else if (d.dof == LBFSI_BODY_PITCH_PLUNGE) {
        const double bh = 0.5 * d.length;
        b.m = d.m_star * pi * rho * bh * bh;
        const double wa = U / (d.v_r * bh * std::sqrt(d.m_star));
        const double wh = d.wh_wa * wa;
        b.s_a = d.x_alpha * b.m * bh;
        b.i_a = d.r_alpha * d.r_alpha * b.m * bh * bh;
        b.k_h = b.m * wh * wh;
        b.k_a = b.i_a * wa * wa;
        b.pitch_amp = d.pitch_amp;
        b.w_a = wa;
        b.t_forced = d.forced_periods * 2.0 * pi / wa;
    }
    return b;
}

double flow_u_inf(const lbfsi_flow_params& p) { return p.ma * std::sqrt(p.gamma * p.t_inf); }

int fill_flow(const lbfsi_flow_params& p, SolveDev& s) {
    if (!(p.gamma > 1.0) || !(p.t_inf > 0) || !(p.rho_inf > 0) || !(p.dt > 0) || !(p.re > 0) ||
        !(p.pr > 0) || !(p.length > 0) || p.ma < 0)
        return set_error(LBFSI_EINVAL, "invalid flow parameters");
    const double U = flow_u_inf(p);
    const double mu = p.rho_inf * U * p.length / p.re;
    if (!(mu > 0)) return set_error(LBFSI_EINVAL, "viscosity must be positive (Ma > 0)");
    s.dt = p.dt;
    s.mu = mu;
    s.Cv = 1.0 / (p.gamma - 1.0);
    s.Pr = p.pr;
    s.rho_inf = p.rho_inf;
    s.uinf_x = U;
    s.uinf_y = 0.0;
    s.T_inf = p.t_inf;
    s.dt_f = (float)s.dt;
    s.mu_f = (float)s.mu;
    s.Cv_f = (float)s.Cv;
    s.Pr_f = (float)s.Pr;
    s.iPr_f = (float)(1.0 / s.Pr);
    s.rho_inf_f = (float)s.rho_inf;
    s.uinf_x_f = (float)s.uinf_x;
    s.uinf_y_f = 0.0f;
    s.T_inf_f = (float)s.T_inf;
    double fr[9], gr[9];
    f_equilibrium<double>(s.rho_inf, s.uinf_x, s.uinf_y, s.T_inf, fr);
    g_equilibrium<double>(s.rho_inf, s.uinf_x, s.uinf_y, s.T_inf, s.Cv, gr);
    for (int q = 0; q < 9; ++q) {
        s.fgref[2 * q] = (float)fr[q];
        s.fgref[2 * q + 1] = (float)gr[q];
    }
    return LBFSI_OK;
}

void* CudaMallocMemory::alloc(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void CudaMallocMemory::release(void* p) {
    if (p) cudaFree(p);
}

int upload_mesh(const HostMesh& h, int precision, DevMemory& mem, cudaStream_t s, DeviceMesh& out) {
    const size_t es = precision == LBFSI_FP64 ? sizeof(double) : sizeof(float);
    auto put = [&](const std::vector<double>& v, bool typed, void** dst) -> int {
        const size_t bytes = v.size() * (typed ? es : sizeof(double));
        void* p = mem.alloc(bytes);
        if (!p) return set_error(LBFSI_ENOMEM, "device allocation of the mesh geometry failed");
        out.blocks.push_back(p);
        out.bytes += bytes;
        cudaError_t e;
        if (typed && precision == LBFSI_FP32) {
            std::vector<float> f(v.begin(), v.end());
            e = cudaMemcpyAsync(p, f.data(), bytes, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        } else {
            e = cudaMemcpyAsync(p, v.data(), bytes, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        if (e != cudaSuccess) return set_error(LBFSI_ECUDA, std::string("mesh upload: ") + cudaGetErrorString(e));
        *dst = p;
        return LBFSI_OK;
    };
    MeshDev& d = out.dev;
    d.nr = h.nr;
    d.nt = h.nt;
    d.N = h.Nx;
    d.ntj = h.ntj;
    d.xm = h.xm;
    d.ym = h.ym;
    d.xm_f = (float)h.xm;
    d.ym_f = (float)h.ym;
    d.emin = 0.0;
    if (!h.general) {
        d.emin = 1e300;
        for (int j = 0; j < h.nt; ++j) d.emin = std::min(d.emin, std::hypot(h.e[2 * j], h.e[2 * j + 1]));
    }
    d.emin_f = (float)d.emin;
    void *pr = nullptr, *pe = nullptr, *pn = nullptr, *pw = nullptr, *prt = nullptr, *pct = nullptr;
    void *pxw = nullptr, *pfd = nullptr, *px = nullptr, *pj = nullptr, *pc = nullptr, *pfj = nullptr;
    void* pct_ = nullptr;
    int rc = put(h.n0, false, &pn);
    if (!rc) rc = put(h.wall_geo, false, &pw);
    if (!rc) rc = put(h.xw, false, &pxw);
    if (!rc) rc = put(h.fardir, false, &pfd);
    if (h.general) {
        if (!rc) rc = put(h.X, true, &px);
        if (!rc) rc = put(h.jinv, true, &pj);
        if (!rc) rc = put(h.cellc, true, &pc);
        if (!rc && h.cgrid) rc = put(h.fardirj, false, &pfj);
        if (!rc && h.cgrid) {
            const size_t bytes = h.coltype.size() * sizeof(int);
            pct_ = mem.alloc(bytes);
            if (!pct_) {
                rc = set_error(LBFSI_ENOMEM, "device allocation of the mesh geometry failed");
            } else {
                out.blocks.push_back(pct_);
                out.bytes += bytes;
                cudaError_t e = cudaMemcpyAsync(pct_, h.coltype.data(), bytes, cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) rc = set_error(LBFSI_ECUDA, std::string("mesh upload: ") + cudaGetErrorString(e));
            }
        }
    } else {
        if (!rc) rc = put(h.r, false, &pr);
        if (!rc) rc = put(h.e, false, &pe);
        if (!rc) rc = put(h.rowtab, true, &prt);
        if (!rc) rc = put(h.coltab, true, &pct);
    }
    if (rc) {
        release_mesh(out, mem);
        return rc;
    }
    d.r = (const double*)pr;
    d.e = (const double*)pe;
    d.n0 = (const double*)pn;
    d.wall_geo = (const double*)pw;
    d.rowtab = prt;
    d.coltab = pct;
    d.xw = (const double*)pxw;
    d.fardir = (const double*)pfd;
    d.general = h.general ? 1 : 0;
    // general-mesh arrays: pointers at row 0 (a C-grid's mirrored rows before it)
    const size_t g0 = (size_t)h.G * h.nt;
    d.nodex = px ? (const char*)px + g0 * 2 * es : nullptr;
    d.jinv = pj ? (const char*)pj + g0 * 4 * es : nullptr;
    d.cellc = pc ? (const char*)pc + g0 * CELLC * es : nullptr;
    d.cgrid = h.cgrid ? 1 : 0;
    d.box = h.box ? 1 : 0;
    d.fardirj = (const double*)pfj;
    d.coltype = (const int*)pct_;
    return LBFSI_OK;
}

void release_mesh(DeviceMesh& m, DevMemory& mem) {
    for (void* p : m.blocks) mem.release(p);
    m.blocks.clear();
    m.bytes = 0;
}

size_t solve_bytes(int N, int ntj, int precision) {
    const size_t es = precision == LBFSI_FP64 ? sizeof(double) : sizeof(float);
    const size_t pops = 2 * 2 * 9 * (size_t)N * es;  // f, g ping-pong
    const size_t mom = 2 * 4 * (size_t)N * es;
    return pops + mom + 2 * sizeof(StepMaps) + (size_t)ntj * 3 * sizeof(double) + 256 +
           sizeof(BodyDev) + 5 * 256;  // alignment slack
}

size_t mesh_bytes(int nr, int nt, int precision) {
    const size_t es = precision == LBFSI_FP64 ? sizeof(double) : sizeof(float);
    return (size_t)nr * sizeof(double) + (size_t)nt * 14 * sizeof(double) +
           ((size_t)nr * ROWTAB + (size_t)nt * COLTAB) * es + 8 * 256;
}

}  // namespace lbfsi
