// C-ABI of the library (declared in include/lbfsi.h): handle, device memory,
// host-side mesh geometry and the launch sequence of the coupled step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lbfsi.h"
#include "lbfsi_internal.h"

using lbfsi::BodyDev;
using lbfsi::BodyStateDev;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(LBFSI_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

int lbfsi::set_error(int code, const std::string& msg) { return fail(code, msg); }

struct lbfsi_mesh_s {
    int nr = 0, nt = 0, N = 0, nbatch = 0, precision = 0, ntj = 0;
    double xm = 0, ym = 0;
    cudaStream_t stream = nullptr;
    size_t esize = 8;
    std::vector<double> r, e, n0, wall_geo;
    std::vector<lbfsi_body_desc> bodies;
    double* d_r = nullptr;
    double* d_e = nullptr;
    double* d_n0 = nullptr;
    double* d_wall_geo = nullptr;
    void* d_rowtab = nullptr;
    void* d_coltab = nullptr;
    BodyDev* d_bodies = nullptr;
    void* d_f[2] = {nullptr, nullptr};
    void* d_g[2] = {nullptr, nullptr};
    void* d_M[2] = {nullptr, nullptr};
    void* d_fpost = nullptr;
    void* d_gpost = nullptr;
    double* d_stage = nullptr;  // [nbatch][4][N] float64 staging
    lbfsi::StepMaps* d_maps[2] = {nullptr, nullptr};  // maps of the next launch (cur) / scratch
    BodyStateDev* d_state_a = nullptr;                // host-given states staging
    BodyStateDev* d_state_b = nullptr;
    double* d_loads_tmp = nullptr;
    double* d_part = nullptr;        // [nbatch][ntj][3] load partials
    unsigned* d_counter = nullptr;   // [nbatch] CTA completion counters
    unsigned* d_status = nullptr;
    int cur = 0, curM = 0;
    int variant = 0;                 // tile shape of the float step kernel
    bool initialized = false, first = true;
    double dt = 0, mu = 0, Cv = 0, Pr = 0, rho_inf = 0, uinf = 0, T_inf = 0;
    int64_t launches = 0;
};

namespace {

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

int check_status(lbfsi_mesh m) {
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    unsigned st = 0;
    e = cudaMemcpy(&st, m->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (st & lbfsi::ST_DEPARTURE)
        return fail(LBFSI_EDEPARTURE, "departure point outside the cells adjacent to its node (CFL)");
    if (st & lbfsi::ST_BPOINT)
        return fail(LBFSI_EDEPARTURE, "wall target point outside the first element row");
    if (st & lbfsi::ST_NONPHYS) return fail(LBFSI_ENONPHYS, "non-physical state (rho<=0, T<=0 or NaN)");
    return LBFSI_OK;
}

void to_double(const void* src, double* dst, size_t n, int precision) {
    if (precision == LBFSI_FP64) {
        std::memcpy(dst, src, n * sizeof(double));
    } else {
        const float* s = static_cast<const float*>(src);
        for (size_t k = 0; k < n; ++k) dst[k] = (double)s[k];
    }
}

int download(lbfsi_mesh m, const void* dsrc, double* host, size_t n) {
    std::vector<unsigned char> tmp(n * m->esize);
    cudaError_t e = cudaMemcpyAsync(tmp.data(), dsrc, n * m->esize, cudaMemcpyDeviceToHost, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "download");
    e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "download sync");
    to_double(tmp.data(), host, n, m->precision);
    return LBFSI_OK;
}

int upload(lbfsi_mesh m, const double* host, void* ddst, size_t n) {
    std::vector<unsigned char> tmp(n * m->esize);
    if (m->precision == LBFSI_FP64) {
        std::memcpy(tmp.data(), host, n * sizeof(double));
    } else {
        float* t = reinterpret_cast<float*>(tmp.data());
        for (size_t k = 0; k < n; ++k) t[k] = (float)host[k];
    }
    cudaError_t e = cudaMemcpyAsync(ddst, tmp.data(), n * m->esize, cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload");
    e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload sync");
    return LBFSI_OK;
}

// Wall polygon of the O-grid (Sec. III): the wall edges are the straight
// element edges between even-indexed wall nodes.  For every wall node: the unit
// normal n0 out of the body (odd node: its edge's normal; even node: the
// normalised sum of its two edges' normals) and its Simpson share of the
// adjacent edges (weight*length and edge normal, up to two edges).
void wall_geometry(lbfsi_mesh m) {
    const int nt = m->nt, ne = nt / 2;
    std::vector<double> X(2 * nt);
    for (int j = 0; j < nt; ++j) {
        X[2 * j] = m->xm + m->r[0] * m->e[2 * j];
        X[2 * j + 1] = m->ym + m->r[0] * m->e[2 * j + 1];
    }
    std::vector<double> en(2 * ne), ds(ne);
    for (int k = 0; k < ne; ++k) {
        const int a = 2 * k, c = (2 * k + 2) % nt;
        const double tx = X[2 * c] - X[2 * a], ty = X[2 * c + 1] - X[2 * a + 1];
        const double L = std::sqrt(tx * tx + ty * ty);
        ds[k] = L;
        en[2 * k] = ty / L;
        en[2 * k + 1] = -tx / L;
    }
    m->n0.assign(2 * nt, 0.0);
    m->wall_geo.assign(6 * nt, 0.0);
    for (int j = 0; j < nt; ++j) {
        double* g = &m->wall_geo[6 * j];
        if (j % 2) {
            const int k = j / 2;
            m->n0[2 * j] = en[2 * k];
            m->n0[2 * j + 1] = en[2 * k + 1];
            g[0] = 4.0 / 6.0 * ds[k];
            g[1] = en[2 * k];
            g[2] = en[2 * k + 1];
        } else {
            const int k2 = j / 2, k1 = (j / 2 - 1 + ne) % ne;
            const double vx = en[2 * k1] + en[2 * k2], vy = en[2 * k1 + 1] + en[2 * k2 + 1];
            const double L = std::sqrt(vx * vx + vy * vy);
            m->n0[2 * j] = vx / L;
            m->n0[2 * j + 1] = vy / L;
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
// the step kernel (float64 here, stored in the element type of the path):
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
void geometry_tables(lbfsi_mesh m, std::vector<double>& row, std::vector<double>& col) {
    const int nr = m->nr, nt = m->nt;
    const double* r = m->r.data();
    const double* e = m->e.data();
    row.assign((size_t)nr * lbfsi::ROWTAB, 0.0);
    for (int i = 0; i < nr; ++i) {
        double drc;
        if (i == 0)
            drc = 0.5 * (-3.0 * r[0] + 4.0 * r[1] - r[2]);
        else if (i == nr - 1)
            drc = 0.5 * (3.0 * r[nr - 1] - 4.0 * r[nr - 2] + r[nr - 3]);
        else
            drc = 0.5 * (r[i + 1] - r[i - 1]);
        double* t = &row[(size_t)i * lbfsi::ROWTAB];
        t[0] = r[i];
        t[1] = 1.0 / drc;
        t[2] = 1.0 / r[i];
        for (int c = 0; c < 2; ++c) {
            const int a = i - 1 + c;
            if (a < 0 || a > nr - 2) continue;
            const int wa = std::min(2 * (a / 2), nr - 3);
            t[3 + 2 * c] = (double)(i - wa - 1);
            t[4 + 2 * c] = 2.0 / (r[wa + 2] - r[wa]);
        }
    }
    col.assign((size_t)nt * lbfsi::COLTAB, 0.0);
    auto wr = [nt](int j) { return ((j % nt) + nt) % nt; };
    for (int j = 0; j < nt; ++j) {
        const double ex = e[2 * j], ey = e[2 * j + 1];
        const int jp = wr(j + 1), jm = wr(j - 1);
        const double dex = 0.5 * (e[2 * jp] - e[2 * jm]), dey = 0.5 * (e[2 * jp + 1] - e[2 * jm + 1]);
        const double cr = ex * dey - ey * dex;
        double* t = &col[(size_t)j * lbfsi::COLTAB];
        t[0] = ex;
        t[1] = ey;
        t[2] = dey / cr;
        t[3] = ey / cr;
        t[4] = dex / cr;
        t[5] = ex / cr;
        for (int c = 0; c < 2; ++c) {
            const int b = j - 1 + c;
            const int wb = (b >= 0) ? 2 * (b / 2) : -2 * ((-b + 1) / 2);
            const int w0 = wr(wb), w2 = wr(wb + 2);
            const double dEx = 0.5 * (e[2 * w2] - e[2 * w0]), dEy = 0.5 * (e[2 * w2 + 1] - e[2 * w0 + 1]);
            t[6 + 4 * c] = (double)(j - wb - 1);
            t[7 + 4 * c] = dEx;
            t[8 + 4 * c] = dEy;
            t[9 + 4 * c] = dEx * ey - dEy * ex;
        }
    }
}

// Dimensional ODE coefficients from the paper's nondimensional groups
// (Sec. IV A for the transverse model, Sec. IV D for pitch-plunge).
BodyDev body_dev(const lbfsi_body_desc& d, double rho, double U) {
    BodyDev b{};
    b.dof = d.dof;
    b.xc = d.xc; b.yc = d.yc; b.xp = d.xp; b.yp = d.yp;
    b.r_in = d.r_in; b.r_out = d.r_out;
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
    }
    return b;
}

void free_all(lbfsi_mesh m) {
    void* ptrs[] = {m->d_r, m->d_e, m->d_n0, m->d_wall_geo, m->d_rowtab, m->d_coltab, m->d_bodies,
                    m->d_f[0], m->d_f[1], m->d_g[0], m->d_g[1], m->d_M[0], m->d_M[1], m->d_fpost,
                    m->d_gpost, m->d_stage, m->d_maps[0], m->d_maps[1], m->d_state_a, m->d_state_b,
                    m->d_loads_tmp, m->d_part, m->d_counter, m->d_status};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

}  // namespace

extern "C" {

const char* lbfsi_last_error(void) { return g_last_error.c_str(); }

int lbfsi_create_mesh(const lbfsi_mesh_desc* d, void* cuda_stream, lbfsi_mesh* out) {
    g_last_error.clear();
    if (!d || !out) return fail(LBFSI_EINVAL, "null argument");
    *out = nullptr;
    if (d->nr < 5) return fail(LBFSI_EINVAL, "nr must be >= 5");
    if (d->ntheta < 4 || d->ntheta % 2) return fail(LBFSI_EINVAL, "ntheta must be even and >= 4");
    if (d->precision != LBFSI_FP64 && d->precision != LBFSI_FP32)
        return fail(LBFSI_EINVAL, "precision must be LBFSI_FP64 or LBFSI_FP32");
    if (d->nbatch < 1) return fail(LBFSI_EINVAL, "nbatch must be >= 1");
    if (!d->r || !d->e || !d->bodies) return fail(LBFSI_EINVAL, "null table or body pointer");
    const long long Nll = (long long)d->nr * d->ntheta;
    if (Nll * 9 * d->nbatch > (1ll << 31)) return fail(LBFSI_EINVAL, "mesh too large for 32-bit node indexing");
    auto m = new lbfsi_mesh_s();
    m->nr = d->nr;
    m->nt = d->ntheta;
    m->N = (int)Nll;
    m->nbatch = d->nbatch;
    m->precision = d->precision;
    m->esize = d->precision == LBFSI_FP64 ? sizeof(double) : sizeof(float);
    m->ntj = lbfsi::tiles_j(m->nt);
    m->xm = d->xc;
    m->ym = d->yc;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    // tile shape of the float kernel (a tuning knob, every variant computes the
    // same result): LBFSI_STEP_VARIANT 0: 8 x 32 nodes, 2 CTAs/SM; 1: 16 x 32,
    // 2 CTAs/SM; 2: 8 x 32, 3 CTAs/SM; 3: 12 x 32, 384 threads (default)
    m->variant = 3;
    if (const char* v = std::getenv("LBFSI_STEP_VARIANT")) {
        const int k = std::atoi(v);
        m->variant = (k >= 0 && k <= 3) ? k : 3;
    }
    m->r.assign(d->r, d->r + d->nr);
    m->e.assign(d->e, d->e + 2 * d->ntheta);
    m->bodies.assign(d->bodies, d->bodies + d->nbatch);
    for (int i = 1; i < m->nr; ++i)
        if (!(m->r[i] > m->r[i - 1])) {
            delete m;
            return fail(LBFSI_EINVAL, "radial table must increase");
        }
    // subparametric tables: odd entries are the averages of their even
    // neighbours (and, for even nr, the clamped last window is uniform), so
    // every window is the bilinear image of the reference square
    auto near = [](double a, double b, double scale) { return std::fabs(a - b) <= 1e-12 * scale; };
    bool sub = true;
    for (int i = 1; i + 1 < m->nr; i += 2)
        sub = sub && near(m->r[i], 0.5 * (m->r[i - 1] + m->r[i + 1]), std::fabs(m->r[i + 1]));
    if (m->nr % 2 == 0)
        sub = sub && near(m->r[m->nr - 2], 0.5 * (m->r[m->nr - 3] + m->r[m->nr - 1]), std::fabs(m->r[m->nr - 1]));
    for (int j = 1; j < m->nt; j += 2)
        for (int c = 0; c < 2; ++c)
            sub = sub && near(m->e[2 * j + c], 0.5 * (m->e[2 * (j - 1) + c] + m->e[2 * ((j + 1) % m->nt) + c]), 1.0);
    if (!sub) {
        delete m;
        return fail(LBFSI_EINVAL, "r and e tables must be subparametric (odd entries = mean of even neighbours)");
    }
    for (const auto& b : m->bodies) {
        if (b.dof < 0 || b.dof > 2) {
            delete m;
            return fail(LBFSI_EINVAL, "body dof must be 0, 1 or 2");
        }
        if (b.dof != 0) {
            if (!(b.r_out > b.r_in) || !(b.length > 0) || !(b.m_star > 0) || !(b.v_r > 0)) {
                delete m;
                return fail(LBFSI_EINVAL, "moving body needs r_out > r_in, length, m_star, v_r > 0");
            }
            for (int j = 0; j < m->nt; ++j) {
                const double x = m->xm + m->r[0] * m->e[2 * j] - b.xc;
                const double y = m->ym + m->r[0] * m->e[2 * j + 1] - b.yc;
                if (std::sqrt(x * x + y * y) >= b.r_in) {
                    delete m;
                    return fail(LBFSI_EINVAL, "the wall must lie inside the rigid zone (r_in)");
                }
            }
        }
    }
    wall_geometry(m);
    std::vector<double> rowt, colt;
    geometry_tables(m, rowt, colt);
    const size_t N = (size_t)m->N, nb = (size_t)m->nbatch;
    cudaError_t e = cudaSuccess;
#define LB_ALLOC(ptr, cnt)                                   \
    if (e == cudaSuccess) e = dalloc(&(ptr), (cnt));
    LB_ALLOC(m->d_r, (size_t)m->nr);
    LB_ALLOC(m->d_e, 2 * (size_t)m->nt);
    LB_ALLOC(m->d_n0, 2 * (size_t)m->nt);
    LB_ALLOC(m->d_wall_geo, 6 * (size_t)m->nt);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_rowtab, rowt.size() * m->esize);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_coltab, colt.size() * m->esize);
    LB_ALLOC(m->d_bodies, nb);
    LB_ALLOC(m->d_stage, nb * 4 * N);
    LB_ALLOC(m->d_maps[0], nb);
    LB_ALLOC(m->d_maps[1], nb);
    LB_ALLOC(m->d_state_a, nb);
    LB_ALLOC(m->d_state_b, nb);
    LB_ALLOC(m->d_loads_tmp, nb * 3);
    LB_ALLOC(m->d_part, nb * m->ntj * 3);
    LB_ALLOC(m->d_counter, nb);
    LB_ALLOC(m->d_status, 1);
#undef LB_ALLOC
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMalloc(&m->d_f[k], nb * 9 * N * m->esize);
        if (e == cudaSuccess) e = cudaMalloc(&m->d_g[k], nb * 9 * N * m->esize);
        if (e == cudaSuccess) e = cudaMalloc(&m->d_M[k], nb * 4 * N * m->esize);
    }
    if (e != cudaSuccess) {
        free_all(m);
        delete m;
        cudaGetLastError();
        return fail(LBFSI_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(m->d_r, m->r.data(), m->nr * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_e, m->e.data(), 2 * m->nt * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_n0, m->n0.data(), 2 * m->nt * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(m->d_wall_geo, m->wall_geo.data(), 6 * m->nt * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(m->d_counter, 0, nb * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(m->d_part, 0, nb * m->ntj * 3 * sizeof(double));
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        const std::vector<double>& src = k ? colt : rowt;
        void* dst = k ? m->d_coltab : m->d_rowtab;
        if (m->precision == LBFSI_FP64) {
            e = cudaMemcpy(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice);
        } else {
            std::vector<float> tf(src.begin(), src.end());
            e = cudaMemcpy(dst, tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) {
        free_all(m);
        delete m;
        return cuda_fail(e, "create_mesh copy");
    }
    *out = m;
    return LBFSI_OK;
}

int lbfsi_destroy_mesh(lbfsi_mesh m) {
    if (!m) return fail(LBFSI_EINVAL, "null mesh");
    cudaStreamSynchronize(m->stream);
    free_all(m);
    delete m;
    return LBFSI_OK;
}

int lbfsi_init_fields(lbfsi_mesh m, const lbfsi_flow_params* p, const double* rho_u_T) {
    if (!m || !p) return fail(LBFSI_EINVAL, "null argument");
    if (!(p->gamma > 1.0) || !(p->t_inf > 0) || !(p->rho_inf > 0) || !(p->dt > 0) || !(p->re > 0) ||
        !(p->pr > 0) || !(p->length > 0) || p->ma < 0)
        return fail(LBFSI_EINVAL, "invalid flow parameters");
    m->dt = p->dt;
    m->Cv = 1.0 / (p->gamma - 1.0);
    m->Pr = p->pr;
    m->rho_inf = p->rho_inf;
    m->T_inf = p->t_inf;
    m->uinf = p->ma * std::sqrt(p->gamma * p->t_inf);
    m->mu = p->rho_inf * m->uinf * p->length / p->re;
    if (!(m->mu > 0)) return fail(LBFSI_EINVAL, "viscosity must be positive (Ma > 0)");
    const size_t N = (size_t)m->N, nb = (size_t)m->nbatch;
    std::vector<BodyDev> bd(nb);
    for (size_t b = 0; b < nb; ++b) bd[b] = body_dev(m->bodies[b], m->rho_inf, m->uinf);
    std::vector<double> M(nb * 4 * N);
    if (rho_u_T) {
        std::memcpy(M.data(), rho_u_T, M.size() * sizeof(double));
    } else {
        for (size_t b = 0; b < nb; ++b)
            for (size_t n = 0; n < N; ++n) {
                M[(b * 4 + 0) * N + n] = m->rho_inf;
                M[(b * 4 + 1) * N + n] = m->uinf;
                M[(b * 4 + 2) * N + n] = 0.0;
                M[(b * 4 + 3) * N + n] = m->T_inf;
            }
    }
    std::vector<BodyStateDev> zero(nb, BodyStateDev{0.0, 0.0, 0.0, 0.0});
    std::vector<double> zl(nb * 3, 0.0);
    cudaError_t e = cudaMemcpyAsync(m->d_bodies, bd.data(), nb * sizeof(BodyDev), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->d_stage, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->d_state_a, zero.data(), nb * sizeof(BodyStateDev), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->d_loads_tmp, zl.data(), zl.size() * sizeof(double), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_status, 0, sizeof(unsigned), m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_counter, 0, nb * sizeof(unsigned), m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "init_fields upload");
    m->cur = m->curM = 0;
    e = lbfsi::launch_prepare(m->d_bodies, m->d_state_a, m->d_state_a, m->d_state_a, m->d_loads_tmp,
                              m->dt, m->nbatch, m->d_maps[0], m->stream);
    m->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "prepare kernel");
    e = lbfsi::launch_init(m->precision, m->d_stage, m->d_f[0], m->d_g[0], m->d_M[0], m->N, m->nbatch,
                           m->Cv, m->stream);
    m->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "init sync");
    m->initialized = true;
    m->first = true;
    return LBFSI_OK;
}

int lbfsi_blend_mesh(lbfsi_mesh m, const lbfsi_body_state* state, const lbfsi_body_state* prev) {
    if (!m || !state) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    const size_t nb = (size_t)m->nbatch;
    static_assert(sizeof(lbfsi_body_state) == sizeof(BodyStateDev), "layout");
    const lbfsi_body_state* pv = prev ? prev : state;
    cudaError_t e = cudaMemcpyAsync(m->d_state_a, state, nb * sizeof(BodyStateDev), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->d_state_b, pv, nb * sizeof(BodyStateDev), cudaMemcpyHostToDevice, m->stream);
    // before the first step the collision map is unused; later it stays the
    // state of the last streamed step
    if (e == cudaSuccess)
        e = lbfsi::launch_prepare(m->d_bodies, m->first ? m->d_state_a : nullptr, m->d_state_a,
                                  m->d_state_b, nullptr, m->dt, m->nbatch, m->d_maps[m->curM], m->stream);
    m->launches++;
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "blend_mesh");
    return LBFSI_OK;
}

static lbfsi::StepArgs make_args(lbfsi_mesh m, int mode) {
    lbfsi::StepArgs a{};
    a.nr = m->nr; a.nt = m->nt; a.N = m->N; a.nbatch = m->nbatch; a.ntj = m->ntj;
    a.xm = m->xm; a.ym = m->ym;
    a.r = m->d_r; a.e = m->d_e; a.n0 = m->d_n0; a.wall_geo = m->d_wall_geo;
    a.rowtab = m->d_rowtab; a.coltab = m->d_coltab;
    a.dt = m->dt; a.mu = m->mu; a.Cv = m->Cv; a.Pr = m->Pr; a.rho_inf = m->rho_inf;
    a.uinf_x = m->uinf; a.uinf_y = 0.0; a.T_inf = m->T_inf;
    a.dt_f = (float)m->dt; a.mu_f = (float)m->mu; a.Cv_f = (float)m->Cv; a.Pr_f = (float)m->Pr;
    a.iPr_f = (float)(1.0 / m->Pr); a.xm_f = (float)m->xm; a.ym_f = (float)m->ym;
    a.rho_inf_f = (float)m->rho_inf; a.uinf_x_f = (float)m->uinf; a.uinf_y_f = 0.0f;
    a.T_inf_f = (float)m->T_inf;
    a.f_in = m->d_f[m->cur]; a.g_in = m->d_g[m->cur];
    a.f_out = m->d_f[m->cur ^ 1]; a.g_out = m->d_g[m->cur ^ 1];
    a.M_in = m->d_M[m->cur]; a.M_out = m->d_M[m->cur ^ 1];
    a.bodies = m->d_bodies;
    a.maps_in = m->d_maps[m->curM];
    a.maps_out = m->d_maps[m->curM ^ 1];
    a.part = m->d_part;
    a.counter = m->d_counter;
    a.mode = mode;
    a.status = m->d_status;
    return a;
}

int lbfsi_step(lbfsi_mesh m, int nsteps) {
    if (!m) return fail(LBFSI_EINVAL, "null mesh");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    if (nsteps < 0) return fail(LBFSI_EINVAL, "nsteps must be >= 0");
    for (int s = 0; s < nsteps; ++s) {
        lbfsi::StepArgs a = make_args(m, m->first ? lbfsi::MODE_STREAM_ONLY : lbfsi::MODE_COLLIDE_STREAM);
        cudaError_t e = lbfsi::launch_step(a, m->precision, m->variant, m->stream);
        m->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
        m->cur ^= 1;
        m->curM ^= 1;
        m->first = false;
    }
    return LBFSI_OK;
}

int lbfsi_synchronize(lbfsi_mesh m) {
    if (!m) return fail(LBFSI_EINVAL, "null mesh");
    return check_status(m);
}

static int download_maps(lbfsi_mesh m, std::vector<lbfsi::StepMaps>& out) {
    out.resize(m->nbatch);
    cudaError_t e = cudaMemcpyAsync(out.data(), m->d_maps[m->curM], out.size() * sizeof(lbfsi::StepMaps),
                                    cudaMemcpyDeviceToHost, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "maps copy");
    return check_status(m);
}

int lbfsi_body_forces(lbfsi_mesh m, double* out) {
    if (!m || !out) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    std::vector<lbfsi::StepMaps> mp;
    const int rc = download_maps(m, mp);
    if (rc) return rc;
    for (int b = 0; b < m->nbatch; ++b)
        for (int c = 0; c < 3; ++c) out[b * 3 + c] = mp[b].loads[c];
    return LBFSI_OK;
}

int lbfsi_advance_bodies(lbfsi_mesh m, const double* loads, double dt) {
    if (!m) return fail(LBFSI_EINVAL, "null mesh");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    const size_t nb = (size_t)m->nbatch;
    std::vector<double> ld(nb * 3);
    if (loads) {
        std::memcpy(ld.data(), loads, ld.size() * sizeof(double));
    } else {
        std::vector<lbfsi::StepMaps> mp;
        const int rc = download_maps(m, mp);
        if (rc) return rc;
        for (size_t b = 0; b < nb; ++b)
            for (int c = 0; c < 3; ++c) ld[b * 3 + c] = mp[b].loads[c];
    }
    cudaError_t e = cudaMemcpyAsync(m->d_loads_tmp, ld.data(), ld.size() * sizeof(double), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = lbfsi::launch_advance(m->d_bodies, m->d_loads_tmp, dt, m->nbatch, m->d_maps[m->curM], m->stream);
    m->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "advance_bodies");
    return check_status(m);
}

int lbfsi_get_body_state(lbfsi_mesh m, lbfsi_body_state* out) {
    if (!m || !out) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    std::vector<lbfsi::StepMaps> mp;
    const int rc = download_maps(m, mp);
    if (rc) return rc;
    for (int b = 0; b < m->nbatch; ++b) {
        out[b].h = mp[b].S_next.h;
        out[b].alpha = mp[b].S_next.alpha;
        out[b].hdot = mp[b].S_next.hdot;
        out[b].adot = mp[b].S_next.adot;
    }
    return LBFSI_OK;
}

int lbfsi_get_fields(lbfsi_mesh m, double* rho_u_T) {
    if (!m || !rho_u_T) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    int rc = download(m, m->d_M[m->cur], rho_u_T, (size_t)m->nbatch * 4 * m->N);
    if (rc) return rc;
    return check_status(m);
}

int lbfsi_get_populations(lbfsi_mesh m, int which, double* f, double* g) {
    if (!m || !f || !g) return fail(LBFSI_EINVAL, "null argument");
    if (which != 0 && which != 1) return fail(LBFSI_EINVAL, "which must be 0 or 1");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    const size_t cnt = (size_t)m->nbatch * 9 * m->N;
    const void* fs = m->d_f[m->cur];
    const void* gs = m->d_g[m->cur];
    if (which == 1 && !m->first) {
        cudaError_t e = cudaSuccess;
        if (!m->d_fpost) e = cudaMalloc(&m->d_fpost, cnt * m->esize);
        if (e == cudaSuccess && !m->d_gpost) e = cudaMalloc(&m->d_gpost, cnt * m->esize);
        if (e != cudaSuccess) return fail(LBFSI_ENOMEM, "post-collision staging allocation failed");
        lbfsi::StepArgs a = make_args(m, lbfsi::MODE_COLLIDE_ONLY);
        a.f_out = m->d_fpost;
        a.g_out = m->d_gpost;
        e = lbfsi::launch_step(a, m->precision, m->variant, m->stream);
        m->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "collide kernel launch");
        fs = m->d_fpost;
        gs = m->d_gpost;
    }
    int rc = download(m, fs, f, cnt);
    if (rc) return rc;
    rc = download(m, gs, g, cnt);
    if (rc) return rc;
    return check_status(m);
}

int lbfsi_set_populations(lbfsi_mesh m, const double* f, const double* g, const double* rho_u_T) {
    if (!m || !f || !g || !rho_u_T) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    const size_t cnt = (size_t)m->nbatch * 9 * m->N;
    int rc = upload(m, f, m->d_f[m->cur], cnt);
    if (!rc) rc = upload(m, g, m->d_g[m->cur], cnt);
    if (!rc) rc = upload(m, rho_u_T, m->d_M[m->cur], (size_t)m->nbatch * 4 * m->N);
    if (rc) return rc;
    m->first = false;
    return LBFSI_OK;
}

int64_t lbfsi_launch_count(lbfsi_mesh m) { return m ? m->launches : -1; }

}  // extern "C"
