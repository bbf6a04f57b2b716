// Fused time-step kernel of the two-population compressible semi-Lagrangian
// LBM on a blended O-grid (Sec. II-III of the paper), for sm_103a.
//
// One launch L_k advances the solver by one step in the order
//     collide(step k)  ->  stream(step k+1)
// which is the paper's stream-then-collide cycle shifted by half a step: the
// state kept in HBM between launches is the post-propagation (pre-collision)
// population set of step k, plus its moment field M^k.  Doing the collision
// first lets the correction term phi (a second derivative of moments of the
// *current* step, Sec. II C) use the moment field written by the previous
// launch, so the whole step is one kernel with no grid-wide dependency:
//
//   prologue   per-body RK4 with the loads of step k (Sec. III B), redundantly
//              in every CTA (identical, deterministic), and the blended maps
//              of steps k and k+1 (Sec. II D)
//   phase 1    stage M^k and the node coordinates of the tile +-4 nodes, and
//              the populations of the tile +-2 nodes, in shared memory
//   phase 2    correction fields: dQ on +-4, D = (mu/p) d(dQ) on +-3 (FE
//              gradients, Eq. ddx+fem, mapped by g^{-1}), collision of the
//              +-2 region in place (Eq. f_boltz)
//   phase 3    stream every tile node: c_hat = g^{-T} c - V_G, departure point,
//              bilinear inverse (Eq. depPnt) and Q2 interpolation (Eq.
//              SemiLagrProp) from the collided tile; wall nodes rebuild their
//              missing populations by Grad's approximation (Sec. III A); far
//              field nodes take equilibria at their targets; write the
//              populations and M^{k+1}; wall nodes add their share of the
//              force and moment (Sec. III) into a per-CTA partial.
//
// The redundant work is the collision of the 2-node halo; the HBM traffic per
// node is the 18 populations read and written once plus the 4-value moment
// field.
#include <cstdio>

#include "lbfsi_device.cuh"
#include "lbfsi_internal.h"

namespace lbfsi {

template <typename R>
struct Tol;
template <>
struct Tol<double> {
    static constexpr double newton = 1e-13;
    static constexpr double inside = 1e-12;
    static constexpr int maxit = 50;
};
template <>
struct Tol<float> {
    static constexpr float newton = 2e-7f;
    static constexpr float inside = 1e-4f;
    static constexpr int maxit = 8;
};

template <int TI, int TJ>
struct Tile {
    static constexpr int HP = 2, HD = 3, HM = 4;
    static constexpr int PH = TI + 2 * HP, PW = TJ + 2 * HP, PS = PH * PW;
    static constexpr int DH = TI + 2 * HD, DW = TJ + 2 * HD, DS = DH * DW;
    static constexpr int MH = TI + 2 * HM, MW = TJ + 2 * HM, MS = MH * MW;
    static constexpr int NT = TI * TJ;
};

template <typename R, int TI, int TJ>
constexpr size_t step_smem_bytes() {
    using T = Tile<TI, TJ>;
    return sizeof(R) * (size_t)(18 * T::PS + 4 * T::MS + 2 * T::MS + 2 * T::MS + 4 * T::DS + 2 * T::DS);
}

__device__ __forceinline__ int wrapj(int j, int nt) {
    j %= nt;
    return j < 0 ? j + nt : j;
}

// Derivative along an index direction of the 1-D quadratic Lagrange interpolant
// through a node and its neighbours, evaluated at the node: central inside,
// one-sided (-3 c0 + 4 c1 - c2)/2 on the first row, (3 cN - 4 cN-1 + cN-2)/2 on the
// last.  p points at the node, stride is the row pitch.
template <typename R>
__device__ __forceinline__ R d_row(const R* p, int stride, int i, int nr) {
    if (i == 0) return R(0.5) * (R(-3) * p[0] + R(4) * p[stride] - p[2 * stride]);
    if (i == nr - 1) return R(0.5) * (R(3) * p[0] - R(4) * p[-stride] + p[-2 * stride]);
    return R(0.5) * (p[stride] - p[-stride]);
}
template <typename R>
__device__ __forceinline__ R d_col(const R* p) {
    return R(0.5) * (p[1] - p[-1]);
}

// Locate P (relative to the node) in cell (ac, bc) (bc unwrapped) by Newton
// on the window's bilinear map (Eq. depPnt).  sX holds node coordinates
// relative to the tile reference on the +-HM region, (mi0, mj0) = global index
// of its first entry.  Returns true if P lies in that cell.
template <typename R, int MW>
__device__ __forceinline__ bool locate_cell(int ac, int bc, int nr, const R* sX, int MS, int mi0,
                                            int mj0, R nx, R ny, R Px, R Py, R gxi, R geta,
                                            bool use_guess, int& wa, int& wb, R& xi, R& eta) {
    if (ac < 0 || ac > nr - 2) return false;
    wa = min((ac >> 1) * 2, nr - 3);
    wb = (bc >> 1) * 2;  // arithmetic shift: floor for negative bc
    const int li = wa - mi0, lj = wb - mj0;
    const R* X0 = sX + li * MW + lj;
    const R* Y0 = X0 + MS;
    const R c00x = X0[0] - nx, c00y = Y0[0] - ny;
    const R c10x = X0[2 * MW] - nx, c10y = Y0[2 * MW] - ny;
    const R c01x = X0[2] - nx, c01y = Y0[2] - ny;
    const R c11x = X0[2 * MW + 2] - nx, c11y = Y0[2 * MW + 2] - ny;
    R x = R(0), y = R(0);
    if (use_guess) {
        x = gxi - R(wa + 1);
        y = geta - R(wb + 1);
    }
    for (int it = 0; it < Tol<R>::maxit; ++it) {
        const R n00 = R(0.25) * (R(1) - x) * (R(1) - y), n10 = R(0.25) * (R(1) + x) * (R(1) - y);
        const R n01 = R(0.25) * (R(1) - x) * (R(1) + y), n11 = R(0.25) * (R(1) + x) * (R(1) + y);
        const R rx = n00 * c00x + n10 * c10x + n01 * c01x + n11 * c11x - Px;
        const R ry = n00 * c00y + n10 * c10y + n01 * c01y + n11 * c11y - Py;
        const R dxix = R(0.25) * ((c10x - c00x) * (R(1) - y) + (c11x - c01x) * (R(1) + y));
        const R dxiy = R(0.25) * ((c10y - c00y) * (R(1) - y) + (c11y - c01y) * (R(1) + y));
        const R detx = R(0.25) * ((c01x - c00x) * (R(1) - x) + (c11x - c10x) * (R(1) + x));
        const R dety = R(0.25) * ((c01y - c00y) * (R(1) - x) + (c11y - c10y) * (R(1) + x));
        const R det = dxix * dety - dxiy * detx;
        const R sx = -(dety * rx - detx * ry) / det;
        const R sy = -(-dxiy * rx + dxix * ry) / det;
        x += sx;
        y += sy;
        if (!(fabs(sx) >= Tol<R>::newton || fabs(sy) >= Tol<R>::newton)) break;
        if (!(fabs(x) < R(4) && fabs(y) < R(4))) break;
    }
    xi = x;
    eta = y;
    const R la = R(ac - wa), lb = R(bc - wb);
    const R t = Tol<R>::inside;
    return (x >= la - R(1) - t) && (x <= la + t) && (y >= lb - R(1) - t) && (y <= lb + t);
}

// Try the guessed cell first, then the four cells around node (i, j) in the
// fixed order (i-1,j-1), (i-1,j), (i,j-1), (i,j).
template <typename R, int MW>
__device__ __forceinline__ bool locate(int i, int j, int nr, const R* sX, int MS, int mi0, int mj0,
                                       R nx, R ny, R Px, R Py, R dxi, R deta, bool use_guess,
                                       int& wa, int& wb, R& xi, R& eta) {
    int ga = -2, gb = -2;
    if (use_guess) {
        ga = dxi < R(0) ? -1 : 0;
        gb = deta < R(0) ? -1 : 0;
        if (locate_cell<R, MW>(i + ga, j + gb, nr, sX, MS, mi0, mj0, nx, ny, Px, Py, R(i) + dxi,
                               R(j) + deta, true, wa, wb, xi, eta))
            return true;
    }
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
        const int da = (c < 2) ? -1 : 0, db = (c & 1) ? 0 : -1;
        if (da == ga && db == gb) continue;
        if (locate_cell<R, MW>(i + da, j + db, nr, sX, MS, mi0, mj0, nx, ny, Px, Py, R(0), R(0),
                               false, wa, wb, xi, eta))
            return true;
    }
    return false;
}

template <typename R>
__device__ __forceinline__ void lagrange3(R t, R* L) {
    L[0] = R(0.5) * t * (t - R(1));
    L[1] = R(1) - t * t;
    L[2] = R(0.5) * t * (t + R(1));
}

template <typename R, int TI, int TJ>
__global__ void __launch_bounds__(TI* TJ) k_step(const StepArgs a) {
    using T = Tile<TI, TJ>;
    extern __shared__ __align__(16) unsigned char smraw[];
    R* sp = reinterpret_cast<R*>(smraw);   // [18][PS] populations (f then g)
    R* sM = sp + 18 * T::PS;               // [4][MS]  rho, ux, uy, T of step k
    R* sX = sM + 4 * T::MS;                // [2][MS]  node coordinates - X(i0, j0)
    R* sQ = sX + 2 * T::MS;                // [2][MS]  dQ_x, dQ_y
    R* sG = sQ + 2 * T::MS;                // [4][DS]  g^{-1} J^{-1}: (C_xi, C_eta) -> grad_x C
    R* sD = sG + 4 * T::DS;                // [2][DS]  D_x, D_y

    __shared__ BodyMap<R> mapK, mapS;
    __shared__ BodyMap<double> mapSd;
    __shared__ R s_dr[T::MH];
    __shared__ R s_ex[T::MW], s_ey[T::MW], s_dex[T::MW], s_dey[T::MW];
    __shared__ R s_X0[2];
    __shared__ double s_red[3][TJ];

    const int tid = threadIdx.x;
    const int b = blockIdx.z;
    const int j0 = blockIdx.x * TJ, i0 = blockIdx.y * TI;
    const int nr = a.nr, nt = a.nt, N = a.N;
    const size_t off9 = (size_t)b * 9 * N, off4 = (size_t)b * 4 * N;
    const R* __restrict__ f_in = reinterpret_cast<const R*>(a.f_in) + off9;
    const R* __restrict__ g_in = reinterpret_cast<const R*>(a.g_in) + off9;
    R* __restrict__ f_out = reinterpret_cast<R*>(a.f_out) + off9;
    R* __restrict__ g_out = reinterpret_cast<R*>(a.g_out) + off9;
    const R* __restrict__ M_in = reinterpret_cast<const R*>(a.M_in) + off4;
    R* __restrict__ M_out = reinterpret_cast<R*>(a.M_out) + off4;
    const R dt = (R)a.dt, mu = (R)a.mu, Cv = (R)a.Cv, Pr = (R)a.Pr;
    const bool collide = a.mode != MODE_STREAM_ONLY;
    const bool stream = a.mode != MODE_COLLIDE_ONLY;

    // ---- prologue: body update and blended maps --------------------------
    if (tid == 0) {
        const BodyDev bd = a.bodies[b];
        const BodyStateDev Sk = a.S_in[b];
        BodyStateDev Snew = Sk, Sold = Sk;
        double F[3] = {0.0, 0.0, 0.0};
        if (a.mode == MODE_COLLIDE_STREAM) {
            for (int t = 0; t < a.ntj; ++t)
                for (int c = 0; c < 3; ++c) F[c] += a.part_in[((size_t)b * a.ntj + t) * 3 + c];
            Snew = a.S_force ? a.S_force[b] : rk4_body(bd, Sk, F[1], F[2], a.dt);
            Sold = Sk;
        } else if (a.mode == MODE_STREAM_ONLY) {
            Sold = a.S_prev0[b];
        }
        mapK = make_body_map<R>(bd, Sk, Sk, a.dt);
        mapS = make_body_map<R>(bd, Snew, Sold, a.dt);
        mapSd = make_body_map<double>(bd, Snew, Sold, a.dt);
        if (blockIdx.x == 0 && blockIdx.y == 0 && stream) {
            a.S_out[b] = Snew;
            if (a.loads_out)
                for (int c = 0; c < 3; ++c) a.loads_out[b * 3 + c] = F[c];
        }
        s_X0[0] = (R)(a.xm + a.r[i0] * a.e[2 * j0]);
        s_X0[1] = (R)(a.ym + a.r[i0] * a.e[2 * j0 + 1]);
    }
    const int mi0 = i0 - T::HM, mj0 = j0 - T::HM;   // global index of sM/sX entry (0,0)
    for (int t = tid; t < T::MH; t += T::NT) {
        const int i = min(max(mi0 + t, 0), nr - 1);
        s_dr[t] = (R)(a.r[i] - a.r[i0]);
    }
    for (int t = tid; t < T::MW; t += T::NT) {
        const int j = wrapj(mj0 + t, nt);
        s_ex[t] = (R)a.e[2 * j];
        s_ey[t] = (R)a.e[2 * j + 1];
        s_dex[t] = (R)(a.e[2 * j] - a.e[2 * j0]);
        s_dey[t] = (R)(a.e[2 * j + 1] - a.e[2 * j0 + 1]);
    }
    __syncthreads();

    // ---- phase 1: stage coordinates, M^k and populations ------------------
    const R r0 = (R)a.r[i0];
    for (int idx = tid; idx < T::MS; idx += T::NT) {
        const int li = idx / T::MW, lj = idx - li * T::MW;
        const int i = mi0 + li;
        sX[idx] = s_dr[li] * s_ex[lj] + r0 * s_dex[lj];
        sX[T::MS + idx] = s_dr[li] * s_ey[lj] + r0 * s_dey[lj];
        if (i >= 0 && i < nr) {
            const int n = i * nt + wrapj(mj0 + lj, nt);
#pragma unroll
            for (int c = 0; c < 4; ++c) sM[c * T::MS + idx] = M_in[(size_t)c * N + n];
        }
    }
    const int pi0 = i0 - T::HP, pj0 = j0 - T::HP;
    for (int idx = tid; idx < T::PS; idx += T::NT) {
        const int li = idx / T::PW, lj = idx - li * T::PW;
        const int i = pi0 + li;
        if (i >= 0 && i < nr) {
            const int n = i * nt + wrapj(pj0 + lj, nt);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                sp[q * T::PS + idx] = f_in[(size_t)q * N + n];
                sp[(9 + q) * T::PS + idx] = g_in[(size_t)q * N + n];
            }
        }
    }
    __syncthreads();

    // ---- phase 2: correction fields and collision of step k --------------
    if (collide) {
        for (int idx = tid; idx < T::MS; idx += T::NT) {
            const int i = mi0 + idx / T::MW;
            if (i < 0 || i >= nr) continue;
            const R rho = sM[idx], ux = sM[T::MS + idx], uy = sM[2 * T::MS + idx], Tn = sM[3 * T::MS + idx];
            sQ[idx] = rho * ux * (R(1) - R(3) * Tn) - rho * ux * ux * ux;
            sQ[T::MS + idx] = rho * uy * (R(1) - R(3) * Tn) - rho * uy * uy * uy;
        }
        // gradient maps G = F^{-T} J^{-1} on the +-3 region (step-k kinematics)
        for (int idx = tid; idx < T::DS; idx += T::NT) {
            const int li = idx / T::DW, lj = idx - li * T::DW;
            const int i = i0 - T::HD + li;
            if (i < 0 || i >= nr) continue;
            const int m = (li + 1) * T::MW + (lj + 1);
            const R xxi = d_row(sX + m, T::MW, i, nr), yxi = d_row(sX + T::MS + m, T::MW, i, nr);
            const R xet = d_col(sX + m), yet = d_col(sX + T::MS + m);
            const R detJ = xxi * yet - yxi * xet;
            const R j00 = yet / detJ, j01 = -yxi / detJ, j10 = -xet / detJ, j11 = xxi / detJ;
            R F00, F01, F10, F11, vx, vy;
            kinematics(mapK, s_X0[0] + sX[m], s_X0[1] + sX[T::MS + m], F00, F01, F10, F11, vx, vy);
            const R dF = F00 * F11 - F01 * F10;
            const R i00 = F11 / dF, i01 = -F01 / dF, i10 = -F10 / dF, i11 = F00 / dF;  // F^{-1}
            // grad_x = F^{-T} grad_X, grad_X = Jinv (C_xi, C_eta)
            sG[idx] = i00 * j00 + i10 * j10;
            sG[T::DS + idx] = i00 * j01 + i10 * j11;
            sG[2 * T::DS + idx] = i01 * j00 + i11 * j10;
            sG[3 * T::DS + idx] = i01 * j01 + i11 * j11;
        }
        __syncthreads();
        for (int idx = tid; idx < T::DS; idx += T::NT) {
            const int li = idx / T::DW, lj = idx - li * T::DW;
            const int i = i0 - T::HD + li;
            if (i < 0 || i >= nr) continue;
            const int m = (li + 1) * T::MW + (lj + 1);
            const R mup = mu / (sM[m] * sM[3 * T::MS + m]);
            const R qx_xi = d_row(sQ + m, T::MW, i, nr), qx_et = d_col(sQ + m);
            const R qy_xi = d_row(sQ + T::MS + m, T::MW, i, nr), qy_et = d_col(sQ + T::MS + m);
            sD[idx] = mup * (sG[idx] * qx_xi + sG[T::DS + idx] * qx_et);
            sD[T::DS + idx] = mup * (sG[2 * T::DS + idx] * qy_xi + sG[3 * T::DS + idx] * qy_et);
        }
        __syncthreads();
        for (int idx = tid; idx < T::PS; idx += T::NT) {
            const int li = idx / T::PW, lj = idx - li * T::PW;
            const int i = pi0 + li;
            if (i < 0 || i >= nr) continue;
            R f[9], g[9];
            if (i == nr - 1) {
                const int m = (li + 2) * T::MW + (lj + 2);
                f_equilibrium(sM[m], sM[T::MS + m], sM[2 * T::MS + m], sM[3 * T::MS + m], f);
                g_equilibrium(sM[m], sM[T::MS + m], sM[2 * T::MS + m], sM[3 * T::MS + m], Cv, g);
            } else {
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    f[q] = sp[q * T::PS + idx];
                    g[q] = sp[(9 + q) * T::PS + idx];
                }
                const int d = (li + 1) * T::DW + (lj + 1);
                const R dx_xi = d_row(sD + d, T::DW, i, nr), dx_et = d_col(sD + d);
                const R dy_xi = d_row(sD + T::DS + d, T::DW, i, nr), dy_et = d_col(sD + T::DS + d);
                const R Yx = sG[d] * dx_xi + sG[T::DS + d] * dx_et;
                const R Yy = sG[2 * T::DS + d] * dy_xi + sG[3 * T::DS + d] * dy_et;
                collide_node(f, g, Yx, Yy, mu, dt, Cv, Pr);
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                sp[q * T::PS + idx] = f[q];
                sp[(9 + q) * T::PS + idx] = g[q];
            }
        }
        __syncthreads();
        if (!stream) {
            const int ti = tid / TJ, tj = tid - (tid / TJ) * TJ;
            const int i = i0 + ti, j = j0 + tj;
            if (i < nr && j < nt) {
                const int n = i * nt + j;
                const int p = (ti + T::HP) * T::PW + tj + T::HP;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    f_out[(size_t)q * N + n] = sp[q * T::PS + p];
                    g_out[(size_t)q * N + n] = sp[(9 + q) * T::PS + p];
                }
            }
            return;
        }
    }

    // ---- phase 3: stream step k+1 ----------------------------------------
    const int ti = tid / TJ, tj = tid - (tid / TJ) * TJ;
    const int i = i0 + ti, j = j0 + tj;
    double fcx = 0.0, fcy = 0.0, fcm = 0.0;
    if (i < nr && j < nt) {
        const int n = i * nt + j;
        const int m = (ti + T::HM) * T::MW + tj + T::HM;   // node in M/X coords
        if (i == nr - 1) {
            // far field (Sec. III A 2): inlet where the free stream enters,
            // zero-gradient outlet elsewhere (targets of the previous step)
            const double un = a.uinf_x * a.e[2 * j] + a.uinf_y * a.e[2 * j + 1];
            R rho, ux, uy, Tt;
            if (un < 0.0) {
                rho = (R)a.rho_inf; ux = (R)a.uinf_x; uy = (R)a.uinf_y; Tt = (R)a.T_inf;
            } else {
                const int mm = m - T::MW;
                rho = sM[mm]; ux = sM[T::MS + mm]; uy = sM[2 * T::MS + mm]; Tt = sM[3 * T::MS + mm];
            }
            R f[9], g[9];
            f_equilibrium(rho, ux, uy, Tt, f);
            g_equilibrium(rho, ux, uy, Tt, Cv, g);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                f_out[(size_t)q * N + n] = f[q];
                g_out[(size_t)q * N + n] = g[q];
            }
            M_out[n] = rho; M_out[(size_t)N + n] = ux; M_out[(size_t)2 * N + n] = uy;
            M_out[(size_t)3 * N + n] = Tt;
        } else {
            const R nx = sX[m], ny = sX[T::MS + m];
            R F00, F01, F10, F11, vx, vy;
            kinematics(mapS, s_X0[0] + nx, s_X0[1] + ny, F00, F01, F10, F11, vx, vy);
            const R dF = F00 * F11 - F01 * F10;
            const R i00 = F11 / dF, i01 = -F01 / dF, i10 = -F10 / dF, i11 = F00 / dF;
            // node-centred metric for the index-space guess of each departure cell
            const R xxi = d_row(sX + m, T::MW, i, nr), yxi = d_row(sX + T::MS + m, T::MW, i, nr);
            const R xet = d_col(sX + m), yet = d_col(sX + T::MS + m);
            const R detJ = xxi * yet - yxi * xet;
            unsigned missing = 0u;
            R fw[9], gw[9];
            if (i == 0) {
                // missing populations: departure point inside the body,
                // c_hat . n0 > 0, decided in float64 (Sec. III A)
                const double Xd = a.xm + a.r[0] * a.e[2 * j], Yd = a.ym + a.r[0] * a.e[2 * j + 1];
                double D00, D01, D10, D11, dvx, dvy;
                kinematics(mapSd, Xd, Yd, D00, D01, D10, D11, dvx, dvy);
                const double dd = D00 * D11 - D01 * D10;
                const double n0x = a.n0[2 * j], n0y = a.n0[2 * j + 1];
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const double cx = cxq(q), cy = cyq(q);
                    const double hx = (D11 * cx - D01 * cy) / dd - dvx;
                    const double hy = (-D10 * cx + D00 * cy) / dd - dvy;
                    if (hx * n0x + hy * n0y > 1e-12) missing |= 1u << q;
                }
                if (missing) {
                    // targets: rho, T at B = A + dt n0 by Q2 interpolation of
                    // M^k; u = wall velocity; gradients of M^k at the wall node
                    const R Px = dt * (R)n0x, Py = dt * (R)n0y;
                    int wa, wb;
                    R xi, eta;
                    bool ok = locate<R, T::MW>(0, j, nr, sX, T::MS, mi0, mj0, nx, ny, Px, Py, R(0),
                                               R(0), false, wa, wb, xi, eta);
                    R rhoB = sM[m], TB = sM[3 * T::MS + m];
                    if (ok) {
                        R Lx[3], Ly[3];
                        lagrange3(xi, Lx);
                        lagrange3(eta, Ly);
                        const int w0 = (wa - mi0) * T::MW + (wb - mj0);
                        rhoB = R(0);
                        TB = R(0);
#pragma unroll
                        for (int aa = 0; aa < 3; ++aa)
#pragma unroll
                            for (int bb = 0; bb < 3; ++bb) {
                                const R wgt = Lx[aa] * Ly[bb];
                                rhoB += wgt * sM[w0 + aa * T::MW + bb];
                                TB += wgt * sM[3 * T::MS + w0 + aa * T::MW + bb];
                            }
                    } else {
                        atomicOr(a.status, ST_BPOINT);
                    }
                    const R j00 = yet / detJ, j01 = -yxi / detJ, j10 = -xet / detJ, j11 = xxi / detJ;
                    const R G00 = i00 * j00 + i10 * j10, G01 = i00 * j01 + i10 * j11;
                    const R G10 = i01 * j00 + i11 * j10, G11 = i01 * j01 + i11 * j11;
                    R gr[3][2];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const R* p = sM + (c + 1) * T::MS + m;
                        const R cxi = d_row(p, T::MW, 0, nr), cet = d_col(p);
                        gr[c][0] = G00 * cxi + G01 * cet;
                        gr[c][1] = G10 * cxi + G11 * cet;
                    }
                    grad_populations(rhoB, vx, vy, TB, gr[0][0], gr[0][1], gr[1][0], gr[1][1],
                                     gr[2][0], gr[2][1], mu, dt, Cv, Pr, fw, gw);
                }
            }
            R f[9], g[9];
            bool lost = false;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                if (missing & (1u << q)) {
                    f[q] = fw[q];
                    g[q] = gw[q];
                    continue;
                }
                const R cx = (R)cxq(q), cy = (R)cyq(q);
                const R hx = i00 * cx + i01 * cy - vx, hy = i10 * cx + i11 * cy - vy;
                const R Px = -dt * hx, Py = -dt * hy;
                const R dxi = (yet * Px - xet * Py) / detJ;
                const R deta = (-yxi * Px + xxi * Py) / detJ;
                int wa, wb;
                R xi, eta;
                if (locate<R, T::MW>(i, j, nr, sX, T::MS, mi0, mj0, nx, ny, Px, Py, dxi, deta, true,
                                     wa, wb, xi, eta)) {
                    R Lx[3], Ly[3];
                    lagrange3(xi, Lx);
                    lagrange3(eta, Ly);
                    const int p0 = (wa - pi0) * T::PW + (wb - pj0);
                    R sf = R(0), sg = R(0);
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
                        for (int bb = 0; bb < 3; ++bb) {
                            const R wgt = Lx[aa] * Ly[bb];
                            const int p = p0 + aa * T::PW + bb;
                            sf += wgt * sp[q * T::PS + p];
                            sg += wgt * sp[(9 + q) * T::PS + p];
                        }
                    f[q] = sf;
                    g[q] = sg;
                } else {
                    lost = true;
                    const int p = (ti + T::HP) * T::PW + tj + T::HP;
                    f[q] = sp[q * T::PS + p];
                    g[q] = sp[(9 + q) * T::PS + p];
                }
            }
            if (lost) atomicOr(a.status, ST_DEPARTURE);
            const Macro<R> mc = moments(f, g, Cv);
            if (!(mc.rho > R(0)) || !(mc.T > R(0)) || !isfinite(mc.ux) || !isfinite(mc.uy))
                atomicOr(a.status, ST_NONPHYS);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                f_out[(size_t)q * N + n] = f[q];
                g_out[(size_t)q * N + n] = g[q];
            }
            M_out[n] = mc.rho; M_out[(size_t)N + n] = mc.ux; M_out[(size_t)2 * N + n] = mc.uy;
            M_out[(size_t)3 * N + n] = mc.T;
            if (i == 0) {
                // wall stress sigma = -p I - (1 - omega/2) P^(1), P^(1) = sum (f - f^eq) c c
                // (Sec. III), this node's Simpson share of its edges, float64
                R feq[9];
                f_equilibrium(mc.rho, mc.ux, mc.uy, mc.T, feq);
                double pxx = 0, pxy = 0, pyy = 0;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const double fn = (double)f[q] - (double)feq[q];
                    pxx += cxq(q) * cxq(q) * fn;
                    pxy += cxq(q) * cyq(q) * fn;
                    pyy += cyq(q) * cyq(q) * fn;
                }
                const double rho = mc.rho, Tn = mc.T;
                const double om = 1.0 / (0.5 + a.mu / (rho * Tn * a.dt));
                const double p = rho * Tn, am = 1.0 - 0.5 * om;
                const double sxx = -p - am * pxx, sxy = -am * pxy, syy = -p - am * pyy;
                const double R00 = 1.0 + mapSd.a00, R01 = mapSd.a01, R10 = mapSd.a10, R11 = 1.0 + mapSd.a11;
                const BodyDev& bd = a.bodies[b];
                const double Xd = a.xm + a.r[0] * a.e[2 * j] - bd.xp;
                const double Yd = a.ym + a.r[0] * a.e[2 * j + 1] - bd.yp;
                const double rx = R00 * Xd + R01 * Yd, ry = R10 * Xd + R11 * Yd;
                const double* wg = a.wall_geo + 6 * j;
#pragma unroll
                for (int e2 = 0; e2 < 2; ++e2) {
                    const double wds = wg[3 * e2], ex = wg[3 * e2 + 1], ey = wg[3 * e2 + 2];
                    const double nxr = R00 * ex + R01 * ey, nyr = R10 * ex + R11 * ey;
                    const double tx = sxx * nxr + sxy * nyr, ty = sxy * nxr + syy * nyr;
                    fcx += wds * tx;
                    fcy += wds * ty;
                    fcm += wds * (rx * ty - ry * tx);
                }
            }
        }
    }
    if (blockIdx.y == 0) {
        if (ti == 0) {
            s_red[0][tj] = fcx;
            s_red[1][tj] = fcy;
            s_red[2][tj] = fcm;
        }
        __syncthreads();
        if (tid == 0) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            for (int t = 0; t < TJ; ++t) {
                s0 += s_red[0][t];
                s1 += s_red[1][t];
                s2 += s_red[2][t];
            }
            double* po = a.part_out + ((size_t)b * a.ntj + blockIdx.x) * 3;
            po[0] = s0;
            po[1] = s1;
            po[2] = s2;
        }
    }
}

// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_init(const double* __restrict__ M, R* __restrict__ f, R* __restrict__ g,
                       R* __restrict__ Mout, int N, int nbatch, double Cv) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)N * nbatch) return;
    const size_t b = t / N, n = t - b * N;
    const double* Mb = M + b * 4 * N;
    const R rho = (R)Mb[n], ux = (R)Mb[N + n], uy = (R)Mb[2 * (size_t)N + n], T = (R)Mb[3 * (size_t)N + n];
    R fe[9], ge[9];
    f_equilibrium(rho, ux, uy, T, fe);
    g_equilibrium(rho, ux, uy, T, (R)Cv, ge);
    for (int q = 0; q < 9; ++q) {
        f[(b * 9 + q) * N + n] = fe[q];
        g[(b * 9 + q) * N + n] = ge[q];
    }
    for (int c = 0; c < 4; ++c) Mout[(b * 4 + c) * N + n] = (R)Mb[c * (size_t)N + n];
}

__global__ void k_reduce_loads(const double* __restrict__ part, int ntj, int nbatch,
                               double* __restrict__ loads) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbatch) return;
    double s[3] = {0.0, 0.0, 0.0};
    for (int t = 0; t < ntj; ++t)
        for (int c = 0; c < 3; ++c) s[c] += part[((size_t)b * ntj + t) * 3 + c];
    for (int c = 0; c < 3; ++c) loads[b * 3 + c] = s[c];
}

__global__ void k_advance(const BodyDev* __restrict__ bodies, const BodyStateDev* __restrict__ S,
                          const double* __restrict__ loads, double dt, int nbatch,
                          BodyStateDev* __restrict__ S_out, BodyStateDev* __restrict__ S_prev_out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbatch) return;
    const BodyStateDev s = S[b];
    const BodyStateDev n = rk4_body(bodies[b], s, loads[b * 3 + 1], loads[b * 3 + 2], dt);
    if (S_prev_out) S_prev_out[b] = s;
    S_out[b] = n;
}

// Tile shapes: 8 radial x 32 angular nodes (one warp per radial row).
constexpr int TI = 8, TJ = 32;

template <typename R>
static cudaError_t launch_step_t(const StepArgs& a, cudaStream_t s) {
    const size_t smem = step_smem_bytes<R, TI, TJ>();
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_step<R, TI, TJ>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((a.nt + TJ - 1) / TJ, (a.nr + TI - 1) / TI, a.nbatch);
    k_step<R, TI, TJ><<<grid, TI * TJ, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_step(const StepArgs& a, int precision, cudaStream_t s) {
    return precision == 0 ? launch_step_t<double>(a, s) : launch_step_t<float>(a, s);
}

int tiles_j(int nt) { return (nt + TJ - 1) / TJ; }

cudaError_t launch_init(int precision, const double* M, void* f, void* g, void* Mout, int N,
                        int nbatch, double Cv, cudaStream_t s) {
    const size_t total = (size_t)N * nbatch;
    const int bs = 256;
    const unsigned nb = (unsigned)((total + bs - 1) / bs);
    if (precision == 0)
        k_init<double><<<nb, bs, 0, s>>>(M, (double*)f, (double*)g, (double*)Mout, N, nbatch, Cv);
    else
        k_init<float><<<nb, bs, 0, s>>>(M, (float*)f, (float*)g, (float*)Mout, N, nbatch, Cv);
    return cudaGetLastError();
}

cudaError_t launch_reduce_loads(const double* part, int ntj, int nbatch, double* loads,
                                cudaStream_t s) {
    k_reduce_loads<<<(nbatch + 127) / 128, 128, 0, s>>>(part, ntj, nbatch, loads);
    return cudaGetLastError();
}

cudaError_t launch_advance(const BodyDev* bodies, const BodyStateDev* S, const double* loads,
                           double dt, int nbatch, BodyStateDev* S_out, BodyStateDev* S_prev_out,
                           cudaStream_t s) {
    k_advance<<<(nbatch + 127) / 128, 128, 0, s>>>(bodies, S, loads, dt, nbatch, S_out, S_prev_out);
    return cudaGetLastError();
}

}  // namespace lbfsi
