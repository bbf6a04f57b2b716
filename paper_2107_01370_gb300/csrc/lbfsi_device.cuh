// Device-side physics of the two-population compressible lattice Boltzmann
// step (Sec. II C of the paper): equilibria, correction terms, collision,
// Grad's approximation (Sec. III A), blended-mesh kinematics (Sec. II A, II D)
// and the rigid-body RK4 (Sec. III B).  Templated on the arithmetic type R
// (double for the FP64 path, float for the FP32 path).
#pragma once

#include <cuda_runtime.h>
#include "lbfsi_internal.h"

namespace lbfsi {

// D2Q9 velocity of index q: 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1)
// 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).  Resolved at compile time in unrolled loops.
__host__ __device__ constexpr int cxq(int q) {
    return (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cyq(int q) {
    return (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0);
}

// Reciprocal and square root in the precision of the path: the hardware
// approximations (relative error about 2^-23) on the float path, IEEE
// operations on the float64 path.
__device__ __forceinline__ float rcp_(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__host__ __device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float sqrt_(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float abs_(float x) { return fabsf(x); }
__device__ __forceinline__ double abs_(double x) { return fabs(x); }
// Arithmetic with its rounding fixed: the compiler neither fuses nor splits
// these, so an expression written with them rounds the same way in every
// kernel it is inlined into (a Newton iterate then converges to the same
// last bit whatever the tile shape or launch form).
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

template <typename R>
struct Macro {
    R rho, ux, uy, T, E;
};

// rho = sum f, rho u = sum f c, 2 rho E = sum g, T = (E - u^2/2) / Cv.
template <typename R>
__device__ __forceinline__ Macro<R> moments(const R* f, const R* g, R Cv) {
    R rho = 0, jx = 0, jy = 0, s2 = 0;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        rho += f[q];
        jx += (R)cxq(q) * f[q];
        jy += (R)cyq(q) * f[q];
        s2 += g[q];
    }
    Macro<R> m;
    const R ir = rcp_(rho);
    m.rho = rho;
    m.ux = jx * ir;
    m.uy = jy * ir;
    m.E = R(0.5) * s2 * ir;
    m.T = (m.E - R(0.5) * (m.ux * m.ux + m.uy * m.uy)) * rcp_(Cv);
    return m;
}

// Product-form equilibrium f_i^eq = rho Phi_{cx}(u_x) Phi_{cy}(u_y) (Eq. feq).
template <typename R>
__host__ __device__ __forceinline__ void f_equilibrium(R rho, R ux, R uy, R T, R* f) {
    R ax = ux * ux + T, ay = uy * uy + T;
    R px[3] = {R(0.5) * (ax - ux), R(1) - ax, R(0.5) * (ax + ux)};   // index c+1
    R py[3] = {R(0.5) * (ay - uy), R(1) - ay, R(0.5) * (ay + uy)};
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q] = rho * px[cxq(q) + 1] * py[cyq(q) + 1];
}

// g = W_i (2 rho E + q.c/T + (R^eq - 2 rho E T I):(c c - T I)/(2T^2)) + Psi_i
// (Eqs. geq, gstar).  H = E + T (energy flux of the enthalpy), R^eq as printed,
// Psi_i = B_i . X with B_0 = (1,1), B_{1,3} = (-1/2,0), B_{2,4} = (0,-1/2).
template <typename R>
__host__ __device__ __forceinline__ void g_hermite(R rho, R ux, R uy, R T, R E, R qx, R qy, R* g) {
    const R uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    // A = R^eq - 2 rho E T I
    const R axx = R(2) * rho * E * uxx + R(2) * rho * T * (T + R(2) * uxx);
    const R ayy = R(2) * rho * E * uyy + R(2) * rho * T * (T + R(2) * uyy);
    const R axy = R(2) * rho * E * uxy + R(4) * rho * T * uxy;
    const R invT = rcp_(T);
    const R inv2T2 = R(0.5) * invT * invT;
    const R pre = rho * (R(1) - R(3) * T) * invT;
    const R Xx = pre * (T * T + R(2) * uxx * T + E * uxx);
    const R Xy = pre * (T * T + R(2) * uyy * T + E * uyy);
    const R w[3] = {R(0.5) * T, R(1) - T, R(0.5) * T};
    const R twoRhoE = R(2) * rho * E;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int cx = cxq(q), cy = cyq(q);
        const R herm = (axx * (R(cx * cx) - T) + R(2) * axy * R(cx * cy) + ayy * (R(cy * cy) - T)) * inv2T2;
        R v = w[cx + 1] * w[cy + 1] * (twoRhoE + (qx * R(cx) + qy * R(cy)) * invT + herm);
        if (q == 0) v += Xx + Xy;
        if (q == 1 || q == 3) v -= R(0.5) * Xx;
        if (q == 2 || q == 4) v -= R(0.5) * Xy;
        g[q] = v;
    }
}

template <typename R>
__host__ __device__ __forceinline__ void g_equilibrium(R rho, R ux, R uy, R T, R Cv, R* g) {
    const R E = Cv * T + R(0.5) * (ux * ux + uy * uy);
    const R H2 = R(2) * rho * (E + T);
    g_hermite(rho, ux, uy, T, E, H2 * ux, H2 * uy, g);
}

// Lane-wise arithmetic on (f_q, g_q) pairs: packed FP32x2 instructions on the
// float path (one instruction for both populations of a direction).
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 psub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 pair(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 pair(double a, double b) { return make_double2(a, b); }

// Collision at one node (Eq. f_boltz) on its (f_q, g_q) pairs p[9]:
// f* = f + w (f^eq - f) + dt phi, g* = g + w (g^eq - g) + (w1 - w)(g^qe - g).
// phi_i = -(1/2) c_i . Y on the axis velocities; q* = q^eq + 2 u.(P - P^eq);
// 1/w = 1/2 + mu/(rho T dt), 1/w1 = 1/2 + (1/w - 1/2)/Pr.  g^qe differs from
// g^eq only in the heat flux, so both come from one Hermite expansion, whose
// (R^eq - 2 rho E T I):(c c - T I)/(2T^2) term takes five values (rest,
// x-axis, y-axis and the two diagonal pairs).
template <typename R, typename R2>
__device__ __forceinline__ void collide_pairs(R2* p, R Yx, R Yy, R mu, R dt, R Cv, R iPr) {
    // rho = sum f, 2 rho E = sum g, rho u = sum f c, P = sum f c c
    R2 s = p[0];
#pragma unroll
    for (int q = 1; q < 9; ++q) s = padd(s, p[q]);
    const R rho = s.x, twoRhoE = s.y;
    const R jx = ((p[1].x - p[3].x) + (p[5].x - p[6].x)) + (p[8].x - p[7].x);
    const R jy = ((p[2].x - p[4].x) + (p[5].x - p[8].x)) + (p[6].x - p[7].x);
    const R sd = (p[5].x + p[6].x) + (p[7].x + p[8].x);
    const R pxx = (p[1].x + p[3].x) + sd, pyy = (p[2].x + p[4].x) + sd;
    const R pxy = (p[5].x - p[6].x) + (p[7].x - p[8].x);
    const R ir = rcp_(rho);
    const R ux = jx * ir, uy = jy * ir;
    const R E = R(0.5) * twoRhoE * ir;
    const R uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    const R T = (E - R(0.5) * (uxx + uyy)) * rcp_(Cv);
    const R tau = R(0.5) + mu * rcp_(rho * T * dt);
    const R om = rcp_(tau);
    const R om1 = rcp_(R(0.5) + (tau - R(0.5)) * iPr);
    const R dom = om1 - om;
    const R dxx = pxx - rho * (uxx + T);
    const R dxy = pxy - rho * uxy;
    const R dyy = pyy - rho * (uyy + T);
    const R invT = rcp_(T);
    // heat flux of g^eq (2 rho H u) and the quasi-equilibrium shift
    // q* - q^eq = 2 u.(P - P^eq), both over T
    const R H2 = R(2) * rho * (E + T) * invT;
    const R qx = H2 * ux, qy = H2 * uy;
    const R dqx = R(2) * (ux * dxx + uy * dxy) * invT, dqy = R(2) * (ux * dxy + uy * dyy) * invT;
    const R rT2 = R(2) * rho * T;
    const R axx = twoRhoE * uxx + rT2 * (T + R(2) * uxx);
    const R ayy = twoRhoE * uyy + rT2 * (T + R(2) * uyy);
    const R axy = twoRhoE * uxy + R(2) * rT2 * uxy;
    const R inv2T2 = R(0.5) * invT * invT;
    const R A = axx + ayy, TA = T * A;
    const R h0 = -TA * inv2T2, hx = (axx - TA) * inv2T2, hy = (ayy - TA) * inv2T2;
    const R hd = (A - TA) * inv2T2, hxy = R(2) * axy * inv2T2;
    const R pre = rho * (R(1) - R(3) * T) * invT;
    const R Xx = pre * (T * T + R(2) * uxx * T + E * uxx);
    const R Xy = pre * (T * T + R(2) * uyy * T + E * uyy);
    const R ax = uxx + T, ay = uyy + T;
    const R px[3] = {R(0.5) * (ax - ux), R(1) - ax, R(0.5) * (ax + ux)};
    const R py[3] = {R(0.5) * (ay - uy), R(1) - ay, R(0.5) * (ay + uy)};
    const R w0 = R(0.5) * T, w1 = R(1) - T;
    const R Wr = w1 * w1, Wa = w0 * w1, Wd = w0 * w0;
    const R2 om2 = pair(om, om);
    R2 d[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int cx = cxq(q), cy = cyq(q);
        const R feq = rho * px[cx + 1] * py[cy + 1];
        const R herm = q == 0 ? h0 : (cy == 0 ? hx : (cx == 0 ? hy : hd + R(cx * cy) * hxy));
        const R W = q == 0 ? Wr : (cx == 0 || cy == 0 ? Wa : Wd);
        const R flux = (cx ? R(cx) * qx : R(0)) + (cy ? R(cy) * qy : R(0));
        R geq = W * (twoRhoE + flux + herm);
        if (q == 0) geq += Xx + Xy;
        if (q == 1 || q == 3) geq -= R(0.5) * Xx;
        if (q == 2 || q == 4) geq -= R(0.5) * Xy;
        const R shift = (cx ? R(cx) * dqx : R(0)) + (cy ? R(cy) * dqy : R(0));
        const R gqe = geq + W * shift;
        // (w (f^eq - f), w (g^eq - g) + (w1 - w)(g^qe - g))
        d[q] = pfma(om2, psub(pair(feq, geq), p[q]), pair(R(0), dom * (gqe - p[q].y)));
    }
    if constexpr (sizeof(R) == 4) {
        // The relaxation leaves mass, momentum and energy unchanged in exact
        // arithmetic (sum f^eq = rho, sum f^eq c = rho u, sum g^eq = sum g^qe =
        // 2 rho E).  In float the rounded equilibria miss that by an ulp, and
        // at a node whose state barely changes the miss has the same sign at
        // every step, so it accumulates.  Its sums over the small changes are
        // exact to far below the populations' ulp: take them out of the rest
        // population (mass, energy) and of the axis pairs (momentum; their
        // sum, hence the mass, unchanged).
        R2 e = d[0];
#pragma unroll
        for (int q = 1; q < 9; ++q) e = padd(e, d[q]);
        const R ex = ((d[1].x - d[3].x) + (d[5].x - d[6].x)) + (d[8].x - d[7].x);
        const R ey = ((d[2].x - d[4].x) + (d[5].x - d[8].x)) + (d[6].x - d[7].x);
        d[0] = psub(d[0], e);
        d[1].x -= R(0.5) * ex;
        d[3].x += R(0.5) * ex;
        d[2].x -= R(0.5) * ey;
        d[4].x += R(0.5) * ey;
    }
    // dt phi on the axis velocities
    const R hyx = R(0.5) * dt * Yx, hyy = R(0.5) * dt * Yy;
    d[1].x -= hyx;
    d[3].x += hyx;
    d[2].x -= hyy;
    d[4].x += hyy;
#pragma unroll
    for (int q = 0; q < 9; ++q) p[q] = padd(p[q], d[q]);
}

// Grad's approximation at wall targets (Sec. III A, Eqs. fnoneq, gnoneq,
// strainrate): f = f^eq + dt f1, g = g^eq + dt g1.  grad u as (d_x u_x, d_y u_x,
// d_x u_y, d_y u_y), grad T as (d_x T, d_y T).
template <typename R>
__device__ __forceinline__ void grad_populations(R rho, R ux, R uy, R T, R dudx, R dudy, R dvdx,
                                                 R dvdy, R dTdx, R dTdy, R mu, R dt, R Cv, R Pr,
                                                 R* f, R* g) {
    const R Cp = Cv + R(1);
    const R iom = R(0.5) + mu * rcp_(rho * T * dt);      // 1/omega
    const R iom1 = R(0.5) + (iom - R(0.5)) * rcp_(Pr);  // 1/omega_1
    const R E = Cv * T + R(0.5) * (ux * ux + uy * uy);
    const R sxx = R(2) * dudx, syy = R(2) * dvdy, sxy = dvdx + dudy;
    const R div = dudx + dvdy;
    const R iCv = rcp_(Cv);
    const R cP = -iom * rho * T;
    const R p1xx = cP * (sxx - div * iCv), p1yy = cP * (syy - div * iCv), p1xy = cP * sxy;
    const R dEdx = Cv * dTdx + ux * dudx + uy * dvdx;
    const R dEdy = Cv * dTdy + ux * dudy + uy * dvdy;
    const R cq = -R(2) * iom1 * rho * Cp * T;
    const R q1x = cq * dTdx + R(2) * (ux * p1xx + uy * p1xy);
    const R q1y = cq * dTdy + R(2) * (ux * p1xy + uy * p1yy);
    const R cR = -R(2) * iom1 * rho * T;
    const R EpT = E + R(2) * T;
    const R r1xx = cR * (sxx * EpT + R(2) * ux * dEdx);
    const R r1yy = cR * (syy * EpT + R(2) * uy * dEdy);
    const R r1xy = cR * (sxy * EpT + ux * dEdy + dEdx * uy);
    f_equilibrium(rho, ux, uy, T, f);
    g_equilibrium(rho, ux, uy, T, Cv, g);
    const R w[3] = {R(0.5) * T, R(1) - T, R(0.5) * T};
    const R invT = rcp_(T);
    const R inv2T2 = R(0.5) * invT * invT;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int cx = cxq(q), cy = cyq(q);
        const R W = w[cx + 1] * w[cy + 1];
        const R dxx = R(cx * cx) - T, dyy = R(cy * cy) - T, dxy = R(cx * cy);
        const R hp = (p1xx * dxx + R(2) * p1xy * dxy + p1yy * dyy) * inv2T2;
        const R hr = (r1xx * dxx + R(2) * r1xy * dxy + r1yy * dyy) * inv2T2;
        f[q] += dt * W * hp;
        g[q] += dt * W * ((q1x * R(cx) + q1y * R(cy)) * invT + hr);
    }
}

// Rotation part of a body state: sin(alpha) and cos(alpha) - 1 written as
// -2 sin^2(alpha/2) (no cancellation for small angles).  A state without
// rotation (every state of a transverse body) takes no transcendental call:
// sin(+-0) = +-0 exactly, so the values are the same.
struct BodyRot {
    double sa, cm1;
};
__host__ __device__ inline BodyRot body_rot(double alpha) {
    double sa = alpha, h = 0.5 * alpha;
    if (alpha != 0.0) {
        sa = sin(alpha);
        h = sin(0.5 * alpha);
    }
    return BodyRot{sa, -2.0 * h * h};
}

// Blended rigid map of one body (Sec. II D) for one body state s with
// previous state sp:  d(X) = A (X - Xp) + t with A = R(alpha) - I,
// t = (0, h);  x = X + (1 - r_blend) d(X).  The va.., vt. fields are the
// (state - previous state) differences times inv_dt, for V_G.
__host__ __device__ inline BodyMap<double> make_body_map(const BodyDev& b, const BodyStateDev& s,
                                                         BodyRot rs, const BodyStateDev& sp,
                                                         BodyRot rp, double inv_dt) {
    BodyMap<double> m;
    m.active = b.dof != 0;
    m.xc = b.xc; m.yc = b.yc; m.xp = b.xp; m.yp = b.yp;
    m.r_in = b.r_in;
    m.inv_w = b.inv_w;
    m.a00 = rs.cm1; m.a01 = -rs.sa; m.a10 = rs.sa; m.a11 = rs.cm1;
    m.tx = 0.0; m.ty = s.h;
    m.va00 = (rs.cm1 - rp.cm1) * inv_dt; m.va01 = -(rs.sa - rp.sa) * inv_dt;
    m.va10 = (rs.sa - rp.sa) * inv_dt; m.va11 = (rs.cm1 - rp.cm1) * inv_dt;
    m.vtx = 0.0; m.vty = (s.h - sp.h) * inv_dt;
    return m;
}

__host__ __device__ inline BodyMap<float> to_float(const BodyMap<double>& d) {
    BodyMap<float> m;
    m.active = d.active;
    m.xc = (float)d.xc; m.yc = (float)d.yc; m.xp = (float)d.xp; m.yp = (float)d.yp;
    m.r_in = (float)d.r_in; m.inv_w = (float)d.inv_w;
    m.a00 = (float)d.a00; m.a01 = (float)d.a01; m.a10 = (float)d.a10; m.a11 = (float)d.a11;
    m.tx = (float)d.tx; m.ty = (float)d.ty;
    m.va00 = (float)d.va00; m.va01 = (float)d.va01; m.va10 = (float)d.va10; m.va11 = (float)d.va11;
    m.vtx = (float)d.vtx; m.vty = (float)d.vty;
    return m;
}

// F = dx/dX of the blended map (analytic, includes the gradient of the blend
// factor) and V_G at absolute position (X, Y).  Outside the blended region
// F = I and V_G = 0 exactly, and the result is false.
template <typename R>
__device__ __forceinline__ bool kinematics(const BodyMap<R>& bm, R X, R Y, R& F00, R& F01, R& F10,
                                           R& F11, R& vx, R& vy) {
    F00 = R(1); F01 = R(0); F10 = R(0); F11 = R(1); vx = R(0); vy = R(0);
    if (!bm.active) return false;
    const R dx = X - bm.xc, dy = Y - bm.yc;
    const R dist = sqrt_(dx * dx + dy * dy);
    const R s = (dist - bm.r_in) * bm.inv_w;
    if (s > R(1)) return false;
    R w, drx = R(0), dry = R(0);
    if (s < R(0)) {
        w = R(1);
    } else {
        const R r5 = s * s * s * (R(10) - R(15) * s + R(6) * s * s);
        const R d5 = R(30) * s * s * (R(1) - s) * (R(1) - s);
        w = R(1) - r5;
        const R gq = d5 * bm.inv_w * rcp_(dist);
        drx = gq * dx;
        dry = gq * dy;
    }
    const R px = X - bm.xp, py = Y - bm.yp;
    const R ux = bm.a00 * px + bm.a01 * py + bm.tx;
    const R uy = bm.a10 * px + bm.a11 * py + bm.ty;
    F00 = R(1) + w * bm.a00 - ux * drx;
    F01 = w * bm.a01 - ux * dry;
    F10 = w * bm.a10 - uy * drx;
    F11 = R(1) + w * bm.a11 - uy * dry;
    vx = w * (bm.va00 * px + bm.va01 * py + bm.vtx);
    vy = w * (bm.va10 * px + bm.va11 * py + bm.vty);
    return true;
}

// Kinematics of several bodies' blended maps: the displacements add
// (Sec. II D), so F = I + sum_b (F_b - I) and V_G = sum_b V_b; a body whose
// blended region does not hold the point adds nothing.
template <typename R>
__device__ __forceinline__ bool kinematics_sum(const BodyMap<R>* bm, int nb, R X, R Y, R& F00, R& F01,
                                               R& F10, R& F11, R& vx, R& vy) {
    bool moved = kinematics(bm[0], X, Y, F00, F01, F10, F11, vx, vy);
    for (int b = 1; b < nb; ++b) {
        R g00, g01, g10, g11, wx, wy;
        if (!kinematics(bm[b], X, Y, g00, g01, g10, g11, wx, wy)) continue;
        if (moved) {
            F00 += g00 - R(1); F01 += g01; F10 += g10; F11 += g11 - R(1);
            vx += wx; vy += wy;
        } else {
            F00 = g00; F01 = g01; F10 = g10; F11 = g11; vx = wx; vy = wy;
        }
        moved = true;
    }
    return moved;
}

// Fill a maps record: collision map from S_cur, stream maps from
// (S_next, S_vgprev); the float maps are the float64 ones rounded.
__host__ __device__ inline void build_maps(const BodyDev& b, const BodyStateDev& S_cur,
                                           const BodyStateDev& S_next,
                                           const BodyStateDev& S_vgprev, double dt, StepMaps& m) {
    m.S_cur = S_cur;
    m.S_next = S_next;
    m.S_vgprev = S_vgprev;
    const double inv_dt = 1.0 / dt;
    const BodyRot rc = body_rot(S_cur.alpha), rn = body_rot(S_next.alpha), rp = body_rot(S_vgprev.alpha);
    m.Kd = make_body_map(b, S_cur, rc, S_cur, rc, inv_dt);
    m.Sd = make_body_map(b, S_next, rn, S_vgprev, rp, inv_dt);
    m.Kf = to_float(m.Kd);
    m.Sf = to_float(m.Sd);
}

// Classical RK4 of the body ODE over dt with the load (Fx, Fy, M) held fixed
// (Sec. III B; weak coupling of Sec. III), for step n (from n dt to (n+1) dt).
// A pitch-plunge body in its forcing interval (Sec. IV D) has the pitch
// prescribed, alpha = amp sin(w_a t): the plunge row is integrated with the
// prescribed pitch acceleration at the stage times and alpha, alpha' are set
// to their values at (n+1) dt.
__host__ __device__ inline BodyStateDev rk4_body(const BodyDev& b, BodyStateDev s, double fy,
                                                 double mz, double dt, long long n) {
    if (b.dof == 2 && (double)(n + 1) * dt <= b.t_forced) {
        const double w = b.w_a, amp = b.pitch_amp;
        auto acc = [&](double t, double h, double v) {
            const double acc_a = -amp * w * w * sin(w * t);
            return (fy - b.k_h * h - b.s_a * acc_a) / b.m;
        };
        const double t0 = (double)n * dt, tm = ((double)n + 0.5) * dt, t1 = (double)(n + 1) * dt;
        const double h0 = s.h, v0 = s.hdot;
        const double k1h = v0, k1v = acc(t0, h0, v0);
        const double k2h = v0 + 0.5 * dt * k1v, k2v = acc(tm, h0 + 0.5 * dt * k1h, v0 + 0.5 * dt * k1v);
        const double k3h = v0 + 0.5 * dt * k2v, k3v = acc(tm, h0 + 0.5 * dt * k2h, v0 + 0.5 * dt * k2v);
        const double k4h = v0 + dt * k3v, k4v = acc(t1, h0 + dt * k3h, v0 + dt * k3v);
        s.h = h0 + dt / 6.0 * (k1h + 2.0 * k2h + 2.0 * k3h + k4h);
        s.hdot = v0 + dt / 6.0 * (k1v + 2.0 * k2v + 2.0 * k3v + k4v);
        s.alpha = amp * sin(w * t1);
        s.adot = amp * w * cos(w * t1);
        return s;
    }
    if (b.dof == 1) {
        auto acc = [&](double h, double v) { return (fy - b.k * h - b.c * v) / b.m; };
        const double h0 = s.h, v0 = s.hdot;
        const double k1h = v0, k1v = acc(h0, v0);
        const double k2h = v0 + 0.5 * dt * k1v, k2v = acc(h0 + 0.5 * dt * k1h, v0 + 0.5 * dt * k1v);
        const double k3h = v0 + 0.5 * dt * k2v, k3v = acc(h0 + 0.5 * dt * k2h, v0 + 0.5 * dt * k2v);
        const double k4h = v0 + dt * k3v, k4v = acc(h0 + dt * k3h, v0 + dt * k3v);
        s.h = h0 + dt / 6.0 * (k1h + 2.0 * k2h + 2.0 * k3h + k4h);
        s.hdot = v0 + dt / 6.0 * (k1v + 2.0 * k2v + 2.0 * k3v + k4v);
    } else if (b.dof == 2) {
        const double det = b.m * b.i_a - b.s_a * b.s_a;
        auto accel = [&](const double* y, double* a) {
            const double r0 = fy - b.k_h * y[0], r1 = mz - b.k_a * y[1];
            a[0] = (b.i_a * r0 - b.s_a * r1) / det;
            a[1] = (-b.s_a * r0 + b.m * r1) / det;
        };
        double y0[4] = {s.h, s.alpha, s.hdot, s.adot}, k[4][4], yt[4], acc2[2];
        for (int st = 0; st < 4; ++st) {
            const double c = (st == 0) ? 0.0 : (st == 3 ? 1.0 : 0.5);
            for (int n = 0; n < 4; ++n) yt[n] = y0[n] + (st ? c * dt * k[st - 1][n] : 0.0);
            accel(yt, acc2);
            k[st][0] = yt[2]; k[st][1] = yt[3]; k[st][2] = acc2[0]; k[st][3] = acc2[1];
        }
        double y1[4];
        for (int n = 0; n < 4; ++n)
            y1[n] = y0[n] + dt / 6.0 * (k[0][n] + 2.0 * k[1][n] + 2.0 * k[2][n] + k[3][n]);
        s.h = y1[0]; s.alpha = y1[1]; s.hdot = y1[2]; s.adot = y1[3];
    }
    return s;
}

}  // namespace lbfsi
