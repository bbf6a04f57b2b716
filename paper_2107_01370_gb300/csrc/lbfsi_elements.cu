// The coupled step on an unstructured Q2 element list (the paper's mesh type,
// Sec. II B; the structured meshes of lbfsi_step.cu are its special cases).
//
// A node's neighbourhood is no longer a tile of an index grid, so the step is
// four launches over node lists, each node's data read from global memory
// (the mesh tables and the step's fields stay in L2 for meshes of this size):
//
//   D        correction field D = (mu/p) grad dQ at every node (Sec. II C),
//            with the mesh's nodal gradient operator (Eq. ddx+fem; reading
//            R33, or R18 for a renumbered index grid) mapped by g^{-1}
//   collide  Y = grad D, collision of every node (Eq. f_boltz) into a
//            post-collision buffer; far-field nodes take the equilibria of
//            their targets.  The float path stores deviations from the free
//            stream's pairs there, so that the Q2 weights' round-off acts on
//            deviations (as in the tiled kernel)
//   stream   per node and direction: c_hat = g^{-T} c - V_G, the departure
//            point searched in the node's elements in increasing index
//            (Eq. depPnt; readings R8, R9) by Newton's method on each
//            element's bilinear map relative to the node, the Q2 gather of
//            the nine element nodes (Eq. SemiLagrProp); wall nodes rebuild
//            their missing populations by Grad's approximation at the
//            target point B = A + dt n0, far-field nodes take equilibria at
//            the targets at B = A - dt n_out (Sec. III A; readings R19, R20,
//            R34); moments; the wall nodes' Simpson shares of the load (FP64)
//            summed per block in thread order
//   finish   per solve: the block partials summed in block order, RK4 of the
//            body (Sec. III B), the next step's blended maps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "lbfsi.h"
#include "lbfsi_device.cuh"
#include "lbfsi_host.h"
#include "lbfsi_internal.h"

namespace lbfsi {
namespace {

constexpr int EM_THREADS = 256;
constexpr int EN_STRIDE = 12;

// Node kinds (kind[n]): 0 interior, w + 1 the wall chain's node w, -(f + 1)
// the far-field chain's node f.
struct EArgs {
    int N, nbatch, nblk, kstep, collide;
    const void* X;        // [N][2] node coordinates (element type of the path)
    const int* E;         // [Ne][EN_STRIDE] element nodes, entry a * 3 + b (then padding, so
                          // that a gather reads an element's nodes in three 16-byte loads)
    const void* ecoef;    // [Ne][6] bilinear map: (b_x, b_y, c_x, c_y, d_x, d_y)
    const int* hptr;      // [N + 1] holding elements of each node
    const int* hold;      // [.] element * 16 + the node's entry in it
    const int* gptr;      // [N + 1] gradient operator rows
    const int* gcol;      // [.] neighbour node
    const void* gw;       // [.][2] weights of d/dX and d/dY
    const int* kind;      // [N]
    const double* xw;     // [nwall][2] wall node coordinates
    const double* n0;     // [nwall][2] wall normals (undeformed)
    const double* wgeo;   // [nwall][6] Simpson shares
    const double* nfar;   // [nfar][2] outward directions of the far field
    // departures of the interior nodes for a node the blend does not move
    // (the displacement of direction q is then -dt c_q at every step),
    // solved once for the flow's dt: the position in hold of the holding
    // element [9][N] (-1: none holds the point) and (xi, eta) [9][N]; null:
    // solved every step
    int* dep_e;
    void* dep_xe;
    const void* p_in;     // [nbatch][9][N] pairs: pre-collision state of step k
    void* ppost;          // [nbatch][9][N] pairs: post-collision (float: deviations)
    void* p_out;          // [nbatch][9][N] pairs: pre-collision state of step k + 1
    const void* M_in;     // [nbatch][4][N] moments of step k
    void* M_out;          // [nbatch][4][N] moments of step k + 1
    void* D;              // [nbatch][2][N]
    void* dQ;             // [nbatch][2][N] dQ of the moments the stream writes (the next
                          // step's correction field reads it at every neighbour)
    const StepMaps* maps_in;   // [nbatch]
    StepMaps* maps_out;        // [nbatch]
    const BodyDev* bodies;     // [nbatch]
    double* part;         // [nbatch][nblk][3]
    SolveDev flow;        // flow parameters (buffers unused)
    unsigned* status;
};

template <typename R>
struct EVec;
template <>
struct EVec<float> {
    using T2 = float2;
};
template <>
struct EVec<double> {
    using T2 = double2;
};

template <typename R>
__device__ __forceinline__ R flowv(const SolveDev& s, double d, float f) {
    return sizeof(R) == 4 ? (R)f : (R)d;
}

template <typename R>
__device__ __forceinline__ const BodyMap<R>& kmap(const StepMaps& m);
template <>
__device__ __forceinline__ const BodyMap<float>& kmap<float>(const StepMaps& m) { return m.Kf; }
template <>
__device__ __forceinline__ const BodyMap<double>& kmap<double>(const StepMaps& m) { return m.Kd; }
template <typename R>
__device__ __forceinline__ const BodyMap<R>& smap(const StepMaps& m);
template <>
__device__ __forceinline__ const BodyMap<float>& smap<float>(const StepMaps& m) { return m.Sf; }
template <>
__device__ __forceinline__ const BodyMap<double>& smap<double>(const StepMaps& m) { return m.Sd; }

// F^{-1} of the blended map at node n for a map (Sec. II A, II D); false
// where the blend does not move the node (F = I, V_G = 0).
template <typename R>
__device__ __forceinline__ bool inv_map(const BodyMap<R>& bm, R X, R Y, R& i00, R& i01, R& i10, R& i11, R& vx,
                                        R& vy) {
    R F00, F01, F10, F11;
    const bool moved = kinematics(bm, X, Y, F00, F01, F10, F11, vx, vy);
    const R idF = rcp_(F00 * F11 - F01 * F10);
    i00 = F11 * idF;
    i01 = -F01 * idF;
    i10 = -F10 * idF;
    i11 = F00 * idF;
    return moved;
}

// Newton's method for the point (dx, dy) relative to a node at reference
// position (xi0, eta0) of an element with bilinear map X0 + b xi + c eta +
// d xi eta, c = (b_x, b_y, c_x, c_y, d_x, d_y): (b + d eta0) u + (c + d xi0) v
// + d u v = (dx, dy).  Returns the point's reference coordinates.  Written
// with fixed rounding (fma_rn, mul_rn, add_rn) so that the departures cached
// by k_em_record equal, bit for bit, the ones k_em_stream solves.
template <typename R>
__device__ __forceinline__ void em_newton(const R* c, R xi0, R et0, R dx, R dy, R& x, R& y) {
    const R Bx = fma_rn(c[4], et0, c[0]), By = fma_rn(c[5], et0, c[1]);
    const R Cx = fma_rn(c[4], xi0, c[2]), Cy = fma_rn(c[5], xi0, c[3]);
    R u = R(0), v = R(0);
    constexpr int ITS = sizeof(R) == 4 ? 4 : 20;
#pragma unroll 1
    for (int it = 0; it < ITS; ++it) {
        const R uv = mul_rn(u, v);
        const R rx = fma_rn(c[4], uv, fma_rn(Cx, v, fma_rn(Bx, u, -dx)));
        const R ry = fma_rn(c[5], uv, fma_rn(Cy, v, fma_rn(By, u, -dy)));
        const R a11 = fma_rn(c[4], v, Bx), a12 = fma_rn(c[4], u, Cx);
        const R a21 = fma_rn(c[5], v, By), a22 = fma_rn(c[5], u, Cy);
        const R idet = rcp_(fma_rn(a11, a22, -mul_rn(a12, a21)));
        const R du = mul_rn(fma_rn(a22, rx, -mul_rn(a12, ry)), idet);
        const R dv = mul_rn(fma_rn(a11, ry, -mul_rn(a21, rx)), idet);
        u = add_rn(u, -du);
        v = add_rn(v, -dv);
        if (sizeof(R) == 8 && abs_(du) + abs_(dv) < R(1e-15)) break;
    }
    x = add_rn(xi0, u);
    y = add_rn(et0, v);
}

// Containment tolerance of pass 0 / 1 (reading R8): 1e-12 of the element
// (float: 1e-5), then 1e-9.
template <typename R>
__device__ __forceinline__ R em_tol(int pass) {
    return R(1) + (pass ? R(1e-9) : (sizeof(R) == 4 ? R(1e-5) : R(1e-12)));
}
template <typename R>
__host__ __device__ constexpr int em_passes() {
    return sizeof(R) == 4 ? 1 : 2;
}

// Departure point of node n displaced by (dx, dy): the first element holding
// the node (increasing index) that contains it (Eq. depPnt; readings R8, R9).
template <typename R>
__device__ bool em_locate(const EArgs& a, int n, R dx, R dy, int& elem, R& xi, R& eta) {
    const R* ec = static_cast<const R*>(a.ecoef);
    const int h0 = a.hptr[n], h1 = a.hptr[n + 1];
#pragma unroll 1
    for (int pass = 0; pass < em_passes<R>(); ++pass) {
        const R tin = em_tol<R>(pass);
#pragma unroll 1
        for (int h = h0; h < h1; ++h) {
            const int code = __ldg(a.hold + h), e = code >> 4, ent = code & 15;
            R x, y;
            em_newton<R>(ec + 6 * (size_t)e, R(ent / 3 - 1), R(ent % 3 - 1), dx, dy, x, y);
            if (abs_(x) <= tin && abs_(y) <= tin) {
                elem = e;
                xi = x;
                eta = y;
                return true;
            }
        }
    }
    return false;
}

// The nodal gradient operator applied to two fields in one pass over the
// operator's row: fld(m, v0, v1) gives both at node m.  Each field's sums
// run in the same order as in em_grad.
template <typename R, typename Fn>
__device__ __forceinline__ void em_grad2(const EArgs& a, int n, Fn fld, R& g0X, R& g0Y, R& g1X, R& g1Y) {
    const R* w = static_cast<const R*>(a.gw);
    g0X = R(0);
    g0Y = R(0);
    g1X = R(0);
    g1Y = R(0);
    for (int k = a.gptr[n]; k < a.gptr[n + 1]; ++k) {
        R v0, v1;
        fld(a.gcol[k], v0, v1);
        const R wX = w[2 * k], wY = w[2 * k + 1];
        g0X += wX * v0;
        g0Y += wY * v0;
        g1X += wX * v1;
        g1Y += wY * v1;
    }
}

// The nodal gradient operator applied to a field given by a functor.
template <typename R, typename Fn>
__device__ __forceinline__ void em_grad(const EArgs& a, int n, Fn fld, R& gX, R& gY) {
    const R* w = static_cast<const R*>(a.gw);
    gX = R(0);
    gY = R(0);
    for (int k = a.gptr[n]; k < a.gptr[n + 1]; ++k) {
        const R v = fld(a.gcol[k]);
        gX += w[2 * k] * v;
        gY += w[2 * k + 1] * v;
    }
}

template <typename R>
__device__ __forceinline__ typename EVec<R>::T2 ref_pair(const SolveDev& s, int q) {
    typename EVec<R>::T2 r;
    if constexpr (sizeof(R) == 4) {
        r.x = s.fgref[2 * q];
        r.y = s.fgref[2 * q + 1];
    } else {
        r.x = R(0);
        r.y = R(0);
    }
    return r;
}

// ---- launch 1: D = (mu/p) grad dQ (Sec. II C), dQ_a = rho u_a (1 - 3T) - rho u_a^3
// (dQ written with the moments by the previous stream launch, em_dq)
template <typename R>
__global__ void __launch_bounds__(EM_THREADS) k_em_D(const EArgs a) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (n >= a.N) return;
    const size_t N = (size_t)a.N;
    const R* M = static_cast<const R*>(a.M_in) + (size_t)b * 4 * N;
    const R* X = static_cast<const R*>(a.X);
    R i00, i01, i10, i11, vx, vy;
    inv_map(kmap<R>(a.maps_in[b]), X[2 * n], X[2 * n + 1], i00, i01, i10, i11, vx, vy);
    const R* Q = static_cast<const R*>(a.dQ) + (size_t)b * 2 * N;
    R xX, xY, yX, yY;
    em_grad2<R>(a, n, [&](int m, R& v0, R& v1) {
        v0 = Q[m];
        v1 = Q[N + m];
    }, xX, xY, yX, yY);
    const R mup = flowv<R>(a.flow, a.flow.mu, a.flow.mu_f) * rcp_(M[n] * M[3 * N + n]);
    R* D = static_cast<R*>(a.D) + (size_t)b * 2 * N;
    D[n] = mup * (i00 * xX + i10 * xY);
    D[N + n] = mup * (i01 * yX + i11 * yY);
}

// dQ_a = rho u_a (1 - 3T) - rho u_a^3 of a node's moments (Sec. II C).
template <typename R>
__device__ __forceinline__ void em_dq(R* Q, size_t N, int n, R rho, R ux, R uy, R T) {
    Q[n] = rho * ux * (R(1) - R(3) * T) - rho * ux * ux * ux;
    Q[N + n] = rho * uy * (R(1) - R(3) * T) - rho * uy * uy * uy;
}

// ---- launch 2: Y = grad D and the collision (Eq. f_boltz) into ppost;
// step 0 only copies the initial state
template <typename R>
__global__ void __launch_bounds__(EM_THREADS) k_em_collide(const EArgs a) {
    using R2 = typename EVec<R>::T2;
    const int n = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (n >= a.N) return;
    const size_t N = (size_t)a.N;
    const R2* pin = static_cast<const R2*>(a.p_in) + (size_t)b * 9 * N;
    R2* pout = static_cast<R2*>(a.ppost) + (size_t)b * 9 * N;
    R2 pq[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) pq[q] = pin[q * N + n];
    if (a.collide) {
        const R* M = static_cast<const R*>(a.M_in) + (size_t)b * 4 * N;
        const R Cv = flowv<R>(a.flow, a.flow.Cv, a.flow.Cv_f);
        if (a.kind[n] < 0) {
            R f[9], g[9];
            f_equilibrium(M[n], M[N + n], M[2 * N + n], M[3 * N + n], f);
            g_equilibrium(M[n], M[N + n], M[2 * N + n], M[3 * N + n], Cv, g);
#pragma unroll
            for (int q = 0; q < 9; ++q) pq[q] = pair(f[q], g[q]);
        } else {
            const R* X = static_cast<const R*>(a.X);
            R i00, i01, i10, i11, vx, vy;
            inv_map(kmap<R>(a.maps_in[b]), X[2 * n], X[2 * n + 1], i00, i01, i10, i11, vx, vy);
            const R* D = static_cast<const R*>(a.D) + (size_t)b * 2 * N;
            R xX, xY, yX, yY;
            em_grad2<R>(a, n, [&](int m, R& v0, R& v1) {
                v0 = D[m];
                v1 = D[N + m];
            }, xX, xY, yX, yY);
            const R Yx = i00 * xX + i10 * xY, Yy = i01 * yX + i11 * yY;
            collide_pairs(pq, Yx, Yy, flowv<R>(a.flow, a.flow.mu, a.flow.mu_f),
                          flowv<R>(a.flow, a.flow.dt, a.flow.dt_f), Cv,
                          flowv<R>(a.flow, 1.0 / a.flow.Pr, a.flow.iPr_f));
        }
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) pout[q * N + n] = psub(pq[q], ref_pair<R>(a.flow, q));
}

// Q2 interpolation of direction q's post-collision pairs over element e.
template <typename R>
__device__ __forceinline__ typename EVec<R>::T2 em_gather(const EArgs& a, const typename EVec<R>::T2* pp, int e,
                                                          R xi, R eta) {
    using R2 = typename EVec<R>::T2;
    R Lx[3], Ly[3];
    Lx[0] = xi * (R(0.5) * xi - R(0.5));
    Lx[1] = R(1) - xi * xi;
    Lx[2] = xi * (R(0.5) * xi + R(0.5));
    Ly[0] = eta * (R(0.5) * eta - R(0.5));
    Ly[1] = R(1) - eta * eta;
    Ly[2] = eta * (R(0.5) * eta + R(0.5));
    const int4* e4 = reinterpret_cast<const int4*>(a.E + EN_STRIDE * (size_t)e);
    const int4 n0 = __ldg(e4), n1 = __ldg(e4 + 1), n2 = __ldg(e4 + 2);
    const int nd[9] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w, n2.x};
    R2 acc = pair(R(0), R(0));
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
        R2 t = pmul(pair(Ly[0], Ly[0]), pp[nd[3 * aa]]);
        t = pfma(pair(Ly[1], Ly[1]), pp[nd[3 * aa + 1]], t);
        t = pfma(pair(Ly[2], Ly[2]), pp[nd[3 * aa + 2]], t);
        acc = pfma(pair(Lx[aa], Lx[aa]), t, acc);
    }
    return acc;
}

// Moments rho, u, T at a point of element e: the node's own values plus the
// Q2-weighted differences from them (the weights' round-off then acts on
// small differences).
template <typename R>
__device__ __forceinline__ void em_interp_M(const EArgs& a, const R* M, size_t N, int n, int e, R xi, R eta,
                                            R* out) {
    R Lx[3], Ly[3];
    Lx[0] = xi * (R(0.5) * xi - R(0.5));
    Lx[1] = R(1) - xi * xi;
    Lx[2] = xi * (R(0.5) * xi + R(0.5));
    Ly[0] = eta * (R(0.5) * eta - R(0.5));
    Ly[1] = R(1) - eta * eta;
    Ly[2] = eta * (R(0.5) * eta + R(0.5));
    const int* en = a.E + EN_STRIDE * (size_t)e;
    R d[4] = {R(0), R(0), R(0), R(0)};
    R own[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) own[c] = M[c * N + n];
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        const R w = Lx[s / 3] * Ly[s % 3];
        const int m = en[s];
#pragma unroll
        for (int c = 0; c < 4; ++c) d[c] += w * (M[c * N + m] - own[c]);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) out[c] = own[c] + d[c];
}

// ---- launch 3: stream step k + 1.  Bound by the latency of its dependent
// loads: the float kernel is held to 40 registers so that six blocks (48
// warps) share an SM (measured: 64 registers and four blocks 2506 MLUPS,
// 48 and five 2635, 40 and six 2700)
template <typename R>
__global__ void __launch_bounds__(EM_THREADS, sizeof(R) == 4 ? 6 : 2) k_em_stream(const EArgs a) {
    using R2 = typename EVec<R>::T2;
    const int n = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    const size_t N = (size_t)a.N;
    double fcx = 0.0, fcy = 0.0, fcm = 0.0;
    bool wallnode = false;
    if (n < a.N) {
        const SolveDev& fl = a.flow;
        const R dt = flowv<R>(fl, fl.dt, fl.dt_f), Cv = flowv<R>(fl, fl.Cv, fl.Cv_f);
        const R* M = static_cast<const R*>(a.M_in) + (size_t)b * 4 * N;
        const R2* pp = static_cast<const R2*>(a.ppost) + (size_t)b * 9 * N;
        R2* po = static_cast<R2*>(a.p_out) + (size_t)b * 9 * N;
        R* Mo = static_cast<R*>(a.M_out) + (size_t)b * 4 * N;
        R* Qo = static_cast<R*>(a.dQ) + (size_t)b * 2 * N;
        const R* X = static_cast<const R*>(a.X);
        const int kd = a.kind[n];
        wallnode = kd > 0;
        if (kd < 0) {
            // far field: targets at B = A - dt n_out; the inlet prescribes the
            // free stream's u and T (reading R20)
            const double* nf = a.nfar + 2 * (size_t)(-kd - 1);
            R t[4];
            int e;
            R xi, eta;
            if (em_locate<R>(a, n, -dt * (R)nf[0], -dt * (R)nf[1], e, xi, eta)) {
                em_interp_M<R>(a, M, N, n, e, xi, eta, t);
            } else {
                atomicOr(a.status, ST_BPOINT);
                for (int c = 0; c < 4; ++c) t[c] = M[c * N + n];
            }
            if (fl.uinf_x * nf[0] + fl.uinf_y * nf[1] < 0.0) {
                t[1] = flowv<R>(fl, fl.uinf_x, fl.uinf_x_f);
                t[2] = flowv<R>(fl, fl.uinf_y, fl.uinf_y_f);
                t[3] = flowv<R>(fl, fl.T_inf, fl.T_inf_f);
            }
            R f[9], g[9];
            f_equilibrium(t[0], t[1], t[2], t[3], f);
            g_equilibrium(t[0], t[1], t[2], t[3], Cv, g);
#pragma unroll
            for (int q = 0; q < 9; ++q) po[q * N + n] = pair(f[q], g[q]);
#pragma unroll
            for (int c = 0; c < 4; ++c) Mo[c * N + n] = t[c];
            em_dq<R>(Qo, N, n, t[0], t[1], t[2], t[3]);
        } else {
            const StepMaps& mp = a.maps_in[b];
            R i00, i01, i10, i11, vx, vy;
            const bool moved = inv_map(smap<R>(mp), X[2 * n], X[2 * n + 1], i00, i01, i10, i11, vx, vy);
            // an interior node the blend does not move takes its cached
            // departures (the same solves, made once for the flow's dt)
            const bool cached = a.dep_e != nullptr && kd == 0 && !moved;
            const R2* dxe = static_cast<const R2*>(a.dep_xe);
            unsigned missing = 0u;
            const int w = kd - 1;
            if (kd > 0) {
                // missing populations: c_hat . n0 > 0, decided in float64 (reading R10)
                double D00, D01, D10, D11, dvx, dvy;
                kinematics(mp.Sd, a.xw[2 * w], a.xw[2 * w + 1], D00, D01, D10, D11, dvx, dvy);
                const double idd = 1.0 / (D00 * D11 - D01 * D10);
                const double n0x = a.n0[2 * w], n0y = a.n0[2 * w + 1];
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const double cx = cxq(q), cy = cyq(q);
                    const double hx = (D11 * cx - D01 * cy) * idd - dvx;
                    const double hy = (-D10 * cx + D00 * cy) * idd - dvy;
                    if (hx * n0x + hy * n0y > 1e-12) missing |= 1u << q;
                }
            }
            R f[9], g[9];
            bool lost = false;
#pragma unroll 1
            for (int q = 0; q < 9; ++q) {
                f[q] = R(0);
                g[q] = R(0);
                if (missing & (1u << q)) continue;
                const R cx = (R)cxq(q), cy = (R)cyq(q);
                const R hx = i00 * cx + i01 * cy - vx, hy = i10 * cx + i11 * cy - vy;
                int e;
                R xi, eta;
                R2 v;
                bool found;
                if (cached) {
                    e = __ldg(a.dep_e + (size_t)q * N + n);
                    found = e >= 0;
                    const R2 xe = __ldg(dxe + (size_t)q * N + n);
                    xi = xe.x;
                    eta = xe.y;
                } else {
                    found = em_locate<R>(a, n, -dt * hx, -dt * hy, e, xi, eta);
                }
                if (found) {
                    v = em_gather<R>(a, pp + (size_t)q * N, e, xi, eta);
                } else {
                    lost = true;
                    v = pp[q * N + n];
                }
                v = padd(v, ref_pair<R>(fl, q));
                f[q] = v.x;
                g[q] = v.y;
            }
            if (lost) atomicOr(a.status, ST_DEPARTURE);
            if (missing) {
                // wall targets: rho, T at B = A + dt n0 (previous field), u =
                // wall velocity, gradients at the node; Grad's approximation
                // of the missing populations (Sec. III A)
                R t[4];
                int e;
                R xi, eta;
                if (em_locate<R>(a, n, dt * (R)a.n0[2 * w], dt * (R)a.n0[2 * w + 1], e, xi, eta)) {
                    em_interp_M<R>(a, M, N, n, e, xi, eta, t);
                } else {
                    atomicOr(a.status, ST_BPOINT);
                    for (int c = 0; c < 4; ++c) t[c] = M[c * N + n];
                }
                R gr[3][2];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    R gX, gY;
                    em_grad<R>(a, n, [&](int m) { return M[(1 + c) * N + m]; }, gX, gY);
                    gr[c][0] = i00 * gX + i10 * gY;
                    gr[c][1] = i01 * gX + i11 * gY;
                }
                R fw[9], gw[9];
                grad_populations(t[0], vx, vy, t[3], gr[0][0], gr[0][1], gr[1][0], gr[1][1], gr[2][0], gr[2][1],
                                 flowv<R>(fl, fl.mu, fl.mu_f), dt, Cv, flowv<R>(fl, fl.Pr, fl.Pr_f), fw, gw);
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    if (missing & (1u << q)) {
                        f[q] = fw[q];
                        g[q] = gw[q];
                    }
            }
            const Macro<R> mc = moments(f, g, Cv);
            if (!(mc.rho > R(0)) || !(mc.T > R(0)) || !isfinite(mc.ux) || !isfinite(mc.uy))
                atomicOr(a.status, ST_NONPHYS);
#pragma unroll
            for (int q = 0; q < 9; ++q) po[q * N + n] = pair(f[q], g[q]);
            Mo[n] = mc.rho;
            Mo[N + n] = mc.ux;
            Mo[2 * N + n] = mc.uy;
            Mo[3 * N + n] = mc.T;
            em_dq<R>(Qo, N, n, mc.rho, mc.ux, mc.uy, mc.T);
            if (kd > 0) {
                // wall stress sigma = -p I - (1 - omega/2) sum (f - f^eq) c c
                // (Sec. III) in float64, this node's Simpson shares
                double fd[9], gd[9], feq[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    fd[q] = (double)f[q];
                    gd[q] = (double)g[q];
                }
                const Macro<double> md = moments(fd, gd, fl.Cv);
                f_equilibrium(md.rho, md.ux, md.uy, md.T, feq);
                double pxx = 0, pxy = 0, pyy = 0;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const double fn = fd[q] - feq[q];
                    pxx += cxq(q) * cxq(q) * fn;
                    pxy += cxq(q) * cyq(q) * fn;
                    pyy += cyq(q) * cyq(q) * fn;
                }
                const double om = 1.0 / (0.5 + fl.mu / (md.rho * md.T * fl.dt));
                const double p = md.rho * md.T, am = 1.0 - 0.5 * om;
                const double sxx = -p - am * pxx, sxy = -am * pxy, syy = -p - am * pyy;
                const BodyMap<double>& mw = mp.Sd;
                const double R00 = 1.0 + mw.a00, R01 = mw.a01, R10 = mw.a10, R11 = 1.0 + mw.a11;
                const BodyDev& bd = a.bodies[b];
                const double Xd = a.xw[2 * w] - bd.xp, Yd = a.xw[2 * w + 1] - bd.yp;
                const double rx = R00 * Xd + R01 * Yd, ry = R10 * Xd + R11 * Yd;
                const double* wg = a.wgeo + 6 * (size_t)w;
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
    // this block's share of the load, summed in thread order (a block with
    // no wall node writes the zeros that sum would give)
    __shared__ double red[3][EM_THREADS];
    double* pt0 = a.part + ((size_t)b * a.nblk + blockIdx.x) * 3;
    if (!__syncthreads_or(wallnode)) {
        if (threadIdx.x == 0) pt0[0] = pt0[1] = pt0[2] = 0.0;
        return;
    }
    red[0][threadIdx.x] = fcx;
    red[1][threadIdx.x] = fcy;
    red[2][threadIdx.x] = fcm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int t = 0; t < EM_THREADS; ++t) {
            s0 += red[0][t];
            s1 += red[1][t];
            s2 += red[2][t];
        }
        double* pt = a.part + ((size_t)b * a.nblk + blockIdx.x) * 3;
        pt[0] = s0;
        pt[1] = s1;
        pt[2] = s2;
    }
}

// ---- once per flow dt (init_fields): the departures of every interior node
// for the displacement of a node the blend does not move, by the same solves
// as k_em_stream (an inactive map gives its F = I and V_G = 0)
template <typename R>
__global__ void __launch_bounds__(EM_THREADS) k_em_record(const EArgs a) {
    using R2 = typename EVec<R>::T2;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= a.N) return;
    const size_t N = (size_t)a.N;
    R2* dxe = static_cast<R2*>(a.dep_xe);
    if (a.kind[n] != 0) {
        for (int q = 0; q < 9; ++q) {
            a.dep_e[q * N + n] = -1;
            dxe[q * N + n] = pair(R(0), R(0));
        }
        return;
    }
    const SolveDev& fl = a.flow;
    const R dt = flowv<R>(fl, fl.dt, fl.dt_f);
    const R* X = static_cast<const R*>(a.X);
    BodyMap<R> still{};
    still.active = 0;
    R i00, i01, i10, i11, vx, vy;
    inv_map(still, X[2 * n], X[2 * n + 1], i00, i01, i10, i11, vx, vy);
#pragma unroll 1
    for (int q = 0; q < 9; ++q) {
        const R cx = (R)cxq(q), cy = (R)cyq(q);
        const R hx = i00 * cx + i01 * cy - vx, hy = i10 * cx + i11 * cy - vy;
        int e;
        R xi, eta;
        if (em_locate<R>(a, n, -dt * hx, -dt * hy, e, xi, eta)) {
            a.dep_e[q * N + n] = e;
            dxe[q * N + n] = pair(xi, eta);
        } else {
            a.dep_e[q * N + n] = -1;
            dxe[q * N + n] = pair(R(0), R(0));
        }
    }
}

// ---- launch 4: one warp per solve: the load from the block partials in a
// fixed order (lane t sums blocks t, t + 32, ...; then the lanes in order),
// RK4 (Sec. III B) and the next step's blended maps
__global__ void k_em_finish(const EArgs a) {
    const int b = blockIdx.x, l = threadIdx.x;
    const double* pt = a.part + (size_t)b * a.nblk * 3;
    double v[3] = {0.0, 0.0, 0.0};
    for (int k = l; k < a.nblk; k += 32)
        for (int c = 0; c < 3; ++c) v[c] += pt[3 * k + c];
    double F[3] = {0.0, 0.0, 0.0};
    for (int t = 0; t < 32; ++t)
        for (int c = 0; c < 3; ++c) F[c] += __shfl_sync(0xffffffffu, v[c], t);
    if (l != 0) return;
    const BodyDev bd = a.bodies[b];
    const BodyStateDev Sn = a.maps_in[b].S_next;
    const BodyStateDev Snew = rk4_body(bd, Sn, F[1], F[2], a.flow.dt, (long long)a.kstep);
    StepMaps mo;
    build_maps(bd, Sn, Snew, Sn, a.flow.dt, mo);
    for (int c = 0; c < 3; ++c) mo.loads[c] = F[c];
    a.maps_out[b] = mo;
}

}  // namespace
}  // namespace lbfsi

using lbfsi::BodyDev;
using lbfsi::BodyStateDev;
using lbfsi::SolveDev;
using lbfsi::StepMaps;

struct lbfsi_emesh_s {
    int N = 0, Ne = 0, nwall = 0, nfarn = 0, nbatch = 0, precision = 0, nblk = 0;
    size_t es = 8;   // element size of the path
    cudaStream_t stream = nullptr;
    std::vector<lbfsi_body_desc> bodies;
    std::vector<void*> blocks;   // every device allocation
    // mesh
    void* X = nullptr;
    int* E = nullptr;
    void* ecoef = nullptr;
    int *hptr = nullptr, *hold = nullptr, *gptr = nullptr, *gcol = nullptr, *kind = nullptr;
    void* gw = nullptr;
    double *xw = nullptr, *n0 = nullptr, *wgeo = nullptr, *nfar = nullptr;
    // cached departures of the interior nodes the blend does not move
    // ([9][N] position in hold of the holding element, [9][N] (xi, eta)),
    // or null
    int* dep_e = nullptr;
    void* dep_xe = nullptr;
    // solves
    void* p[2] = {nullptr, nullptr};
    void* ppost = nullptr;
    void* M[2] = {nullptr, nullptr};
    void* D = nullptr;
    void* dQ = nullptr;   // [nbatch][2][N] dQ of the last streamed moments
    StepMaps* maps[2] = {nullptr, nullptr};
    BodyDev* dbodies = nullptr;
    double* part = nullptr;
    double* stage = nullptr;   // [nbatch][4][N] float64 staging
    BodyStateDev *st_a = nullptr, *st_b = nullptr;
    double* zl = nullptr;
    unsigned* status = nullptr;
    SolveDev flow{};
    std::vector<int> perm;   // library node i is the caller's node perm[i]
    bool initialized = false;
    unsigned k = 0;
    int64_t launches = 0;
    int cur() const { return (int)(k & 1u); }
};

namespace {

int efail(int code, const std::string& msg) { return lbfsi::set_error(code, msg); }
int ecuda(cudaError_t e, const char* where) {
    cudaGetLastError();
    return lbfsi::set_error(LBFSI_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
cudaError_t ealloc(lbfsi_emesh m, T** p, size_t count) {
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) {
        m->blocks.push_back(q);
        *p = static_cast<T*>(q);
    }
    return e;
}

void release(lbfsi_emesh m) {
    for (void* q : m->blocks) cudaFree(q);
    m->blocks.clear();
}

// Values of a float64 vector in the element type of the path.
std::vector<unsigned char> typed(const std::vector<double>& v, int precision) {
    std::vector<unsigned char> out;
    if (precision == LBFSI_FP64) {
        out.resize(v.size() * sizeof(double));
        std::memcpy(out.data(), v.data(), out.size());
    } else {
        std::vector<float> f(v.begin(), v.end());
        out.resize(f.size() * sizeof(float));
        std::memcpy(out.data(), f.data(), out.size());
    }
    return out;
}

// 1-D Q2 Lagrange derivatives at t (nodes -1, 0, 1).
void lagrange_d(double t, double* d) {
    d[0] = t - 0.5;
    d[1] = -2.0 * t;
    d[2] = t + 0.5;
}

// Nodal gradient operator, reading R33: for each node, the mean over its
// holding elements of the element's Q2 derivative at the node's reference
// position mapped by that element's Q2 metric there.  Rows: node -> (col,
// w_X, w_Y) with repeated columns merged in first-seen order.
// Z-order (Morton) numbering of N points: perm[i] is the point at position
// i of the curve through the bounding box quantised to 2^16 x 2^16 cells
// (ties in input order), inv its inverse.
void zorder(int N, const double* X, std::vector<int>& perm, std::vector<int>& inv) {
    double lo[2] = {X[0], X[1]}, hi[2] = {X[0], X[1]};
    for (int n = 0; n < N; ++n)
        for (int c = 0; c < 2; ++c) {
            lo[c] = std::min(lo[c], X[2 * (size_t)n + c]);
            hi[c] = std::max(hi[c], X[2 * (size_t)n + c]);
        }
    auto spread = [](unsigned v) {   // the 16 bits of v to the even bit positions
        v &= 0xffffu;
        v = (v | (v << 8)) & 0x00ff00ffu;
        v = (v | (v << 4)) & 0x0f0f0f0fu;
        v = (v | (v << 2)) & 0x33333333u;
        v = (v | (v << 1)) & 0x55555555u;
        return v;
    };
    std::vector<unsigned> code((size_t)N);
    for (int n = 0; n < N; ++n) {
        unsigned qc[2];
        for (int c = 0; c < 2; ++c) {
            const double w = hi[c] > lo[c] ? (X[2 * (size_t)n + c] - lo[c]) / (hi[c] - lo[c]) : 0.0;
            qc[c] = (unsigned)std::min(65535.0, std::max(0.0, std::floor(w * 65536.0)));
        }
        code[n] = spread(qc[0]) | (spread(qc[1]) << 1);
    }
    perm.resize((size_t)N);
    for (int n = 0; n < N; ++n) perm[n] = n;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return code[a] < code[b]; });
    inv.assign((size_t)N, 0);
    for (int i = 0; i < N; ++i) inv[perm[i]] = i;
}

int gradient_r33(int N, const std::vector<int>& E, const double* X, const std::vector<int>& hptr,
                 const std::vector<int>& hold, std::vector<int>& gptr, std::vector<int>& gcol,
                 std::vector<double>& gw) {
    gptr.assign(N + 1, 0);
    gcol.clear();
    gw.clear();
    for (int n = 0; n < N; ++n) {
        std::vector<int> cols;
        std::vector<double> wx, wy;
        auto add = [&](int m, double ax, double ay) {
            for (size_t k = 0; k < cols.size(); ++k)
                if (cols[k] == m) {
                    wx[k] += ax;
                    wy[k] += ay;
                    return;
                }
            cols.push_back(m);
            wx.push_back(ax);
            wy.push_back(ay);
        };
        const int nh = hptr[n + 1] - hptr[n];
        for (int h = hptr[n]; h < hptr[n + 1]; ++h) {
            const int e = hold[h] >> 4, ent = hold[h] & 15, a = ent / 3, b = ent % 3;
            double dxi[3], deta[3];
            lagrange_d(a - 1.0, dxi);
            lagrange_d(b - 1.0, deta);
            const int* en = &E[9 * (size_t)e];
            double xx = 0, xy = 0, ex = 0, ey = 0;   // x_xi, y_xi, x_eta, y_eta
            for (int k = 0; k < 3; ++k) {
                xx += dxi[k] * X[2 * en[3 * k + b]];
                xy += dxi[k] * X[2 * en[3 * k + b] + 1];
                ex += deta[k] * X[2 * en[3 * a + k]];
                ey += deta[k] * X[2 * en[3 * a + k] + 1];
            }
            const double det = xx * ey - xy * ex;
            if (!(det > 0.0)) return efail(LBFSI_EINVAL, "element not positively oriented at a node");
            const double s = 1.0 / nh;
            for (int k = 0; k < 3; ++k) {
                // d/dX = (y_eta d/dxi - y_xi d/deta) / det, d/dY = (-x_eta d/dxi + x_xi d/deta) / det
                add(en[3 * k + b], s * ey * dxi[k] / det, -s * ex * dxi[k] / det);
                add(en[3 * a + k], -s * xy * deta[k] / det, s * xx * deta[k] / det);
            }
        }
        for (size_t k = 0; k < cols.size(); ++k) {
            gcol.push_back(cols[k]);
            gw.push_back(wx[k]);
            gw.push_back(wy[k]);
        }
        gptr[n + 1] = (int)gcol.size();
    }
    return LBFSI_OK;
}

// Nodal gradient operator of reading R18 on an index grid (nr x nt, periodic
// in j): the derivative of the 1-D quadratic through a node and its
// neighbours along each index direction (one-sided on rows 0 and nr - 1),
// mapped by the inverse of the metric taken with the same stencils.
int gradient_r18(int N, const int* ij, int nr, int nt, const double* X, std::vector<int>& gptr,
                 std::vector<int>& gcol, std::vector<double>& gw) {
    if (nr < 3 || nt < 4 || (long long)nr * nt != N)
        return efail(LBFSI_EINVAL, "grid_nr x grid_nt must equal the node count");
    std::vector<int> at((size_t)N, -1);
    for (int n = 0; n < N; ++n) {
        const int i = ij[2 * n], j = ij[2 * n + 1];
        if (i < 0 || i >= nr || j < 0 || j >= nt || at[(size_t)i * nt + j] >= 0)
            return efail(LBFSI_EINVAL, "grid_ij must map the nodes one to one onto the grid");
        at[(size_t)i * nt + j] = n;
    }
    gptr.assign(N + 1, 0);
    gcol.clear();
    gw.clear();
    for (int n = 0; n < N; ++n) {
        const int i = ij[2 * n], j = ij[2 * n + 1];
        int ci[3];
        double wi[3];
        if (i == 0) {
            ci[0] = 0; ci[1] = 1; ci[2] = 2;
            wi[0] = -1.5; wi[1] = 2.0; wi[2] = -0.5;
        } else if (i == nr - 1) {
            ci[0] = nr - 1; ci[1] = nr - 2; ci[2] = nr - 3;
            wi[0] = 1.5; wi[1] = -2.0; wi[2] = 0.5;
        } else {
            ci[0] = i + 1; ci[1] = i - 1; ci[2] = i;
            wi[0] = 0.5; wi[1] = -0.5; wi[2] = 0.0;
        }
        const int jp = at[(size_t)i * nt + (j + 1) % nt], jm = at[(size_t)i * nt + (j + nt - 1) % nt];
        double xx = 0, xy = 0;
        for (int k = 0; k < 3; ++k) {
            const int m = at[(size_t)ci[k] * nt + j];
            xx += wi[k] * X[2 * m];
            xy += wi[k] * X[2 * m + 1];
        }
        const double ex = 0.5 * (X[2 * jp] - X[2 * jm]), ey = 0.5 * (X[2 * jp + 1] - X[2 * jm + 1]);
        const double det = xx * ey - xy * ex;
        if (!(det > 0.0)) return efail(LBFSI_EINVAL, "grid not positively oriented");
        for (int k = 0; k < 3; ++k) {
            if (wi[k] == 0.0) continue;
            gcol.push_back(at[(size_t)ci[k] * nt + j]);
            gw.push_back(ey * wi[k] / det);
            gw.push_back(-ex * wi[k] / det);
        }
        gcol.push_back(jp);
        gw.push_back(-xy * 0.5 / det);
        gw.push_back(xx * 0.5 / det);
        gcol.push_back(jm);
        gw.push_back(xy * 0.5 / det);
        gw.push_back(-xx * 0.5 / det);
        gptr[n + 1] = (int)gcol.size();
    }
    return LBFSI_OK;
}

template <typename R>
lbfsi::EArgs make_eargs(lbfsi_emesh m) {
    lbfsi::EArgs a{};
    a.N = m->N;
    a.nbatch = m->nbatch;
    a.nblk = m->nblk;
    a.kstep = (int)m->k;
    a.collide = m->k > 0u;
    a.X = m->X;
    a.E = m->E;
    a.ecoef = m->ecoef;
    a.hptr = m->hptr;
    a.hold = m->hold;
    a.gptr = m->gptr;
    a.gcol = m->gcol;
    a.gw = m->gw;
    a.kind = m->kind;
    a.xw = m->xw;
    a.n0 = m->n0;
    a.wgeo = m->wgeo;
    a.nfar = m->nfar;
    a.dep_e = m->dep_e;
    a.dep_xe = m->dep_xe;
    const int c = m->cur();
    a.p_in = m->p[c];
    a.ppost = m->ppost;
    a.p_out = m->p[c ^ 1];
    a.M_in = m->M[c];
    a.M_out = m->M[c ^ 1];
    a.D = m->D;
    a.dQ = m->dQ;
    a.maps_in = m->maps[c];
    a.maps_out = m->maps[c ^ 1];
    a.bodies = m->dbodies;
    a.part = m->part;
    a.flow = m->flow;
    a.status = m->status;
    return a;
}

// The correction field and the collision of the current step into ppost
// (at step 0, the initial state copied).
template <typename R>
cudaError_t launch_em_collide(lbfsi_emesh m) {
    const lbfsi::EArgs a = make_eargs<R>(m);
    const dim3 grid((unsigned)m->nblk, (unsigned)m->nbatch);
    if (a.collide) {
        lbfsi::k_em_D<R><<<grid, lbfsi::EM_THREADS, 0, m->stream>>>(a);
        m->launches++;
    }
    lbfsi::k_em_collide<R><<<grid, lbfsi::EM_THREADS, 0, m->stream>>>(a);
    m->launches++;
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_em_step(lbfsi_emesh m) {
    cudaError_t e = launch_em_collide<R>(m);
    if (e != cudaSuccess) return e;
    const lbfsi::EArgs a = make_eargs<R>(m);
    const dim3 grid((unsigned)m->nblk, (unsigned)m->nbatch);
    lbfsi::k_em_stream<R><<<grid, lbfsi::EM_THREADS, 0, m->stream>>>(a);
    lbfsi::k_em_finish<<<m->nbatch, 32, 0, m->stream>>>(a);
    m->launches += 2;
    return cudaGetLastError();
}

int em_status(lbfsi_emesh m) {
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return ecuda(e, "stream synchronize");
    unsigned st = 0;
    e = cudaMemcpy(&st, m->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ecuda(e, "status read");
    if (st & lbfsi::ST_DEPARTURE)
        return efail(LBFSI_EDEPARTURE, "departure point outside the elements holding its node (CFL)");
    if (st & lbfsi::ST_BPOINT)
        return efail(LBFSI_EDEPARTURE, "wall or far-field target point B outside the elements holding its node");
    if (st & lbfsi::ST_NONPHYS) return efail(LBFSI_ENONPHYS, "non-physical state (rho<=0, T<=0 or NaN)");
    return LBFSI_OK;
}

// Device array of the path's element type -> float64 host array.
int download(lbfsi_emesh m, const void* src, double* dst, size_t count) {
    int rc = em_status(m);
    if (rc) return rc;
    if (m->precision == LBFSI_FP64) {
        const cudaError_t e = cudaMemcpy(dst, src, count * sizeof(double), cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? LBFSI_OK : ecuda(e, "download");
    }
    std::vector<float> f(count);
    const cudaError_t e = cudaMemcpy(f.data(), src, count * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ecuda(e, "download");
    for (size_t i = 0; i < count; ++i) dst[i] = f[i];
    return LBFSI_OK;
}

}  // namespace

extern "C" {

int lbfsi_create_mesh_elements(const lbfsi_mesh_elements_desc* d, void* cuda_stream, lbfsi_emesh* out) {
    lbfsi::TraceRange trace_("lbfsi_create_mesh_elements");
    if (!d || !out) return efail(LBFSI_EINVAL, "null argument");
    *out = nullptr;
    const int N = d->nnode, Ne = d->nelem;
    if (N < 9 || Ne < 1 || !d->X || !d->elements) return efail(LBFSI_EINVAL, "empty node or element list");
    if (d->precision != LBFSI_FP64 && d->precision != LBFSI_FP32)
        return efail(LBFSI_EINVAL, "precision must be LBFSI_FP64 or LBFSI_FP32");
    if (d->nbatch < 1 || !d->bodies) return efail(LBFSI_EINVAL, "nbatch >= 1 bodies required");
    if (d->nwall < 4 || d->nwall % 2 || !d->wall || d->nfar < 4 || d->nfar % 2 || !d->far)
        return efail(LBFSI_EINVAL, "wall and far-field chains must have an even length >= 4");
    if ((long long)N * 9 > (1ll << 31) / 2) return efail(LBFSI_EINVAL, "mesh too large");
    double scale = 0.0;
    for (int k = 0; k < 2 * N; ++k) {
        if (!std::isfinite(d->X[k])) return efail(LBFSI_EINVAL, "node coordinates must be finite");
        scale = std::max(scale, std::fabs(d->X[k]));
    }
    std::vector<int> E(d->elements, d->elements + 9 * (size_t)Ne);
    for (int v : E)
        if (v < 0 || v >= N) return efail(LBFSI_EINVAL, "element node index out of range");
    // The library numbers the nodes along a Z-order curve of their
    // coordinates: the EM_THREADS consecutive nodes of a stream block are then
    // close in space, so the nodes their gathers read stay few (and in
    // cache) and the block's writes coalesce.  Elements keep the caller's
    // order (the departure search visits them in it); the calls that take or
    // return node fields map between the two numberings.
    std::vector<int> perm, inv;
    zorder(N, d->X, perm, inv);
    std::vector<double> Xr(2 * (size_t)N);
    for (int i = 0; i < N; ++i) {
        Xr[2 * (size_t)i] = d->X[2 * (size_t)perm[i]];
        Xr[2 * (size_t)i + 1] = d->X[2 * (size_t)perm[i] + 1];
    }
    const double* X = Xr.data();
    for (int& v : E) v = inv[v];
    std::vector<int> ijr;
    if (d->grid_ij) {
        ijr.resize(2 * (size_t)N);
        for (int i = 0; i < N; ++i) {
            ijr[2 * (size_t)i] = d->grid_ij[2 * (size_t)perm[i]];
            ijr[2 * (size_t)i + 1] = d->grid_ij[2 * (size_t)perm[i] + 1];
        }
    }
    // subparametric elements: every node at the bilinear position of the corners
    std::vector<double> ecoef(6 * (size_t)Ne);
    for (int e = 0; e < Ne; ++e) {
        const int* en = &E[9 * (size_t)e];
        for (int c = 0; c < 2; ++c) {
            const double c00 = X[2 * en[0] + c], c10 = X[2 * en[6] + c], c01 = X[2 * en[2] + c],
                         c11 = X[2 * en[8] + c];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const double xi = a - 1.0, et = b - 1.0;
                    const double v = 0.25 * ((1 - xi) * (1 - et) * c00 + (1 + xi) * (1 - et) * c10 +
                                             (1 - xi) * (1 + et) * c01 + (1 + xi) * (1 + et) * c11);
                    if (std::fabs(v - X[2 * en[3 * a + b] + c]) > 1e-12 * scale)
                        return efail(LBFSI_EINVAL, "elements must be subparametric (mid nodes at the bilinear "
                                                   "positions of the corners)");
                }
            ecoef[6 * (size_t)e + c] = 0.25 * (-c00 + c10 - c01 + c11);
            ecoef[6 * (size_t)e + 2 + c] = 0.25 * (-c00 - c10 + c01 + c11);
            ecoef[6 * (size_t)e + 4 + c] = 0.25 * (c00 - c10 - c01 + c11);
        }
    }
    // node -> holding elements, in increasing element index
    std::vector<int> hcount(N + 1, 0);
    for (int e = 0; e < Ne; ++e)
        for (int s = 0; s < 9; ++s) hcount[E[9 * (size_t)e + s] + 1]++;
    std::vector<int> hptr(N + 1, 0);
    for (int n = 0; n < N; ++n) {
        if (hcount[n + 1] == 0) return efail(LBFSI_EINVAL, "every node must belong to an element");
        hptr[n + 1] = hptr[n] + hcount[n + 1];
    }
    std::vector<int> hold((size_t)hptr[N]), fill(hptr.begin(), hptr.end() - 1);
    for (int e = 0; e < Ne; ++e)
        for (int s = 0; s < 9; ++s) {
            const int n = E[9 * (size_t)e + s];
            hold[fill[n]++] = e * 16 + s;
        }
    // gradient operator
    std::vector<int> gptr, gcol;
    std::vector<double> gw;
    int rc = d->grid_ij ? gradient_r18(N, ijr.data(), d->grid_nr, d->grid_nt, X, gptr, gcol, gw)
                        : gradient_r33(N, E, X, hptr, hold, gptr, gcol, gw);
    if (rc) return rc;
    // elements stored in the order of their centre nodes (so along the same
    // curve as the nodes); each node's list of holding elements keeps the
    // caller's element order, the order of the departure search
    std::vector<int> eperm((size_t)Ne), einv((size_t)Ne);
    for (int e2 = 0; e2 < Ne; ++e2) eperm[e2] = e2;
    std::stable_sort(eperm.begin(), eperm.end(),
                     [&](int a, int b) { return E[9 * (size_t)a + 4] < E[9 * (size_t)b + 4]; });
    for (int k = 0; k < Ne; ++k) einv[eperm[k]] = k;
    {
        std::vector<int> Es(E.size());
        std::vector<double> cs(ecoef.size());
        for (int k = 0; k < Ne; ++k) {
            std::copy_n(&E[9 * (size_t)eperm[k]], 9, &Es[9 * (size_t)k]);
            std::copy_n(&ecoef[6 * (size_t)eperm[k]], 6, &cs[6 * (size_t)k]);
        }
        E.swap(Es);
        ecoef.swap(cs);
        for (int& h : hold) h = einv[h >> 4] * 16 + (h & 15);
    }
    // chains
    std::vector<int> kind(N, 0);
    std::vector<double> pw(2 * (size_t)d->nwall), pf(2 * (size_t)d->nfar);
    for (int w = 0; w < d->nwall; ++w) {
        const int n = d->wall[w] >= 0 && d->wall[w] < N ? inv[d->wall[w]] : -1;
        if (n < 0 || kind[n] != 0) return efail(LBFSI_EINVAL, "wall chain: bad or repeated node");
        kind[n] = w + 1;
        pw[2 * w] = X[2 * n];
        pw[2 * w + 1] = X[2 * n + 1];
    }
    for (int f = 0; f < d->nfar; ++f) {
        const int n = d->far[f] >= 0 && d->far[f] < N ? inv[d->far[f]] : -1;
        if (n < 0 || kind[n] != 0) return efail(LBFSI_EINVAL, "far-field chain: bad or repeated node");
        kind[n] = -(f + 1);
        pf[2 * f] = X[2 * n];
        pf[2 * f + 1] = X[2 * n + 1];
    }
    std::vector<double> n0, wgeo, nfar, fgeo;
    lbfsi::chain_geometry(pw, n0, wgeo);
    lbfsi::chain_geometry(pf, nfar, fgeo);
    // bodies: the wall inside each body's rigid zone
    for (int b = 0; b < d->nbatch; ++b) {
        const lbfsi_body_desc& bd = d->bodies[b];
        if (bd.dof < 0 || bd.dof > 2) return efail(LBFSI_EINVAL, "body dof must be 0, 1 or 2");
        if (bd.dof != 0) {
            if (!(bd.r_out > bd.r_in && bd.r_in > 0)) return efail(LBFSI_EINVAL, "blend radii: 0 < r_in < r_out");
            for (int w = 0; w < d->nwall; ++w)
                if (std::hypot(pw[2 * w] - bd.xc, pw[2 * w + 1] - bd.yc) >= bd.r_in)
                    return efail(LBFSI_EINVAL, "the wall must lie inside the body's rigid zone (r < r_in)");
        }
    }
    lbfsi_emesh m = new lbfsi_emesh_s();
    m->N = N;
    m->Ne = Ne;
    m->nwall = d->nwall;
    m->nfarn = d->nfar;
    m->nbatch = d->nbatch;
    m->precision = d->precision;
    m->es = d->precision == LBFSI_FP64 ? sizeof(double) : sizeof(float);
    m->nblk = (N + lbfsi::EM_THREADS - 1) / lbfsi::EM_THREADS;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    m->bodies.assign(d->bodies, d->bodies + d->nbatch);
    m->perm = perm;
    const size_t es = m->es, nb = (size_t)d->nbatch;
    std::vector<double> Xv(X, X + 2 * (size_t)N);
    auto put = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
        unsigned char* q = nullptr;
        cudaError_t e = ealloc(m, &q, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(q, src, bytes, cudaMemcpyHostToDevice);
        *dst = q;
        return e;
    };
    const std::vector<unsigned char> Xt = typed(Xv, d->precision), ect = typed(ecoef, d->precision),
                                     gwt = typed(gw, d->precision);
    cudaError_t e = put(&m->X, Xt.data(), Xt.size());
    std::vector<int> Ep((size_t)Ne * lbfsi::EN_STRIDE, 0);
    for (size_t k = 0; k < (size_t)Ne; ++k)
        for (int s = 0; s < 9; ++s) Ep[k * lbfsi::EN_STRIDE + s] = E[9 * k + s];
    if (e == cudaSuccess) e = put((void**)&m->E, Ep.data(), Ep.size() * sizeof(int));
    if (e == cudaSuccess) e = put(&m->ecoef, ect.data(), ect.size());
    if (e == cudaSuccess) e = put((void**)&m->hptr, hptr.data(), hptr.size() * sizeof(int));
    if (e == cudaSuccess) e = put((void**)&m->hold, hold.data(), hold.size() * sizeof(int));
    if (e == cudaSuccess) e = put((void**)&m->gptr, gptr.data(), gptr.size() * sizeof(int));
    if (e == cudaSuccess) e = put((void**)&m->gcol, gcol.data(), std::max<size_t>(gcol.size(), 1) * sizeof(int));
    if (e == cudaSuccess) e = put(&m->gw, gwt.data(), std::max<size_t>(gwt.size(), 1));
    if (e == cudaSuccess) e = put((void**)&m->kind, kind.data(), kind.size() * sizeof(int));
    if (e == cudaSuccess) e = put((void**)&m->xw, pw.data(), pw.size() * sizeof(double));
    if (e == cudaSuccess) e = put((void**)&m->n0, n0.data(), n0.size() * sizeof(double));
    if (e == cudaSuccess) e = put((void**)&m->wgeo, wgeo.data(), wgeo.size() * sizeof(double));
    if (e == cudaSuccess) e = put((void**)&m->nfar, nfar.data(), nfar.size() * sizeof(double));
    unsigned char* q = nullptr;
    for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
        e = ealloc(m, &q, nb * 9 * N * 2 * es);
        m->p[c] = q;
        if (e == cudaSuccess) e = ealloc(m, &q, nb * 4 * N * es);
        m->M[c] = q;
        if (e == cudaSuccess) e = ealloc(m, &m->maps[c], nb);
    }
    if (e == cudaSuccess) e = ealloc(m, &q, nb * 9 * N * 2 * es);
    m->ppost = q;
    if (e == cudaSuccess) e = ealloc(m, &q, nb * 2 * N * es);
    m->D = q;
    if (e == cudaSuccess) e = ealloc(m, &q, nb * 2 * N * es);
    m->dQ = q;
    if (e == cudaSuccess) e = ealloc(m, &m->dbodies, nb);
    if (e == cudaSuccess) e = ealloc(m, &m->part, nb * m->nblk * 3);
    if (e == cudaSuccess) e = ealloc(m, &m->stage, nb * 4 * N);
    if (e == cudaSuccess) e = ealloc(m, &m->st_a, nb);
    if (e == cudaSuccess) e = ealloc(m, &m->st_b, nb);
    if (e == cudaSuccess) e = ealloc(m, &m->zl, nb * 3);
    if (e == cudaSuccess) e = ealloc(m, &m->status, 1);
    if (e == cudaSuccess) e = cudaMemset(m->status, 0, sizeof(unsigned));
    // departures of the static interior nodes, solved once per time step
    // size (LBFSI_NO_DEPARTURE_CACHE=1 solves them every step instead; the
    // results are the same)
    const char* nc = std::getenv("LBFSI_NO_DEPARTURE_CACHE");
    if (e == cudaSuccess && !(nc && std::atoi(nc) != 0)) {
        e = ealloc(m, &m->dep_e, 9 * (size_t)N);
        if (e == cudaSuccess) e = ealloc(m, &q, 9 * (size_t)N * 2 * es);
        m->dep_xe = q;
    }
    if (e != cudaSuccess) {
        release(m);
        delete m;
        cudaGetLastError();
        return efail(e == cudaErrorMemoryAllocation ? LBFSI_ENOMEM : LBFSI_ECUDA,
                     std::string("element mesh upload: ") + cudaGetErrorString(e));
    }
    *out = m;
    return LBFSI_OK;
}

int lbfsi_emesh_destroy(lbfsi_emesh m) {
    if (!m) return LBFSI_OK;
    cudaStreamSynchronize(m->stream);
    release(m);
    delete m;
    return LBFSI_OK;
}

int lbfsi_emesh_init_fields(lbfsi_emesh m, const lbfsi_flow_params* p, const double* rho_u_T) {
    lbfsi::TraceRange trace_("lbfsi_emesh_init_fields");
    if (!m || !p) return efail(LBFSI_EINVAL, "null argument");
    SolveDev proto{};
    int rc = lbfsi::fill_flow(*p, proto);
    if (rc) return rc;
    m->flow = proto;
    const size_t N = (size_t)m->N, nb = (size_t)m->nbatch;
    std::vector<BodyDev> bd(nb);
    for (size_t b = 0; b < nb; ++b) bd[b] = lbfsi::body_dev(m->bodies[b], proto.rho_inf, proto.uinf_x);
    std::vector<double> Mh;
    if (rho_u_T) {
        // the caller's node order -> the library's
        Mh.resize(nb * 4 * N);
        for (size_t r = 0; r < nb * 4; ++r)
            for (size_t i = 0; i < N; ++i) Mh[r * N + i] = rho_u_T[r * N + (size_t)m->perm[i]];
    } else {
        Mh.resize(nb * 4 * N);
        for (size_t b = 0; b < nb; ++b)
            for (size_t n = 0; n < N; ++n) {
                Mh[(b * 4 + 0) * N + n] = proto.rho_inf;
                Mh[(b * 4 + 1) * N + n] = proto.uinf_x;
                Mh[(b * 4 + 2) * N + n] = 0.0;
                Mh[(b * 4 + 3) * N + n] = proto.T_inf;
            }
    }
    std::vector<BodyStateDev> zero(nb, BodyStateDev{0.0, 0.0, 0.0, 0.0});
    std::vector<double> zl(nb * 3, 0.0);
    cudaError_t e = cudaMemcpyAsync(m->dbodies, bd.data(), nb * sizeof(BodyDev), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->stage, Mh.data(), nb * 4 * N * sizeof(double), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->st_a, zero.data(), nb * sizeof(BodyStateDev), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->zl, zl.data(), zl.size() * sizeof(double), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, sizeof(unsigned), m->stream);
    if (e != cudaSuccess) return ecuda(e, "init_fields upload");
    m->k = 0;
    e = lbfsi::launch_init(m->precision, m->stage, m->p[0], m->M[0], m->N, m->nbatch, proto.Cv, m->stream);
    if (e == cudaSuccess)
        e = lbfsi::launch_prepare(m->dbodies, m->st_a, m->st_a, m->st_a, m->zl, proto.dt, m->nbatch, m->maps[0],
                                  m->stream);
    m->launches += 2;
    if (e == cudaSuccess && m->dep_e) {
        const unsigned blocks = (unsigned)m->nblk;
        if (m->precision == LBFSI_FP64)
            lbfsi::k_em_record<double><<<blocks, lbfsi::EM_THREADS, 0, m->stream>>>(make_eargs<double>(m));
        else
            lbfsi::k_em_record<float><<<blocks, lbfsi::EM_THREADS, 0, m->stream>>>(make_eargs<float>(m));
        m->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return ecuda(e, "init_fields");
    m->initialized = true;
    return LBFSI_OK;
}

int lbfsi_emesh_blend_mesh(lbfsi_emesh m, const lbfsi_body_state* state, const lbfsi_body_state* prev) {
    if (!m || !state) return efail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return efail(LBFSI_ESTATE, "init_fields first");
    static_assert(sizeof(lbfsi_body_state) == sizeof(BodyStateDev), "layout");
    const size_t nb = (size_t)m->nbatch;
    cudaError_t e = cudaMemcpyAsync(m->st_a, state, nb * sizeof(BodyStateDev), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->st_b, prev ? prev : state, nb * sizeof(BodyStateDev), cudaMemcpyHostToDevice,
                            m->stream);
    if (e == cudaSuccess)
        e = lbfsi::launch_prepare(m->dbodies, m->k == 0u ? m->st_a : nullptr, m->st_a, m->st_b, nullptr,
                                  m->flow.dt, m->nbatch, m->maps[m->cur()], m->stream);
    m->launches++;
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return ecuda(e, "blend_mesh");
    return LBFSI_OK;
}

int lbfsi_emesh_step(lbfsi_emesh m, int nsteps) {
    lbfsi::TraceRange trace_("lbfsi_emesh_step");
    if (!m) return efail(LBFSI_EINVAL, "null mesh");
    if (!m->initialized) return efail(LBFSI_ESTATE, "init_fields first");
    if (nsteps < 0) return efail(LBFSI_EINVAL, "nsteps must be >= 0");
    for (int s = 0; s < nsteps; ++s) {
        const cudaError_t e = m->precision == LBFSI_FP64 ? launch_em_step<double>(m) : launch_em_step<float>(m);
        if (e != cudaSuccess) return ecuda(e, "element step launch");
        m->k++;
    }
    return LBFSI_OK;
}

int lbfsi_emesh_synchronize(lbfsi_emesh m) {
    if (!m) return efail(LBFSI_EINVAL, "null mesh");
    return em_status(m);
}

int lbfsi_emesh_body_forces(lbfsi_emesh m, double* out) {
    if (!m || !out) return efail(LBFSI_EINVAL, "null argument");
    const int rc = em_status(m);
    if (rc) return rc;
    std::vector<StepMaps> mp((size_t)m->nbatch);
    const cudaError_t e = cudaMemcpy(mp.data(), m->maps[m->cur()], mp.size() * sizeof(StepMaps), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ecuda(e, "loads download");
    for (int b = 0; b < m->nbatch; ++b)
        for (int c = 0; c < 3; ++c) out[3 * b + c] = mp[b].loads[c];
    return LBFSI_OK;
}

int lbfsi_emesh_get_body_state(lbfsi_emesh m, lbfsi_body_state* out) {
    if (!m || !out) return efail(LBFSI_EINVAL, "null argument");
    const int rc = em_status(m);
    if (rc) return rc;
    std::vector<StepMaps> mp((size_t)m->nbatch);
    const cudaError_t e = cudaMemcpy(mp.data(), m->maps[m->cur()], mp.size() * sizeof(StepMaps), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ecuda(e, "state download");
    for (int b = 0; b < m->nbatch; ++b) {
        out[b].h = mp[b].S_next.h;
        out[b].alpha = mp[b].S_next.alpha;
        out[b].hdot = mp[b].S_next.hdot;
        out[b].adot = mp[b].S_next.adot;
    }
    return LBFSI_OK;
}

int lbfsi_emesh_get_fields(lbfsi_emesh m, double* rho_u_T) {
    if (!m || !rho_u_T) return efail(LBFSI_EINVAL, "null argument");
    const size_t N = (size_t)m->N, rows = (size_t)m->nbatch * 4;
    std::vector<double> v(rows * N);
    const int rc = download(m, m->M[m->cur()], v.data(), rows * N);
    if (rc) return rc;
    for (size_t r = 0; r < rows; ++r)
        for (size_t i = 0; i < N; ++i) rho_u_T[r * N + (size_t)m->perm[i]] = v[r * N + i];
    return LBFSI_OK;
}

int lbfsi_emesh_get_populations(lbfsi_emesh m, int which, double* f, double* g) {
    if (!m || !f || !g) return efail(LBFSI_EINVAL, "null argument");
    if (which != 0 && which != 1) return efail(LBFSI_EINVAL, "which must be 0 or 1");
    if (!m->initialized) return efail(LBFSI_ESTATE, "init_fields first");
    const size_t cnt = (size_t)m->nbatch * 9 * m->N;
    if (which == 1) {
        // the collision of the current step into the post-collision buffer
        // (which the next step's collision overwrites anyway)
        cudaError_t e = m->precision == LBFSI_FP64 ? launch_em_collide<double>(m) : launch_em_collide<float>(m);
        if (e != cudaSuccess) return ecuda(e, "collision launch");
    }
    std::vector<double> pairs(2 * cnt);
    const int rc = download(m, which == 0 ? m->p[m->cur()] : m->ppost, pairs.data(), 2 * cnt);
    if (rc) return rc;
    for (size_t k = 0; k < cnt; ++k) {
        double fv = pairs[2 * k], gv = pairs[2 * k + 1];
        if (which == 1 && m->precision == LBFSI_FP32) {
            // the float path keeps the post-collision pairs as deviations
            // from the free stream's
            const int q = (int)((k / m->N) % 9);
            fv += (double)m->flow.fgref[2 * q];
            gv += (double)m->flow.fgref[2 * q + 1];
        }
        const size_t row = k / m->N, to = row * m->N + (size_t)m->perm[k - row * m->N];
        f[to] = fv;
        g[to] = gv;
    }
    return LBFSI_OK;
}

int64_t lbfsi_emesh_launch_count(lbfsi_emesh m) { return m ? m->launches : -1; }

}  // extern "C"
