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
//   prologue   the solve's step number; the blended maps of steps k and k+1
//              (Sec. II D), built by the previous launch
//   phase 1    stage M^k of the tile +-4 nodes, the per-row / per-column
//              geometry, and the populations of the tile +-2 nodes in shared
//              memory, all as 16-byte asynchronous copies
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
//   epilogue   the last CTA of each solve reduces the partials and advances
//              the body by RK4 (Sec. III B) into the next launch's maps.
//
// Populations are kept in HBM as (f_q, g_q) pairs, [q][node] (both share the
// departure point and the interpolation weights), so staging moves 16-byte
// chunks and the stream writes one 64-bit pair per direction.  The redundant
// work is the collision of the 2-node halo; the HBM traffic per node is the
// 18 populations read and written once plus the 4-value moment field.
#include <climits>
#include <cstdio>
#include <type_traits>

#include "lbfsi_device.cuh"
#include "lbfsi_internal.h"

namespace lbfsi {

template <int TI, int TJ>
struct Tile {
    static constexpr int HP = 2, HD = 3, HM = 4;
    static constexpr int PH = TI + 2 * HP, PW = TJ + 2 * HP, PS = PH * PW;
    // staged populations: rows of PWS nodes from j0 - 4 (16-byte aligned
    // chunks), so the +-2 region starts at column 2 of a row
    static constexpr int PWS = TJ + 8, PSS = PH * PWS, PC = 2;
    static constexpr int DH = TI + 2 * HD, DW = TJ + 2 * HD, DS = DH * DW;
    static constexpr int MH = TI + 2 * HM, MW = TJ + 2 * HM, MS = MH * MW;
    static constexpr int NT = TI * TJ;
};

template <typename R>
struct Vec2;
template <>
struct Vec2<float> {
    using T = float2;
};
template <>
struct Vec2<double> {
    using T = double2;
};

// Shared-memory strides of the geometry tables: a row is read by whole warps
// (broadcast); consecutive columns are 20 words apart, so the 16-byte loads of
// eight threads (one shared-memory wavefront) cover distinct banks.
constexpr int RS = ROWTAB;
constexpr int CS = COLTAB + 4;

// Four consecutive table entries (16-byte aligned) in one or two loads.
__device__ __forceinline__ void ld4(const float* p, float& a, float& b, float& c, float& d) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double& a, double& b, double& c, double& d) {
    const double2 u = *reinterpret_cast<const double2*>(p);
    const double2 v = *reinterpret_cast<const double2*>(p + 2);
    a = u.x; b = u.y; c = v.x; d = v.y;
}

// Per-cell element coefficients of a general mesh (entries per cell).
constexpr int CELLC = 8;

template <typename R, int TI, int TJ, bool GEN>
constexpr size_t step_smem_bytes() {
    using T = Tile<TI, TJ>;
    return sizeof(R) * (size_t)(18 * T::PSS + 4 * T::MS + 2 * T::MS + 4 * T::DS + 2 * T::DS +
                                (GEN ? 6 * T::DS + (TI + 1) * (TJ + 1) * CELLC : T::MH * RS + T::MW * CS));
}

// Bounds-checked build (LBFSI_BOUNDS_CHECK): the shared-memory windows the
// step reads and the global slots it writes are checked; an index outside
// its buffer sets ST_BOUNDS and the access is skipped.  The substitute for a
// memory checker where none can run; without the macro every check is true.
#ifdef LBFSI_BOUNDS_CHECK
__device__ __forceinline__ bool in_bounds(bool ok, unsigned* st) {
    if (!ok) atomicOr(st, ST_BOUNDS);
    return ok;
}
#else
__device__ __forceinline__ bool in_bounds(bool, unsigned*) { return true; }
#endif

// Derivative along an index direction of the 1-D quadratic Lagrange interpolant
// through a node and its neighbours, evaluated at the node (Eq. ddx+fem):
// central inside, one-sided (-3 c0 + 4 c1 - c2)/2 on the first row,
// (3 cN - 4 cN-1 + cN-2)/2 on the last.  p points at the node.
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
// The same stencils on a general mesh that may be a C-grid (cg): central
// along i at row-0 nodes whose row below is the mirrored row across the cut
// (across), one-sided along j at the outlet columns and, at the two copies of
// the rear point, along the cut.  With cg == 0 and across == false they are
// d_row and d_col.
template <typename R>
__device__ __forceinline__ R d_row_c(const R* p, int stride, int i, int nr, bool across, bool wrap_rows = false) {
    if (!wrap_rows) {   // a periodic box has no first or last row
        if (i == 0 && !across) return R(0.5) * (R(-3) * p[0] + R(4) * p[stride] - p[2 * stride]);
        if (i == nr - 1) return R(0.5) * (R(3) * p[0] - R(4) * p[-stride] + p[-2 * stride]);
    }
    return R(0.5) * (p[stride] - p[-stride]);
}
// jdir: at a row-0 junction of a C-grid, +1 (the cut is the next column) or
// -1 (the previous one); 0 elsewhere.
template <typename R>
__device__ __forceinline__ R d_col_c(const R* p, int j, int nt, int cg, int jdir) {
    if (cg) {
        if (j == 0 || jdir > 0) return R(0.5) * (R(-3) * p[0] + R(4) * p[1] - p[2]);
        if (j == nt - 1 || jdir < 0) return R(0.5) * (R(3) * p[0] - R(4) * p[-1] + p[-2]);
    }
    return R(0.5) * (p[1] - p[-1]);
}

template <typename R>
__device__ __forceinline__ void lagrange3(R t, R* L) {
    L[0] = t * (R(0.5) * t - R(0.5));
    L[1] = R(1) - t * t;
    L[2] = t * (R(0.5) * t + R(0.5));
}

// Departure point of node (i, j) displaced by d, in the reference coordinates
// of its element (Eq. depPnt).  On the subparametric O-grid the bilinear map
// of every element factorises, X(xi, eta) = R(xi) E(eta) with R linear in xi
// (radius) and E linear in eta (a point on the chord between two direction
// vectors), so the inverse is closed-form and relative to the node:
//   eta - eta_node = s = -(e_j x d) / (r_i (dE x e_j) + dE x d)
//   R - r_i = (d . E - r_i s dE . E) / |E|^2,   E = e_j + s dE
// with dE = dE/deta of the element.  The adjacent cell is picked by the signs
// of e_j x d (which side of the ray through the node) and of R - r_i (which
// side of the ring through the node); lines of constant eta are rays and of
// constant xi are rings, so this choice is exact.
//
// NodeGeo holds the table entries of one node and, for the four candidate
// cells (da, db) in {-1, 0}^2, the shared-memory node offset of their
// element's first node, so that the nine directions only select among them.
template <typename R>
struct NodeGeo {
    R ex, ey, ri;
    R eta0, dEx0, dEy0, cq0, eta1, dEx1, dEy1, cq1;   // angular cells j-1 (0) and j (1)
    R xin0, idR0, xin1, idR1;                       // radial cells i-1 (0) and i (1)
    int b00, b01, b10, b11;                         // element origins, [da][db]
};

template <typename R>
__device__ __forceinline__ void node_geo(int i, int j, int nr, const R* row, const R* col, int pi0,
                                         int sj0, int PWS, NodeGeo<R>& G) {
    R u0, u1;
    ld4(col + CT_E, G.ex, G.ey, u0, u1);
    G.ri = row[RT_R];
    ld4(col + CT_C0, G.eta0, G.dEx0, G.dEy0, G.cq0);
    ld4(col + CT_C1, G.eta1, G.dEx1, G.dEy1, G.cq1);
    ld4(row + RT_XIN0, G.xin0, G.idR0, G.xin1, G.idR1);
    const int wa0 = min((max(i - 1, 0) >> 1) * 2, nr - 3);   // the wall row has no cell i-1
    const int wa1 = min((i >> 1) * 2, nr - 3);
    const int wb0 = ((j - 1) >> 1) * 2, wb1 = (j >> 1) * 2;
    G.b00 = (wa0 - pi0) * PWS + (wb0 - sj0);
    G.b01 = (wa0 - pi0) * PWS + (wb1 - sj0);
    G.b10 = (wa1 - pi0) * PWS + (wb0 - sj0);
    G.b11 = (wa1 - pi0) * PWS + (wb1 - sj0);
}

template <typename R>
__device__ __forceinline__ bool depart(const NodeGeo<R>& G, int i, R dx, R dy, int& base, R& xi,
                                       R& eta) {
    const R cr = G.ex * dy - G.ey * dx;
    const bool db = !(cr < R(0));
    const R dEx = db ? G.dEx1 : G.dEx0, dEy = db ? G.dEy1 : G.dEy0;
    const R s = -cr * rcp_(G.ri * (db ? G.cq1 : G.cq0) + (dEx * dy - dEy * dx));
    const R Ex = G.ex + s * dEx, Ey = G.ey + s * dEy;
    const R dR = (dx * Ex + dy * Ey - G.ri * s * (dEx * Ex + dEy * Ey)) * rcp_(Ex * Ex + Ey * Ey);
    const bool da = !(dR < R(0)) || i == 0;   // on the wall: round-off of a tangential departure
    const R dxi = dR * (da ? G.idR1 : G.idR0);
    xi = (da ? G.xin1 : G.xin0) + dxi;
    eta = (db ? G.eta1 : G.eta0) + s;
    base = da ? (db ? G.b11 : G.b10) : (db ? G.b01 : G.b00);
    const R lim = R(1) + R(1e-4);
    return abs_(s) <= lim && abs_(dxi) <= lim;
}

// The same solve for a node the blend does not move (g = I, V_G = 0), where
// the displacement is the constant d = -dt c for the lattice velocity
// c = (CX, CY): the products with d reduce to sums of table entries.
template <int CX, int CY, typename R>
__device__ __forceinline__ bool depart_static(const NodeGeo<R>& G, R dt, int& base, R& xi, R& eta) {
    // e x c and dE x c for the two angular cells; d = -dt c
    const R exc = (CY ? G.ex * R(CY) : R(0)) - (CX ? G.ey * R(CX) : R(0));
    const R cr = -dt * exc;
    const bool db = !(cr < R(0));
    const R dEx = db ? G.dEx1 : G.dEx0, dEy = db ? G.dEy1 : G.dEy0;
    const R dexc = (CY ? dEx * R(CY) : R(0)) - (CX ? dEy * R(CX) : R(0));
    const R s = -cr * rcp_(G.ri * (db ? G.cq1 : G.cq0) - dt * dexc);
    const R Ex = G.ex + s * dEx, Ey = G.ey + s * dEy;
    const R cE = (CX ? R(CX) * Ex : R(0)) + (CY ? R(CY) * Ey : R(0));
    const R dR = (-dt * cE - G.ri * s * (dEx * Ex + dEy * Ey)) * rcp_(Ex * Ex + Ey * Ey);
    const bool da = !(dR < R(0));
    const R dxi = dR * (da ? G.idR1 : G.idR0);
    xi = (da ? G.xin1 : G.xin0) + dxi;
    eta = (db ? G.eta1 : G.eta0) + s;
    base = da ? (db ? G.b11 : G.b10) : (db ? G.b01 : G.b00);
    const R lim = R(1) + R(1e-4);
    return abs_(s) <= lim && abs_(dxi) <= lim;
}

// Map from index derivatives (C_xi, C_eta) at a node to the physical gradient:
// grad_X C = J^{-1} (C_xi, C_eta) (Eq. ddx+fem) with the separable O-grid
// metric, then grad_x = g^{-1} grad_X = F^{-T} grad_X (Eq. dx_ref).
template <typename R>
__device__ __forceinline__ void grad_map_j(R j00, R j01, R j10, R j11, R F00, R F01, R F10, R F11,
                                           R* G) {
    const R idet = rcp_(F00 * F11 - F01 * F10);
    const R i00 = F11 * idet, i01 = -F01 * idet, i10 = -F10 * idet, i11 = F00 * idet;
    G[0] = i00 * j00 + i10 * j10;
    G[1] = i00 * j01 + i10 * j11;
    G[2] = i01 * j00 + i11 * j10;
    G[3] = i01 * j01 + i11 * j11;
}

// J^{-1} of the separable O-grid from its row and column tables.
template <typename R>
__device__ __forceinline__ void grad_map(const R* row, const R* col, R F00, R F01, R F10, R F11,
                                         R* G) {
    R c0, c1, c2, c3;
    ld4(col + CT_G, c0, c1, c2, c3);
    grad_map_j(row[RT_IDRC] * c0, -row[RT_IR] * c1, -row[RT_IDRC] * c2, row[RT_IR] * c3, F00, F01, F10,
               F11, G);
}

// Departure point on a general mesh (Eq. depPnt): the node's Q2 element for
// the adjacent cell (a, b) the displacement d points into (its index-space
// direction J^{-1} d at the node), then Newton's method on the element's
// bilinear map X0 + b xi + c eta + d xi eta relative to the node's own local
// coordinates (xi0, eta0): (b + d eta0) u + (c + d xi0) v + d u v = d, which
// involves no absolute coordinates.  If the point falls outside that element
// the other adjacent cell is tried in the direction it left by; a point in no
// adjacent cell is a CFL violation.  jn: the node's (j00, j01, j10, j11) with
// d/dX = j00 d/di + j01 d/dj, d/dY = j10 d/di + j11 d/dj.
template <typename R, int TI, int TJ>
__device__ __forceinline__ bool depart_gen(const R* sC, const R* jn, int i, int j, int i0, int j0,
                                           int nr, int pi0, int sj0, int PWS, R dx, R dy, int& base,
                                           R& xi, R& eta, bool below = false, bool wrap_rows = false,
                                           unsigned* st = nullptr, int cbmax = -1) {
    // below: the node has cells below row 0 (the mirrored cells across a
    // C-grid's cut, or the wrapped rows of a periodic box); otherwise a row-0
    // node only has the cells of row 0.  wrap_rows: no last window to clamp to.
    // cbmax >= 0: only the cell columns 0..cbmax exist (a C-grid's outlet
    // columns, whose points on the column line may round to either side)
    // (written with fixed rounding: see fma_rn)
    const R di = fma_rn(jn[0], dx, mul_rn(jn[2], dy)), dj = fma_rn(jn[1], dx, mul_rn(jn[3], dy));
    const bool down = i > 0 || below;
    auto cb_ok = [&](int d) { return cbmax < 0 || (unsigned)(j + d) <= (unsigned)cbmax; };
    int da = (!(di < R(0)) || !down) ? 0 : -1;
    int db = !(dj < R(0)) ? 0 : -1;
    if (!cb_ok(db)) db = -1 - db;
    // an element is taken when the point lies in it up to round-off (tin);
    // failing that, the first candidate within the CFL margin (lim), as for
    // a wall departure that grazes the body
    const R tin = R(1) + (sizeof(R) == 4 ? R(1e-5) : R(1e-12));
    const R lim = R(1) + R(1e-4);
    bool have = false;
    int b_base = 0;
    R b_xi = R(0), b_eta = R(0), b_du = R(2);
#pragma unroll 1
    for (int attempt = 0; attempt < 3; ++attempt) {
        const int ca = i + da, cb = j + db;
        const int wa = wrap_rows ? (ca >> 1) * 2 : min((ca >> 1) * 2, nr - 3), wb = (cb >> 1) * 2;
        if (!in_bounds(ca - (i0 - 1) >= 0 && ca - (i0 - 1) <= TI && cb - (j0 - 1) >= 0 && cb - (j0 - 1) <= TJ, st))
            break;
        const R* c = sC + ((ca - (i0 - 1)) * (TJ + 1) + (cb - (j0 - 1))) * CELLC;
        const R xi0 = R(i - wa - 1), et0 = R(j - wb - 1);
        const R Bx = fma_rn(c[4], et0, c[0]), By = fma_rn(c[5], et0, c[1]);
        const R Cx = fma_rn(c[4], xi0, c[2]), Cy = fma_rn(c[5], xi0, c[3]);
        R u = R(0), v = R(0);
        constexpr int ITS = sizeof(R) == 4 ? 3 : 16;
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
        const R x = add_rn(xi0, u), e = add_rn(et0, v);
        const R du = max(abs_(u), abs_(v));   // displacement in cells (CFL)
        if (abs_(x) <= tin && abs_(e) <= tin) {
            base = (wa - pi0) * PWS + (wb - sj0);
            xi = x;
            eta = e;
            return du <= lim;
        }
        if (!have && abs_(x) <= lim && abs_(e) <= lim) {
            have = true;
            b_base = (wa - pi0) * PWS + (wb - sj0);
            b_xi = x;
            b_eta = e;
            b_du = du;
        }
        bool next = false;
        if (x > tin && da == -1) { da = 0; next = true; }
        else if (x < -tin && da == 0 && down) { da = -1; next = true; }
        if (e > tin && db == -1 && cb_ok(0)) { db = 0; next = true; }
        else if (e < -tin && db == 0 && cb_ok(-1)) { db = -1; next = true; }
        if (!next) break;
    }
    base = b_base;
    xi = b_xi;
    eta = b_eta;
    return have && b_du <= lim;
}

// Asynchronous 4- or 8-byte copy global -> shared (cp.async): no register
// round trip, so every copy of the tile is in flight at once.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(float* dst, const float* src) { cp_async4(dst, src); }
__device__ __forceinline__ void cp_async(double* dst, const double* src) { cp_async8(dst, src); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Wait until at most N of this thread's committed groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
// A record of 4-byte words copied by the 32 lanes of one warp.
__device__ __forceinline__ void cp_async_words(void* dst, const void* src, int words, int lane) {
    for (int q = lane; q < words; q += 32)
        cp_async4(static_cast<unsigned*>(dst) + q, static_cast<const unsigned*>(src) + q);
}

// Tensor copies (TMA): one thread moves a whole 4-D box global -> shared, the
// bytes arriving on a shared-memory transaction barrier (mbarrier) that every
// reader waits on.  Each barrier of a CTA is used for one phase (parity 0).
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(b) : "memory");
}
// make the initialised barriers visible to the tensor-copy (async) proxy
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\nfence.proxy.async.shared::cta;\n" ::: "memory");
}
// the one arrival of the phase, announcing the bytes the copies will deliver
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait0(unsigned long long* bar) {
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(b)
        : "memory");
    return done != 0u;
}
// Wait for phase 0 of a barrier with an iteration limit; a wait that runs out
// flags the launch (the host then reports the step as failed) and returns.
constexpr int TMA_WAIT_LIMIT = 1 << 22;
__device__ __forceinline__ void mbar_wait0(unsigned long long* bar, unsigned* status) {
    for (int it = 0; it < TMA_WAIT_LIMIT; ++it)
        if (mbar_try_wait0(bar)) return;
    atomicOr(status, ST_TMA);
}
// Box of a 4-D tensor map at element coordinates (x innermost) into shared
// memory; x times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, unsigned long long* bar, int x,
                                            int y, int z, int w) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(d),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(b)
        : "memory");
}

// Angular index modulo nt (the tile's halo may wrap more than once on very
// coarse rings).
__device__ __forceinline__ int wrap_nt(int j, int nt) {
    if ((unsigned)j >= (unsigned)nt) {
        j %= nt;
        if (j < 0) j += nt;
    }
    return j;
}

template <typename R>
__device__ __forceinline__ R pick(double d, float f);
template <>
__device__ __forceinline__ float pick<float>(double, float f) {
    return f;
}
template <>
__device__ __forceinline__ double pick<double>(double d, float) {
    return d;
}


// Q2 interpolation of one (f, g) pair over a 3x3 window (rows rowstride
// apart, columns adjacent): separable sums t_a = sum_b L_b(eta) v(a, b), then
// sum_a L_a(xi) t_a (Eq. SemiLagrProp); on the float path with packed
// two-wide FMAs (f and g share the weights).
template <typename R2>
__device__ __forceinline__ R2 gather9(const R2* p, int rowstride, const float* Lx, const float* Ly);
// The float path reads the first two pairs of a window row with one 16-byte
// load: window origins are even columns of a staged row that starts on a
// 16-byte boundary.
template <>
__device__ __forceinline__ float2 gather9<float2>(const float2* p, int rowstride, const float* Lx,
                                                  const float* Ly) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
        const float2* pr = p + aa * rowstride;
        const float4 p01 = *reinterpret_cast<const float4*>(pr);
        float2 t = __fmul2_rn(make_float2(Ly[0], Ly[0]), make_float2(p01.x, p01.y));
        t = __ffma2_rn(make_float2(Ly[1], Ly[1]), make_float2(p01.z, p01.w), t);
        t = __ffma2_rn(make_float2(Ly[2], Ly[2]), pr[2], t);
        acc = __ffma2_rn(make_float2(Lx[aa], Lx[aa]), t, acc);
    }
    return acc;
}
template <typename R2>
__device__ __forceinline__ R2 gather9(const R2* p, int rowstride, const double* Lx, const double* Ly) {
    R2 acc;
    acc.x = 0.0;
    acc.y = 0.0;
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
        const R2* pr = p + aa * rowstride;
        double tx = 0.0, ty = 0.0;
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
            tx += Ly[bb] * pr[bb].x;
            ty += Ly[bb] * pr[bb].y;
        }
        acc.x += Lx[aa] * tx;
        acc.y += Lx[aa] * ty;
    }
    return acc;
}

// Q2 interpolation over a window whose last row is given (v20, v21, v22)
// instead of read from the staged tile: the rear point's mirrored cell on a
// C-grid, whose element's row 0 is the other side's (Eq. SemiLagrProp).
template <typename R, typename R2>
__device__ __forceinline__ R2 gather9_last(const R2* p, int rowstride, const R* Lx, const R* Ly, R2 v20,
                                           R2 v21, R2 v22) {
    R2 acc;
    acc.x = R(0);
    acc.y = R(0);
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
        const R2* pr = p + aa * rowstride;
        const R2 u0 = aa == 2 ? v20 : pr[0], u1 = aa == 2 ? v21 : pr[1], u2 = aa == 2 ? v22 : pr[2];
        const R tx = Ly[0] * u0.x + Ly[1] * u1.x + Ly[2] * u2.x;
        const R ty = Ly[0] * u0.y + Ly[1] * u1.y + Ly[2] * u2.y;
        acc.x += Lx[aa] * tx;
        acc.y += Lx[aa] * ty;
    }
    return acc;
}

// The same over a window below row 0 at a C-grid junction, whose row 0 may
// hold the other side's wall nodes (read from the node's own global row 0,
// p0, at the mirrored column): out of line, since only junction nodes take
// it and an inline copy in each of the nine directions would only swell
// the kernel.
template <typename R, typename R2>
__device__ __noinline__ R2 gather9_mirror(const R2* p, int rowstride, R lx0, R lx1, R lx2, R ly0, R ly1, R ly2,
                                          const R2* p0, const int* ctab, int wb, int nt, R2 ref) {
    // ref: the pair the staged tile is a deviation from (zero on the float64
    // path); the values read from global memory are full populations
    R2 e[3];
#pragma unroll
    for (int b2 = 0; b2 < 3; ++b2) {
        const int c = wb + b2, ct = ctab[c];
        if ((ct & CT_WALL) && !(ct & CT_JUNC)) {
            e[b2] = p0[nt - 1 - c];
            e[b2].x -= ref.x;
            e[b2].y -= ref.y;
        } else {
            e[b2] = p[2 * rowstride + b2];
        }
    }
    const R Lx[3] = {lx0, lx1, lx2}, Ly[3] = {ly0, ly1, ly2};
    return gather9_last(p, rowstride, Lx, Ly, e[0], e[1], e[2]);
}

template <typename R, int TI, int TJ, int NT, int MINB, bool UNIFORM, bool GEN>
__global__ void __launch_bounds__(NT, MINB) k_step(const __grid_constant__ StepArgs a) {
    using T = Tile<TI, TJ>;
    using R2 = typename Vec2<R>::T;
    // tile nodes streamed per thread (the float64 tiles of 2 and 4 rows have
    // more threads than nodes: the rest only stage and collide)
    constexpr int NPT = (TI * TJ + NT - 1) / NT;
    constexpr bool RAGGED = NPT * NT != TI * TJ;
    static_assert(NT >= TJ && NT >= 192 && (!RAGGED || NPT == 1), "tile / thread count");
    extern __shared__ __align__(128) unsigned char smraw[];
    R2* sp = reinterpret_cast<R2*>(smraw);          // [9][PH][PWS] (f_q, g_q) pairs
    R* sM = reinterpret_cast<R*>(sp + 9 * T::PSS);  // [4][MS]  rho, ux, uy, T of step k
    R* sQ = sM + 4 * T::MS;                         // [2][MS]  dQ_x, dQ_y
    R* sG = sQ + 2 * T::MS;                         // [4][DS]  gradient maps
    R* sD = sG + 4 * T::DS;                         // [2][DS]  D_x, D_y
    R* srow = sD + 2 * T::DS;                       // separable: [MH][ROWTAB] (stride RS)
    R* scol = srow + T::MH * RS;                    // separable: [MW][COLTAB] (stride CS)
    R* sX = sD + 2 * T::DS;                         // general: [DS][2] node coordinates
    R* sJ = sX + 2 * T::DS;                         // general: [DS][4] inverse metric
    R* sC = sJ + 4 * T::DS;                         // general: [TI+1][TJ+1][CELLC] cells

    // blended maps of the solve's bodies (several only on general meshes)
    constexpr int MB = GEN ? MAX_BODIES : 1;
    __shared__ BodyMap<R> mapK[MB], mapS[MB];
    __shared__ BodyMap<double> mapSd[MB];
    __shared__ double s_red[3][TJ];
    __shared__ int s_bid[GEN ? TJ : 1];
    __shared__ SolveDev s_sol;
    __shared__ MeshDev s_mesh;
    __shared__ __align__(8) unsigned long long s_bar[2];   // tensor copies: [0] M^k, [1] populations

    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    // ---- prologue: this CTA's tile and solve; the solve's step number k
    // (current buffer k & 1; k == 0 streams the initial state without
    // colliding).  Every thread reads what it needs to address its copies
    // itself, so the whole staging below is one batch of asynchronous copies
    // and one barrier.
    int sb, i0, j0, tjx, nr, nt, N;
    int ttma = 0, tsol = 0;   // table launch: the tile's tensor-copy flag and solve
    const SolveDev* sg = nullptr;   // table launch: the solve and mesh records
    const MeshDev* mg = nullptr;
    unsigned* ctr;
    StepMaps* const* mptr;
    if constexpr (UNIFORM) {
        sb = a.uorder ? (int)blockIdx.x : (int)blockIdx.z;
        tjx = a.uorder ? (int)blockIdx.y : (int)blockIdx.x;
        j0 = tjx * TJ;
        i0 = (a.uorder ? (int)blockIdx.z : (int)blockIdx.y) * TI;
        nr = a.umesh.nr; nt = a.umesh.nt; N = a.umesh.N;
        ctr = a.usol.counter + 2 * sb;
        mptr = a.usol.maps;
    } else {
        const TileDev* tg = a.tiles + blockIdx.x;
        sb = 0;
        tjx = tg->tj; j0 = tg->j0; i0 = tg->i0;
        ttma = tg->tma; tsol = tg->solve;
        sg = a.solves + tg->solve;
        mg = a.meshes + tg->mesh;
        nr = mg->nr; nt = mg->nt; N = mg->N;
        ctr = tg->counter;
        mptr = tg->maps;
    }
    // bodies of the solve (maps, body records and load partials per body)
    int nb = 1;
    if constexpr (GEN) nb = UNIFORM ? a.usol.nbody : __ldg(&sg->nbody);
    // C-grid (general meshes): rows from -4 are stored (the mirrored rows),
    // the angular index does not wrap
    int cg = 0, pb = 0;
    const int* ctab = nullptr;
    if constexpr (GEN) {
        cg = UNIFORM ? a.umesh.cgrid : mg->cgrid;
        ctab = UNIFORM ? a.umesh.coltype : mg->coltype;
        pb = UNIFORM ? a.umesh.box : mg->box;
    }
    // class of a C-grid's row-0 column (CT_*); the one-sided direction of a
    // row-0 junction's derivative along j
    auto ctype = [&](int j) -> int { return cg ? __ldg(ctab + j) : 0; };
    auto jdir_of = [&](int c) -> int { return (c & CT_JUNC) ? ((c & CT_JFWD) ? 1 : -1) : 0; };
    const int rlo = cg ? -CGRID_GHOST_ROWS : 0;
    // rows that exist (a periodic box: all, wrapped) and their stored index
    auto rowok = [&](int i) { return pb || (i >= rlo && i < nr); };
    auto rw = [&](int i) { return pb ? wrap_nt(i, nr) : i; };
    // a uniform launch from the host knows the step number; otherwise it is
    // the solve's device counter
    const unsigned kstep = (UNIFORM && a.ustep >= 0) ? (unsigned)a.ustep : __ldcg(ctr + 1);
    const int cur = (int)(kstep & 1u);
    // C-grid step (general meshes), two launches: the first collides the
    // rows below CGRID_PRE_ROWS into ppost; in the second the first row of
    // tiles, whose +-2 window reaches across the cut, streams that collided
    // state, and every other tile collides and streams in one pass
    if (GEN && a.collide_only && a.cgrid_pre && i0 >= CGRID_PRE_ROWS) return;
    const bool split = GEN && a.stream_post && i0 + TI + 2 <= CGRID_PRE_ROWS;
    const int mode = a.collide_only ? MODE_COLLIDE_ONLY
                     : (kstep == 0u || split) ? MODE_STREAM_ONLY : MODE_COLLIDE_STREAM;
    const bool from_post = split && kstep != 0u && !a.collide_only;
    {
        const StepMaps* mi = (cur ? mptr[1] : mptr[0]) + (size_t)sb * nb;
        if (!UNIFORM && w == 1) cp_async_words(&s_sol, sg, (int)(sizeof(SolveDev) / 4), l);
        if (!UNIFORM && w == 2) cp_async_words(&s_mesh, mg, (int)(sizeof(MeshDev) / 4), l);
        for (int b = 0; b < nb; ++b) {
            if (w == 3) {
                if constexpr (sizeof(R) == 4) cp_async_words(&mapK[b], &mi[b].Kf, (int)(sizeof(BodyMap<R>) / 4), l);
                else cp_async_words(&mapK[b], &mi[b].Kd, (int)(sizeof(BodyMap<R>) / 4), l);
            }
            if (w == 4) {
                if constexpr (sizeof(R) == 4) cp_async_words(&mapS[b], &mi[b].Sf, (int)(sizeof(BodyMap<R>) / 4), l);
                else cp_async_words(&mapS[b], &mi[b].Sd, (int)(sizeof(BodyMap<R>) / 4), l);
            }
            if (w == 5) cp_async_words(&mapSd[b], &mi[b].Sd, (int)(sizeof(BodyMap<double>) / 4), l);
        }
    }
    // solve / mesh fields: kernel parameters for a uniform launch, the copied
    // records for a table launch (valid after the staging barrier)
#define SD(x) (UNIFORM ? a.usol.x : s_sol.x)
#define MD(x) (UNIFORM ? a.umesh.x : s_mesh.x)
    const size_t o9 = (size_t)sb * 9 * N, o4 = (size_t)sb * 4 * N;
    const void* psrc = from_post ? (UNIFORM ? a.usol.ppost : sg->ppost)
                                 : UNIFORM ? (cur ? a.usol.p[1] : a.usol.p[0]) : sg->p[cur];
    const void* Msrc = UNIFORM ? (cur ? a.usol.M[1] : a.usol.M[0]) : sg->M[cur];
    const R2* __restrict__ p_in = reinterpret_cast<const R2*>(psrc) + o9;
    const R* __restrict__ M_in = reinterpret_cast<const R*>(Msrc) + o4;
    const R* __restrict__ rowtab = reinterpret_cast<const R*>(UNIFORM ? a.umesh.rowtab : mg->rowtab);
    const R* __restrict__ coltab = reinterpret_cast<const R*>(UNIFORM ? a.umesh.coltab : mg->coltab);
    const int mi0 = i0 - T::HM, mj0 = j0 - T::HM;   // global index of sM entry (0,0)
    const int pi0 = i0 - T::HP, sj0 = j0 - 4;       // global index of sp row 0, column 0
    // float launches: the M^k and population boxes of a tile whose columns do
    // not wrap (every tile of a C-grid, whose columns never wrap) come by two
    // tensor copies that one thread issues (rows and columns outside the mesh
    // arrive as zeros and are never read; a C-grid's arrays start tma_g
    // mirrored rows below row 0); uniform launches through the handle's maps,
    // the batch's separable table launches through each solve's own.  The
    // other tiles, a step that streams the collide-only buffer, the
    // departure-cache pass and the general kernel's table launches stage by
    // per-thread copies
    bool use_tma = false;
    if constexpr (sizeof(R) == 4 && (UNIFORM || !GEN)) {
        // (the boxes' shared-memory destinations are 128-byte aligned by the
        // layout; checked, so that another layout falls back instead of faulting)
        const unsigned sa = (unsigned)__cvta_generic_to_shared(sp), ma = (unsigned)__cvta_generic_to_shared(sM);
        const bool aligned = ((sa | ma) & 127u) == 0u;
        const CUtensorMap *tmM, *tmP;
        int g = 0, w = 0;
        if constexpr (UNIFORM) {
            use_tma = a.tma != 0 && (cg || (mj0 >= 0 && mj0 + T::MW <= nt)) && !pb && !from_post &&
                      !(GEN && a.record) && aligned;
            tmM = &a.tm_M[cur];
            tmP = &a.tm_p[cur];
            g = a.tma_g;
            w = sb;
        } else {
            // a separable solve of the batch runtime: its own maps, one solve each
            use_tma = ttma != 0 && a.tmaps != nullptr && mj0 >= 0 && mj0 + T::MW <= nt && aligned;
            tmP = a.tmaps + 4 * tsol + cur;
            tmM = a.tmaps + 4 * tsol + 2 + cur;
        }
        if (use_tma && tid == 0) {
            mbar_init(&s_bar[0]);
            mbar_init(&s_bar[1]);
            mbar_fence_init();
            mbar_expect_tx(&s_bar[0], 4u * T::MS * (unsigned)sizeof(R));
            tma_load_4d(sM, tmM, &s_bar[0], mj0, mi0 + g, 0, w);
            mbar_expect_tx(&s_bar[1], 9u * T::PSS * (unsigned)sizeof(R2));
            tma_load_4d(sp, tmP, &s_bar[1], 2 * sj0, pi0 + g, 0, w);
        }
    }

    // ---- phase 1: stage the geometry tables, M^k and the populations ------
    if constexpr (GEN) {
        // node coordinates and inverse metric on the +-3 region, element
        // coefficients of the cells adjacent to the tile's nodes
        const R* gx = reinterpret_cast<const R*>(UNIFORM ? a.umesh.nodex : mg->nodex);
        const R* gj = reinterpret_cast<const R*>(UNIFORM ? a.umesh.jinv : mg->jinv);
        const R* gc = reinterpret_cast<const R*>(UNIFORM ? a.umesh.cellc : mg->cellc);
        for (int idx = tid; idx < T::DS; idx += NT) {
            const int li = idx / T::DW, lj = idx - li * T::DW;
            const int i = i0 - T::HD + li, jj = j0 - T::HD + lj;
            if (!rowok(i) || (cg && (unsigned)jj >= (unsigned)nt)) continue;
            const ptrdiff_t n = (ptrdiff_t)rw(i) * nt + (cg ? jj : wrap_nt(jj, nt));
            if (!in_bounds(n >= (ptrdiff_t)rlo * nt && n < (ptrdiff_t)nr * nt, a.status)) continue;
            if constexpr (sizeof(R) == 4) {
                cp_async8(sX + 2 * idx, gx + 2 * n);
                cp_async16(sJ + 4 * idx, gj + 4 * n);
            } else {
                cp_async16(sX + 2 * idx, gx + 2 * n);
                cp_async16(sJ + 4 * idx, gj + 4 * n);
                cp_async16(sJ + 4 * idx + 2, gj + 4 * n + 2);
            }
        }
        constexpr int CE = 16 / (int)sizeof(R), NCC = CELLC / CE;
        for (int t = tid; t < (TI + 1) * (TJ + 1) * NCC; t += NT) {
            const int cell = t / NCC, ch = t - cell * NCC;
            const int la = cell / (TJ + 1), lb = cell - la * (TJ + 1);
            const int ca = i0 - 1 + la, cb = j0 - 1 + lb;
            if (!pb && (ca < (cg ? -1 : 0) || ca > nr - 2)) continue;
            if (cg && (unsigned)cb > (unsigned)(nt - 2)) continue;
            const ptrdiff_t g = ((ptrdiff_t)rw(ca) * nt + (cg ? cb : wrap_nt(cb, nt))) * CELLC + ch * CE;
            if (!in_bounds(g >= (ptrdiff_t)(cg ? -nt : 0) * CELLC && g < (ptrdiff_t)nr * nt * CELLC, a.status)) continue;
            cp_async16(sC + cell * CELLC + ch * CE, gc + g);
        }
    } else {
        constexpr int CE = 16 / (int)sizeof(R);   // table entries per 16-byte chunk
        for (int t = tid; t < T::MH * (ROWTAB / CE); t += NT) {
            const int li = t / (ROWTAB / CE), c = (t - li * (ROWTAB / CE)) * CE;
            const int i = min(max(mi0 + li, 0), nr - 1);
            cp_async16(srow + li * RS + c, rowtab + i * ROWTAB + c);
        }
        for (int t = tid; t < T::MW * (COLTAB / CE); t += NT) {
            const int lj = t / (COLTAB / CE), c = (t - lj * (COLTAB / CE)) * CE;
            cp_async16(scol + lj * CS + c, coltab + wrap_nt(mj0 + lj, nt) * COLTAB + c);
        }
    }
    // M^k in 16-byte chunks of consecutive columns (element-wise when Ntheta
    // is not a multiple of the chunk); one thread per (row, chunk), the four
    // components N apart
    {
        constexpr int CM = 16 / (int)sizeof(R), NCH = T::MW / CM;
        const bool vec = nt % CM == 0 && !cg;
        for (int idx = use_tma ? T::MH * NCH : tid; idx < T::MH * NCH; idx += NT) {
            const int ch = idx % NCH, li = idx / NCH;
            const int i = mi0 + li;
            if (!rowok(i)) continue;
            R* dst = sM + li * T::MW + ch * CM;
            const R* src = M_in + (ptrdiff_t)rw(i) * nt;
            if (vec) {
                src += wrap_nt(mj0 + ch * CM, nt);
#pragma unroll
                for (int c = 0; c < 4; ++c) cp_async16(dst + c * T::MS, src + (size_t)c * N);
            } else {
#pragma unroll
                for (int e = 0; e < CM; ++e) {
                    const int jj = mj0 + ch * CM + e;
                    if (cg && (unsigned)jj >= (unsigned)nt) continue;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        cp_async(dst + c * T::MS + e, src + (size_t)c * N + (cg ? jj : wrap_nt(jj, nt)));
                }
            }
        }
    }
    // the copies so far (records, maps, geometry, M^k) form the first group:
    // the correction fields need only them and start while the populations
    // (the second group) are still arriving
    cp_async_commit();
    // populations: rows of PWS (f, g) pairs per direction in 16-byte chunks
    // (two float pairs or one double pair); one thread per (row, chunk), the
    // nine directions N apart
    {
        constexpr int CP = 16 / (int)sizeof(R2), NCH = T::PWS / CP;
        const bool vec = nt % CP == 0 && !cg;
        for (int idx = use_tma ? T::PH * NCH : tid; idx < T::PH * NCH; idx += NT) {
            const int ch = idx % NCH, li = idx / NCH;
            const int i = pi0 + li;
            if (!rowok(i)) continue;
            R2* dst = sp + li * T::PWS + ch * CP;
            const R2* src = p_in + (ptrdiff_t)rw(i) * nt;
            if (vec) {
                src += wrap_nt(sj0 + ch * CP, nt);
#pragma unroll
                for (int q = 0; q < 9; ++q) cp_async16(dst + q * T::PSS, src + (size_t)q * N);
            } else {
#pragma unroll
                for (int e = 0; e < CP; ++e) {
                    const int jj = sj0 + ch * CP + e;
                    if (cg && (unsigned)jj >= (unsigned)nt) continue;
                    const R2* se = src + (cg ? jj : wrap_nt(jj, nt));
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        if constexpr (sizeof(R2) == 16)
                            cp_async16(dst + q * T::PSS + e, se + (size_t)q * N);
                        else
                            cp_async8(dst + q * T::PSS + e, se + (size_t)q * N);
                    }
                }
            }
        }
    }
    // general meshes: the cached static departures are read per node in the
    // stream phase (the solves of a handle share them, so they are mostly
    // L2 hits); here a prefetch of the tile's entries into L2
    const bool dcache = GEN && UNIFORM && !a.record && mode != MODE_COLLIDE_ONLY && a.usol.dep_code != nullptr;
    if (dcache) {
        const int len = min(TJ, nt - j0);
        for (int t = tid; t < 2 * 10 * TI; t += NT) {
            const int c = t / (2 * TI), r = (t >> 1) % TI, end = t & 1;
            const int i = i0 + r;
            if (i >= nr || len <= 0) continue;
            const size_t off = (size_t)i * nt + j0 + (end ? len - 1 : 0);
            const void* ad = c < 9 ? (const void*)(reinterpret_cast<const R2*>(a.usol.dep_xe) + (size_t)c * N + off)
                                   : (const void*)(a.usol.dep_code + off);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ad));
        }
    }
    if constexpr (UNIFORM) {
        // L2 prefetch of the tile that the CTA one resident wave later will
        // stage (CTAs start in linear block order): its populations and
        // moments move from HBM while this CTA computes, so its staging hits
        // L2.  The first and last address of every row segment cover its
        // lines (a segment is at most two lines); the prefetch is a hint and
        // changes no result.
        const unsigned nx = gridDim.x, ny = gridDim.y;
        const unsigned lin = blockIdx.x + nx * (blockIdx.y + ny * blockIdx.z) + (unsigned)a.pf_dist;
        if (a.pf_dist > 0 && lin < nx * ny * gridDim.z) {
            const int gx = (int)(lin % nx), gy = (int)((lin / nx) % ny), gz = (int)(lin / (nx * ny));
            const int xn = a.uorder ? gy : gx, yn = a.uorder ? gz : gy, zn = a.uorder ? gx : gz;
            const int jb = xn * TJ;
            const int len = min(TJ, nt - jb);
            for (int t = tid; t < 2 * 13 * TI; t += NT) {
                const int c = t / (2 * TI), r = (t >> 1) % TI, end = t & 1;
                const int i = yn * TI + r;
                if (i >= nr) continue;
                const size_t off = (size_t)i * nt + jb + (end ? len - 1 : 0);
                const void* ad = c < 9 ? (const void*)(reinterpret_cast<const R2*>(psrc) + ((size_t)zn * 9 + c) * N + off)
                                       : (const void*)(reinterpret_cast<const R*>(Msrc) + ((size_t)zn * 4 + c - 9) * N + off);
                asm volatile("prefetch.global.L2 [%0];" ::"l"(ad));
            }
        }
    }
    cp_async_commit();
    cp_async_wait_group<1>();
    __syncthreads();
    if (use_tma) mbar_wait0(&s_bar[0], a.status);   // M^k (the barrier above ordered the init)
    R2* __restrict__ p_out = reinterpret_cast<R2*>(mode == MODE_COLLIDE_ONLY ? SD(ppost) : SD(p[cur ^ 1])) + o9;
    R* __restrict__ M_out = reinterpret_cast<R*>(SD(M[cur ^ 1])) + o4;
    const R dt = pick<R>(SD(dt), SD(dt_f)), mu = pick<R>(SD(mu), SD(mu_f)), Cv = pick<R>(SD(Cv), SD(Cv_f));
    const R Pr = pick<R>(SD(Pr), SD(Pr_f)), iPr = pick<R>(1.0 / SD(Pr), SD(iPr_f));
    const R xm = pick<R>(MD(xm), MD(xm_f)), ym = pick<R>(MD(ym), MD(ym_f));
    // float path: shared memory holds the post-collision pairs as deviations
    // from the free-stream pair of their direction, so that the Q2 weights
    // (which sum to 1 only up to round-off, the same way at every step of a
    // node that does not move) act on the deviation; an interpolated pair
    // gets the reference back.  The float64 path keeps full values.
    constexpr bool DEV = sizeof(R) == 4;
    auto ref_of = [&](int q) -> R2 {
        R2 r;
        if constexpr (DEV) {
            r.x = SD(fgref)[2 * q];
            r.y = SD(fgref)[2 * q + 1];
        } else {
            r.x = R(0);
            r.y = R(0);
        }
        return r;
    };
    auto add_ref = [&](int q, R2 v) -> R2 {
        if constexpr (DEV) v = padd(v, ref_of(q));
        return v;
    };
    const bool collide = mode != MODE_STREAM_ONLY;
    const bool stream = mode != MODE_COLLIDE_ONLY;
    // static tile: no node of the tile's +-4 region lies in the blended
    // region of the body (F = I, V_G = 0 there), from a lower bound of the
    // distance to the blend centre on the separable O-grid (r of the first
    // staged row x min |e_j| - |mesh centre - blend centre|) with a margin;
    // such tiles skip the kinematics.  Tiles near the boundary take the
    // general path, which gives the same result.
    bool tile_static = false;
    if constexpr (!GEN) {
        if (!mapS[0].active) {
            tile_static = true;
        } else {
            // in the element type of the path (no float64 on the float path),
            // with a margin well above its rounding
            const R rmin = srow[RT_R] * pick<R>(MD(emin), MD(emin_f));   // first staged row
            const R ox = xm - mapS[0].xc, oy = ym - mapS[0].yc;
            const R r_out = mapS[0].r_in + rcp_(mapS[0].inv_w);
            tile_static = rmin - sqrt_(ox * ox + oy * oy) > r_out * (R(1) + R(1e-4)) + R(1e-5);
        }
    }

    // ---- phase 2: correction fields and collision of step k --------------
    // a collide-only launch of a general mesh (a C-grid's first launch)
    // writes the tile's nodes only: the collision is needed there, the
    // correction field D and the gradient maps on +-2 (a junction's or an
    // outlet's one-sided stencil along j reaches two nodes), dQ on +-4
    const bool shrink = GEN && mode == MODE_COLLIDE_ONLY;
    // a C-grid step's collide-only launch: the tiles that stream its output
    // are the first row of tiles, whose windows reach row TI + 1, so rows
    // from TI + 2 on are neither collided nor written (nor D and the maps
    // from TI + 3, nor dQ from TI + 4); ci: the row, e: 0 collision, 1 D, 2 dQ
    const int rcap = (GEN && a.collide_only && a.cgrid_pre) ? TI + 2 : INT_MAX;
    auto capped = [&](int ci, int e) { return ci - e >= rcap; };
    auto outside = [&](int li, int lj, int h, int w) {
        return shrink && (li < h - w || li >= h + TI + w || lj < h - w || lj >= h + TJ + w);
    };
    if (collide) {
        for (int idx = tid; idx < T::MS; idx += NT) {
            const int i = mi0 + idx / T::MW;
            if (!rowok(i) || capped(i, 2)) continue;
            if (cg && (unsigned)(mj0 + idx % T::MW) >= (unsigned)nt) continue;
            const R rho = sM[idx], ux = sM[T::MS + idx], uy = sM[2 * T::MS + idx], Tn = sM[3 * T::MS + idx];
            sQ[idx] = rho * ux * (R(1) - R(3) * Tn) - rho * ux * ux * ux;
            sQ[T::MS + idx] = rho * uy * (R(1) - R(3) * Tn) - rho * uy * uy * uy;
        }
        // static separable tile (F = I): the gradient maps are products of the
        // mesh tables, formed where they are used instead of stored
        const bool gtab = !GEN && tile_static;
        auto gstatic = [&](int li, int lj, R* G) {   // li, lj: coordinates in the +-3 region
            const R* row = srow + (li + 1) * RS;
            const R* col = scol + (lj + 1) * CS;
            R c0, c1, c2, c3;
            ld4(col + CT_G, c0, c1, c2, c3);
            G[0] = row[RT_IDRC] * c0;
            G[1] = -row[RT_IR] * c1;
            G[2] = -row[RT_IDRC] * c2;
            G[3] = row[RT_IR] * c3;
        };
        // gradient maps on the +-3 region with the step-k kinematics
        for (int idx = gtab ? T::DS : tid; idx < T::DS; idx += NT) {
            const int li = idx / T::DW, lj = idx - li * T::DW;
            const int i = i0 - T::HD + li;
            if (!rowok(i) || capped(i, 1)) continue;
            if (cg && (unsigned)(j0 - T::HD + lj) >= (unsigned)nt) continue;
            if (outside(li, lj, T::HD, 2)) continue;
            R F00, F01, F10, F11, vx, vy;
            R G[4];
            if constexpr (GEN) {
                kinematics_sum(mapK, nb, sX[2 * idx], sX[2 * idx + 1], F00, F01, F10, F11, vx, vy);
                R j00, j01, j10, j11;
                ld4(sJ + 4 * idx, j00, j01, j10, j11);
                grad_map_j(j00, j01, j10, j11, F00, F01, F10, F11, G);
            } else {
                const R* row = srow + (li + 1) * RS;
                const R* col = scol + (lj + 1) * CS;
                if (tile_static) {
                    // F = I: the inverse metric of the mesh alone
                    R c0, c1, c2, c3;
                    ld4(col + CT_G, c0, c1, c2, c3);
                    G[0] = row[RT_IDRC] * c0;
                    G[1] = -row[RT_IR] * c1;
                    G[2] = -row[RT_IDRC] * c2;
                    G[3] = row[RT_IR] * c3;
                } else {
                    R ex, ey, u0, u1;
                    ld4(col + CT_E, ex, ey, u0, u1);
                    kinematics(mapK[0], xm + row[RT_R] * ex, ym + row[RT_R] * ey, F00, F01, F10, F11, vx, vy);
                    grad_map(row, col, F00, F01, F10, F11, G);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) sG[c * T::DS + idx] = G[c];
        }
        __syncthreads();
        for (int idx = tid; idx < T::DS; idx += NT) {
            const int li = idx / T::DW, lj = idx - li * T::DW;
            const int i = i0 - T::HD + li, jj = j0 - T::HD + lj;
            if (!rowok(i) || capped(i, 1)) continue;
            if (cg && (unsigned)jj >= (unsigned)nt) continue;
            if (outside(li, lj, T::HD, 2)) continue;
            const int m = (li + 1) * T::MW + (lj + 1);
            const R mup = mu * rcp_(sM[m] * sM[3 * T::MS + m]);
            R qx_xi, qx_et, qy_xi, qy_et;
            if constexpr (GEN) {
                const int ct = (cg && i == 0) ? ctype(jj) : 0;
                const bool across = (ct & (CT_CUT | CT_JUNC)) != 0;
                qx_xi = d_row_c(sQ + m, T::MW, i, nr, across, pb);
                qx_et = d_col_c(sQ + m, jj, nt, cg, jdir_of(ct));
                qy_xi = d_row_c(sQ + T::MS + m, T::MW, i, nr, across, pb);
                qy_et = d_col_c(sQ + T::MS + m, jj, nt, cg, jdir_of(ct));
            } else {
                qx_xi = d_row(sQ + m, T::MW, i, nr);
                qx_et = d_col(sQ + m);
                qy_xi = d_row(sQ + T::MS + m, T::MW, i, nr);
                qy_et = d_col(sQ + T::MS + m);
            }
            R G[4];
            if (gtab) {
                gstatic(li, lj, G);
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) G[c] = sG[c * T::DS + idx];
            }
            sD[idx] = mup * (G[0] * qx_xi + G[1] * qx_et);
            sD[T::DS + idx] = mup * (G[2] * qy_xi + G[3] * qy_et);
        }
        cp_async_wait_all();   // the populations
        if (use_tma) mbar_wait0(&s_bar[1], a.status);
        __syncthreads();
        for (int idx = tid; idx < T::PS; idx += NT) {
            const int li = idx / T::PW, lj = idx - li * T::PW;
            const int i = pi0 + li, jj = j0 - T::HP + lj;
            if (!(pb || (i >= 0 && i < nr)) || capped(i, 0)) continue;
            if (cg && (unsigned)jj >= (unsigned)nt) continue;
            if (outside(li, lj, T::HP, 0)) continue;
            const int sn = li * T::PWS + lj + 2;   // staged node
            R2 pq[9];
            if ((!pb && i == nr - 1) || (cg && (jj == 0 || jj == nt - 1))) {
                const int m = (li + 2) * T::MW + (lj + 2);
                R f[9], g[9];
                f_equilibrium(sM[m], sM[T::MS + m], sM[2 * T::MS + m], sM[3 * T::MS + m], f);
                g_equilibrium(sM[m], sM[T::MS + m], sM[2 * T::MS + m], sM[3 * T::MS + m], Cv, g);
#pragma unroll
                for (int q = 0; q < 9; ++q) pq[q] = pair(f[q], g[q]);
            } else {
#pragma unroll
                for (int q = 0; q < 9; ++q) pq[q] = sp[q * T::PSS + sn];
                const int d = (li + 1) * T::DW + (lj + 1);
                R dx_xi, dx_et, dy_xi, dy_et;
                if constexpr (GEN) {
                    const int ct = (cg && i == 0) ? ctype(jj) : 0;
                    const bool across = (ct & (CT_CUT | CT_JUNC)) != 0;
                    dx_xi = d_row_c(sD + d, T::DW, i, nr, across, pb);
                    dx_et = d_col_c(sD + d, jj, nt, cg, jdir_of(ct));
                    dy_xi = d_row_c(sD + T::DS + d, T::DW, i, nr, across, pb);
                    dy_et = d_col_c(sD + T::DS + d, jj, nt, cg, jdir_of(ct));
                } else {
                    dx_xi = d_row(sD + d, T::DW, i, nr);
                    dx_et = d_col(sD + d);
                    dy_xi = d_row(sD + T::DS + d, T::DW, i, nr);
                    dy_et = d_col(sD + T::DS + d);
                }
                R G[4];
                if (gtab) {
                    gstatic(li + 1, lj + 1, G);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) G[c] = sG[c * T::DS + d];
                }
                const R Yx = G[0] * dx_xi + G[1] * dx_et;
                const R Yy = G[2] * dy_xi + G[3] * dy_et;
                collide_pairs(pq, Yx, Yy, mu, dt, Cv, iPr);
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) sp[q * T::PSS + sn] = psub(pq[q], ref_of(q));
        }
        __syncthreads();
        if (!stream) {
            for (int k = 0; k < NPT; ++k) {
                const int t = tid + k * NT;
                const int ti = t / TJ, tj = t - (t / TJ) * TJ;
                const int i = i0 + ti, j = j0 + tj;
                if ((!RAGGED || ti < TI) && i < nr && j < nt && !capped(i, 0)) {
                    const int n = i * nt + j;
                    const int sn = (ti + T::HP) * T::PWS + tj + T::HP + 2;
                    // C-grid: the first copy of a cut node also writes the
                    // second (which writes nothing), rows 1 and 2 their
                    // mirrored slots (the next stream's rows below row 0)
                    const int ct = (cg && i == 0) ? ctype(j) : 0;
                    if (ct & CT_DUP) continue;
                    const int n2 = i == 0 ? nt - 1 - j : -i * nt + (nt - 1 - j);
                    const bool two = ((ct & (CT_CUT | CT_JUNC)) || (cg && (i == 1 || i == 2))) &&
                                     in_bounds(n2 >= rlo * nt && n2 < nr * nt, a.status);
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        const R2 v = add_ref(q, sp[q * T::PSS + sn]);
                        p_out[(ptrdiff_t)q * N + n] = v;
                        if (two) p_out[(ptrdiff_t)q * N + n2] = v;
                    }
                }
            }
            return;
        }
    }

    // ---- phase 3: stream step k+1 ----------------------------------------
    if (!collide) {
        cp_async_wait_all();   // the populations
        if (use_tma) mbar_wait0(&s_bar[1], a.status);
        __syncthreads();
        if constexpr (DEV) {
            // the staged pairs are full values here (nothing collided them):
            // make them deviations like the collided ones
            for (int idx = tid; idx < 9 * T::PSS; idx += NT) {
                const R2 r = ref_of(idx / T::PSS);
                R2 v = sp[idx];
                v.x -= r.x;
                v.y -= r.y;
                sp[idx] = v;
            }
            __syncthreads();
        }
    }
    double fcx = 0.0, fcy = 0.0, fcm = 0.0;   // this thread's wall share (node row 0)
    int fbid = 0;                              // the body of that wall node
#pragma unroll 1
    for (int k = 0; k < NPT; ++k) {
        const int t = tid + k * NT;
        const int ti = t / TJ, tj = t - (t / TJ) * TJ;
        const int i = i0 + ti, j = j0 + tj;
        if ((RAGGED && ti >= TI) || i >= nr || j >= nt) continue;
        // C-grid: the second copies of the row-0 cut nodes (and of the rear
        // point) are written by their first copies; rows 1-4 also write
        // their moments into their mirrored slots below row 0
        const int ct = (cg && i == 0) ? ctype(j) : 0;
        if (ct & CT_DUP) continue;
        const int n2 = i == 0 ? nt - 1 - j : -i * nt + (nt - 1 - j);
        const bool dup2_ = (ct & (CT_CUT | CT_JUNC)) != 0, mir_ = cg && i >= 1 && i <= CGRID_GHOST_ROWS;
        const bool n2ok = !(dup2_ || mir_) || in_bounds(n2 >= rlo * nt && n2 < nr * nt, a.status);
        const bool dup2 = dup2_ && n2ok;
        const bool mir = mir_ && n2ok;
        const int n = i * nt + j;
        const int m = (ti + T::HM) * T::MW + tj + T::HM;   // node in M coords
        const R* row = srow + (ti + T::HM) * RS;
        const R* col = scol + (tj + T::HM) * CS;
        const bool farj = cg && i < nr - 1 && (j == 0 || j == nt - 1);
        if ((!pb && i == nr - 1) || farj) {
            if (GEN && a.record) continue;
            // far field (Sec. III A 2), targets built like the wall's: a
            // quantity the boundary does not prescribe takes a zero normal
            // gradient through the point B = A - dt n_out one step inside
            // along the outward unit direction, by Q2 interpolation of M^k
            // (the previous step's field).  An inlet (where the free stream
            // enters) prescribes the free stream's u and T, its density is
            // the value at B; an outlet prescribes nothing.  On a C-grid
            // also the outlet columns (direction along j)
            const double* fd = farj ? MD(fardirj) + 4 * i + (j == 0 ? 0 : 2) : MD(fardir) + 2 * j;
            const double un = SD(uinf_x) * fd[0] + SD(uinf_y) * fd[1];
            R rho, ux, uy, Tt;
            {
                const R bx = -dt * (R)fd[0], by = -dt * (R)fd[1];
                int base;
                R xi, eta;
                bool ok;
                if constexpr (GEN) {
                    const int dn = (ti + T::HD) * T::DW + tj + T::HD;
                    ok = depart_gen<R, TI, TJ>(sC, sJ + 4 * dn, i, j, i0, j0, nr, pi0, sj0, T::PWS, bx, by, base, xi,
                                               eta, dup2 || pb, pb, a.status, cg ? nt - 2 : -1);
                } else {
                    NodeGeo<R> fg;
                    node_geo(i, j, nr, row, col, pi0, sj0, T::PWS, fg);
                    ok = depart(fg, i, bx, by, base, xi, eta);
                }
                const int wa = base / T::PWS + pi0, wb = base - (base / T::PWS) * T::PWS + sj0;
                const int w0 = (wa - mi0) * T::MW + (wb - mj0);
                ok = ok && in_bounds(w0 >= 0 && w0 + 2 * T::MW + 2 < T::MS, a.status);
                rho = sM[m]; ux = sM[T::MS + m]; uy = sM[2 * T::MS + m]; Tt = sM[3 * T::MS + m];
                if (ok) {
                    // interpolated as the node's own value plus the weighted
                    // differences from it: B lies a fraction of a cell from
                    // the node, and the weights' round-off (their sum is 1 to
                    // an ulp, the same at every step) then acts on the small
                    // differences, not on the values
                    R Lx[3], Ly[3];
                    lagrange3(xi, Lx);
                    lagrange3(eta, Ly);
                    R drho = R(0), dux = R(0), duy = R(0), dT = R(0);
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
                        for (int bb = 0; bb < 3; ++bb) {
                            const R wgt = Lx[aa] * Ly[bb];
                            const int o = w0 + aa * T::MW + bb;
                            drho += wgt * (sM[o] - rho);
                            dux += wgt * (sM[T::MS + o] - ux);
                            duy += wgt * (sM[2 * T::MS + o] - uy);
                            dT += wgt * (sM[3 * T::MS + o] - Tt);
                        }
                    rho += drho; ux += dux; uy += duy; Tt += dT;
                } else {
                    atomicOr(a.status, ST_BPOINT);
                }
                if (un < 0.0) {
                    ux = pick<R>(SD(uinf_x), SD(uinf_x_f));
                    uy = pick<R>(SD(uinf_y), SD(uinf_y_f));
                    Tt = pick<R>(SD(T_inf), SD(T_inf_f));
                }
            }
            R f[9], g[9];
            f_equilibrium(rho, ux, uy, Tt, f);
            g_equilibrium(rho, ux, uy, Tt, Cv, g);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                R2 v;
                v.x = f[q];
                v.y = g[q];
                p_out[(size_t)q * N + n] = v;
                if (dup2) p_out[(ptrdiff_t)q * N + n2] = v;
            }
            M_out[n] = rho; M_out[(size_t)N + n] = ux; M_out[(size_t)2 * N + n] = uy;
            M_out[(size_t)3 * N + n] = Tt;
            if (dup2 || mir) {
                M_out[n2] = rho; M_out[(ptrdiff_t)N + n2] = ux; M_out[(ptrdiff_t)2 * N + n2] = uy;
                M_out[(ptrdiff_t)3 * N + n2] = Tt;
            }
            continue;
        }
        const bool wall = !pb && i == 0 && (!cg || (ct & CT_WALL));
        const bool rear = (ct & CT_JUNC) != 0;   // a junction (first copy)
        // a window below row 0 is the mirror of one on the other side of the
        // cut, its row 0 included: next to a junction that row can lie on the
        // other side's wall, whose nodes are then read from global memory (only
        // a junction's windows can reach a wall column)
        const int rbase_row = -2 - pi0;   // staged row of global row -2
        NodeGeo<R> geo;
        R F00, F01, F10, F11, vx, vy;
        bool moved;
        const int dn = (ti + T::HD) * T::DW + tj + T::HD;   // this node in the +-3 region
        if constexpr (GEN) {
            moved = kinematics_sum(mapS, nb, sX[2 * dn], sX[2 * dn + 1], F00, F01, F10, F11, vx, vy);
        } else {
            node_geo(i, j, nr, row, col, pi0, sj0, T::PWS, geo);
            if (tile_static) {
                F00 = R(1); F01 = R(0); F10 = R(0); F11 = R(1); vx = R(0); vy = R(0);
                moved = false;
            } else {
                moved = kinematics(mapS[0], xm + geo.ri * geo.ex, ym + geo.ri * geo.ey, F00, F01, F10, F11, vx, vy);
            }
        }
        const R idF = rcp_(F00 * F11 - F01 * F10);
        const R i00 = F11 * idF, i01 = -F01 * idF, i10 = -F10 * idF, i11 = F00 * idF;
        unsigned missing = 0u;
        if (wall) {
            // missing populations: departure point inside the body,
            // c_hat . n0 > 0, decided in float64 (Sec. III A)
            const double Xd = MD(xw)[2 * j], Yd = MD(xw)[2 * j + 1];
            double D00, D01, D10, D11, dvx, dvy;
            if constexpr (GEN) kinematics_sum(mapSd, nb, Xd, Yd, D00, D01, D10, D11, dvx, dvy);
            else kinematics(mapSd[0], Xd, Yd, D00, D01, D10, D11, dvx, dvy);
            const double idd = 1.0 / (D00 * D11 - D01 * D10);
            const double n0x = MD(n0)[2 * j], n0y = MD(n0)[2 * j + 1];
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
        const int own = (ti + T::HP) * T::PWS + tj + T::HP + 2;   // this node in the staged tile
        // departure solve of this node for a displacement (dx, dy)
        auto departure = [&](int inode, R dx, R dy, int& base, R& xi, R& eta) -> bool {
            if constexpr (GEN)
                return depart_gen<R, TI, TJ>(sC, sJ + 4 * dn, inode, j, i0, j0, nr, pi0, sj0, T::PWS, dx, dy, base, xi, eta,
                                         dup2 || pb, pb, a.status) &&
                       in_bounds(base >= 0 && base + 2 * T::PWS + 2 < T::PSS, a.status);
            else
                return depart(geo, inode, dx, dy, base, xi, eta) &&
                       in_bounds(base >= 0 && base + 2 * T::PWS + 2 < T::PSS, a.status);
        };
        // general meshes: a node the blend does not move takes its cached
        // departures (the same solves, made once for the handle's dt)
        unsigned long long dcode = ~0ull;
        if constexpr (GEN) {
            if (a.record) {
                if (!moved && i > 0) {
                    R2* gxe = reinterpret_cast<R2*>(a.usol.dep_xe);
                    unsigned long long code = 0ull;
                    bool ok = true;
#pragma unroll 1
                    for (int q = 0; q < 9; ++q) {
                        const R cx = (R)cxq(q), cy = (R)cyq(q);
                        const R hx = i00 * cx + i01 * cy - vx, hy = i10 * cx + i11 * cy - vy;
                        int base;
                        R2 xe;
                        unsigned nib = 16u;   // a lost departure
                        if (departure(i, -dt * hx, -dt * hy, base, xe.x, xe.y)) {
                            const int dr = base / T::PWS - (i - pi0), dc = base % T::PWS - (j - sj0);
                            if (dr < -3 || dr > 0 || dc < -3 || dc > 0) ok = false;
                            nib = (unsigned)(((dr + 3) << 2) | (dc + 3));
                        }
                        code |= (unsigned long long)nib << (5 * q);
                        gxe[(size_t)q * N + n] = xe;
                    }
                    a.usol.dep_code[n] = ok ? code : ~0ull;
                }
                continue;
            }
            if (dcache && !moved && i > 0) dcode = __ldg(a.usol.dep_code + n);
        }
        if (GEN && dcode != ~0ull) {
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const unsigned nib = (unsigned)(dcode >> (5 * q)) & 31u;
                R2 v;
                if (nib & 16u) {
                    lost = true;
                    v = add_ref(q, sp[q * T::PSS + own]);
                } else {
                    const int base = own + ((int)(nib >> 2) - 3) * T::PWS + ((int)(nib & 3u) - 3);
                    const R2 xe = __ldg(reinterpret_cast<const R2*>(a.usol.dep_xe) + (size_t)q * N + n);
                    R Lx[3], Ly[3];
                    lagrange3(xe.x, Lx);
                    lagrange3(xe.y, Ly);
                    v = add_ref(q, gather9(sp + q * T::PSS + base, T::PWS, Lx, Ly));
                }
                f[q] = v.x;
                g[q] = v.y;
            }
        } else if (!GEN && !moved && i > 0) {
            // a node the blend does not move: c_hat = c, and the rest
            // population's departure point is the node itself
            {
                const R2 v = add_ref(0, sp[own]);
                f[0] = v.x;
                g[0] = v.y;
            }
            auto pull = [&](auto cxc, auto cyc, int q) {
                int base;
                R xi, eta;
                R2 v;
                if (depart_static<decltype(cxc)::value, decltype(cyc)::value>(geo, dt, base, xi, eta) &&
                    in_bounds(base >= 0 && base + 2 * T::PWS + 2 < T::PSS, a.status)) {
                    R Lx[3], Ly[3];
                    lagrange3(xi, Lx);
                    lagrange3(eta, Ly);
                    v = gather9(sp + q * T::PSS + base, T::PWS, Lx, Ly);
                } else {
                    lost = true;
                    v = sp[q * T::PSS + own];
                }
                v = add_ref(q, v);
                f[q] = v.x;
                g[q] = v.y;
            };
            using P1 = std::integral_constant<int, 1>;
            using Z0 = std::integral_constant<int, 0>;
            using M1 = std::integral_constant<int, -1>;
            pull(P1{}, Z0{}, 1);
            pull(Z0{}, P1{}, 2);
            pull(M1{}, Z0{}, 3);
            pull(Z0{}, M1{}, 4);
            pull(P1{}, P1{}, 5);
            pull(M1{}, P1{}, 6);
            pull(M1{}, M1{}, 7);
            pull(P1{}, M1{}, 8);
        } else {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            f[q] = R(0);
            g[q] = R(0);
            if (missing & (1u << q)) continue;
            const R cx = (R)cxq(q), cy = (R)cyq(q);
            const R hx = i00 * cx + i01 * cy - vx, hy = i10 * cx + i11 * cy - vy;
            int base;
            R xi, eta;
            if (departure(i, -dt * hx, -dt * hy, base, xi, eta)) {
                R Lx[3], Ly[3];
                lagrange3(xi, Lx);
                lagrange3(eta, Ly);
                R2 v;
                if (GEN && rear && base / T::PWS == rbase_row)
                    v = gather9_mirror<R, R2>(sp + q * T::PSS + base, T::PWS, Lx[0], Lx[1], Lx[2], Ly[0], Ly[1], Ly[2],
                                              p_in + (size_t)q * N, ctab, base - rbase_row * T::PWS + sj0, nt,
                                              ref_of(q));
                else
                    v = gather9(sp + q * T::PSS + base, T::PWS, Lx, Ly);
                v = add_ref(q, v);
                f[q] = v.x;
                g[q] = v.y;
            } else {
                lost = true;
                const R2 v = add_ref(q, sp[q * T::PSS + own]);
                f[q] = v.x;
                g[q] = v.y;
            }
        }
        }
        if (missing) {
            // wall targets: rho, T at B = A + dt n0 by Q2 interpolation of
            // M^k; u = wall velocity; gradients of M^k at the wall node; the
            // missing populations by Grad's approximation (Sec. III A)
            int base;
            R xi, eta;
            R rhoB = sM[m], TB = sM[3 * T::MS + m];
            if (departure(0, dt * (R)MD(n0)[2 * j], dt * (R)MD(n0)[2 * j + 1], base, xi, eta)) {
                R Lx[3], Ly[3];
                lagrange3(xi, Lx);
                lagrange3(eta, Ly);
                // element origin in the staged tile -> in the moment tile
                const int wa = base / T::PWS + pi0, wb = base - (base / T::PWS) * T::PWS + sj0;
                const int w0 = (wa - mi0) * T::MW + (wb - mj0);
                rhoB = R(0);
                TB = R(0);
                // row 0 from the other side (a junction's window below row 0)
                unsigned mw = 0u;
                if (GEN && rear && wa == -2)
                    for (int b2 = 0; b2 < 3; ++b2) {
                        const int c2 = ctype(wb + b2);
                        if ((c2 & CT_WALL) && !(c2 & CT_JUNC)) mw |= 1u << b2;
                    }
                const bool wok = in_bounds(w0 >= 0 && w0 + 2 * T::MW + 2 < T::MS, a.status);
                // the wall node's own value plus the weighted differences from
                // it (as for the outlet targets: the weights' round-off then
                // acts on small differences)
                const R rhoA = sM[m], TA = sM[3 * T::MS + m];
#pragma unroll
                for (int aa = 0; aa < 3; ++aa)
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb) {
                        if (!wok) continue;
                        const R wgt = Lx[aa] * Ly[bb];
                        const bool far = aa == 2 && ((mw >> bb) & 1u);
                        const int c2 = nt - 1 - wb - bb;
                        rhoB += wgt * ((far ? M_in[c2] : sM[w0 + aa * T::MW + bb]) - rhoA);
                        TB += wgt * ((far ? M_in[(size_t)3 * N + c2] : sM[3 * T::MS + w0 + aa * T::MW + bb]) - TA);
                    }
                rhoB += rhoA;
                TB += TA;
            } else {
                atomicOr(a.status, ST_BPOINT);
            }
            R G[4];
            if constexpr (GEN) {
                R j00, j01, j10, j11;
                ld4(sJ + 4 * dn, j00, j01, j10, j11);
                grad_map_j(j00, j01, j10, j11, F00, F01, F10, F11, G);
            } else {
                grad_map(row, col, F00, F01, F10, F11, G);
            }
            R gr[3][2];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const R* p = sM + (c + 1) * T::MS + m;
                R cxi, cet;
                if constexpr (GEN) {
                    cxi = d_row_c(p, T::MW, 0, nr, rear);
                    cet = d_col_c(p, j, nt, cg, jdir_of(ct));
                } else {
                    cxi = d_row(p, T::MW, 0, nr);
                    cet = d_col(p);
                }
                gr[c][0] = G[0] * cxi + G[1] * cet;
                gr[c][1] = G[2] * cxi + G[3] * cet;
            }
            R fw[9], gw[9];
            grad_populations(rhoB, vx, vy, TB, gr[0][0], gr[0][1], gr[1][0], gr[1][1], gr[2][0],
                             gr[2][1], mu, dt, Cv, Pr, fw, gw);
#pragma unroll
            for (int q = 0; q < 9; ++q)
                if (missing & (1u << q)) {
                    f[q] = fw[q];
                    g[q] = gw[q];
                }
        }
        if (lost) atomicOr(a.status, ST_DEPARTURE);
        const Macro<R> mc = moments(f, g, Cv);
        if (!(mc.rho > R(0)) || !(mc.T > R(0)) || !isfinite(mc.ux) || !isfinite(mc.uy))
            atomicOr(a.status, ST_NONPHYS);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            R2 v;
            v.x = f[q];
            v.y = g[q];
            p_out[(size_t)q * N + n] = v;
            if (dup2) p_out[(ptrdiff_t)q * N + n2] = v;
        }
        M_out[n] = mc.rho; M_out[(size_t)N + n] = mc.ux; M_out[(size_t)2 * N + n] = mc.uy;
        M_out[(size_t)3 * N + n] = mc.T;
        if (dup2 || mir) {
            M_out[n2] = mc.rho; M_out[(ptrdiff_t)N + n2] = mc.ux; M_out[(ptrdiff_t)2 * N + n2] = mc.uy;
            M_out[(ptrdiff_t)3 * N + n2] = mc.T;
        }
        if (wall) {
            // wall stress sigma = -p I - (1 - omega/2) P^(1), P^(1) = sum (f - f^eq) c c
            // (Sec. III), this node's Simpson share of its edges: float64 from
            // the populations on (their moments, f^eq and f - f^eq too)
            double fd[9], gd[9], feq[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                fd[q] = (double)f[q];
                gd[q] = (double)g[q];
            }
            const Macro<double> md = moments(fd, gd, SD(Cv));
            f_equilibrium(md.rho, md.ux, md.uy, md.T, feq);
            double pxx = 0, pxy = 0, pyy = 0;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const double fn = fd[q] - feq[q];
                pxx += cxq(q) * cxq(q) * fn;
                pxy += cxq(q) * cyq(q) * fn;
                pyy += cyq(q) * cyq(q) * fn;
            }
            const double rho = md.rho, Tn = md.T;
            const double om = 1.0 / (0.5 + SD(mu) / (rho * Tn * SD(dt)));
            const double p = rho * Tn, am = 1.0 - 0.5 * om;
            const double sxx = -p - am * pxx, sxy = -am * pxy, syy = -p - am * pyy;
            // the wall node moves with its own body (its chain's body on a
            // C-grid with several bodies): rotation and moment reference of
            // that body
            if constexpr (GEN) fbid = (ct >> CT_BODY_SHIFT) & (MAX_BODIES - 1);
            const BodyMap<double>& mw = mapSd[fbid];
            const double R00 = 1.0 + mw.a00, R01 = mw.a01, R10 = mw.a10, R11 = 1.0 + mw.a11;
            const BodyDev& bd = *(SD(body) + (size_t)sb * nb + fbid);
            const double Xd = MD(xw)[2 * j] - bd.xp;
            const double Yd = MD(xw)[2 * j + 1] - bd.yp;
            const double rx = R00 * Xd + R01 * Yd, ry = R10 * Xd + R11 * Yd;
            const double* wg = MD(wall_geo) + 6 * j;
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
    if (GEN && a.record) return;
    if (i0 == 0) {
        if (tid < TJ) {
            s_red[0][tid] = fcx;
            s_red[1][tid] = fcy;
            s_red[2][tid] = fcm;
            if constexpr (GEN) s_bid[tid] = fbid;
        }
        __syncthreads();
        if (tid == 0) {
            // per body, in column order
            for (int b = 0; b < nb; ++b) {
                double s0 = 0.0, s1 = 0.0, s2 = 0.0;
                for (int t = 0; t < TJ; ++t) {
                    if (GEN && s_bid[GEN ? t : 0] != b) continue;
                    s0 += s_red[0][t];
                    s1 += s_red[1][t];
                    s2 += s_red[2][t];
                }
                double* po = SD(part) + ((size_t)sb * nb + b) * MD(ntj) * 3 + (size_t)tjx * 3;
                po[0] = s0;
                po[1] = s1;
                po[2] = s2;
            }
        }
    }
    if (w == 0) {
        // ---- epilogue: the last CTA of this solve sums the load partials in a
        // fixed order, advances the body by RK4 (Sec. III B, weak coupling:
        // load of this step held over the next), builds the next launch's
        // maps and advances the solve's step number.  The acquire-release
        // count publishes this CTA's partial (written by thread 0) and, for
        // the last CTA, makes every other CTA's partial visible.  When the
        // step number is a launch argument no CTA reads the counter, so only
        // the wall-row tiles (the ones with a partial) take part; otherwise
        // every tile does, so that the step number advances after the last
        // CTA of the solve has read it.
        const bool host_step = UNIFORM && a.ustep >= 0;
        const unsigned ntiles = host_step ? (unsigned)MD(ntj)
                              : UNIFORM ? (unsigned)a.usol.ntiles : (unsigned)s_sol.ntiles;
        unsigned done = 0u;
        if (l == 0 && (!host_step || i0 == 0))
            asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(done) : "l"(ctr) : "memory");
        done = __shfl_sync(0xffffffffu, done, 0);
        if ((!host_step || i0 == 0) && done == ntiles - 1u) {
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            const int ntj = MD(ntj);
            for (int b = 0; b < nb; ++b) {
                const size_t sbb = (size_t)sb * nb + b;
                const double* part = SD(part) + sbb * ntj * 3;
                // lane t holds the partials of tiles t, t + 32, ...; the sum
                // runs over lanes in order (for ntj <= 32: tile order)
                double v[3] = {0.0, 0.0, 0.0};
                for (int t = l; t < ntj; t += 32)
                    for (int c = 0; c < 3; ++c) v[c] += __ldcg(part + (size_t)t * 3 + c);
                double F[3] = {0.0, 0.0, 0.0};
                for (int t = 0; t < 32; ++t)
                    for (int c = 0; c < 3; ++c) F[c] += __shfl_sync(0xffffffffu, v[c], t);
                if (l == 0) {
                    const BodyDev bd = *(SD(body) + sbb);
                    const BodyStateDev Sn = ((cur ? mptr[1] : mptr[0]) + sbb)->S_next;
                    const BodyStateDev Snew = rk4_body(bd, Sn, F[1], F[2], SD(dt), (long long)kstep);
                    StepMaps mo;
                    build_maps(bd, Sn, Snew, Sn, SD(dt), mo);
                    for (int c = 0; c < 3; ++c) mo.loads[c] = F[c];
                    *((cur ? mptr[0] : mptr[1]) + sbb) = mo;
                }
            }
            if (l == 0) {
                ctr[0] = 0u;
                ctr[1] = kstep + 1u;
            }
        }
    }
}

#undef SD
#undef MD

// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_init(const double* __restrict__ M, typename Vec2<R>::T* __restrict__ P,
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
        typename Vec2<R>::T v;
        v.x = fe[q];
        v.y = ge[q];
        P[(b * 9 + q) * N + n] = v;
    }
    for (int c = 0; c < 4; ++c) Mout[(b * 4 + c) * N + n] = (R)Mb[c * (size_t)N + n];
}

__global__ void k_prepare(const BodyDev* __restrict__ bodies, const BodyStateDev* S_cur,
                          const BodyStateDev* S_next, const BodyStateDev* S_vgprev,
                          const double* loads, double dt, int nbatch, StepMaps* maps) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbatch) return;
    StepMaps m = maps[b];
    const BodyStateDev sc = S_cur ? S_cur[b] : m.S_cur;
    const BodyStateDev sn = S_next ? S_next[b] : m.S_next;
    const BodyStateDev sp = S_vgprev ? S_vgprev[b] : m.S_vgprev;
    build_maps(bodies[b], sc, sn, sp, dt, m);
    if (loads)
        for (int c = 0; c < 3; ++c) m.loads[c] = loads[b * 3 + c];
    maps[b] = m;
}

__global__ void k_advance(const BodyDev* __restrict__ bodies, const double* __restrict__ loads,
                          double dt, long long n, int nbatch, StepMaps* maps) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbatch) return;
    StepMaps m = maps[b];
    const BodyStateDev s = m.S_next;
    const BodyStateDev ns = rk4_body(bodies[b], s, loads[b * 3 + 1], loads[b * 3 + 2], dt, n);
    build_maps(bodies[b], m.S_cur, ns, s, dt, m);
    maps[b] = m;
}

// Tile shapes of the step kernel (angular tile width one warp).
constexpr int TJ = TILE_J;

template <typename R, int TI, int NT, int MINB, bool UNIFORM, bool GEN = false>
struct StepKernel {
    static inline int resident = -1;   // CTAs resident on the whole GPU at once

    static cudaError_t configure() {
        if (resident >= 0) return cudaSuccess;
        const size_t smem = step_smem_bytes<R, TI, TJ, GEN>();
        cudaError_t e = cudaFuncSetAttribute(k_step<R, TI, TJ, NT, MINB, UNIFORM, GEN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<R, TI, TJ, NT, MINB, UNIFORM, GEN>, NT, smem);
        if (e != cudaSuccess) return e;
        resident = sms * per_sm;
        return cudaSuccess;
    }

    static cudaError_t launch(const StepArgs& a, int nbatch, cudaStream_t s) {
        cudaError_t e = configure();
        if (e != cudaSuccess) return e;
        const size_t smem = step_smem_bytes<R, TI, TJ, GEN>();
        if (UNIFORM) {
            // prefetch distance: one resident wave for the separable kernel
            // staging by per-thread copies only; none where tensor copies
            // stage the tiles, nor in the general kernel (measured faster
            // without, C-grids included)
            StepArgs b = a;
            b.pf_dist = (a.tma || GEN) ? 0 : resident;
            int nti = (a.umesh.nr + TI - 1) / TI;
            if (GEN && a.collide_only && a.cgrid_pre) nti = std::min(nti, (CGRID_PRE_ROWS + TI - 1) / TI);
            const dim3 grid = a.uorder ? dim3(nbatch, a.umesh.ntj, nti) : dim3(a.umesh.ntj, nti, nbatch);
            k_step<R, TI, TJ, NT, MINB, UNIFORM, GEN><<<grid, NT, smem, s>>>(b);
        } else {
            k_step<R, TI, TJ, NT, MINB, UNIFORM, GEN><<<a.ntiles, NT, smem, s>>>(a);
        }
        return cudaGetLastError();
    }
};

template <typename R, int TI, int NT, int MINB, bool UNIFORM>
static cudaError_t launch_step_t(const StepArgs& a, int nbatch, cudaStream_t s) {
    return StepKernel<R, TI, NT, MINB, UNIFORM>::launch(a, nbatch, s);
}

// General meshes (node coordinates given): one tile shape per precision
// (general_tile_rows rows), in uniform and in table launches.
static cudaError_t launch_general(const StepArgs& a, int precision, int nbatch, cudaStream_t s) {
    static_assert(GEN_TILE_ROWS == 8 && GEN_TILE_ROWS_FP32 == 12, "tile shapes of the general kernel");
    if (precision == 0) return StepKernel<double, 8, 256, 1, true, true>::launch(a, nbatch, s);
    return StepKernel<float, 12, 384, 2, true, true>::launch(a, nbatch, s);
}

template <bool UNIFORM>
static cudaError_t configure_any(int precision, int variant) {
    if (precision == 0) {
        switch (variant) {
            case 1: return StepKernel<double, 4, 256, 1, UNIFORM>::configure();
            case 2: return StepKernel<double, 2, 256, 1, UNIFORM>::configure();
            default: return StepKernel<double, 8, 256, 1, UNIFORM>::configure();
        }
    }
    switch (variant) {
        case 1: return StepKernel<float, 16, 256, 2, UNIFORM>::configure();
        case 2: return StepKernel<float, 8, 256, 3, UNIFORM>::configure();
        case 3: return StepKernel<float, 12, 384, 2, UNIFORM>::configure();
        case 4: return StepKernel<float, 16, 512, 2, UNIFORM>::configure();
        default: return StepKernel<float, 8, 256, 2, UNIFORM>::configure();
    }
}

cudaError_t launch_step_general_table(const StepArgs& a, int precision, cudaStream_t s) {
    if (precision == 0) return StepKernel<double, 8, 256, 1, false, true>::launch(a, 0, s);
    return StepKernel<float, 12, 384, 2, false, true>::launch(a, 0, s);
}

cudaError_t prepare_step(int precision, int variant, bool uniform, bool general) {
    if (general && !uniform)
        return precision == 0 ? StepKernel<double, 8, 256, 1, false, true>::configure()
                              : StepKernel<float, 12, 384, 2, false, true>::configure();
    if (general)
        return precision == 0 ? StepKernel<double, 8, 256, 1, true, true>::configure()
                              : StepKernel<float, 12, 384, 2, true, true>::configure();
    return uniform ? configure_any<true>(precision, variant) : configure_any<false>(precision, variant);
}

int step_variants(int precision) { return precision == 0 ? 3 : 5; }

template <bool UNIFORM>
static cudaError_t launch_any(const StepArgs& a, int precision, int variant, int nbatch, cudaStream_t s) {
    if (precision == 0) {
        // float64: 8-row tiles, or 4 and 2 rows to spread a small mesh over
        // more SMs (the float64 rate per SM bounds it)
        switch (variant) {
            case 1: return launch_step_t<double, 4, 256, 1, UNIFORM>(a, nbatch, s);
            case 2: return launch_step_t<double, 2, 256, 1, UNIFORM>(a, nbatch, s);
            default: return launch_step_t<double, 8, 256, 1, UNIFORM>(a, nbatch, s);
        }
    }
    switch (variant) {
        case 1: return launch_step_t<float, 16, 256, 2, UNIFORM>(a, nbatch, s);
        case 2: return launch_step_t<float, 8, 256, 3, UNIFORM>(a, nbatch, s);
        case 3: return launch_step_t<float, 12, 384, 2, UNIFORM>(a, nbatch, s);
        case 4: return launch_step_t<float, 16, 512, 2, UNIFORM>(a, nbatch, s);
        default: return launch_step_t<float, 8, 256, 2, UNIFORM>(a, nbatch, s);
    }
}

cudaError_t launch_step(const StepArgs& a, int precision, int variant, cudaStream_t s) {
    return launch_any<false>(a, precision, variant, 0, s);
}

cudaError_t launch_step_uniform(const StepArgs& a, int precision, int variant, int nbatch,
                                cudaStream_t s) {
    if (a.umesh.general) return launch_general(a, precision, nbatch, s);
    return launch_any<true>(a, precision, variant, nbatch, s);
}

int tile_rows(int precision, int variant) {
    if (precision == 0) return variant == 1 ? 4 : variant == 2 ? 2 : 8;
    switch (variant) {
        case 1: return 16;
        case 3: return 12;
        case 4: return 16;
        default: return 8;
    }
}

cudaError_t launch_init(int precision, const double* M, void* P, void* Mout, int N, int nbatch,
                        double Cv, cudaStream_t s) {
    const size_t total = (size_t)N * nbatch;
    const int bs = 256;
    const unsigned nb = (unsigned)((total + bs - 1) / bs);
    if (precision == 0)
        k_init<double><<<nb, bs, 0, s>>>(M, (double2*)P, (double*)Mout, N, nbatch, Cv);
    else
        k_init<float><<<nb, bs, 0, s>>>(M, (float2*)P, (float*)Mout, N, nbatch, Cv);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const BodyDev* bodies, const BodyStateDev* S_cur,
                           const BodyStateDev* S_next, const BodyStateDev* S_vgprev,
                           const double* loads, double dt, int nbatch, StepMaps* maps,
                           cudaStream_t s) {
    k_prepare<<<(nbatch + 127) / 128, 128, 0, s>>>(bodies, S_cur, S_next, S_vgprev, loads, dt, nbatch, maps);
    return cudaGetLastError();
}

cudaError_t launch_advance(const BodyDev* bodies, const double* loads, double dt, long long n,
                           int nbatch, StepMaps* maps, cudaStream_t s) {
    k_advance<<<(nbatch + 127) / 128, 128, 0, s>>>(bodies, loads, dt, n, nbatch, maps);
    return cudaGetLastError();
}

}  // namespace lbfsi
