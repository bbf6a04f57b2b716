// Allocation-free wall-load entry point (lbfsi_wall_loads_noalloc).
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// want the loads -- code that runs while another owner (a framework's caching
// allocator, a real-time loop that forbids allocation after start-up, a
// process that must not grow its device footprint) controls every byte of
// device memory, or that must not trigger the implicit device synchronisation
// a cudaMalloc/cudaFree can cause.  They pass their own input and output
// buffers; the only other memory this entry point touches is the fixed
// scratch array below.
//
// It is the load reduction of the step kernel on its own: the same wall
// stress and Simpson shares per wall node, summed per CTA, then the CTA
// partials summed in a fixed order by the last CTA of each solve.  Its
// scratch (the CTA partials and the per-solve completion counters) lives in a
// file-scope __device__ array instead of handle-owned cudaMalloc memory.
#include <cuda_runtime.h>

#include <mutex>

#include "lbfsi.h"
#include "lbfsi_device.cuh"
#include "lbfsi_internal.h"

namespace {

constexpr int NA_TJ = 32;            // wall nodes per CTA
constexpr int NA_MAX_BATCH = 256;    // solves per call
constexpr int NA_MAX_PARTIALS = 4096;  // nbatch * ceil(ntheta / 32)
constexpr int NA_MAX_DEVICES = 64;

struct NoAllocScratch {
    double part[NA_MAX_PARTIALS * 3];
    unsigned counter[NA_MAX_BATCH];
};

// Held by every GPU that loads the library, until the process exits
// (about 97 KB).  Host code must not pass the symbol itself to a kernel: its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_ptr[NA_MAX_DEVICES] = {};

template <typename R>
__global__ void __launch_bounds__(NA_TJ) k_wall_loads_noalloc(
    int nr, int nt, const double* __restrict__ r, const double* __restrict__ e, double xm,
    double ym, const R* __restrict__ f, const R* __restrict__ g,
    const double* __restrict__ body_ref, double mu, double dt, double Cv,
    double* __restrict__ loads, NoAllocScratch* sc) {
    const int b = blockIdx.y, tile = blockIdx.x, ntj = gridDim.x;
    const int j = tile * NA_TJ + threadIdx.x;
    const size_t N = (size_t)nr * nt;
    __shared__ double red[3][NA_TJ];
    double c0 = 0.0, c1 = 0.0, c2 = 0.0;
    if (j < nt) {
        double fq[9], gq[9];
        for (int q = 0; q < 9; ++q) {
            fq[q] = (double)f[((size_t)b * 9 + q) * N + j];
            gq[q] = (double)g[((size_t)b * 9 + q) * N + j];
        }
        // sigma = -p I - (1 - omega/2) P^(1), P^(1) = sum (f - f^eq) c c (Sec. III),
        // float64 from the populations on, as in the step kernel
        const lbfsi::Macro<double> mc = lbfsi::moments(fq, gq, Cv);
        double feq[9];
        lbfsi::f_equilibrium(mc.rho, mc.ux, mc.uy, mc.T, feq);
        double pxx = 0, pxy = 0, pyy = 0;
        for (int q = 0; q < 9; ++q) {
            const double fn = fq[q] - feq[q];
            pxx += lbfsi::cxq(q) * lbfsi::cxq(q) * fn;
            pxy += lbfsi::cxq(q) * lbfsi::cyq(q) * fn;
            pyy += lbfsi::cyq(q) * lbfsi::cyq(q) * fn;
        }
        const double rho = mc.rho, Tn = mc.T;
        const double om = 1.0 / (0.5 + mu / (rho * Tn * dt));
        const double p = rho * Tn, am = 1.0 - 0.5 * om;
        const double sxx = -p - am * pxx, sxy = -am * pxy, syy = -p - am * pyy;
        // body pose: pitch about its reference point, rigid near the wall
        const double xp = body_ref[3 * b], yp = body_ref[3 * b + 1], al = body_ref[3 * b + 2];
        const double sh = sin(0.5 * al);
        const double R00 = 1.0 - 2.0 * sh * sh, R01 = -sin(al), R10 = sin(al), R11 = R00;
        auto wx = [&](int k) { k = ((k % nt) + nt) % nt; return xm + r[0] * e[2 * k]; };
        auto wy = [&](int k) { k = ((k % nt) + nt) % nt; return ym + r[0] * e[2 * k + 1]; };
        const double Xd = wx(j) - xp, Yd = wy(j) - yp;
        const double rx = R00 * Xd + R01 * Yd, ry = R10 * Xd + R11 * Yd;
        // the wall edges of this node (straight element edges between
        // even-indexed wall nodes) with Simpson weights 1/6 (ends), 4/6 (middle)
        int ea[2], eb[2];
        double w[2];
        int ne;
        if (j % 2) {
            ea[0] = j - 1; eb[0] = j + 1; w[0] = 4.0 / 6.0; ne = 1;
        } else {
            ea[0] = j; eb[0] = j + 2; w[0] = 1.0 / 6.0;
            ea[1] = j - 2; eb[1] = j; w[1] = 1.0 / 6.0; ne = 2;
        }
        for (int k = 0; k < ne; ++k) {
            const double tx = wx(eb[k]) - wx(ea[k]), ty = wy(eb[k]) - wy(ea[k]);
            const double ds = sqrt(tx * tx + ty * ty);
            const double ex = ty / ds, ey = -tx / ds;
            const double nxr = R00 * ex + R01 * ey, nyr = R10 * ex + R11 * ey;
            const double trx = sxx * nxr + sxy * nyr, try_ = sxy * nxr + syy * nyr;
            const double wds = w[k] * ds;
            c0 += wds * trx;
            c1 += wds * try_;
            c2 += wds * (rx * try_ - ry * trx);
        }
    }
    red[0][threadIdx.x] = c0;
    red[1][threadIdx.x] = c1;
    red[2][threadIdx.x] = c2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[3] = {0.0, 0.0, 0.0};
        for (int t = 0; t < NA_TJ; ++t)
            for (int c = 0; c < 3; ++c) s[c] += red[c][t];
        double* po = sc->part + ((size_t)b * ntj + tile) * 3;
        for (int c = 0; c < 3; ++c) po[c] = s[c];
        __threadfence();
        const unsigned done = atomicAdd(&sc->counter[b], 1u);
        if (done == (unsigned)ntj - 1u) {
            __threadfence();
            double F[3] = {0.0, 0.0, 0.0};
            for (int t = 0; t < ntj; ++t)
                for (int c = 0; c < 3; ++c) F[c] += __ldcg(sc->part + ((size_t)b * ntj + t) * 3 + c);
            for (int c = 0; c < 3; ++c) loads[3 * b + c] = F[c];
            sc->counter[b] = 0u;   // leave the counter at zero for the next call
        }
    }
}

// Device address of the scratch array on the current device, looked up once
// per device (with that device current).  The array needs no clearing here:
// each call clears the counters it uses on its own stream.
int scratch_for_current_device(NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lbfsi::set_error(LBFSI_ECUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= NA_MAX_DEVICES) return lbfsi::set_error(LBFSI_EINVAL, "device index too large");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return lbfsi::set_error(LBFSI_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_scratch_ptr[dev];
    return LBFSI_OK;
}

}  // namespace

extern "C" int lbfsi_wall_loads_noalloc(int nr, int ntheta, int nbatch, int precision,
                                        const double* r, const double* e, double xc, double yc,
                                        const void* f, const void* g, const double* body_ref,
                                        double mu, double dt, double gamma, double* loads,
                                        void* cuda_stream) {
    if (nr < 5 || ntheta < 4 || ntheta % 2)
        return lbfsi::set_error(LBFSI_EINVAL, "nr must be >= 5 and ntheta even and >= 4");
    if (precision != LBFSI_FP64 && precision != LBFSI_FP32)
        return lbfsi::set_error(LBFSI_EINVAL, "precision must be LBFSI_FP64 or LBFSI_FP32");
    if (nbatch < 1 || nbatch > NA_MAX_BATCH)
        return lbfsi::set_error(LBFSI_EINVAL, "nbatch must be in [1, 256] for the allocation-free loads");
    const int ntj = (ntheta + NA_TJ - 1) / NA_TJ;
    if ((long long)nbatch * ntj > NA_MAX_PARTIALS)
        return lbfsi::set_error(LBFSI_EINVAL,
                                "nbatch * ceil(ntheta / 32) exceeds 4096, the size of the fixed scratch");
    if (!r || !e || !f || !g || !body_ref || !loads) return lbfsi::set_error(LBFSI_EINVAL, "null pointer");
    if (!(mu > 0) || !(dt > 0) || !(gamma > 1.0)) return lbfsi::set_error(LBFSI_EINVAL, "invalid flow parameters");
    NoAllocScratch* sc = nullptr;
    int rc = scratch_for_current_device(&sc);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the completion counters of this call's solves start at zero (the last
    // CTA of a solve also leaves its counter at zero; clearing them here, in
    // stream order, keeps a call independent of whatever the array held)
    cudaError_t err = cudaMemsetAsync(sc->counter, 0, sizeof(unsigned) * (size_t)nbatch, s);
    if (err != cudaSuccess)
        return lbfsi::set_error(LBFSI_ECUDA, std::string("scratch clear: ") + cudaGetErrorString(err));
    const dim3 grid(ntj, nbatch);
    const double Cv = 1.0 / (gamma - 1.0);
    if (precision == LBFSI_FP64)
        k_wall_loads_noalloc<double><<<grid, NA_TJ, 0, s>>>(nr, ntheta, r, e, xc, yc, (const double*)f,
                                                           (const double*)g, body_ref, mu, dt, Cv, loads, sc);
    else
        k_wall_loads_noalloc<float><<<grid, NA_TJ, 0, s>>>(nr, ntheta, r, e, xc, yc, (const float*)f,
                                                          (const float*)g, body_ref, mu, dt, Cv, loads, sc);
    err = cudaGetLastError();
    if (err != cudaSuccess)
        return lbfsi::set_error(LBFSI_ECUDA, std::string("wall loads launch: ") + cudaGetErrorString(err));
    return LBFSI_OK;
}
