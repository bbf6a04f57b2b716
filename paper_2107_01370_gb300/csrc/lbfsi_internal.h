// Internal declarations shared by the kernels and the C-ABI layer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbfsi {

// Status bits written by the kernels (OR-ed into a device word).
enum : unsigned {
    ST_DEPARTURE = 1u,   // departure point outside the adjacent cells
    ST_NONPHYS = 2u,     // rho <= 0, T <= 0 or NaN
    ST_BPOINT = 4u,      // wall target point outside the first element row
};

// Body model with dimensional ODE coefficients (Sec. III, Sec. IV).
struct BodyDev {
    int dof;                 // 0 fixed, 1 transverse, 2 pitch-plunge
    double xc, yc, xp, yp;   // blend centre, reference point
    double r_in, r_out;
    double m, k, c;          // transverse: m h'' + c h' + k h = F_y
    double s_a, i_a, k_h, k_a;  // pitch-plunge: [m S; S I] y'' + diag(k_h, k_a) y = [F_y; M]
};

struct BodyStateDev {
    double h, alpha, hdot, adot;
};

enum StepMode : int { MODE_STREAM_ONLY = 0, MODE_COLLIDE_STREAM = 1, MODE_COLLIDE_ONLY = 2 };

// Arguments of the fused step kernel (one launch = collide step k in shared
// memory, then stream step k+1).
struct StepArgs {
    int nr, nt, N, nbatch, ntj;
    double xm, ym;             // mesh centre
    const double* r;           // [nr]
    const double* e;           // [nt][2]
    const double* n0;          // [nt][2] wall normals (undeformed)
    const double* wall_geo;    // [nt][6]: per wall node (w1 ds1 n1x n1y, w2 ds2) see api
    // flow
    double dt, mu, Cv, Pr, rho_inf, uinf_x, uinf_y, T_inf;
    // state buffers (element type set by the template)
    const void* f_in;
    const void* g_in;
    void* f_out;
    void* g_out;
    const void* M_in;
    void* M_out;
    // bodies
    const BodyDev* bodies;          // [nbatch]
    const BodyStateDev* S_in;       // [nbatch] state S^k
    const BodyStateDev* S_prev0;    // [nbatch] previous state (stream-only mode)
    const BodyStateDev* S_force;    // [nbatch] prescribed next state (nullptr = RK4)
    BodyStateDev* S_out;            // [nbatch] state S^{k+1}
    const double* part_in;          // [nbatch][ntj][3] load partials of step k
    double* part_out;               // [nbatch][ntj][3] load partials of step k+1
    double* loads_out;              // [nbatch][3] loads of step k (written by tile 0)
    int mode;
    unsigned* status;
};

// Launchers (defined in lbfsi_step.cu).
cudaError_t launch_step(const StepArgs& a, int precision, cudaStream_t s);
cudaError_t launch_init(int precision, const double* M, void* f, void* g, void* Mout, int N,
                        int nbatch, double Cv, cudaStream_t s);
cudaError_t launch_reduce_loads(const double* part, int ntj, int nbatch, double* loads,
                                cudaStream_t s);
cudaError_t launch_advance(const BodyDev* bodies, const BodyStateDev* S, const double* loads,
                           double dt, int nbatch, BodyStateDev* S_out, BodyStateDev* S_prev_out,
                           cudaStream_t s);
cudaError_t launch_convert(int precision, const void* src, double* dst, size_t n, int to_double,
                           cudaStream_t s);

}  // namespace lbfsi
