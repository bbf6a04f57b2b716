// Internal declarations shared by the kernels and the C-ABI layer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

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

// Per-row and per-column geometry of the O-grid X = centre + r_i e_j (see
// the table builder in lbfsi_api.cu for the meaning of each entry).
constexpr int ROWTAB = 8;
constexpr int COLTAB = 16;

// Blended rigid map of one body for one body state (defined in
// lbfsi_device.cuh); declared here so the per-step record can hold it.
template <typename R>
struct BodyMap {
    int active;
    R xc, yc, xp, yp, r_in, inv_w;
    R a00, a01, a10, a11, tx, ty;
    R va00, va01, va10, va11, vtx, vty;
};

// Per-solve record handed from one launch to the next: the body state of the
// last streamed step (used by the next collision), the state and previous
// state for the next stream (V_G), the loads of the last streamed step and
// the blended maps built from those states.
struct StepMaps {
    BodyStateDev S_cur, S_next, S_vgprev;
    double loads[3];
    BodyMap<double> Kd, Sd;
    BodyMap<float> Kf, Sf;
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
    const double* wall_geo;    // [nt][6]: per wall node two (weight*length, n_x, n_y) edge shares
    const void* rowtab;        // [nr][ROWTAB] per-row geometry (element type of the path)
    const void* coltab;        // [nt][COLTAB] per-column geometry
    // flow (float64, and float copies for the float path so that no thread
    // converts or divides in float64)
    double dt, mu, Cv, Pr, rho_inf, uinf_x, uinf_y, T_inf;
    float dt_f, mu_f, Cv_f, Pr_f, iPr_f, xm_f, ym_f, rho_inf_f, uinf_x_f, uinf_y_f, T_inf_f;
    // state buffers (element type set by the template)
    const void* f_in;
    const void* g_in;
    void* f_out;
    void* g_out;
    const void* M_in;
    void* M_out;
    // bodies
    const BodyDev* bodies;          // [nbatch]
    const StepMaps* maps_in;        // [nbatch] maps of this launch
    StepMaps* maps_out;             // [nbatch] maps of the next launch (written by the last CTA)
    double* part;                   // [nbatch][ntj][3] load partials of the streamed step
    unsigned* counter;              // [nbatch] CTA completion counters (zero between launches)
    int mode;
    unsigned* status;
};

// Record msg as the calling thread's last error and return code (defined in
// lbfsi_api.cu).
int set_error(int code, const std::string& msg);

// Launchers (defined in lbfsi_step.cu).  variant selects the tile shape of
// the step kernel (0: 8 x 32 nodes, 1: 16 x 32 nodes with two rows per thread).
cudaError_t launch_step(const StepArgs& a, int precision, int variant, cudaStream_t s);
int tiles_j(int nt);
cudaError_t launch_init(int precision, const double* M, void* f, void* g, void* Mout, int N,
                        int nbatch, double Cv, cudaStream_t s);
// Build the maps record from explicit states: S_cur (collision), S_next and
// S_vgprev (stream); loads copied from 'loads' if non-null.
cudaError_t launch_prepare(const BodyDev* bodies, const BodyStateDev* S_cur,
                           const BodyStateDev* S_next, const BodyStateDev* S_vgprev,
                           const double* loads, double dt, int nbatch, StepMaps* maps,
                           cudaStream_t s);
// RK4 of every body over dt with the given loads from maps->S_next; the
// result becomes S_next and the old S_next S_vgprev and S_cur.
cudaError_t launch_advance(const BodyDev* bodies, const double* loads, double dt, int nbatch,
                           StepMaps* maps, cudaStream_t s);

}  // namespace lbfsi
