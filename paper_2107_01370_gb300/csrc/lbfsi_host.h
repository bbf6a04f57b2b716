// Host-side helpers shared by the mesh handle (lbfsi_api.cu) and the batch
// runtime (lbfsi_batch.cu): mesh validation and derived geometry tables,
// body and flow parameters, device allocation of a mesh's geometry.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <string>
#include <vector>

#include "lbfsi.h"
#include "lbfsi_internal.h"

namespace lbfsi {

// NVTX range over a host call of the library (shown by profilers that
// collect NVTX; without one attached, a push and a pop that do nothing).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// A validated O-grid shape with its derived tables (float64, host).  Either
// separable (X = centre + r_i e_j: r, e, rowtab, coltab) or general (node
// coordinates X, per-node inverse metric jinv, per-cell element coefficients
// cellc).  Both: wall node coordinates xw, far-field outward directions
// fardir, wall normals n0 and Simpson shares wall_geo.
struct HostMesh {
    int nr = 0, nt = 0, N = 0, ntj = 0;
    // node slots per field component: N, plus G mirrored rows below row 0 on
    // a C-grid (row 0 starts at slot G nt)
    int Nx = 0, G = 0;
    double xm = 0, ym = 0;
    bool general = false;
    // C-grid: the wall chains (inclusive row-0 column ranges) and the class
    // of every row-0 column (CT_*, a wall column's body from CT_BODY_SHIFT);
    // nbody: bodies per solve (the chains' owners)
    bool cgrid = false;
    std::vector<int> walls, coltype;
    int nbody = 1;
    // doubly periodic box (no wall, no far field): rows wrap as well
    bool box = false;
    std::vector<double> r, e, n0, wall_geo, rowtab, coltab, xw, fardir, X, jinv, cellc;
    std::vector<double> fardirj;   // C-grid: [nr][2][2] outward directions of the outlet columns
};


// Per-cell element coefficients of a general mesh: 8 entries per cell (a, b),
// a in [0, nr-2], b in [0, nt-1], row-major: the bilinear map of the cell's
// Q2 element, X(xi, eta) = X0 + b xi + c eta + d xi eta, as (b_x, b_y, c_x,
// c_y, d_x, d_y, 0, 0).
constexpr int CELLC = 8;

// Validate (sizes, increasing radii, subparametric tables) and derive the
// wall geometry and the per-row / per-column tables.  Returns an lbfsi_status
// and sets the thread's last error on failure.
int build_host_mesh(int nr, int nt, const double* r, const double* e, double xc, double yc,
                    HostMesh& out);

// The same for an O-grid given by its node coordinates X [nr][nt][2]
// (subparametric, positive Jacobian): wall geometry, far-field directions,
// per-node inverse metric and per-cell element coefficients.
int build_host_mesh_xy(int nr, int nt, const double* X, double xc, double yc, HostMesh& out);

// The same for a C-grid given by its node coordinates X [nr][nt][2] (nt
// odd) and its wall chains walls[2 k], walls[2 k + 1] (inclusive row-0
// column ranges, even ends; the rest of row 0 is cut, symmetric in
// j -> nt-1-j, its nodes and the chains' ends one point with their mirrors):
// the arrays carry G mirrored rows below row 0 (node (-k, j) = node
// (k, nt-1-j)).  wall_body (NULL: every chain body 0) names the body of each
// chain among nbody independent bodies; mirrored chains share their body.
int build_host_mesh_c(int nr, int nt, int nwalls, const int* walls, const double* X, double xc, double yc,
                      HostMesh& out, int nbody = 1, const int* wall_body = nullptr);

// A doubly periodic box given by the node coordinates X [ni][nj][2] of one
// period and the period vectors along i and j (node (i + ni, j) = node (i, j)
// + shift_i): no wall, no far field; bodies must be fixed.
int build_host_mesh_box(int ni, int nj, const double* X, const double* shift_i, const double* shift_j,
                        HostMesh& out);

// Normals and Simpson shares of a closed chain of points P [n][2] (even n,
// counterclockwise around what it bounds, even entries the vertices of its
// straight edges): n0 [n][2] the unit normals out of the bounded region (at a
// vertex the normalised sum of its two edge normals), wgeo [n][6] the node's
// (weight x length, n_x, n_y) share of each of its edges (one edge for a
// midpoint, 4/6; two for a vertex, 1/6 each).
void chain_geometry(const std::vector<double>& P, std::vector<double>& n0, std::vector<double>& wgeo);

// Check the bodies of n solves ([n][m.nbody]) against a mesh: dof range,
// blend radii, each wall inside its own body's rigid zone and outside every
// other body's blended region, blended regions of moving bodies disjoint.
int validate_bodies(const HostMesh& m, const lbfsi_body_desc* bodies, int n);

// Dimensional ODE coefficients from the nondimensional groups.
BodyDev body_dev(const lbfsi_body_desc& d, double rho, double U);

// Validate flow parameters and fill the flow fields of a solve descriptor.
int fill_flow(const lbfsi_flow_params& p, SolveDev& s);

// Free-stream speed and viscosity of a flow.
double flow_u_inf(const lbfsi_flow_params& p);

// Simple device memory source: a plain cudaMalloc allocator, or a
// first-fit arena carved from one cudaMalloc (the batch runtime's pool).
struct DevMemory {
    virtual ~DevMemory() {}
    virtual void* alloc(size_t bytes) = 0;
    virtual void release(void* p) = 0;
};

struct CudaMallocMemory : DevMemory {
    void* alloc(size_t bytes) override;
    void release(void* p) override;
};

// Device copy of a mesh's geometry (tables in the path's element type).
struct DeviceMesh {
    MeshDev dev{};
    std::vector<void*> blocks;
    size_t bytes = 0;
};

int upload_mesh(const HostMesh& h, int precision, DevMemory& mem, cudaStream_t s, DeviceMesh& out);
void release_mesh(DeviceMesh& m, DevMemory& mem);

// Bytes of device memory one solve on an N-node mesh needs (populations,
// moment fields, maps, partials, counter, body), and of a mesh's geometry.
size_t solve_bytes(int N, int ntj, int precision);
size_t mesh_bytes(int nr, int nt, int precision);

}  // namespace lbfsi
