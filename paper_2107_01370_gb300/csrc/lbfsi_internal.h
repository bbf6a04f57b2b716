// Internal declarations shared by the kernels and the C-ABI layer.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace lbfsi {

// Status bits written by the kernels (OR-ed into a device word).
enum : unsigned {
    ST_DEPARTURE = 1u,   // departure point outside the adjacent cells
    ST_NONPHYS = 2u,     // rho <= 0, T <= 0 or NaN
    ST_BPOINT = 4u,      // wall or outlet target point B outside the cells next to its node
    ST_BOUNDS = 8u,      // bounds-checked build: an index outside its buffer (access skipped)
    ST_TMA = 16u,        // a tensor-copy wait of the step ran out of iterations
};

// Body model with dimensional ODE coefficients (Sec. III, Sec. IV).
struct BodyDev {
    int dof;                 // 0 fixed, 1 transverse, 2 pitch-plunge
    double xc, yc, xp, yp;   // blend centre, reference point
    double r_in, r_out, inv_w;   // blend radii, 1 / (r_out - r_in)
    double m, k, c;          // transverse: m h'' + c h' + k h = F_y
    double s_a, i_a, k_h, k_a;  // pitch-plunge: [m S; S I] y'' + diag(k_h, k_a) y = [F_y; M]
    double pitch_amp, w_a, t_forced;  // forced pitch amp sin(w_a t) while (n + 1) dt <= t_forced
};

struct BodyStateDev {
    double h, alpha, hdot, adot;
};

// Per-row and per-column geometry of the O-grid X = centre + r_i e_j (see
// the table builder in lbfsi_api.cu for the meaning of each entry).
// Entries are grouped in fours so that a kernel reads each group with one
// 16-byte load.
constexpr int ROWTAB = 8;
constexpr int COLTAB = 16;
// row i: [0..3] xi of the node and 1 / (dR/dxi) in the cells i-1 and i
// (element coordinates), [4] r_i, [5] 1 / (dr/dxi) at the node (centred),
// [6] 1 / r_i, [7] unused
enum : int { RT_XIN0 = 0, RT_IDR0 = 1, RT_XIN1 = 2, RT_IDR1 = 3, RT_R = 4, RT_IDRC = 5, RT_IR = 6 };
// column j: [0..3] (de_y, e_y, de_x, e_x) / (e x de) with de the centred
// difference of the direction vectors (inverse metric), [4..5] e_j, [6..7]
// unused, [8..11] and [12..15] for the cells j-1 and j: eta of the node,
// dE/deta (x, y) and dE x e_j
enum : int { CT_G = 0, CT_E = 4, CT_C0 = 8, CT_C1 = 12 };

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

// Mirrored rows kept below row 0 of a C-grid (the +-4 staging halo).
constexpr int CGRID_GHOST_ROWS = 4;
// Rows whose post-collision state a C-grid step's first launch writes: the
// tiles of the first row of tiles stream from it (their +-2 window reaches
// the mirrored rows, i.e. the other side's collided nodes); every other tile
// collides its own window in the second launch.
constexpr int CGRID_PRE_ROWS = 16;
// Classes of a C-grid's row-0 columns: on the cut, on a wall chain, a
// junction (a chain's end next to the cut, one point with its mirror), a
// second copy of the mirrored column's node (past the middle of row 0), and
// for a junction whether its cut neighbour is the next column (else the
// previous one).
enum : int { CT_CUT = 1, CT_WALL = 2, CT_JUNC = 4, CT_DUP = 8, CT_JFWD = 16 };
// A wall column's body (C-grids with independent bodies): bits from
// CT_BODY_SHIFT of its class.  At most MAX_BODIES bodies per solve.
constexpr int MAX_BODIES = 4;
enum : int { CT_BODY_SHIFT = 5 };

// Geometry of one O-grid mesh shape, shared by every solve on it (device).
struct MeshDev {
    int nr, nt, N, ntj;            // N: node slots per field component (nr nt, plus the
                                   // mirrored rows of a C-grid)
    double xm, ym;                 // mesh centre
    const double* r;               // [nr]
    const double* e;               // [nt][2]
    const double* n0;              // [nt][2] wall normals (undeformed)
    const double* wall_geo;        // [nt][6] two (weight*length, n_x, n_y) edge shares per wall node
    const void* rowtab;            // [nr][ROWTAB] per-row geometry (element type of the path)
    const void* coltab;            // [nt][COLTAB] per-column geometry
    float xm_f, ym_f;
    double emin;                   // separable O-grid: min over j of |e_j| (static-tile test)
    float emin_f;
    const double* xw;              // [nt][2] wall node coordinates
    const double* fardir;          // [nt][2] outward unit direction at the far-field row
    // general meshes (node coordinates given): element type of the path
    int general;
    const void* nodex;             // [N][2] node coordinates
    const void* jinv;              // [N][4] inverse metric (index derivatives -> d/dX, d/dY)
    const void* cellc;             // [(nr-1) nt][8] element coefficients per cell
    // C-grid (general meshes only): the node, metric and cell arrays and every
    // field component hold mirrored rows -4..-1 below row 0 (their pointers
    // point at row 0); coltype classes the row-0 columns (CT_*); columns 0
    // and nt-1 are outlets
    int cgrid;
    const int* coltype;            // [nt]
    const double* fardirj;         // [nr][2][2] outward unit directions of columns 0 and nt-1
    // doubly periodic box (general meshes only): rows wrap like columns,
    // every node is interior (no wall, no far field)
    int box;
};

// One solve (one set of fields on one mesh and its bodies: nbody > 1 only on
// general meshes, where the maps, body and load-partial arrays hold nbody
// consecutive records).  Buffers are
// ping-pong pairs; which one holds the current state follows from the solve's
// step number k (counter[1]): after k step launches the state is in buffer
// k & 1, and the launch with k == 0 streams from the initial (post-collision)
// state without colliding.  counter[0] counts the CTAs of the solve that have
// finished the current launch; the last one advances the body, resets
// counter[0] and writes k + 1.
struct SolveDev {
    int mesh;
    int ntiles;                    // CTAs of this solve in every step launch
    int nbody = 1;                 // bodies (maps / body records per solve)
    // flow (float64 and float copies, so that no thread of the float path
    // converts or divides in float64)
    double dt, mu, Cv, Pr, rho_inf, uinf_x, uinf_y, T_inf;
    float dt_f, mu_f, Cv_f, Pr_f, iPr_f, rho_inf_f, uinf_x_f, uinf_y_f, T_inf_f, pad_f;
    // float path: the free-stream equilibrium pairs (f_q, g_q), q = 0..8.  The
    // step interpolates deviations from them, so that the round-off of the
    // float Q2 weights (their sum is 1 only to within an ulp, the same way
    // every step at a node that does not move) scales with the deviation, not
    // with the population
    float fgref[18];
    void* p[2];                    // populations, (f_q, g_q) pairs [9][N]
    void* M[2];                    // moments [4][N]
    StepMaps* maps[2];             // [nbody] each
    void* ppost;                   // collide-only output (post-collision pairs)
    double* part;                  // [nbody][ntj][3] load partials of the streamed step
    unsigned* counter;             // [2]: CTA completion count, step number k
    const BodyDev* body;           // [nbody]
    // general meshes, uniform launches: departure points of the nodes the
    // blend does not move (g = I, V_G = 0, so the displacement of direction q
    // is -dt c_q for every step): (xi, eta) pairs [9][N] in the element type
    // of the path and per node a code [N] (5 bits per direction: the window
    // origin relative to the node, row and column offsets in -3..0, or a lost
    // departure; all ones: not cached), shared by the solves of the handle
    // (one mesh, one dt), or null
    void* dep_xe = nullptr;
    unsigned long long* dep_code = nullptr;
};

// One CTA of a step launch: a tile of one solve.  The entry repeats the
// solve's counter and maps pointers so that a CTA can read its step number
// and fetch its maps without first loading the solve record.  tma: stage the
// tile's M^k and populations by tensor copies (StepArgs::tmaps).
struct TileDev {
    int solve, mesh, i0, j0, tj, tma;
    unsigned* counter;
    StepMaps* maps[2];
};

struct StepArgs {
    MeshDev umesh;                 // uniform launch: the mesh
    SolveDev usol;                 // uniform launch: solve 0 (others by stride)
    const MeshDev* meshes;
    const SolveDev* solves;
    const TileDev* tiles;
    int ntiles;
    int collide_only;              // 1: write the collided current state to ppost only
    int ustep;                     // uniform launch: the solves' step number (they advance
                                   // together), or -1 to read it from the device counters
    int uorder;                    // uniform launch: CTA order, 0 = (tile column, tile row,
                                   // solve), 1 = (solve, tile column, tile row)
    int pf_dist;                   // uniform launch: L2 prefetch distance in CTAs (set by the launcher)
    int stream_post;               // C-grid step, second launch: the tiles next to the cut
                                   // (rows < CGRID_PRE_ROWS - tile - 2) stream from ppost
                                   // (written by the step's collide-only launch) without
                                   // colliding, every other tile collides and streams in one
                                   // pass; the step with k == 0 streams the initial state as
                                   // always
    int cgrid_pre;                 // C-grid collide-only launch of a step: only the tiles of
                                   // rows < CGRID_PRE_ROWS (the others return at once)
    int record;                    // general meshes, uniform: fill usol.dep_* (departures of
                                   // the static nodes of solve 0) and write nothing else
    unsigned* status;
    // uniform launch of the float kernel: stage the populations and M^k of a
    // tile whose columns do not wrap by two tensor copies (TMA) into shared
    // memory instead of per-thread copies.  tm_p[c] / tm_M[c] describe buffer
    // c (c = k & 1) of all solves as 4-D float arrays: populations
    // (2 nt, nr + tma_g, 9, nbatch) with boxes (2 (TJ + 8), TI + 4, 9, 1),
    // moments (nt, nr + tma_g, 4, nbatch) with boxes (TJ + 8, TI + 8, 4, 1);
    // tma_g: the mirrored rows a C-grid stores below row 0 (lbfsi_api.cu).
    int tma;
    int tma_g;
    // table launch of the float separable kernel: per solve the tensor maps of
    // its populations (buffers 0, 1) and moments (buffers 0, 1), in device
    // memory, [solve][4], each a (2 nt, nr, 9, 1) or (nt, nr, 4, 1) float
    // array with the boxes above; used by the tiles whose TileDev::tma is set
    const CUtensorMap* tmaps;
    alignas(64) CUtensorMap tm_p[2];
    alignas(64) CUtensorMap tm_M[2];
};

// Tensor map of a float array of dims (dx, dy, dz, dw), x fastest and dense,
// read in boxes of (bx, by, bz, 1), elements outside the array as zeros;
// false if the map cannot be made (defined in lbfsi_api.cu).
bool encode_box4(CUtensorMap* map, void* base, size_t dx, size_t dy, size_t dz, size_t dw, unsigned bx,
                 unsigned by, unsigned bz);

// Record msg as the calling thread's last error and return code (defined in
// lbfsi_api.cu).
int set_error(int code, const std::string& msg);

// Launchers (defined in lbfsi_step.cu).  variant selects the tile shape of
// the step kernel (see tile_rows): five float shapes, float64 tiles of 8, 4
// or 2 rows.
cudaError_t launch_step(const StepArgs& a, int precision, int variant, cudaStream_t s);
// Uniform launch over nbatch solves of one mesh (see StepArgs).
cudaError_t launch_step_uniform(const StepArgs& a, int precision, int variant, int nbatch,
                                cudaStream_t s);
int tile_rows(int precision, int variant);
// Tile rows of the general-geometry kernel, in uniform (mesh handle) and
// table (batch runtime) launches alike: 8 in float64 (256 threads, one CTA
// per SM), 12 in float (384 threads, two CTAs per SM: 24 resident warps
// where an 8-row tile's registers and shared memory allowed 16).
constexpr int GEN_TILE_ROWS = 8;
constexpr int GEN_TILE_ROWS_FP32 = 12;
inline int general_tile_rows(int precision) { return precision == 0 ? GEN_TILE_ROWS : GEN_TILE_ROWS_FP32; }
// Table launch of the general-geometry kernel (the batch runtime's solves on
// meshes given by node coordinates).
cudaError_t launch_step_general_table(const StepArgs& a, int precision, cudaStream_t s);
// Number of tile shapes of the float step kernel (variants 0 .. n-1); the
// float64 kernel has one.
int step_variants(int precision);
// One-time configuration of a step kernel (shared-memory limit, occupancy);
// done by the first launch, and by this call before a stream capture.
cudaError_t prepare_step(int precision, int variant, bool uniform, bool general = false);
constexpr int TILE_J = 32;
inline int tiles_j(int nt) { return (nt + TILE_J - 1) / TILE_J; }
cudaError_t launch_init(int precision, const double* M, void* P, void* Mout, int N, int nbatch,
                        double Cv, cudaStream_t s);
// Build the maps record from explicit states: S_cur (collision), S_next and
// S_vgprev (stream); loads copied from 'loads' if non-null.
cudaError_t launch_prepare(const BodyDev* bodies, const BodyStateDev* S_cur,
                           const BodyStateDev* S_next, const BodyStateDev* S_vgprev,
                           const double* loads, double dt, int nbatch, StepMaps* maps,
                           cudaStream_t s);
// RK4 of every body over dt with the given loads from maps->S_next; the
// result becomes S_next and the old S_next S_vgprev and S_cur.
cudaError_t launch_advance(const BodyDev* bodies, const double* loads, double dt, long long n,
                           int nbatch, StepMaps* maps, cudaStream_t s);

}  // namespace lbfsi
