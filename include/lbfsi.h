/*
 * lbfsi.h - C ABI of the GB300 implementation of the two-population
 * compressible semi-Lagrangian lattice Boltzmann step with fluid-structure
 * coupling on a blended body-fitted mesh (Bhadauria, Dorschner & Karlin,
 * "Lattice Boltzmann method for fluid-structure interaction in compressible
 * flow").
 *
 * Conventions shared by every entry point
 *  - Every call returns an lbfsi_status (0 = success, negative = error) and
 *    never aborts the process.  lbfsi_last_error() gives a thread-local
 *    message for the last failing call of the calling thread.
 *  - Host pointers passed in are borrowed for the duration of the call only
 *    (their contents are copied before the call returns).  Host pointers passed
 *    out must point to caller-owned memory of the stated size.
 *  - All device memory belongs to the mesh handle and is released by
 *    lbfsi_destroy_mesh.  Work is ordered on the CUDA stream given at creation
 *    (NULL = legacy default stream).  lbfsi_step is asynchronous; errors that
 *    the kernels detect (departure point outside the adjacent cells, a
 *    non-physical state) are recorded in a device status word and returned by
 *    the next synchronising call (lbfsi_synchronize, lbfsi_body_forces,
 *    lbfsi_get_*).
 *
 * Mesh: structured O-grid, node (i, j) at X = (xc, yc) + r[i] e[j], i = 0 on
 * the body wall, i = nr-1 on the far field, j periodic.  Node index
 * n = i * ntheta + j.  Second-order elements are the 3x3-node windows whose
 * first node has even indices (the last radial window is clamped to nr-3 when
 * nr is even).  r and e must be subparametric (odd entries the average of
 * their even neighbours), as produced by the package's mesh generator.
 *
 * Field layouts (host arrays, float64, C order):
 *   macroscopic fields  [nbatch][4][nr*ntheta]   rho, u_x, u_y, T
 *   populations         [nbatch][9][nr*ntheta]   D2Q9 order
 *       i = 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1)
 *           7:(-1,-1) 8:(1,-1)
 *   loads               [nbatch][3]              F_x, F_y, M_z
 */
#ifndef LBFSI_H
#define LBFSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbfsi_mesh_s* lbfsi_mesh;

typedef enum {
    LBFSI_OK = 0,
    LBFSI_EINVAL = -1,      /* invalid argument */
    LBFSI_ENOMEM = -2,      /* device or host allocation failed */
    LBFSI_ECUDA = -3,       /* CUDA runtime error */
    LBFSI_EDEPARTURE = -4,  /* departure point not in a cell adjacent to its node (CFL violated) */
    LBFSI_ENONPHYS = -5,    /* rho <= 0, T <= 0 or NaN produced */
    LBFSI_ETIMEOUT = -6,    /* a bounded device wait ran out */
    LBFSI_ESTATE = -7,      /* call out of order (e.g. step before init_fields) */
    LBFSI_EBOUNDS = -8      /* bounds-checked build only: an index of the step outside its
                               buffer (the access was skipped, the results are invalid) */
} lbfsi_status;

enum { LBFSI_FP64 = 0, LBFSI_FP32 = 1 };
enum { LBFSI_BODY_FIXED = 0, LBFSI_BODY_TRANSVERSE = 1, LBFSI_BODY_PITCH_PLUNGE = 2 };

/* One rigid body and its region of influence (Sec. II D, Sec. III).
 * dof: LBFSI_BODY_*.  The blending region is centred at (xc, yc): nodes with
 * |X - Xc| <= r_in move rigidly with the body, nodes beyond r_out stay fixed,
 * the r5 polynomial blends in between (Eq. blendPol).  (xp, yp) is the
 * reference point of the rigid map, of the moment and of the pitch rotation
 * (cylinder centre / elastic axis).  length = D (cylinder) or chord 2b.
 * Transverse: m_star = 4 m / (rho pi D^2), v_r = U / (f_N D), zeta a damping
 * ratio (0 in the paper).  Pitch-plunge: m_star = m / (pi rho b^2),
 * v_r = U / (b omega_alpha sqrt(m*)), x_alpha, r_alpha, wh_wa = omega_h/omega_alpha. */
typedef struct {
    int dof;
    double xc, yc;
    double xp, yp;
    double r_in, r_out;
    double length;
    double m_star, v_r, zeta;
    double x_alpha, r_alpha, wh_wa;
    /* Forced pitching (pitch-plunge, Sec. IV D): alpha(t) = pitch_amp
     * sin(omega_alpha t) is prescribed during the first forced_periods
     * periods 2 pi / omega_alpha (t = step number x dt; a step is forced when
     * it ends within that time), the plunge responding to the load and to the
     * prescribed pitch acceleration; the body is free afterwards.  0, 0: free
     * from the start. */
    double pitch_amp, forced_periods;
} lbfsi_body_desc;

/* Free stream and transport (Sec. II C): U_inf = ma sqrt(gamma t_inf) along +x,
 * mu = rho_inf U_inf length / re, omega from mu = (1/omega - 1/2) rho T dt,
 * omega_1 from Pr.  gamma > 1 (Cv = 1/(gamma - 1), R = 1). */
typedef struct {
    double ma, re, t_inf, gamma, pr, rho_inf, dt, length;
} lbfsi_flow_params;

typedef struct {
    int nr, ntheta;             /* nr >= 5, ntheta even >= 4 */
    const double* r;            /* [nr]        radial node table (host)        */
    const double* e;            /* [ntheta][2] angular node directions (host)  */
    double xc, yc;              /* mesh centre                                  */
    int precision;              /* LBFSI_FP64 or LBFSI_FP32 populations         */
    int nbatch;                 /* independent solves sharing the mesh, >= 1    */
    const lbfsi_body_desc* bodies;  /* [nbatch]: the body of each solve (host)  */
} lbfsi_mesh_desc;

/* Body state: plunge h (up), pitch alpha (counter-clockwise) and rates. */
typedef struct {
    double h, alpha, hdot, adot;
} lbfsi_body_state;

/* Create a mesh handle: copies the tables, derives the wall geometry, and
 * allocates all device buffers (two population buffers, two moment fields,
 * force partials, body states).  cuda_stream: a cudaStream_t or NULL. */
int lbfsi_create_mesh(const lbfsi_mesh_desc* d, void* cuda_stream, lbfsi_mesh* out);

/* A structured O-grid given by its node coordinates (any body shape whose
 * mesh is a ring topology: ellipses, airfoils, ...).  Ring i = 0 is the wall
 * (the body polygon through the even-indexed wall nodes), ring nr - 1 the far
 * field; the angular index is periodic.  The nodes must be subparametric
 * (reading of Sec. II B with structured Q2 elements: each 3 x 3 window with
 * even first indices -- the last radial window starts at nr - 3 when nr is
 * even -- is the bilinear image of its four corner nodes), so the
 * first-order departure solve of Eq. depPnt is exact for the Q2 geometry;
 * the Jacobian of the index-to-space map must be positive at every node. */
typedef struct {
    int nr, ntheta;             /* nr >= 5, ntheta even >= 4 */
    const double* X;            /* [nr][ntheta][2] node coordinates (host, borrowed) */
    double xc, yc;              /* mesh centre (reference point of the geometry)   */
    int precision;              /* LBFSI_FP64 or LBFSI_FP32 populations             */
    int nbatch;                 /* independent solves sharing the mesh, >= 1        */
    const lbfsi_body_desc* bodies;  /* [nbatch]: the body of each solve (host)      */
} lbfsi_mesh_xy_desc;

/* Create a mesh handle on an O-grid given by node coordinates; otherwise as
 * lbfsi_create_mesh.  The departure points are found by Newton's method on
 * the bilinear element (Eq. depPnt) instead of the closed form of a
 * separable O-grid; one tile shape (lbfsi_set_schedule accepts variant 0).
 * LBFSI_EINVAL for a mesh that is not subparametric or not positively
 * oriented. */
int lbfsi_create_mesh_xy(const lbfsi_mesh_xy_desc* d, void* cuda_stream, lbfsi_mesh* out);

/* A C-grid around one body with a wake cut (the airfoil mesh type of
 * Sec. IV D; node coordinates, subparametric and positively oriented as in
 * lbfsi_mesh_xy_desc).  Row 0 runs counterclockwise: the upper side of the
 * cut from the outlet to the body (j < n_cut), the wall from its rear point
 * over the upper surface and the front back to the rear point
 * (n_cut <= j <= ntheta-1-n_cut), then the lower side of the cut out to the
 * outlet; row-0 nodes j and ntheta-1-j must be the same point for
 * j <= n_cut.  Rows grow away from row 0; row nr - 1 and the columns j = 0
 * and j = ntheta-1 are far field (inlet or outlet by the free stream's
 * direction).  Across the cut the mesh continues as its mirror (the node of
 * row -k, column j is the node of row k, column ntheta-1-j), so departure
 * points of cut nodes may lie on the other side.  Fields read and written
 * through the handle are [nr][ntheta] per component; the second copies of the
 * row-0 nodes along the cut hold the first copies' values. */
typedef struct {
    int nr, ntheta;             /* nr >= 5; ntheta odd >= 7 */
    int n_cut;                  /* row-0 nodes on each side of the cut (even, >= 2; the wall keeps >= 3 nodes) */
    const double* X;            /* [nr][ntheta][2] node coordinates (host, borrowed) */
    double xc, yc;              /* mesh centre (reference point of the geometry)   */
    int precision;              /* LBFSI_FP64 or LBFSI_FP32 populations             */
    int nbatch;                 /* independent solves sharing the mesh, >= 1        */
    const lbfsi_body_desc* bodies;  /* [nbatch]: the body of each solve (host)      */
} lbfsi_mesh_cgrid_desc;

/* A doubly periodic box (the Cartesian periodic mesh kind; the mesh of the
 * Taylor-Green and acoustic checks of Sec. II C): node coordinates of one
 * period, X [ni][nj][2] (subparametric, positively oriented), and the
 * period vectors: node (i + ni, j) is node (i, j) + shift_i, node (i, j + nj)
 * is node (i, j) + shift_j (a parallelogram box when shift_j has an x part).
 * Every node is interior: no wall, no far field, so the bodies must be fixed
 * (dof 0) and the loads are zero. */
typedef struct {
    int ni, nj;                 /* even, >= 4 */
    const double* X;            /* [ni][nj][2] node coordinates (host, borrowed) */
    double shift_i[2], shift_j[2];
    int precision;              /* LBFSI_FP64 or LBFSI_FP32 populations             */
    int nbatch;                 /* independent solves sharing the mesh, >= 1        */
    const lbfsi_body_desc* bodies;  /* [nbatch], dof 0 (host)                       */
} lbfsi_mesh_box_desc;

/* Create a mesh handle on a periodic box; otherwise as lbfsi_create_mesh_xy
 * (general-mesh kernel, one tile shape).  LBFSI_EINVAL for odd or too small
 * sizes, a mesh that is not subparametric or not positively oriented, or a
 * moving body. */
int lbfsi_create_mesh_box(const lbfsi_mesh_box_desc* d, void* cuda_stream, lbfsi_mesh* out);

/* A C-grid around several bodies (bodies in tandem: the cut runs along the
 * gaps and the wake), given by its node coordinates as in
 * lbfsi_mesh_cgrid_desc and its wall chains: walls[2 k], walls[2 k + 1] are
 * the first and last row-0 column of chain k (even, inside the outlet
 * columns, not overlapping), counterclockwise around its body; every other
 * row-0 column is on the cut.  The layout must be symmetric in
 * j -> ntheta-1-j, the cut nodes and the chains' ends (the junctions) one
 * point with their mirrors.  A body that row 0 wraps around is one chain
 * (the single C-grid: walls = {n_cut, ntheta-1-n_cut}); a body downstream of
 * another is an upper and a lower chain.
 * With nbody <= 1 every chain belongs to the solve's one body: its load is
 * the sum over all chains (rigidly linked bodies; the rigid zone must
 * contain every wall).  With nbody in 2..4 the bodies are independent
 * (Sec. II D, one blended map per body, the mesh displacements adding):
 * wall_body[k] names chain k's body (mirrored chains, e.g. the upper and
 * lower chain of a downstream body, name the same one; every body owns a
 * chain), each body has its own degrees of freedom, load (summed over its
 * chains, moment about its own reference point) and RK4 update, and bodies
 * and every per-solve body array are [nbatch][nbody]: lbfsi_blend_mesh,
 * lbfsi_body_forces, lbfsi_advance_bodies, lbfsi_get_body_state and
 * lbfsi_step_record take one entry per (solve, body).  Each wall must lie in
 * its body's rigid zone and outside every other body's blended region
 * (r_out), and the blended regions of moving bodies must not overlap. */
typedef struct {
    int nr, ntheta;             /* nr >= 5; ntheta odd >= 7 */
    int nwalls;                 /* wall chains, >= 1 */
    const int* walls;           /* [nwalls][2] inclusive column ranges (host, borrowed) */
    const double* X;            /* [nr][ntheta][2] node coordinates (host, borrowed) */
    double xc, yc;              /* mesh centre (reference point of the geometry)   */
    int precision;              /* LBFSI_FP64 or LBFSI_FP32 populations             */
    int nbatch;                 /* independent solves sharing the mesh, >= 1        */
    const lbfsi_body_desc* bodies;  /* [nbatch][max(nbody, 1)] (host)               */
    int nbody;                  /* independent bodies per solve (0 or 1: one)       */
    const int* wall_body;       /* [nwalls] body of each chain, or NULL (all body 0) */
} lbfsi_mesh_cgrid_walls_desc;

/* Create a mesh handle on a C-grid with several wall chains; otherwise as
 * lbfsi_create_mesh_cgrid.  LBFSI_EINVAL for chains with odd ends, outside
 * the outlets or overlapping, an asymmetric layout, cut or junction nodes
 * that do not coincide with their mirrors, or a bad mesh. */
int lbfsi_create_mesh_cgrid_walls(const lbfsi_mesh_cgrid_walls_desc* d, void* cuda_stream, lbfsi_mesh* out);

/* Create a mesh handle on a C-grid; otherwise as lbfsi_create_mesh_xy (one
 * tile shape).  A step is two launches here: the collision of step k of the
 * 16 rows next to the cut into a post-collision buffer, then one launch in
 * which the tiles next to the cut stream step k + 1 from it and the others
 * collide and stream.
 * LBFSI_EINVAL for an even ntheta, a bad n_cut, cut nodes that do not
 * coincide, or a mesh that is not subparametric or not positively oriented. */
int lbfsi_create_mesh_cgrid(const lbfsi_mesh_cgrid_desc* d, void* cuda_stream, lbfsi_mesh* out);

/* Release every device buffer of the handle (synchronises its stream). */
int lbfsi_destroy_mesh(lbfsi_mesh m);

/* Initial state (Sec. IV: uniform inflow plus seeded noise): populations set to
 * f^eq, g^eq (Eqs. feq, geq) of the given macroscopic fields; the moment field of
 * "the previous step" used by the boundary targets is that same field.  Body
 * states reset to rest.  rho_u_T: host [nbatch][4][N], or NULL for the uniform
 * free stream.  On a mesh given by node coordinates (xy, C-grid, box) this
 * also solves, once for the flow's dt, the departure points of the nodes that
 * no blended region moves (a device buffer of 80 B per node in FP32, 152 B in
 * FP64, allocated at creation unless the environment sets
 * LBFSI_NO_DEPARTURE_CACHE=1; the steps then read them back instead of
 * solving them, with the same results). */
int lbfsi_init_fields(lbfsi_mesh m, const lbfsi_flow_params* p, const double* rho_u_T);

/* Set the body states used by the next step's blended map (Sec. II D):
 * state [nbatch] is the current one, prev [nbatch] the one of the previous
 * step (V_G = (x(state) - x(prev)) / dt); prev may be NULL (= state). */
int lbfsi_blend_mesh(lbfsi_mesh m, const lbfsi_body_state* state, const lbfsi_body_state* prev);

/* Advance nsteps coupled time steps (Sec. III weak coupling): per step the
 * blended-mesh kinematics, departure points and Q2 interpolation of f and g
 * (Eqs. depPnt, SemiLagrProp), wall and far-field boundaries (Sec. III A), moments,
 * correction terms, collision (Eq. f_boltz), wall force and moment (Sec. III) and
 * the RK4 update of each body.  Asynchronous on the handle's stream. */
int lbfsi_step(lbfsi_mesh m, int nsteps);

/* Loads of the last completed step, host out [nbatch][3] = F_x, F_y, M_z
 * (force on the body, moment about its reference point; [nbatch][nbody][3]
 * for independent bodies).  Synchronises. */
int lbfsi_body_forces(lbfsi_mesh m, double* out);

/* RK4 of the body ODEs only (Sec. III B), with the given host loads
 * [nbatch][3] held constant over dt (NULL = the last step's loads).  Updates
 * the body states (the current state becomes the previous one); a forced
 * pitch is evaluated at the handle's step number x dt. */
int lbfsi_advance_bodies(lbfsi_mesh m, const double* loads, double dt);

/* Body states after the structural update of the last step, host out [nbatch]
 * ([nbatch][nbody] for independent bodies). */
int lbfsi_get_body_state(lbfsi_mesh m, lbfsi_body_state* out);

/* Macroscopic fields rho, u_x, u_y, T of the last step's post-propagation
 * state (far field: its targets), host out [nbatch][4][N] float64.  Synchronises. */
int lbfsi_get_fields(lbfsi_mesh m, double* rho_u_T);

/* Populations of the last step: which = 0 post-propagation (after the wall
 * reconstruction, before collision; far-field rows hold their equilibria),
 * which = 1 post-collision.  Host out [nbatch][9][N] each, float64. */
int lbfsi_get_populations(lbfsi_mesh m, int which, double* f, double* g);

/* Replace the post-propagation populations of the last step (host
 * [nbatch][9][N] float64) and their moment field; used to restart from a
 * checkpoint. */
int lbfsi_set_populations(lbfsi_mesh m, const double* f, const double* g,
                          const double* rho_u_T);

enum { LBFSI_FIELD_MOMENTS = 0, LBFSI_FIELD_POPULATIONS = 1 };

/* Zero-copy device view of the current state (for other GPU code, e.g. a
 * torch tensor over the same memory): which = LBFSI_FIELD_MOMENTS gives the
 * moment field rho, u_x, u_y, T of the last step, [nbatch][4][slots];
 * LBFSI_FIELD_POPULATIONS its post-propagation populations as (f, g) pairs,
 * [nbatch][9][slots][2].  Elements are double (LBFSI_FP64) or float
 * (LBFSI_FP32).  *slots (nullable) receives the slots per component: nr *
 * ntheta, plus 4 * ntheta mirrored rows before row 0 on a C-grid; *row0
 * (nullable) the slot where node (0, 0) starts (0, or 4 * ntheta).  The
 * memory belongs to the handle; the pointer is valid until the handle is
 * destroyed, but the state it holds is the current one only until the next
 * step (the step writes the other buffer of a ping-pong pair and that one
 * becomes current).  Reads must be ordered after the handle's stream
 * (lbfsi_synchronize, or work on the same stream); writes change the next
 * step's input.  LBFSI_EINVAL for a bad 'which' or null ptr,
 * LBFSI_ESTATE before lbfsi_init_fields. */
int lbfsi_field_ptr(lbfsi_mesh m, int which, void** ptr, int64_t* slots, int64_t* row0);

/* Wait for the handle's stream; returns the first device-detected error. */
int lbfsi_synchronize(lbfsi_mesh m);

/* Advance nsteps coupled steps (as lbfsi_step) and record every step's
 * loads and, if states_out is not NULL, body states on the host:
 * loads_out [nsteps][nbatch][3] (Fx, Fy, M as lbfsi_body_forces), states_out
 * [nsteps][nbatch] (as lbfsi_get_body_state).  Each step's record is copied
 * device -> host behind its launch (pinned staging owned by the handle), so
 * the steps are not stalled by the reads; the call synchronises once at the
 * end and returns the device status.  The load and displacement histories
 * (C_D(t), C_L(t), h(t), alpha(t)) of Sec. IV come from this call. */
int lbfsi_step_record(lbfsi_mesh m, int nsteps, double* loads_out, lbfsi_body_state* states_out);

/* ---- Checkpoint / resume (no counterpart in the paper).  A checkpoint is
 * the whole state the next step reads, as raw device bytes: the
 * post-propagation populations and their moment field, every solve's maps
 * record (body state of the last stream, next state, the previous state for
 * the mesh velocity of Sec. II D, last loads, blended maps) and the step
 * number, behind a header naming precision, batch and mesh size.  Restoring
 * it into a handle created with the same mesh and bodies and initialised
 * with the same flow continues the run bit for bit. */

/* Size in bytes of a checkpoint of this handle (0 for a null handle). */
size_t lbfsi_checkpoint_bytes(lbfsi_mesh m);

/* Write the checkpoint into the caller's host buffer of at least
 * lbfsi_checkpoint_bytes bytes.  Synchronises; refuses (with the device
 * status) to save a state the kernels flagged. */
int lbfsi_checkpoint(lbfsi_mesh m, void* host_buf, size_t bytes);

/* Replace the handle's state by a checkpoint (host buffer, borrowed).
 * LBFSI_EINVAL if the buffer is not a checkpoint of a handle with the same
 * precision, batch size and mesh dimensions; LBFSI_ESTATE before
 * lbfsi_init_fields.  Clears the device status word.  Synchronises. */
int lbfsi_restore(lbfsi_mesh m, const void* host_buf, size_t bytes);

/* Loads on the body of each solve from caller-provided post-propagation
 * populations, without allocating anything.  The paper has no counterpart:
 * this is the load reduction of lbfsi_step (wall stress, Simpson shares,
 * fixed-order sum) for callers that cannot call cudaMalloc -- e.g. code that
 * runs while a framework's caching allocator or a real-time loop owns all
 * device memory, or that must avoid the device-wide synchronisation an
 * allocation can cause.  Its scratch (per-CTA partial sums and per-solve
 * completion counters) is a fixed file-scope device array of about 97 KB that
 * every GPU which loads the library keeps until the process exits.
 *   nr, ntheta, xc, yc, r, e   the O-grid as for lbfsi_create_mesh; r [nr] and
 *                              e [ntheta][2] are DEVICE pointers (float64)
 *   precision                  LBFSI_FP64 or LBFSI_FP32: element type of f, g
 *   f, g                       DEVICE [nbatch][9][nr*ntheta] post-propagation
 *                              populations (only the wall row is read)
 *   body_ref                   DEVICE [nbatch][3]: x_p, y_p, alpha of each
 *                              body.  x_p, y_p is the body's reference point
 *                              (cylinder centre or elastic axis) in the
 *                              UNDEFORMED mesh frame -- the value given to
 *                              lbfsi_create_mesh, not its current, plunged
 *                              position; alpha is the pitch angle at which
 *                              the populations were streamed.  Moment arms
 *                              are R(alpha)(X_wall - X_p) with X_wall the
 *                              undeformed wall nodes, so a translated x_p, y_p
 *                              gives a wrong moment without an error.
 *   mu, dt, gamma              viscosity, time step, adiabatic exponent
 *   loads                      DEVICE out [nbatch][3]: F_x, F_y, M_z
 * Limits: nbatch <= 256 and nbatch * ceil(ntheta / 32) <= 4096, else
 * LBFSI_EINVAL.  Asynchronous on cuda_stream: each call clears the completion
 * counters it uses with an asynchronous memset on that stream, then launches
 * one kernel.  The first call on a device (with that device current) looks up
 * the scratch array's device address (cudaGetSymbolAddress, which may load the
 * module and block), so make that first call before any stream capture.
 * Every call shares the one scratch array, which keeps the last call's
 * partial sums: calls that overlap on the GPU (other streams, other threads)
 * race and must be serialised by the caller. */
int lbfsi_wall_loads_noalloc(int nr, int ntheta, int nbatch, int precision, const double* r,
                             const double* e, double xc, double yc, const void* f, const void* g,
                             const double* body_ref, double mu, double dt, double gamma,
                             double* loads, void* cuda_stream);

/* ---- Batch runtime: many solves on meshes of different sizes, admitted and
 * retired while others run, advanced together (one launch per step for all
 * active solves).  Device memory comes from one pool allocated at creation;
 * a solve is admitted only if the pool can hold it (continuous batching with
 * memory-based admission).  Solves on identical O-grids share one device copy
 * of the mesh geometry.  The per-step physics is exactly that of lbfsi_step
 * (same kernel), so a solve's result does not depend on what it is batched
 * with. */
typedef struct lbfsi_batch_s* lbfsi_batch;

/* One solve for the batch runtime: its O-grid (as in lbfsi_mesh_desc, host
 * tables borrowed for the call), its body, flow, initial macroscopic field
 * (host [4][nr*ntheta] or NULL for the uniform free stream) and the number of
 * steps after which it is finished (> 0). */
typedef struct {
    int nr, ntheta;
    const double* r;
    const double* e;
    double xc, yc;
    lbfsi_body_desc body;
    lbfsi_flow_params flow;
    const double* rho_u_T;
    int steps;
} lbfsi_solve_desc;

/* Create a batch runtime whose solves live in a device pool of pool_bytes
 * (one cudaMalloc now; none later except when the tile table outgrows its
 * buffer).  precision: LBFSI_FP64 or LBFSI_FP32 for every solve of the batch. */
int lbfsi_batch_create(size_t pool_bytes, int precision, void* cuda_stream, lbfsi_batch* out);
int lbfsi_batch_destroy(lbfsi_batch b);

/* Admit a solve; on success *slot is its id (>= 0).  LBFSI_ENOMEM means the
 * pool has no room for it now (nothing changed; retry after removing finished
 * solves).  The solve's first step happens in the next lbfsi_batch_step. */
int lbfsi_batch_add(lbfsi_batch b, const lbfsi_solve_desc* d, int* slot);

/* One solve on an O-grid given by its node coordinates (as in
 * lbfsi_mesh_xy_desc: X [nr][ntheta][2] host, borrowed for the call), with
 * its body, flow, initial field and step count as in lbfsi_solve_desc. */
typedef struct {
    int nr, ntheta;
    const double* X;
    double xc, yc;
    lbfsi_body_desc body;
    lbfsi_flow_params flow;
    const double* rho_u_T;
    int steps;
} lbfsi_solve_xy_desc;

/* Admit a solve on a general O-grid (same contract as lbfsi_batch_add).
 * Identical coordinate sets share one device copy.  These solves run on the
 * general-geometry kernel with its one tile shape, in a second launch of
 * every lbfsi_batch_step; lbfsi_batch_set_schedule and the autotuner change
 * the tiles of the separable-mesh solves only. */
int lbfsi_batch_add_xy(lbfsi_batch b, const lbfsi_solve_xy_desc* d, int* slot);

/* One solve on a C-grid (as in lbfsi_mesh_cgrid_desc: X [nr][ntheta][2]
 * host, borrowed for the call, n_cut cut nodes per side), with its body,
 * flow, initial field and step count as in lbfsi_solve_desc. */
typedef struct {
    int nr, ntheta, n_cut;
    const double* X;
    double xc, yc;
    lbfsi_body_desc body;
    lbfsi_flow_params flow;
    const double* rho_u_T;
    int steps;
} lbfsi_solve_cgrid_desc;

/* Admit a solve on a C-grid (same contract as lbfsi_batch_add).  Its tiles
 * form a third part of every lbfsi_batch_step: the collision of the rows next
 * to the cut, then the launch that streams the tiles next to the cut from its
 * output and collides and streams the others. */
int lbfsi_batch_add_cgrid(lbfsi_batch b, const lbfsi_solve_cgrid_desc* d, int* slot);

/* Advance every active solve by up to nsteps coupled steps (one launch per
 * step covering all active solves; a solve stops when it reaches its step
 * count).  *active_after (nullable) receives the number of unfinished solves.
 * Asynchronous except when the set of active solves changes. */
int lbfsi_batch_step(lbfsi_batch b, int nsteps, int* active_after);

/* Steps done and finished flag of a slot (host-side bookkeeping, no sync). */
int lbfsi_batch_poll(lbfsi_batch b, int slot, int* steps_done, int* finished);

/* Results of a slot after its last step: macroscopic fields (host
 * [4][nr*ntheta], nullable), loads of the last step (host [3], nullable) and
 * body state after the structural update (nullable).  Synchronises; returns
 * the batch's device error status as lbfsi_synchronize does. */
int lbfsi_batch_get(lbfsi_batch b, int slot, double* rho_u_T, double* loads, lbfsi_body_state* state);

/* Retire a slot: its device memory returns to the pool (synchronises). */
int lbfsi_batch_remove(lbfsi_batch b, int slot);

/* Free bytes of the pool and its largest free block. */
int lbfsi_batch_memory(lbfsi_batch b, size_t* free_bytes, size_t* largest_free);

/* Tile shape and tile-table order of a batch's step launches (the CTA
 * schedule).  order 0: the tiles of each solve together, in slot order;
 * order 1: tile rows outermost across all solves, so the wall and
 * blending-region tiles (the most expensive) start first.  Synchronises. */
int lbfsi_batch_set_schedule(lbfsi_batch b, int variant, int order);
int lbfsi_batch_get_schedule(lbfsi_batch b, int* variant, int* order);

/* graph_steps > 0: lbfsi_batch_step replays a CUDA graph of graph_steps
 * launches over the current tile table for as long as no solve finishes
 * (the graph is dropped whenever the table changes); 0: plain launches. */
int lbfsi_batch_set_graph_steps(lbfsi_batch b, int graph_steps);

/* Autotuner of the batch: like lbfsi_autotune over the active solves (the
 * trial steps count toward their requested steps); the trials are compared
 * by time per node update, since solves may finish during tuning.
 * ns_per_node: nullable host array [lbfsi_step_variants][2]. */
int lbfsi_batch_autotune(lbfsi_batch b, int steps_per_trial, int* best_variant, int* best_order,
                         float* ns_per_node);

/* Number of kernel launches issued on the handle's stream so far. */
int64_t lbfsi_launch_count(lbfsi_mesh m);

/* ---- Execution schedule, CUDA graphs and the autotuner.  The paper has no
 * counterpart: these choose how the step of Sec. II-III is laid out on the
 * GPU, not what it computes.  Every tile shape and CTA order computes
 * bit-identical fields, loads and body states (each node is computed by the
 * same code from the same inputs; load partials have fixed slots and a fixed
 * summation order), so tuning never changes a solve's result. */

/* Number of tile shapes ("step variants") of the step kernel for a
 * precision (LBFSI_FP32: 5, LBFSI_FP64: 3), or LBFSI_EINVAL.  Float shapes,
 * radial x angular nodes per CTA: 0: 8 x 32, 256 threads, 2 CTAs/SM;
 * 1: 16 x 32, 256 threads; 2: 8 x 32, 3 CTAs/SM; 3: 12 x 32, 384 threads;
 * 4: 16 x 32, 512 threads (default of new mesh handles, with order 1, and of
 * new batches, with order 0).  Float64 shapes (separable O-grids; 256
 * threads, one CTA per SM): 0: 8 x 32 (default), 1: 4 x 32, 2: 2 x 32 -- the
 * smaller tiles spread a small mesh over more SMs, whose float64 rate bounds
 * the step.  Meshes given by node coordinates have one shape (0).
 * Staging (every shape): in a float mesh handle whose Ntheta is a multiple
 * of 4, and for the float solves of a batch on separable O-grids whose Ntheta
 * is a multiple of 4, the moments and populations of each tile whose angular
 * range does not wrap are moved into shared memory by two tensor copies
 * (TMA), the other tiles by per-thread copies; LBFSI_TMA=0 in the environment
 * when a handle first steps (when a batch rebuilds its tile table) stages
 * every tile by per-thread copies.  Both give the same bits. */
int lbfsi_step_variants(int precision);

/* Tile shape (0 .. lbfsi_step_variants - 1) and CTA order of a mesh handle's
 * step launches.  order 0: the tiles of one solve are consecutive CTAs;
 * order 1: the solves of one tile are consecutive CTAs.  EINVAL when out of
 * range.  Synchronises the handle's stream when it changes the schedule. */
int lbfsi_set_schedule(lbfsi_mesh m, int variant, int order);
int lbfsi_get_schedule(lbfsi_mesh m, int* variant, int* order);

/* graph_steps > 0: lbfsi_step replays a CUDA graph of graph_steps step
 * launches (captured at first use on a private stream, recaptured after a
 * schedule change; its launches read the step number from the device),
 * plain launches for the remainder; 0 (default): plain launches only. */
int lbfsi_set_graph_steps(lbfsi_mesh m, int graph_steps);

/* Autotuner: advances the handle's solves by 1 + steps_per_trial steps under
 * every (variant, order) pair, times each trial with CUDA events on the
 * handle's stream, and keeps the fastest pair.  The trial steps are real
 * steps of the solves.  best_variant, best_order: outputs (nullable);
 * ms_per_step: nullable host array [lbfsi_step_variants][2] receiving the
 * measured ms per step.  Synchronises; returns the device status. */
int lbfsi_autotune(lbfsi_mesh m, int steps_per_trial, int* best_variant, int* best_order,
                   float* ms_per_step);

/* ---- Unstructured Q2 meshes (the paper's mesh type, Sec. II B: second-
 * order quadrilateral finite elements over a node list; Sec. IV meshes its
 * cases this way).  A separate handle: the step on an element list runs as
 * four launches per step over node lists (correction field D, collision into
 * a post-collision buffer, stream, load reduction and body update) with the
 * Q2 gathers read from global memory, instead of the structured meshes'
 * one-launch tiled kernel.
 *
 * Mesh: N nodes, elements of 3 x 3 node indices [a][b] (entry (a, b) at
 * reference coordinates (a - 1, b - 1)), subparametric (each element's mid
 * nodes at the bilinear positions of its corners, reading R7).  Boundaries
 * (reading R34): a closed wall chain of node indices counterclockwise around
 * the body and a closed far-field chain counterclockwise around the domain,
 * each of even length with the even entries the vertices of straight element
 * edges; the wall normal and the far field's outward direction are the
 * normals of those polygons, and wall loads are Simpson sums over the wall
 * chain's edges.  A node's departure point (Eq. depPnt) and its boundary
 * target point B are searched in the elements that hold the node, in
 * increasing element index (readings R8, R9).  Nodal gradients (Eq. ddx+fem)
 * are the mean over a node's elements of the element derivative at the node
 * (reading R33), or, when grid_ij is given, the structured stencil of reading
 * R18 on that index grid (a structured mesh renumbered into elements then
 * steps exactly as the structured mesh). */
typedef struct lbfsi_emesh_s* lbfsi_emesh;

typedef struct {
    int nnode;                  /* N                                                   */
    const double* X;            /* [N][2] node coordinates (undeformed), host          */
    int nelem;
    const int* elements;        /* [nelem][3][3] node indices, host                    */
    int nwall;                  /* wall chain length (even, >= 4)                      */
    const int* wall;            /* [nwall] node indices, counterclockwise around body  */
    int nfar;                   /* far-field chain length (even, >= 4)                 */
    const int* far;             /* [nfar] node indices, counterclockwise around domain */
    const int* grid_ij;         /* nullable [N][2]: (i, j) of each node on a grid of
                                   grid_nr x grid_nt, periodic in j, row 0 the wall
                                   and row grid_nr - 1 the far field (reading R18)     */
    int grid_nr, grid_nt;
    int nbatch;                 /* independent solves on this mesh                     */
    const lbfsi_body_desc* bodies;   /* [nbatch], host                                 */
    int precision;              /* LBFSI_FP64 or LBFSI_FP32 populations                */
} lbfsi_mesh_elements_desc;

/* Validate the element list (indices in range, every node in an element,
 * subparametric elements with positive Jacobians, chains of distinct nodes
 * that no element repeats, bodies' walls inside their rigid zones), build the
 * node-to-element table and the gradient operator on the host, upload.
 * Inside the handle the nodes are numbered along a Z-order curve of their
 * coordinates (and the elements in the order of their centre nodes) for
 * memory locality; every call that takes or returns node fields uses the
 * caller's node order, and each node's elements are searched in the
 * caller's element order.  LBFSI_EINVAL on a bad mesh; host arrays are
 * borrowed for the call. */
int lbfsi_create_mesh_elements(const lbfsi_mesh_elements_desc* d, void* cuda_stream, lbfsi_emesh* out);
int lbfsi_emesh_destroy(lbfsi_emesh m);

/* As lbfsi_init_fields: rho_u_T host [nbatch][4][N] (node order of the
 * element list) or NULL for the free stream; populations at equilibrium,
 * bodies at rest.  Also solves, once for the flow's dt, the departure points
 * of the interior nodes that no blended region moves (a device buffer of
 * 108 B per node in FP32, 180 B in FP64, allocated at creation unless the
 * environment sets LBFSI_NO_DEPARTURE_CACHE=1; the steps then read them back
 * instead of solving them, with the same results). */
int lbfsi_emesh_init_fields(lbfsi_emesh m, const lbfsi_flow_params* p, const double* rho_u_T);

/* As lbfsi_blend_mesh: body states [nbatch] of the next step's blended map,
 * prev [nbatch] (nullable: = state) the previous ones (V_G). */
int lbfsi_emesh_blend_mesh(lbfsi_emesh m, const lbfsi_body_state* state, const lbfsi_body_state* prev);

/* As lbfsi_step (Sec. III weak coupling), asynchronous on the handle's
 * stream; errors (departure point outside the node's elements, B point
 * outside, non-physical state) surface at the next synchronising call. */
int lbfsi_emesh_step(lbfsi_emesh m, int nsteps);

/* Synchronise and return the device status (LBFSI_EDEPARTURE,
 * LBFSI_ENONPHYS or LBFSI_OK). */
int lbfsi_emesh_synchronize(lbfsi_emesh m);

/* Loads of the last step, host out [nbatch][3] (F_x, F_y, M_z); body states
 * host out [nbatch]; moment field host out [nbatch][4][N] (rho, u_x, u_y,
 * T); populations host out f, g [nbatch][9][N]: which 0 the post-propagation
 * (pre-collision) state of the current step, 1 its post-collision state
 * (collided by this call; step 0: the initial state).  Each synchronises and
 * returns the device status. */
int lbfsi_emesh_body_forces(lbfsi_emesh m, double* out);
int lbfsi_emesh_get_body_state(lbfsi_emesh m, lbfsi_body_state* out);
int lbfsi_emesh_get_fields(lbfsi_emesh m, double* rho_u_T);
int lbfsi_emesh_get_populations(lbfsi_emesh m, int which, double* f, double* g);

/* Kernel launches issued by the handle so far. */
int64_t lbfsi_emesh_launch_count(lbfsi_emesh m);

/* Thread-local message of the last failing call ("" if none). */
const char* lbfsi_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBFSI_H */
