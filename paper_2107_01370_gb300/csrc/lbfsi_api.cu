// C-ABI of the library (declared in include/lbfsi.h): the mesh handle (one
// O-grid, nbatch independent solves advanced together), its device memory and
// the launch sequence of the coupled step.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lbfsi.h"
#include "lbfsi_host.h"
#include "lbfsi_internal.h"

using lbfsi::BodyDev;
using lbfsi::BodyStateDev;
using lbfsi::SolveDev;
using lbfsi::StepMaps;
using lbfsi::TileDev;

namespace lbfsi {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return static_cast<EncodeTiledFn>(nullptr);
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// A float array of dims (dx, dy, dz, dw), x fastest and dense, read in boxes
// of (bx, by, bz, 1); elements outside the array arrive as zeros.
bool encode_box4(CUtensorMap* map, void* base, size_t dx, size_t dy, size_t dz, size_t dw, unsigned bx,
                 unsigned by, unsigned bz) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[4] = {dx, dy, dz, dw};
    const cuuint64_t strides[3] = {dx * 4, dx * dy * 4, dx * dy * dz * 4};   // bytes, dims 1..3
    const cuuint32_t box[4] = {bx, by, bz, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace lbfsi

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(LBFSI_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

int lbfsi::set_error(int code, const std::string& msg) { return fail(code, msg); }

struct lbfsi_mesh_s {
    lbfsi::HostMesh host;
    lbfsi::DeviceMesh dmesh;
    lbfsi::CudaMallocMemory mem;
    int nbatch = 0, precision = 0, variant = 4, order = 1, tile_rows = 16, tiles_per_solve = 0;
    int nbody = 1;                       // bodies per solve (independent bodies of a C-grid)
    size_t slots() const { return (size_t)nbatch * (size_t)nbody; }   // body records
    size_t esize = 8;
    cudaStream_t stream = nullptr;
    std::vector<lbfsi_body_desc> bodies;
    void* d_p[2] = {nullptr, nullptr};   // populations, (f_q, g_q) pairs [nbatch][9][N]
    void* d_M[2] = {nullptr, nullptr};
    void* d_ppost = nullptr;             // collide-only output, same layout
    void* d_dep = nullptr;               // general meshes: cached static departures ((xi, eta)
                                         // [9][Nx], then codes [Nx]; see SolveDev::dep_xe)
    double* d_stage = nullptr;  // [nbatch][4][N] float64 staging
    StepMaps* d_maps[2] = {nullptr, nullptr};  // [nbatch][nbody] each
    BodyStateDev* d_state_a = nullptr;          // host-given states staging
    BodyStateDev* d_state_b = nullptr;
    double* d_loads_tmp = nullptr;
    double* d_part = nullptr;        // [nbatch][nbody][ntj][3] load partials
    unsigned* d_counter = nullptr;   // [nbatch][2] CTA completion count, step number
    BodyDev* d_bodies = nullptr;     // [nbatch][nbody]
    lbfsi::MeshDev* d_meshdev = nullptr;
    SolveDev* d_solves = nullptr;    // [nbatch]
    unsigned* d_status = nullptr;
    std::vector<SolveDev> solves;
    unsigned host_k = 0;             // step number of every solve (mirror of counter[1])
    bool initialized = false;
    double dt = 0;
    int64_t launches = 0;
    // CUDA graph of graph_steps step launches (step number from the device
    // counters), captured on a private stream and replayed on 'stream'
    int graph_steps = 0;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t cap_stream = nullptr;
    // pinned staging of lbfsi_step_record
    void* h_rec = nullptr;
    size_t h_rec_bytes = 0;
    double* d_rec = nullptr;         // device history of lbfsi_step_record: [steps][records][7]
    size_t d_rec_count = 0;
    // tensor maps of the float step (StepArgs::tm_p, tm_M) for tiles of
    // tma_rows rows: -1 not built yet, 0 not used (float64, periodic boxes,
    // Ntheta not a multiple of 4, LBFSI_TMA=0, or no encoder)
    int tma_rows = -1;
    CUtensorMap tm_p[2], tm_M[2];

    int cur() const { return (int)(host_k & 1u); }
    bool first() const { return host_k == 0u; }
};

namespace {

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

int check_status(lbfsi_mesh m) {
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    unsigned st = 0;
    e = cudaMemcpy(&st, m->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (st & lbfsi::ST_BOUNDS)
        return lbfsi::set_error(LBFSI_EBOUNDS, "an index of the step outside its buffer (bounds-checked build)");
    if (st & lbfsi::ST_TMA)
        return lbfsi::set_error(LBFSI_ECUDA, "a tensor copy of the step did not complete within its wait limit");
    if (st & lbfsi::ST_DEPARTURE)
        return fail(LBFSI_EDEPARTURE, "departure point outside the cells adjacent to its node (CFL)");
    if (st & lbfsi::ST_BPOINT)
        return fail(LBFSI_EDEPARTURE, "wall or outlet target point B outside the cells next to its node");
    if (st & lbfsi::ST_NONPHYS) return fail(LBFSI_ENONPHYS, "non-physical state (rho<=0, T<=0 or NaN)");
    return LBFSI_OK;
}

void to_double(const void* src, double* dst, size_t n, int precision) {
    if (precision == LBFSI_FP64) {
        std::memcpy(dst, src, n * sizeof(double));
    } else {
        const float* s = static_cast<const float*>(src);
        for (size_t k = 0; k < n; ++k) dst[k] = (double)s[k];
    }
}

int download(lbfsi_mesh m, const void* dsrc, double* host, size_t n) {
    std::vector<unsigned char> tmp(n * m->esize);
    cudaError_t e = cudaMemcpyAsync(tmp.data(), dsrc, n * m->esize, cudaMemcpyDeviceToHost, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "download");
    e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "download sync");
    to_double(tmp.data(), host, n, m->precision);
    return LBFSI_OK;
}

int upload(lbfsi_mesh m, const double* host, void* ddst, size_t n) {
    std::vector<unsigned char> tmp(n * m->esize);
    if (m->precision == LBFSI_FP64) {
        std::memcpy(tmp.data(), host, n * sizeof(double));
    } else {
        float* t = reinterpret_cast<float*>(tmp.data());
        for (size_t k = 0; k < n; ++k) t[k] = (float)host[k];
    }
    cudaError_t e = cudaMemcpyAsync(ddst, tmp.data(), n * m->esize, cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload");
    e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload sync");
    return LBFSI_OK;
}

// Field blocks of w values per node: the caller's [blocks][N] layout to the
// device's [blocks][Nx] (a C-grid's mirrored rows below row 0 filled from
// their nodes, node (-k, j) = node (k, nt-1-j)), and back.
std::vector<double> expand_rows(const lbfsi::HostMesh& h, const double* user, size_t blocks, int w) {
    const size_t N = (size_t)h.N, Nx = (size_t)h.Nx, nt = (size_t)h.nt, g0 = (size_t)h.G * nt;
    std::vector<double> dev(blocks * Nx * w);
    for (size_t b = 0; b < blocks; ++b) {
        const double* u = user + b * N * w;
        double* d = dev.data() + b * Nx * w;
        std::memcpy(d + g0 * w, u, N * w * sizeof(double));
        for (int k = 1; k <= h.G; ++k)
            for (size_t j = 0; j < nt; ++j)
                for (int c = 0; c < w; ++c)
                    d[(g0 - k * nt + j) * w + c] = u[(k * nt + (nt - 1 - j)) * w + c];
    }
    return dev;
}

void compact_rows(const lbfsi::HostMesh& h, const double* dev, double* user, size_t blocks, int w) {
    const size_t N = (size_t)h.N, Nx = (size_t)h.Nx, g0 = (size_t)h.G * h.nt;
    for (size_t b = 0; b < blocks; ++b)
        std::memcpy(user + b * N * w, dev + (b * Nx + g0) * w, N * w * sizeof(double));
}

// A C-grid's second copies of the row-0 cut nodes (and of the rear point)
// take the first copies' values in caller-given fields of w values per node.
void unify_cut_copies(const lbfsi::HostMesh& h, double* user, size_t blocks, int w) {
    if (!h.cgrid) return;
    for (size_t b = 0; b < blocks; ++b)
        for (int j = 0; j < h.nt; ++j)
            if (h.coltype[j] & lbfsi::CT_DUP)
                for (int c = 0; c < w; ++c)
                    user[(b * h.N + (size_t)j) * w + c] = user[(b * h.N + (size_t)(h.nt - 1 - j)) * w + c];
}

// One coupled step of every solve: one launch (collide of step k, stream of
// k + 1), or on a C-grid two: the collision of the rows next to the cut into
// ppost, because the mirrored rows of one side need the other side's
// post-collision populations, then the launch in which the first row of tiles
// streams from ppost and every other tile collides and streams.
int launches_per_step(lbfsi_mesh m) { return m->host.cgrid ? 2 : 1; }

cudaError_t launch_one_step(lbfsi_mesh m, lbfsi::StepArgs a, cudaStream_t s) {
    if (!m->host.cgrid) return lbfsi::launch_step_uniform(a, m->precision, m->variant, m->nbatch, s);
    lbfsi::StepArgs c = a;
    c.collide_only = 1;
    c.cgrid_pre = 1;
    cudaError_t e = lbfsi::launch_step_uniform(c, m->precision, m->variant, m->nbatch, s);
    if (e != cudaSuccess) return e;
    a.stream_post = 1;
    return lbfsi::launch_step_uniform(a, m->precision, m->variant, m->nbatch, s);
}

void free_all(lbfsi_mesh m) {
    void* ptrs[] = {m->d_p[0], m->d_p[1], m->d_M[0], m->d_M[1], m->d_ppost, m->d_dep, m->d_stage, m->d_maps[0], m->d_maps[1], m->d_state_a, m->d_state_b,
                    m->d_loads_tmp, m->d_part, m->d_counter, m->d_bodies, m->d_meshdev, m->d_solves,
                    m->d_status};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (m->graph) cudaGraphExecDestroy(m->graph);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    if (m->h_rec) cudaFreeHost(m->h_rec);
    if (m->d_rec) cudaFree(m->d_rec);
    lbfsi::release_mesh(m->dmesh, m->mem);
}

// Per-solve descriptors of the handle: solve b's buffers are slices of the
// batch-contiguous arrays.
int upload_solves(lbfsi_mesh m) {
    // field pointers at row 0 of solve b (a C-grid's mirrored rows before it)
    const size_t N = (size_t)m->host.Nx, es = m->esize, g0 = (size_t)m->host.G * m->host.nt;
    for (int b = 0; b < m->nbatch; ++b) {
        SolveDev& s = m->solves[b];
        s.mesh = 0;
        s.ntiles = m->tiles_per_solve;
        s.nbody = m->nbody;
        const size_t bb = (size_t)b * m->nbody;
        for (int p = 0; p < 2; ++p) {
            s.p[p] = (char*)m->d_p[p] + ((size_t)b * 18 * N + 2 * g0) * es;
            s.M[p] = (char*)m->d_M[p] + ((size_t)b * 4 * N + g0) * es;
            s.maps[p] = m->d_maps[p] + bb;
        }
        s.ppost = m->d_ppost ? (char*)m->d_ppost + ((size_t)b * 18 * N + 2 * g0) * es : nullptr;
        s.part = m->d_part + bb * m->host.ntj * 3;
        s.counter = m->d_counter + 2 * b;
        s.body = m->d_bodies + bb;
        s.dep_xe = m->d_dep ? (char*)m->d_dep + g0 * 2 * es : nullptr;
        s.dep_code = m->d_dep ? reinterpret_cast<unsigned long long*>((char*)m->d_dep + 9 * N * 2 * es) + g0
                              : nullptr;
    }
    cudaError_t e = cudaMemcpyAsync(m->d_solves, m->solves.data(), m->solves.size() * sizeof(SolveDev),
                                    cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "solve descriptors upload");
    return LBFSI_OK;
}

// Tensor maps of the handle's two population and moment buffers for its
// current tile shape (built again after a schedule change); false where the
// step stages by per-thread copies.  Populations: (f, g) float pairs as
// (2 Ntheta, rows stored, 9, nbatch) floats, box (2 (32 + 8), rows + 4, 9, 1);
// moments: (Ntheta, rows stored, 4, nbatch), box (32 + 8, rows + 8, 4, 1) --
// the staged tiles of the step kernel (+-2 and +-4 nodes around the tile).
// The rows stored are nr, and on a C-grid its G mirrored rows below row 0.
bool tma_maps(lbfsi_mesh m) {
    if (m->tma_rows == m->tile_rows) return true;
    if (m->tma_rows == 0) return false;
    const char* env = std::getenv("LBFSI_TMA");
    const bool eligible = m->precision == LBFSI_FP32 && !m->host.box && m->host.nt % 4 == 0 &&
                          !(env && std::atoi(env) == 0);
    bool ok = eligible;
    const size_t nt = (size_t)m->host.nt, nr = (size_t)(m->host.nr + m->host.G), nb = (size_t)m->nbatch;
    const unsigned rows = (unsigned)m->tile_rows, w = (unsigned)(lbfsi::TILE_J + 8);
    for (int c = 0; c < 2 && ok; ++c) {
        ok = lbfsi::encode_box4(&m->tm_p[c], m->d_p[c], 2 * nt, nr, 9, nb, 2 * w, rows + 4, 9) &&
             lbfsi::encode_box4(&m->tm_M[c], m->d_M[c], nt, nr, 4, nb, w, rows + 8, 4);
    }
    m->tma_rows = ok ? m->tile_rows : 0;
    return ok;
}

lbfsi::StepArgs make_args(lbfsi_mesh m, int collide_only) {
    lbfsi::StepArgs a{};
    if (tma_maps(m)) {
        a.tma = 1;
        a.tma_g = m->host.G;
        for (int c = 0; c < 2; ++c) {
            a.tm_p[c] = m->tm_p[c];
            a.tm_M[c] = m->tm_M[c];
        }
    }
    a.umesh = m->dmesh.dev;
    a.usol = m->solves[0];
    a.meshes = m->d_meshdev;
    a.solves = m->d_solves;
    a.tiles = nullptr;
    a.ntiles = m->nbatch * m->tiles_per_solve;
    a.collide_only = collide_only;
    a.ustep = (int)m->host_k;
    a.uorder = m->order;
    a.status = m->d_status;
    return a;
}

// Capture graph_steps step launches that take the step number from the
// device counters (so the same graph serves every replay).
int capture_graph(lbfsi_mesh m) {
    lbfsi::TraceRange trace_("lbfsi graph capture");
    cudaError_t e = lbfsi::prepare_step(m->precision, m->variant, true, m->host.general);
    if (e == cudaSuccess && !m->cap_stream) e = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture setup");
    lbfsi::StepArgs a = make_args(m, 0);
    a.ustep = -1;
    e = cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    cudaError_t le = cudaSuccess;
    for (int g = 0; g < m->graph_steps && le == cudaSuccess; ++g) le = launch_one_step(m, a, m->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(m->cap_stream, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(le != cudaSuccess ? le : e, "step capture");
    }
    e = cudaGraphInstantiate(&m->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        m->graph = nullptr;
        return cuda_fail(e, "graph instantiate");
    }
    return LBFSI_OK;
}

void drop_graph(lbfsi_mesh m) {
    if (m->graph) {
        cudaStreamSynchronize(m->stream);
        cudaGraphExecDestroy(m->graph);
        m->graph = nullptr;
    }
}

}  // namespace

extern "C" {

const char* lbfsi_last_error(void) { return g_last_error.c_str(); }

namespace {

int check_common(int nr, int nt, int precision, int nbatch, const lbfsi_body_desc* bodies, lbfsi_mesh* out) {
    if (!out) return fail(LBFSI_EINVAL, "null argument");
    *out = nullptr;
    if (precision != LBFSI_FP64 && precision != LBFSI_FP32)
        return fail(LBFSI_EINVAL, "precision must be LBFSI_FP64 or LBFSI_FP32");
    if (nbatch < 1) return fail(LBFSI_EINVAL, "nbatch must be >= 1");
    if (!bodies) return fail(LBFSI_EINVAL, "null body pointer");
    const long long Nll = (long long)nr * nt;
    if (nr > 0 && nt > 0 && Nll * 9 * nbatch > (1ll << 31))
        return fail(LBFSI_EINVAL, "mesh too large for 32-bit node indexing");
    return LBFSI_OK;
}

int create_common(lbfsi_mesh m, int precision, int nbatch, const lbfsi_body_desc* bodies, void* cuda_stream,
                  lbfsi_mesh* out);

}  // namespace

int lbfsi_create_mesh(const lbfsi_mesh_desc* d, void* cuda_stream, lbfsi_mesh* out) {
    g_last_error.clear();
    if (!d) return fail(LBFSI_EINVAL, "null argument");
    int rc = check_common(d->nr, d->ntheta, d->precision, d->nbatch, d->bodies, out);
    if (rc) return rc;
    auto m = new lbfsi_mesh_s();
    rc = lbfsi::build_host_mesh(d->nr, d->ntheta, d->r, d->e, d->xc, d->yc, m->host);
    if (rc) {
        delete m;
        return rc;
    }
    return create_common(m, d->precision, d->nbatch, d->bodies, cuda_stream, out);
}

int lbfsi_create_mesh_xy(const lbfsi_mesh_xy_desc* d, void* cuda_stream, lbfsi_mesh* out) {
    g_last_error.clear();
    if (!d) return fail(LBFSI_EINVAL, "null argument");
    int rc = check_common(d->nr, d->ntheta, d->precision, d->nbatch, d->bodies, out);
    if (rc) return rc;
    auto m = new lbfsi_mesh_s();
    rc = lbfsi::build_host_mesh_xy(d->nr, d->ntheta, d->X, d->xc, d->yc, m->host);
    if (rc) {
        delete m;
        return rc;
    }
    return create_common(m, d->precision, d->nbatch, d->bodies, cuda_stream, out);
}

int lbfsi_create_mesh_box(const lbfsi_mesh_box_desc* d, void* cuda_stream, lbfsi_mesh* out) {
    g_last_error.clear();
    if (!d) return fail(LBFSI_EINVAL, "null argument");
    int rc = check_common(d->ni, d->nj, d->precision, d->nbatch, d->bodies, out);
    if (rc) return rc;
    auto m = new lbfsi_mesh_s();
    rc = lbfsi::build_host_mesh_box(d->ni, d->nj, d->X, d->shift_i, d->shift_j, m->host);
    if (rc) {
        delete m;
        return rc;
    }
    return create_common(m, d->precision, d->nbatch, d->bodies, cuda_stream, out);
}

int lbfsi_create_mesh_cgrid(const lbfsi_mesh_cgrid_desc* d, void* cuda_stream, lbfsi_mesh* out) {
    g_last_error.clear();
    if (!d) return fail(LBFSI_EINVAL, "null argument");
    int rc = check_common(d->nr + lbfsi::CGRID_GHOST_ROWS, d->ntheta, d->precision, d->nbatch, d->bodies, out);
    if (rc) return rc;
    auto m = new lbfsi_mesh_s();
    const int walls[2] = {d->n_cut, d->ntheta - 1 - d->n_cut};
    rc = lbfsi::build_host_mesh_c(d->nr, d->ntheta, 1, walls, d->X, d->xc, d->yc, m->host);
    if (rc) {
        delete m;
        return rc;
    }
    return create_common(m, d->precision, d->nbatch, d->bodies, cuda_stream, out);
}

int lbfsi_create_mesh_cgrid_walls(const lbfsi_mesh_cgrid_walls_desc* d, void* cuda_stream, lbfsi_mesh* out) {
    g_last_error.clear();
    if (!d) return fail(LBFSI_EINVAL, "null argument");
    int rc = check_common(d->nr + lbfsi::CGRID_GHOST_ROWS, d->ntheta, d->precision, d->nbatch, d->bodies, out);
    if (rc) return rc;
    auto m = new lbfsi_mesh_s();
    const int nbody = d->nbody < 1 ? 1 : d->nbody;
    rc = lbfsi::build_host_mesh_c(d->nr, d->ntheta, d->nwalls, d->walls, d->X, d->xc, d->yc, m->host, nbody,
                                  d->wall_body);
    if (rc) {
        delete m;
        return rc;
    }
    m->nbody = nbody;
    return create_common(m, d->precision, d->nbatch, d->bodies, cuda_stream, out);
}

namespace {

int create_common(lbfsi_mesh m, int precision, int nbatch, const lbfsi_body_desc* bodies, void* cuda_stream,
                  lbfsi_mesh* out) {
    int rc = lbfsi::validate_bodies(m->host, bodies, nbatch);
    if (rc) {
        delete m;
        return rc;
    }
    m->nbatch = nbatch;
    m->precision = precision;
    m->esize = precision == LBFSI_FP64 ? sizeof(double) : sizeof(float);
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    // tile shape of the float kernel (a tuning knob, every variant computes the
    // same result; see lbfsi_step_variants): default 4 with the solve-minor
    // CTA order (the autotuner's choice on a GB300 for batched meshes), or
    // LBFSI_STEP_VARIANT
    m->variant = 4;
    m->order = 1;
    if (const char* v = std::getenv("LBFSI_STEP_VARIANT")) {
        const int k = std::atoi(v);
        m->variant = (k >= 0 && k < lbfsi::step_variants(LBFSI_FP32)) ? k : 4;
    }
    if (m->precision == LBFSI_FP64 || m->host.general) m->variant = 0;   // 8-row tiles (general: the one shape)
    m->tile_rows = m->host.general ? lbfsi::general_tile_rows(m->precision) : lbfsi::tile_rows(m->precision, m->variant);
    const int nti = (m->host.nr + m->tile_rows - 1) / m->tile_rows;
    m->tiles_per_solve = nti * m->host.ntj;
    m->bodies.assign(bodies, bodies + m->slots());
    m->solves.assign(m->nbatch, SolveDev{});
    rc = lbfsi::upload_mesh(m->host, m->precision, m->mem, m->stream, m->dmesh);
    if (rc) {
        delete m;
        return rc;
    }
    const size_t N = (size_t)m->host.Nx, nb = (size_t)m->nbatch, ns = m->slots();
    const int ntj = m->host.ntj;
    cudaError_t e = cudaSuccess;
#define LB_ALLOC(ptr, cnt) \
    if (e == cudaSuccess) e = dalloc(&(ptr), (cnt));
    LB_ALLOC(m->d_stage, nb * 4 * N);
    LB_ALLOC(m->d_maps[0], ns);
    LB_ALLOC(m->d_maps[1], ns);
    LB_ALLOC(m->d_state_a, ns);
    LB_ALLOC(m->d_state_b, ns);
    LB_ALLOC(m->d_loads_tmp, ns * 3);
    LB_ALLOC(m->d_part, ns * ntj * 3);
    LB_ALLOC(m->d_counter, 2 * nb);
    LB_ALLOC(m->d_bodies, ns);
    LB_ALLOC(m->d_meshdev, 1);
    LB_ALLOC(m->d_solves, nb);
    LB_ALLOC(m->d_status, 1);
#undef LB_ALLOC
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMalloc(&m->d_p[k], nb * 18 * N * m->esize);
        if (e == cudaSuccess) e = cudaMalloc(&m->d_M[k], nb * 4 * N * m->esize);
    }
    if (e == cudaSuccess && m->host.cgrid) e = cudaMalloc(&m->d_ppost, nb * 18 * N * m->esize);
    // general meshes: departures of the static nodes, solved once per time
    // step size (LBFSI_NO_DEPARTURE_CACHE=1 solves them every step instead;
    // the results are the same)
    const char* nc = std::getenv("LBFSI_NO_DEPARTURE_CACHE");
    if (e == cudaSuccess && m->host.general && !(nc && std::atoi(nc) != 0))
        e = cudaMalloc(&m->d_dep, 9 * N * 2 * m->esize + N * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        free_all(m);
        delete m;
        cudaGetLastError();
        return fail(LBFSI_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(m->d_meshdev, &m->dmesh.dev, sizeof(lbfsi::MeshDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(m->d_counter, 0, 2 * nb * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(m->d_part, 0, ns * ntj * 3 * sizeof(double));
    if (e != cudaSuccess) {
        free_all(m);
        delete m;
        return cuda_fail(e, "create_mesh copy");
    }
    *out = m;
    return LBFSI_OK;
}

}  // namespace

int lbfsi_destroy_mesh(lbfsi_mesh m) {
    if (!m) return fail(LBFSI_EINVAL, "null mesh");
    cudaStreamSynchronize(m->stream);
    free_all(m);
    delete m;
    return LBFSI_OK;
}

int lbfsi_init_fields(lbfsi_mesh m, const lbfsi_flow_params* p, const double* rho_u_T) {
    lbfsi::TraceRange trace_("lbfsi_init_fields");
    if (!m || !p) return fail(LBFSI_EINVAL, "null argument");
    SolveDev proto{};
    int rc = lbfsi::fill_flow(*p, proto);
    if (rc) return rc;
    const size_t N = (size_t)m->host.N, nb = (size_t)m->nbatch;
    for (auto& s : m->solves) s = proto;
    m->dt = p->dt;
    const size_t ns = m->slots();
    std::vector<BodyDev> bd(ns);
    for (size_t b = 0; b < ns; ++b) bd[b] = lbfsi::body_dev(m->bodies[b], proto.rho_inf, proto.uinf_x);
    // the caller's field goes to the device as it is unless the C-grid's
    // rows need rearranging (cut copies unified, mirrored rows added)
    const bool direct = rho_u_T && !m->host.cgrid && !m->host.G;
    std::vector<double> M(direct ? 0 : nb * 4 * N);
    if (direct) {
    } else if (rho_u_T) {
        std::memcpy(M.data(), rho_u_T, M.size() * sizeof(double));
    } else {
        for (size_t b = 0; b < nb; ++b)
            for (size_t n = 0; n < N; ++n) {
                M[(b * 4 + 0) * N + n] = proto.rho_inf;
                M[(b * 4 + 1) * N + n] = proto.uinf_x;
                M[(b * 4 + 2) * N + n] = 0.0;
                M[(b * 4 + 3) * N + n] = proto.T_inf;
            }
    }
    std::vector<BodyStateDev> zero(ns, BodyStateDev{0.0, 0.0, 0.0, 0.0});
    std::vector<double> zl(ns * 3, 0.0);
    if (!direct) unify_cut_copies(m->host, M.data(), nb * 4, 1);
    if (m->host.G) M = expand_rows(m->host, M.data(), nb * 4, 1);
    cudaError_t e = cudaMemcpyAsync(m->d_bodies, bd.data(), ns * sizeof(BodyDev), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = direct ? cudaMemcpyAsync(m->d_stage, rho_u_T, nb * 4 * N * sizeof(double), cudaMemcpyHostToDevice, m->stream)
                   : cudaMemcpyAsync(m->d_stage, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->d_state_a, zero.data(), ns * sizeof(BodyStateDev), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->d_loads_tmp, zl.data(), zl.size() * sizeof(double), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_status, 0, sizeof(unsigned), m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_counter, 0, 2 * nb * sizeof(unsigned), m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "init_fields upload");
    m->host_k = 0;
    rc = upload_solves(m);
    if (rc) return rc;
    e = lbfsi::launch_init(m->precision, m->d_stage, m->d_p[0], m->d_M[0], m->host.Nx, m->nbatch,
                           proto.Cv, m->stream);
    m->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    e = lbfsi::launch_prepare(m->d_bodies, m->d_state_a, m->d_state_a, m->d_state_a, m->d_loads_tmp, m->dt,
                              (int)ns, m->d_maps[0], m->stream);
    m->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "prepare kernel");
    if (m->d_dep) {
        // the static nodes' departures for this dt (one pass of the step
        // kernel over solve 0 that writes nothing else)
        const size_t Nx = (size_t)m->host.Nx;
        e = cudaMemsetAsync((char*)m->d_dep + 9 * Nx * 2 * m->esize, 0xff, Nx * sizeof(unsigned long long),
                            m->stream);
        lbfsi::StepArgs a = make_args(m, 0);
        a.ustep = 0;
        a.record = 1;
        if (e == cudaSuccess) e = lbfsi::launch_step_uniform(a, m->precision, m->variant, 1, m->stream);
        m->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "departure cache");
    }
    e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "init sync");
    m->initialized = true;
    return LBFSI_OK;
}

int lbfsi_blend_mesh(lbfsi_mesh m, const lbfsi_body_state* state, const lbfsi_body_state* prev) {
    if (!m || !state) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    const size_t nb = m->slots();
    static_assert(sizeof(lbfsi_body_state) == sizeof(BodyStateDev), "layout");
    const lbfsi_body_state* pv = prev ? prev : state;
    cudaError_t e = cudaMemcpyAsync(m->d_state_a, state, nb * sizeof(BodyStateDev), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->d_state_b, pv, nb * sizeof(BodyStateDev), cudaMemcpyHostToDevice, m->stream);
    // before the first step the collision map is unused; later it stays the
    // state of the last streamed step
    if (e == cudaSuccess)
        e = lbfsi::launch_prepare(m->d_bodies, m->first() ? m->d_state_a : nullptr, m->d_state_a, m->d_state_b,
                                  nullptr, m->dt, (int)nb, m->d_maps[m->cur()], m->stream);
    m->launches++;
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "blend_mesh");
    return LBFSI_OK;
}

int lbfsi_step(lbfsi_mesh m, int nsteps) {
    lbfsi::TraceRange trace_("lbfsi_step");
    if (!m) return fail(LBFSI_EINVAL, "null mesh");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    if (nsteps < 0) return fail(LBFSI_EINVAL, "nsteps must be >= 0");
    int s = 0;
    if (m->graph_steps > 0 && nsteps >= m->graph_steps) {
        if (!m->graph) {
            const int rc = capture_graph(m);
            if (rc) return rc;
        }
        for (; nsteps - s >= m->graph_steps; s += m->graph_steps) {
            const cudaError_t e = cudaGraphLaunch(m->graph, m->stream);
            if (e != cudaSuccess) return cuda_fail(e, "graph launch");
            m->launches += (int64_t)m->graph_steps * launches_per_step(m);
            m->host_k += (unsigned)m->graph_steps;
        }
    }
    lbfsi::StepArgs a = make_args(m, 0);
    for (; s < nsteps; ++s) {
        a.ustep = (int)m->host_k;
        cudaError_t e = launch_one_step(m, a, m->stream);
        m->launches += launches_per_step(m);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
        m->host_k++;
    }
    return LBFSI_OK;
}

int lbfsi_field_ptr(lbfsi_mesh m, int which, void** ptr, int64_t* slots, int64_t* row0) {
    if (!m || !ptr) return fail(LBFSI_EINVAL, "null argument");
    if (which != LBFSI_FIELD_MOMENTS && which != LBFSI_FIELD_POPULATIONS)
        return fail(LBFSI_EINVAL, "which must be LBFSI_FIELD_MOMENTS or LBFSI_FIELD_POPULATIONS");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    *ptr = which == LBFSI_FIELD_MOMENTS ? m->d_M[m->cur()] : m->d_p[m->cur()];
    if (slots) *slots = (int64_t)m->host.Nx;
    if (row0) *row0 = (int64_t)m->host.G * m->host.nt;
    return LBFSI_OK;
}

int lbfsi_synchronize(lbfsi_mesh m) {
    if (!m) return fail(LBFSI_EINVAL, "null mesh");
    return check_status(m);
}

static int download_maps(lbfsi_mesh m, std::vector<StepMaps>& out) {
    out.resize(m->slots());
    cudaError_t e = cudaMemcpyAsync(out.data(), m->d_maps[m->cur()], out.size() * sizeof(StepMaps),
                                    cudaMemcpyDeviceToHost, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "maps copy");
    return check_status(m);
}

namespace {
// The records of one or two consecutive steps, packed: (Fx, Fy, M, h,
// alpha, hdot, adot) of every (solve, body) from the maps records the steps'
// epilogues wrote (the two ping-pong sets hold the last two steps' records):
// prev (may be null) then cur, n records each.
__global__ void k_pack_records(const StepMaps* prev, const StepMaps* cur, int n, double* out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int np = prev ? n : 0;
    if (r >= np + n) return;
    const StepMaps& m = r < np ? prev[r] : cur[r - np];
    double* o = out + (size_t)r * 7;
    o[0] = m.loads[0];
    o[1] = m.loads[1];
    o[2] = m.loads[2];
    o[3] = m.S_next.h;
    o[4] = m.S_next.alpha;
    o[5] = m.S_next.hdot;
    o[6] = m.S_next.adot;
}
}  // namespace

int lbfsi_step_record(lbfsi_mesh m, int nsteps, double* loads_out, lbfsi_body_state* states_out) {
    lbfsi::TraceRange trace_("lbfsi_step_record");
    if (!m || !loads_out) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    if (nsteps < 0) return fail(LBFSI_EINVAL, "nsteps must be >= 0");
    const size_t nb = m->slots();   // one record per (solve, body)
    // the records are packed on the device behind every second launch (one
    // small kernel for two steps: a strided copy of the records per step
    // costs more), and the history comes back in one copy at the end
    const size_t cnt = (size_t)nsteps * nb * 7;
    if (cnt > m->d_rec_count || cnt * sizeof(double) > m->h_rec_bytes) {
        cudaError_t e = cudaStreamSynchronize(m->stream);
        if (e == cudaSuccess && cnt > m->d_rec_count) {
            if (m->d_rec) cudaFree(m->d_rec);
            m->d_rec = nullptr;
            m->d_rec_count = 0;
            e = cudaMalloc(&m->d_rec, cnt * sizeof(double));
            if (e == cudaSuccess) m->d_rec_count = cnt;
        }
        if (e == cudaSuccess && cnt * sizeof(double) > m->h_rec_bytes) {
            if (m->h_rec) cudaFreeHost(m->h_rec);
            m->h_rec = nullptr;
            m->h_rec_bytes = 0;
            e = cudaHostAlloc(&m->h_rec, cnt * sizeof(double), cudaHostAllocDefault);
            if (e == cudaSuccess) m->h_rec_bytes = cnt * sizeof(double);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LBFSI_ENOMEM, "staging for the step records");
        }
    }
    lbfsi::StepArgs a = make_args(m, 0);
    for (int s = 0; s < nsteps; ++s) {
        a.ustep = (int)m->host_k;
        cudaError_t e = launch_one_step(m, a, m->stream);
        m->launches += launches_per_step(m);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
        m->host_k++;
        // the launch's epilogue wrote the step's loads and new body state into
        // the maps record of the next launch; the previous step's records are
        // in the other set until the launch after this one
        const bool pair = (s & 1) != 0;
        if (pair || s == nsteps - 1) {
            const int first = pair ? s - 1 : s;
            const unsigned nrec = (unsigned)((pair ? 2 : 1) * nb);
            k_pack_records<<<(nrec + 127) / 128, 128, 0, m->stream>>>(
                pair ? m->d_maps[m->cur() ^ 1] : nullptr, m->d_maps[m->cur()], (int)nb,
                m->d_rec + (size_t)first * nb * 7);
            m->launches++;
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "step record kernel");
        }
    }
    cudaError_t e = cudaSuccess;
    if (cnt) e = cudaMemcpyAsync(m->h_rec, m->d_rec, cnt * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step record copy");
    static_assert(sizeof(lbfsi_body_state) == sizeof(BodyStateDev), "layout");
    const double* h = static_cast<const double*>(m->h_rec);
    for (size_t r = 0; r < (size_t)nsteps * nb; ++r) {
        std::memcpy(loads_out + 3 * r, h + 7 * r, 3 * sizeof(double));
        if (states_out) std::memcpy(states_out + r, h + 7 * r + 3, sizeof(BodyStateDev));
    }
    return check_status(m);
}

int lbfsi_body_forces(lbfsi_mesh m, double* out) {
    lbfsi::TraceRange trace_("lbfsi_body_forces");
    if (!m || !out) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    std::vector<StepMaps> mp;
    const int rc = download_maps(m, mp);
    if (rc) return rc;
    for (size_t b = 0; b < m->slots(); ++b)
        for (int c = 0; c < 3; ++c) out[b * 3 + c] = mp[b].loads[c];
    return LBFSI_OK;
}

int lbfsi_advance_bodies(lbfsi_mesh m, const double* loads, double dt) {
    if (!m) return fail(LBFSI_EINVAL, "null mesh");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    const size_t nb = m->slots();
    std::vector<double> ld(nb * 3);
    if (loads) {
        std::memcpy(ld.data(), loads, ld.size() * sizeof(double));
    } else {
        std::vector<StepMaps> mp;
        const int rc = download_maps(m, mp);
        if (rc) return rc;
        for (size_t b = 0; b < nb; ++b)
            for (int c = 0; c < 3; ++c) ld[b * 3 + c] = mp[b].loads[c];
    }
    cudaError_t e = cudaMemcpyAsync(m->d_loads_tmp, ld.data(), ld.size() * sizeof(double), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = lbfsi::launch_advance(m->d_bodies, m->d_loads_tmp, dt, (long long)m->host_k, (int)nb,
                                  m->d_maps[m->cur()], m->stream);
    m->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "advance_bodies");
    return check_status(m);
}

int lbfsi_get_body_state(lbfsi_mesh m, lbfsi_body_state* out) {
    if (!m || !out) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    std::vector<StepMaps> mp;
    const int rc = download_maps(m, mp);
    if (rc) return rc;
    for (size_t b = 0; b < m->slots(); ++b) {
        out[b].h = mp[b].S_next.h;
        out[b].alpha = mp[b].S_next.alpha;
        out[b].hdot = mp[b].S_next.hdot;
        out[b].adot = mp[b].S_next.adot;
    }
    return LBFSI_OK;
}

int lbfsi_get_fields(lbfsi_mesh m, double* rho_u_T) {
    if (!m || !rho_u_T) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    int rc;
    if (m->host.G) {
        std::vector<double> all((size_t)m->nbatch * 4 * m->host.Nx);
        rc = download(m, m->d_M[m->cur()], all.data(), all.size());
        if (!rc) compact_rows(m->host, all.data(), rho_u_T, (size_t)m->nbatch * 4, 1);
    } else {
        rc = download(m, m->d_M[m->cur()], rho_u_T, (size_t)m->nbatch * 4 * m->host.N);
    }
    if (rc) return rc;
    return check_status(m);
}

int lbfsi_get_populations(lbfsi_mesh m, int which, double* f, double* g) {
    if (!m || !f || !g) return fail(LBFSI_EINVAL, "null argument");
    if (which != 0 && which != 1) return fail(LBFSI_EINVAL, "which must be 0 or 1");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    const size_t cnt = (size_t)m->nbatch * 9 * m->host.N, cntx = (size_t)m->nbatch * 9 * m->host.Nx;
    const void* ps = m->d_p[m->cur()];
    if (which == 1 && !m->first()) {
        cudaError_t e = cudaSuccess;
        if (!m->d_ppost) {
            e = cudaMalloc(&m->d_ppost, 2 * cntx * m->esize);
            if (e != cudaSuccess) return fail(LBFSI_ENOMEM, "post-collision staging allocation failed");
            const int rc = upload_solves(m);
            if (rc) return rc;
        }
        e = lbfsi::launch_step_uniform(make_args(m, 1), m->precision, m->variant, m->nbatch, m->stream);
        m->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "collide kernel launch");
        ps = m->d_ppost;
    }
    std::vector<double> pairs(2 * cnt);
    int rc;
    if (m->host.G) {
        std::vector<double> all(2 * cntx);
        rc = download(m, ps, all.data(), all.size());
        if (!rc) compact_rows(m->host, all.data(), pairs.data(), (size_t)m->nbatch * 9, 2);
    } else {
        rc = download(m, ps, pairs.data(), 2 * cnt);
    }
    if (rc) return rc;
    for (size_t k = 0; k < cnt; ++k) {
        f[k] = pairs[2 * k];
        g[k] = pairs[2 * k + 1];
    }
    return check_status(m);
}

int lbfsi_set_populations(lbfsi_mesh m, const double* f, const double* g, const double* rho_u_T) {
    if (!m || !f || !g || !rho_u_T) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    const size_t cnt = (size_t)m->nbatch * 9 * m->host.N;
    const int c = m->cur();
    std::vector<double> pairs(2 * cnt);
    for (size_t k = 0; k < cnt; ++k) {
        pairs[2 * k] = f[k];
        pairs[2 * k + 1] = g[k];
    }
    int rc;
    if (m->host.G) {
        std::vector<double> mu(rho_u_T, rho_u_T + (size_t)m->nbatch * 4 * m->host.N);
        unify_cut_copies(m->host, pairs.data(), (size_t)m->nbatch * 9, 2);
        unify_cut_copies(m->host, mu.data(), (size_t)m->nbatch * 4, 1);
        const std::vector<double> px = expand_rows(m->host, pairs.data(), (size_t)m->nbatch * 9, 2);
        const std::vector<double> mx = expand_rows(m->host, mu.data(), (size_t)m->nbatch * 4, 1);
        rc = upload(m, px.data(), m->d_p[c], px.size());
        if (!rc) rc = upload(m, mx.data(), m->d_M[c], mx.size());
    } else {
        rc = upload(m, pairs.data(), m->d_p[c], 2 * cnt);
        if (!rc) rc = upload(m, rho_u_T, m->d_M[c], (size_t)m->nbatch * 4 * m->host.N);
    }
    if (rc) return rc;
    // the restored state is post-propagation: make the next launch collide it
    // (step number >= 2 with the same parity)
    m->host_k = 2u + (unsigned)c;
    std::vector<unsigned> ctr(2 * (size_t)m->nbatch);
    for (int b = 0; b < m->nbatch; ++b) {
        ctr[2 * b] = 0u;
        ctr[2 * b + 1] = m->host_k;
    }
    cudaError_t e = cudaMemcpyAsync(m->d_counter, ctr.data(), ctr.size() * sizeof(unsigned),
                                    cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step number upload");
    return LBFSI_OK;
}

int64_t lbfsi_launch_count(lbfsi_mesh m) { return m ? m->launches : -1; }

namespace {
struct CheckpointHeader {
    char magic[8];
    int32_t version, precision, nbatch, nr, nt, esize;
    uint32_t step;
    uint32_t nbody;   // 0 in checkpoints of one-body handles
};
constexpr char kMagic[8] = {'L', 'B', 'F', 'S', 'I', 'C', 'K', '1'};

size_t checkpoint_bytes(lbfsi_mesh m) {
    const size_t N = (size_t)m->host.Nx, nb = (size_t)m->nbatch;
    return sizeof(CheckpointHeader) + nb * 18 * N * m->esize + nb * 4 * N * m->esize + m->slots() * sizeof(StepMaps);
}
}  // namespace

size_t lbfsi_checkpoint_bytes(lbfsi_mesh m) { return m ? checkpoint_bytes(m) : 0; }

int lbfsi_checkpoint(lbfsi_mesh m, void* buf, size_t bytes) {
    lbfsi::TraceRange trace_("lbfsi_checkpoint");
    if (!m || !buf) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    if (bytes < checkpoint_bytes(m)) return fail(LBFSI_EINVAL, "checkpoint buffer too small");
    const int rc = check_status(m);   // a failed state is not saved
    if (rc) return rc;
    CheckpointHeader h{};
    std::memcpy(h.magic, kMagic, sizeof(kMagic));
    h.version = 1;
    h.precision = m->precision;
    h.nbatch = m->nbatch;
    h.nr = m->host.nr;
    h.nt = m->host.nt;
    h.esize = (int32_t)m->esize;
    h.step = m->host_k;
    h.nbody = m->nbody > 1 ? (uint32_t)m->nbody : 0u;
    const size_t N = (size_t)m->host.Nx, nb = (size_t)m->nbatch;
    char* p = static_cast<char*>(buf);
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const int c = m->cur();
    cudaError_t e = cudaMemcpyAsync(p, m->d_p[c], nb * 18 * N * m->esize, cudaMemcpyDeviceToHost, m->stream);
    p += nb * 18 * N * m->esize;
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, m->d_M[c], nb * 4 * N * m->esize, cudaMemcpyDeviceToHost, m->stream);
    p += nb * 4 * N * m->esize;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p, m->d_maps[c], m->slots() * sizeof(StepMaps), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint copy");
    return LBFSI_OK;
}

int lbfsi_restore(lbfsi_mesh m, const void* buf, size_t bytes) {
    lbfsi::TraceRange trace_("lbfsi_restore");
    if (!m || !buf) return fail(LBFSI_EINVAL, "null argument");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first (the flow of the checkpointed run)");
    if (bytes < checkpoint_bytes(m)) return fail(LBFSI_EINVAL, "checkpoint buffer too small for this handle");
    CheckpointHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kMagic, sizeof(kMagic)) != 0 || h.version != 1)
        return fail(LBFSI_EINVAL, "not a checkpoint of this library");
    if (h.precision != m->precision || h.nbatch != m->nbatch || h.nr != m->host.nr || h.nt != m->host.nt ||
        h.esize != (int32_t)m->esize || (h.nbody > 1 ? (int)h.nbody : 1) != m->nbody)
        return fail(LBFSI_EINVAL, "checkpoint of a different mesh, batch or precision");
    drop_graph(m);
    m->host_k = h.step;
    const size_t N = (size_t)m->host.Nx, nb = (size_t)m->nbatch;
    const char* p = static_cast<const char*>(buf) + sizeof(h);
    const int c = m->cur();
    cudaError_t e = cudaMemcpyAsync(m->d_p[c], p, nb * 18 * N * m->esize, cudaMemcpyHostToDevice, m->stream);
    p += nb * 18 * N * m->esize;
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_M[c], p, nb * 4 * N * m->esize, cudaMemcpyHostToDevice, m->stream);
    p += nb * 4 * N * m->esize;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->d_maps[c], p, m->slots() * sizeof(StepMaps), cudaMemcpyHostToDevice, m->stream);
    std::vector<unsigned> ctr(2 * nb);
    for (size_t b = 0; b < nb; ++b) {
        ctr[2 * b] = 0u;
        ctr[2 * b + 1] = m->host_k;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->d_counter, ctr.data(), ctr.size() * sizeof(unsigned), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_status, 0, sizeof(unsigned), m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "restore copy");
    return LBFSI_OK;
}

int lbfsi_step_variants(int precision) {
    if (precision != LBFSI_FP32 && precision != LBFSI_FP64) return fail(LBFSI_EINVAL, "unknown precision");
    return lbfsi::step_variants(precision);
}

int lbfsi_set_schedule(lbfsi_mesh m, int variant, int order) {
    if (!m) return fail(LBFSI_EINVAL, "null mesh");
    if (variant < 0 || variant >= (m->host.general ? 1 : lbfsi::step_variants(m->precision)) ||
        (order != 0 && order != 1))
        return fail(LBFSI_EINVAL, "variant or order out of range");
    if (variant == m->variant && order == m->order) return LBFSI_OK;
    drop_graph(m);
    m->variant = variant;
    m->order = order;
    m->tile_rows = m->host.general ? lbfsi::general_tile_rows(m->precision) : lbfsi::tile_rows(m->precision, m->variant);
    m->tiles_per_solve = ((m->host.nr + m->tile_rows - 1) / m->tile_rows) * m->host.ntj;
    return m->initialized ? upload_solves(m) : LBFSI_OK;
}

int lbfsi_get_schedule(lbfsi_mesh m, int* variant, int* order) {
    if (!m) return fail(LBFSI_EINVAL, "null mesh");
    if (variant) *variant = m->variant;
    if (order) *order = m->order;
    return LBFSI_OK;
}

int lbfsi_set_graph_steps(lbfsi_mesh m, int graph_steps) {
    if (!m) return fail(LBFSI_EINVAL, "null mesh");
    if (graph_steps < 0) return fail(LBFSI_EINVAL, "graph_steps must be >= 0");
    if (graph_steps != m->graph_steps) drop_graph(m);
    m->graph_steps = graph_steps;
    return LBFSI_OK;
}

int lbfsi_autotune(lbfsi_mesh m, int steps_per_trial, int* best_variant, int* best_order, float* ms_per_step) {
    lbfsi::TraceRange trace_("lbfsi_autotune");
    if (!m) return fail(LBFSI_EINVAL, "null mesh");
    if (!m->initialized) return fail(LBFSI_ESTATE, "init_fields first");
    if (steps_per_trial < 1) return fail(LBFSI_EINVAL, "steps_per_trial must be >= 1");
    const int nv = m->host.general ? 1 : lbfsi::step_variants(m->precision);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_fail(e, "tuner events");
    int bv = m->variant, bo = m->order, rc = LBFSI_OK;
    float best = -1.0f;
    const int graph_steps = m->graph_steps;   // trials use plain launches
    lbfsi_set_graph_steps(m, 0);
    for (int v = 0; v < nv && !rc; ++v)
        for (int o = 0; o < 2 && !rc; ++o) {
            rc = lbfsi_set_schedule(m, v, o);
            if (rc) break;
            lbfsi_step(m, 1);   // first launch of a shape configures it
            cudaEventRecord(e0, m->stream);
            rc = lbfsi_step(m, steps_per_trial);
            cudaEventRecord(e1, m->stream);
            e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "tuner trial");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)steps_per_trial;
            if (ms_per_step) ms_per_step[2 * v + o] = ms;
            if (best < 0.0f || ms < best) {
                best = ms;
                bv = v;
                bo = o;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    lbfsi_set_graph_steps(m, graph_steps);
    if (rc) return rc;
    rc = lbfsi_set_schedule(m, bv, bo);
    if (rc) return rc;
    if (best_variant) *best_variant = bv;
    if (best_order) *best_order = bo;
    return check_status(m);
}

}  // extern "C"
