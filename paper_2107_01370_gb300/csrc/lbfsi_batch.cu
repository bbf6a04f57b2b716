// Batch runtime (declared in include/lbfsi.h): solves on O-grids of different
// sizes admitted into a device memory pool and retired while others run, all
// active solves advanced together by one table launch of the step kernel per
// step.  Native pieces: a first-fit pool allocator over one cudaMalloc, a
// cache of device mesh geometry shared by solves on identical O-grids, slot
// bookkeeping and the tile table (the node-to-CTA schedule) of each launch.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "lbfsi.h"
#include "lbfsi_host.h"
#include "lbfsi_internal.h"

using lbfsi::BodyDev;
using lbfsi::BodyStateDev;
using lbfsi::MeshDev;
using lbfsi::SolveDev;
using lbfsi::StepMaps;
using lbfsi::TileDev;

namespace {

// First-fit allocator over one device block; 256-byte granularity; free
// neighbours coalesce.
class Pool : public lbfsi::DevMemory {
public:
    int init(size_t bytes) {
        size_ = (bytes + 255) & ~size_t(255);
        if (cudaMalloc(&base_, size_) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return lbfsi::set_error(LBFSI_ENOMEM, "device pool allocation failed");
        }
        free_[0] = size_;
        return LBFSI_OK;
    }
    ~Pool() override {
        if (base_) cudaFree(base_);
    }
    void* alloc(size_t bytes) override {
        const size_t need = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > need) free_[off + need] = len - need;
            used_[off] = need;
            return base_ + off;
        }
        return nullptr;
    }
    void release(void* p) override {
        if (!p) return;
        const size_t off = (size_t)((char*)p - base_);
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t start = off, len = u->second;
        used_.erase(u);
        auto next = free_.lower_bound(start);
        if (next != free_.end() && next->first == start + len) {
            len += next->second;
            free_.erase(next);
        }
        auto prev = free_.lower_bound(start);
        if (prev != free_.begin()) {
            --prev;
            if (prev->first + prev->second == start) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
    }
    size_t free_bytes() const {
        size_t s = 0;
        for (auto& kv : free_) s += kv.second;
        return s;
    }
    size_t largest() const {
        size_t s = 0;
        for (auto& kv : free_) s = std::max(s, kv.second);
        return s;
    }

private:
    char* base_ = nullptr;
    size_t size_ = 0;
    std::map<size_t, size_t> free_, used_;
};

struct MeshEntry {
    lbfsi::HostMesh host;
    lbfsi::DeviceMesh dev;
    int refs = 0;
    bool used = false;
};

struct Slot {
    bool used = false, finished = false;
    bool general = false;   // on a mesh given by node coordinates (GEN kernel, 8-row tiles)
    bool cgrid = false;     // on a C-grid (general; two launches per step)
    int mesh = -1;
    int steps_target = 0, steps_done = 0;
    int ntiles = 0;
    SolveDev dev{};
    std::vector<void*> blocks;
    // the tile rows its tensor maps were made for (-1: none yet, 0: not used)
    int tma_rows = -1;
};

}  // namespace

struct lbfsi_batch_s {
    Pool pool;
    int precision = LBFSI_FP32, variant = 4, order = 0, tile_rows = 16;
    size_t esize = 4;
    cudaStream_t stream = nullptr;
    std::vector<MeshEntry> meshes;
    std::vector<Slot> slots;
    MeshDev* d_meshes = nullptr;
    SolveDev* d_solves = nullptr;
    TileDev* d_tiles = nullptr;
    size_t tiles_cap = 0;
    int max_meshes = 256, max_slots = 4096;
    unsigned* d_status = nullptr;
    // float separable solves: tensor maps of each slot's populations and
    // moments, [max_slots][4] (StepArgs::tmaps)
    CUtensorMap* d_tmaps = nullptr;
    BodyStateDev* d_zero_state = nullptr;
    double* d_zero_loads = nullptr;
    int ntiles = 0;    // separable-mesh tiles of the table (first part)
    int ngtiles = 0;   // general-mesh tiles (second part)
    int nctiles = 0;   // C-grid tiles (third part)
    int ncpre = 0;     // leading C-grid tiles that hold every tile of rows < CGRID_PRE_ROWS
    bool dirty = true;
    // CUDA graph of graph_steps launches over the current tile table,
    // captured on a private stream, dropped whenever the table changes
    int graph_steps = 0;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t cap_stream = nullptr;
};

namespace {

int cuda_err(cudaError_t e, const char* where) {
    return lbfsi::set_error(LBFSI_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool same_mesh(const lbfsi::HostMesh& h, const lbfsi_solve_desc& d) {
    return !h.general && h.nr == d.nr && h.nt == d.ntheta && h.xm == d.xc && h.ym == d.yc &&
           std::memcmp(h.r.data(), d.r, sizeof(double) * d.nr) == 0 &&
           std::memcmp(h.e.data(), d.e, sizeof(double) * 2 * d.ntheta) == 0;
}

bool same_mesh_xy(const lbfsi::HostMesh& h, const lbfsi_solve_xy_desc& d) {
    return h.general && !h.cgrid && h.nr == d.nr && h.nt == d.ntheta && h.xm == d.xc && h.ym == d.yc &&
           std::memcmp(h.X.data(), d.X, sizeof(double) * 2 * (size_t)d.nr * d.ntheta) == 0;
}

bool same_mesh_c(const lbfsi::HostMesh& h, const lbfsi_solve_cgrid_desc& d) {
    // the stored coordinates carry the mirrored rows before row 0
    return h.cgrid && h.nr == d.nr && h.nt == d.ntheta && h.walls.size() == 2 && h.walls[0] == d.n_cut &&
           h.xm == d.xc && h.ym == d.yc &&
           std::memcmp(h.X.data() + 2 * (size_t)h.G * h.nt, d.X, sizeof(double) * 2 * (size_t)d.nr * d.ntheta) == 0;
}

// Find or create the device geometry of a mesh (match: an existing entry's
// host mesh equals the request; build: the host mesh of a new one); returns
// the mesh index.
template <typename Match, typename Build>
int acquire_mesh(lbfsi_batch b, Match match, Build build_host, int* out) {
    for (size_t k = 0; k < b->meshes.size(); ++k)
        if (b->meshes[k].used && match(b->meshes[k].host)) {
            b->meshes[k].refs++;
            *out = (int)k;
            return LBFSI_OK;
        }
    int k = -1;
    for (size_t q = 0; q < b->meshes.size(); ++q)
        if (!b->meshes[q].used) {
            k = (int)q;
            break;
        }
    if (k < 0) {
        if ((int)b->meshes.size() >= b->max_meshes) return lbfsi::set_error(LBFSI_ENOMEM, "too many distinct meshes");
        b->meshes.emplace_back();
        k = (int)b->meshes.size() - 1;
    }
    MeshEntry& me = b->meshes[k];
    me = MeshEntry{};
    int rc = build_host(me.host);
    if (rc) return rc;
    rc = lbfsi::upload_mesh(me.host, b->precision, b->pool, b->stream, me.dev);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(b->d_meshes + k, &me.dev.dev, sizeof(MeshDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        lbfsi::release_mesh(me.dev, b->pool);
        return cuda_err(e, "mesh descriptor upload");
    }
    me.used = true;
    me.refs = 1;
    *out = k;
    return LBFSI_OK;
}

void drop_mesh(lbfsi_batch b, int k) {
    MeshEntry& me = b->meshes[k];
    if (--me.refs > 0) return;
    cudaStreamSynchronize(b->stream);
    lbfsi::release_mesh(me.dev, b->pool);
    me.used = false;
}

void release_slot_memory(lbfsi_batch b, Slot& s) {
    for (void* p : s.blocks) b->pool.release(p);
    s.blocks.clear();
}

void drop_graph(lbfsi_batch b) {
    if (b->graph) {
        cudaStreamSynchronize(b->stream);
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

// Tile table of the next launches: every tile of every active solve, in the
// batch's order: 0, the tiles of each solve together; 1, tile rows outermost
// across all solves, so that the wall and blending-region rows (the most
// expensive tiles) start first and the far-field rows fill the tail.
int rebuild_tiles(lbfsi_batch b) {
    lbfsi::TraceRange trace_("lbfsi tile table");
    drop_graph(b);
    // separable-mesh tiles first (tile rows of the batch's shape), then the
    // general-mesh tiles and the C-grid tiles (the general kernel's tile)
    std::vector<TileDev> tiles;
    // float separable solves: tensor maps for the current tile shape (made
    // once per slot and shape, uploaded behind the launches already queued)
    cudaError_t e = cudaSuccess;
    const char* tenv = std::getenv("LBFSI_TMA");
    const bool tma_on = b->precision == LBFSI_FP32 && b->d_tmaps && !(tenv && std::atoi(tenv) == 0);
    for (size_t k = 0; k < b->slots.size() && tma_on; ++k) {
        Slot& s = b->slots[k];
        if (!s.used || s.finished || s.general || s.tma_rows == b->tile_rows) continue;
        const lbfsi::HostMesh& h = b->meshes[s.mesh].host;
        bool ok = h.nt % 4 == 0;
        CUtensorMap maps[4];
        const size_t nt = (size_t)h.nt, nr = (size_t)h.nr;
        const unsigned rows = (unsigned)b->tile_rows, w = (unsigned)(lbfsi::TILE_J + 8);
        for (int c = 0; c < 2 && ok; ++c)
            ok = lbfsi::encode_box4(&maps[c], s.dev.p[c], 2 * nt, nr, 9, 1, 2 * w, rows + 4, 9) &&
                 lbfsi::encode_box4(&maps[2 + c], s.dev.M[c], nt, nr, 4, 1, w, rows + 8, 4);
        if (ok) {
            e = cudaMemcpyAsync(b->d_tmaps + 4 * k, maps, sizeof(maps), cudaMemcpyHostToDevice, b->stream);
            if (e != cudaSuccess) return cuda_err(e, "tensor map upload");
        }
        s.tma_rows = ok ? b->tile_rows : 0;
    }
    auto build = [&](int part) {
        const bool general = part > 0;
        const int rows = general ? lbfsi::general_tile_rows(b->precision) : b->tile_rows;
        auto push = [&](size_t k, int ti, int tj) {
            const Slot& s = b->slots[k];
            TileDev t{};
            t.solve = (int)k;
            t.mesh = s.mesh;
            t.i0 = ti * rows;
            t.j0 = tj * lbfsi::TILE_J;
            t.tj = tj;
            // a separable tile whose columns do not wrap, of a solve with maps
            const int ntm = b->meshes[s.mesh].host.nt;
            t.tma = part == 0 && tma_on && s.tma_rows == rows && t.j0 >= 4 && t.j0 + lbfsi::TILE_J + 4 <= ntm;
            t.counter = s.dev.counter;
            t.maps[0] = s.dev.maps[0];
            t.maps[1] = s.dev.maps[1];
            tiles.push_back(t);
        };
        auto active = [&](size_t k) {
            const Slot& s = b->slots[k];
            return s.used && !s.finished && (s.cgrid ? 2 : s.general ? 1 : 0) == part;
        };
        auto nti_of = [&](size_t k) { return (b->meshes[b->slots[k].mesh].host.nr + rows - 1) / rows; };
        if (b->order == 0) {
            for (size_t k = 0; k < b->slots.size(); ++k) {
                if (!active(k)) continue;
                const int nti = nti_of(k), ntj = b->meshes[b->slots[k].mesh].host.ntj;
                for (int ti = 0; ti < nti; ++ti)
                    for (int tj = 0; tj < ntj; ++tj) push(k, ti, tj);
            }
        } else {
            int max_nti = 0;
            for (size_t k = 0; k < b->slots.size(); ++k)
                if (active(k)) max_nti = std::max(max_nti, nti_of(k));
            for (int ti = 0; ti < max_nti; ++ti)
                for (size_t k = 0; k < b->slots.size(); ++k) {
                    if (!active(k) || ti >= nti_of(k)) continue;
                    const int ntj = b->meshes[b->slots[k].mesh].host.ntj;
                    for (int tj = 0; tj < ntj; ++tj) push(k, ti, tj);
                }
        }
    };
    build(0);
    const size_t nsep = tiles.size();
    build(1);
    const size_t ngen = tiles.size() - nsep;
    build(2);
    if (tiles.size() > b->tiles_cap) {
        e = cudaStreamSynchronize(b->stream);
        if (b->d_tiles) cudaFree(b->d_tiles);
        b->d_tiles = nullptr;
        b->tiles_cap = std::max(tiles.size(), 2 * b->tiles_cap);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles, b->tiles_cap * sizeof(TileDev));
        if (e != cudaSuccess) {
            b->tiles_cap = 0;
            return cuda_err(e, "tile table allocation");
        }
    }
    if (!tiles.empty()) {
        // stream-ordered: launches already queued read the previous table
        e = cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(TileDev), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_err(e, "tile table upload");
    }
    b->ntiles = (int)nsep;
    b->ngtiles = (int)ngen;
    b->nctiles = (int)(tiles.size() - nsep - ngen);
    // tile rows outermost: the tiles of the first rows come first; otherwise
    // the collide-only launch runs over the whole part (the others return)
    b->ncpre = b->nctiles;
    if (b->order == 1) {
        int k = 0;
        while (k < b->nctiles && tiles[nsep + ngen + k].i0 < lbfsi::CGRID_PRE_ROWS) ++k;
        b->ncpre = k;
    }
    b->dirty = false;
    return LBFSI_OK;
}

int check_status(lbfsi_batch b) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_err(e, "stream synchronize");
    unsigned st = 0;
    e = cudaMemcpy(&st, b->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e, "status read");
    if (st & lbfsi::ST_BOUNDS)
        return lbfsi::set_error(LBFSI_EBOUNDS, "an index of the step outside its buffer (bounds-checked build)");
    if (st & (lbfsi::ST_DEPARTURE | lbfsi::ST_BPOINT))
        return lbfsi::set_error(LBFSI_EDEPARTURE, "departure point outside the cells adjacent to its node (CFL)");
    if (st & lbfsi::ST_TMA)
        return lbfsi::set_error(LBFSI_ECUDA, "a tensor copy of the step did not complete within its wait limit");
    if (st & lbfsi::ST_NONPHYS) return lbfsi::set_error(LBFSI_ENONPHYS, "non-physical state (rho<=0, T<=0 or NaN)");
    return LBFSI_OK;
}

// Launch arguments of one part of the tile table (0 separable, 1 general, 2 C-grid).
lbfsi::StepArgs step_args(lbfsi_batch b, int part) {
    lbfsi::StepArgs a{};
    a.meshes = b->d_meshes;
    a.solves = b->d_solves;
    a.tiles = b->d_tiles + (part == 0 ? 0 : part == 1 ? b->ntiles : b->ntiles + b->ngtiles);
    a.ntiles = part == 0 ? b->ntiles : part == 1 ? b->ngtiles : b->nctiles;
    a.collide_only = 0;
    a.ustep = -1;
    a.status = b->d_status;
    a.tmaps = part == 0 && b->precision == LBFSI_FP32 ? b->d_tmaps : nullptr;
    return a;
}

// One step of every active solve: the separable-mesh table launch, the
// general-mesh one and, for C-grids, the collision of the rows next to the
// cut followed by the launch that streams the first row of tiles from it and
// collides and streams the others (independent solves, so the order of the
// parts is free).
cudaError_t launch_all(lbfsi_batch b, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (b->ntiles > 0) e = lbfsi::launch_step(step_args(b, 0), b->precision, b->variant, s);
    if (e == cudaSuccess && b->ngtiles > 0) e = lbfsi::launch_step_general_table(step_args(b, 1), b->precision, s);
    if (e == cudaSuccess && b->nctiles > 0) {
        lbfsi::StepArgs a = step_args(b, 2);
        a.collide_only = 1;
        a.cgrid_pre = 1;
        a.ntiles = b->ncpre;   // the tiles of rows < CGRID_PRE_ROWS lead the C-grid part
        e = lbfsi::launch_step_general_table(a, b->precision, s);
        a = step_args(b, 2);
        a.stream_post = 1;
        if (e == cudaSuccess) e = lbfsi::launch_step_general_table(a, b->precision, s);
    }
    return e;
}

// Capture graph_steps launches over the current tile table (every launch
// reads the step numbers from the device counters, so the graph is valid for
// every replay until the table changes).
int capture_graph(lbfsi_batch b) {
    lbfsi::TraceRange trace_("lbfsi batch graph capture");
    cudaError_t e = lbfsi::prepare_step(b->precision, b->variant, false);
    if (e == cudaSuccess && b->ngtiles + b->nctiles > 0) e = lbfsi::prepare_step(b->precision, 0, false, true);
    if (e == cudaSuccess && !b->cap_stream) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_err(e, "graph capture setup");
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_err(e, "begin capture");
    cudaError_t le = cudaSuccess;
    for (int g = 0; g < b->graph_steps && le == cudaSuccess; ++g) le = launch_all(b, b->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_err(le != cudaSuccess ? le : e, "batch step capture");
    }
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return cuda_err(e, "graph instantiate");
    }
    return LBFSI_OK;
}

}  // namespace

extern "C" {

int lbfsi_batch_create(size_t pool_bytes, int precision, void* cuda_stream, lbfsi_batch* out) {
    if (!out) return lbfsi::set_error(LBFSI_EINVAL, "null argument");
    *out = nullptr;
    if (precision != LBFSI_FP64 && precision != LBFSI_FP32)
        return lbfsi::set_error(LBFSI_EINVAL, "precision must be LBFSI_FP64 or LBFSI_FP32");
    if (pool_bytes < (1u << 20)) return lbfsi::set_error(LBFSI_EINVAL, "pool must be at least 1 MiB");
    auto b = new lbfsi_batch_s();
    b->precision = precision;
    b->esize = precision == LBFSI_FP64 ? sizeof(double) : sizeof(float);
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    if (precision == LBFSI_FP64) b->variant = 0;   // 8-row tiles
    b->tile_rows = lbfsi::tile_rows(precision, b->variant);
    int rc = b->pool.init(pool_bytes);
    if (rc) {
        delete b;
        return rc;
    }
    cudaError_t e = cudaMalloc(&b->d_meshes, b->max_meshes * sizeof(MeshDev));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_solves, b->max_slots * sizeof(SolveDev));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(unsigned));
    if (e == cudaSuccess && precision == LBFSI_FP32)
        e = cudaMalloc(&b->d_tmaps, (size_t)b->max_slots * 4 * sizeof(CUtensorMap));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_zero_state, sizeof(BodyStateDev));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_zero_loads, 3 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_zero_state, 0, sizeof(BodyStateDev));
    if (e == cudaSuccess) e = cudaMemset(b->d_zero_loads, 0, 3 * sizeof(double));
    if (e != cudaSuccess) {
        lbfsi_batch_destroy(b);
        return lbfsi::set_error(LBFSI_ENOMEM, std::string("batch allocation: ") + cudaGetErrorString(e));
    }
    *out = b;
    return LBFSI_OK;
}

int lbfsi_batch_destroy(lbfsi_batch b) {
    if (!b) return lbfsi::set_error(LBFSI_EINVAL, "null batch");
    cudaStreamSynchronize(b->stream);
    void* ptrs[] = {b->d_meshes, b->d_solves, b->d_tiles, b->d_status, b->d_zero_state,
                    b->d_zero_loads, b->d_tmaps};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;   // the pool frees its block
    return LBFSI_OK;
}

}  // extern "C"

namespace {

// Admission of one solve whose mesh is given by 'acquire' (which finds or
// creates its device geometry): pool memory, initial state, slot.
template <typename Acquire>
int add_solve(lbfsi_batch b, const lbfsi_body_desc& body_desc, const lbfsi_flow_params& flow,
              const double* rho_u_T, int steps, int nr, int nt, Acquire acquire, int* slot) {
    if (!slot) return lbfsi::set_error(LBFSI_EINVAL, "null argument");
    *slot = -1;
    if (steps <= 0) return lbfsi::set_error(LBFSI_EINVAL, "steps must be > 0");
    const long long Nll = (long long)nr * nt;
    if (nr < 5 || nt < 4 || Nll * 9 > (1ll << 31)) return lbfsi::set_error(LBFSI_EINVAL, "invalid mesh size");
    SolveDev sd{};
    int rc = lbfsi::fill_flow(flow, sd);
    if (rc) return rc;
    // a free slot
    int k = -1;
    for (size_t q = 0; q < b->slots.size(); ++q)
        if (!b->slots[q].used) {
            k = (int)q;
            break;
        }
    if (k < 0) {
        if ((int)b->slots.size() >= b->max_slots) return lbfsi::set_error(LBFSI_ENOMEM, "no free slot");
        b->slots.emplace_back();
        k = (int)b->slots.size() - 1;
    }
    int mk = -1;
    rc = acquire(&mk);
    if (rc) return rc;
    const lbfsi::HostMesh& h = b->meshes[mk].host;
    rc = lbfsi::validate_bodies(h, &body_desc, 1);
    if (rc) {
        drop_mesh(b, mk);
        return rc;
    }
    Slot s;
    // slots per component: nr nt, plus a C-grid's mirrored rows before row 0
    const size_t N = (size_t)h.N, Nx = (size_t)h.Nx, es = b->esize, g0 = (size_t)h.G * h.nt;
    auto take = [&](size_t bytes) -> void* {
        void* p = b->pool.alloc(bytes);
        if (p) s.blocks.push_back(p);
        return p;
    };
    bool ok = true;
    void* p0 = nullptr;   // first population block (the initial state is written there)
    void* m0 = nullptr;
    for (int p = 0; p < 2 && ok; ++p) {
        void* pb = take(18 * Nx * es);
        void* mb = take(4 * Nx * es);
        ok = ok && pb && mb;
        if (p == 0) {
            p0 = pb;
            m0 = mb;
        }
        if (ok) {
            sd.p[p] = (char*)pb + 2 * g0 * es;   // row 0
            sd.M[p] = (char*)mb + g0 * es;
        }
        ok = ok && (sd.maps[p] = (StepMaps*)take(sizeof(StepMaps))) != nullptr;
    }
    sd.ppost = nullptr;
    if (ok && h.cgrid) {
        void* pp = take(18 * Nx * es);
        ok = pp != nullptr;
        if (ok) sd.ppost = (char*)pp + 2 * g0 * es;
    }
    ok = ok && (sd.part = (double*)take((size_t)h.ntj * 3 * sizeof(double))) != nullptr;
    ok = ok && (sd.counter = (unsigned*)take(2 * sizeof(unsigned))) != nullptr;
    BodyDev* body = nullptr;
    ok = ok && (body = (BodyDev*)take(sizeof(BodyDev))) != nullptr;
    double* stage = nullptr;
    ok = ok && (stage = (double*)take(4 * Nx * sizeof(double))) != nullptr;
    if (!ok) {
        release_slot_memory(b, s);
        drop_mesh(b, mk);
        return lbfsi::set_error(LBFSI_ENOMEM, "the pool has no room for this solve now");
    }
    sd.body = body;
    sd.mesh = mk;
    const int rows = h.general ? lbfsi::general_tile_rows(b->precision) : b->tile_rows;
    sd.ntiles = ((h.nr + rows - 1) / rows) * h.ntj;
    // initial state: equilibria of the initial field, bodies at rest
    std::vector<double> M(4 * N);
    if (rho_u_T) {
        std::memcpy(M.data(), rho_u_T, M.size() * sizeof(double));
    } else {
        for (size_t n = 0; n < N; ++n) {
            M[n] = sd.rho_inf;
            M[N + n] = sd.uinf_x;
            M[2 * N + n] = 0.0;
            M[3 * N + n] = sd.T_inf;
        }
    }
    if (h.cgrid) {
        // the two copies of a cut node start from the first copy's values;
        // the mirrored rows below row 0 from their nodes
        for (int c = 0; c < 4; ++c)
            for (int j = 0; j < h.nt; ++j)
                if (h.coltype[j] & lbfsi::CT_DUP) M[c * N + (size_t)j] = M[c * N + (size_t)(h.nt - 1 - j)];
        std::vector<double> Mx(4 * Nx);
        for (int c = 0; c < 4; ++c) {
            std::memcpy(&Mx[c * Nx + g0], &M[c * N], N * sizeof(double));
            for (int k2 = 1; k2 <= h.G; ++k2)
                for (int j = 0; j < h.nt; ++j)
                    Mx[c * Nx + g0 - (size_t)k2 * h.nt + j] = M[c * N + (size_t)k2 * h.nt + (h.nt - 1 - j)];
        }
        M.swap(Mx);
    }
    const BodyDev bd = lbfsi::body_dev(body_desc, sd.rho_inf, sd.uinf_x);
    cudaError_t e = cudaMemcpyAsync(stage, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(body, &bd, sizeof(BodyDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sd.counter, 0, 2 * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = lbfsi::launch_init(b->precision, stage, p0, m0, (int)Nx, 1, sd.Cv, b->stream);
    if (e == cudaSuccess)
        e = lbfsi::launch_prepare(body, b->d_zero_state, b->d_zero_state, b->d_zero_state, b->d_zero_loads, sd.dt,
                                  1, sd.maps[0], b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_solves + k, &sd, sizeof(SolveDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    // the staging block is no longer needed
    b->pool.release(stage);
    s.blocks.erase(std::remove(s.blocks.begin(), s.blocks.end(), (void*)stage), s.blocks.end());
    if (e != cudaSuccess) {
        release_slot_memory(b, s);
        drop_mesh(b, mk);
        return cuda_err(e, "solve initialisation");
    }
    s.used = true;
    s.finished = false;
    s.general = h.general;
    s.cgrid = h.cgrid;
    s.mesh = mk;
    s.steps_target = steps;
    s.steps_done = 0;
    s.ntiles = sd.ntiles;
    s.dev = sd;
    b->slots[k] = std::move(s);
    b->dirty = true;
    *slot = k;
    return LBFSI_OK;
}

}  // namespace

extern "C" {

int lbfsi_batch_add(lbfsi_batch b, const lbfsi_solve_desc* d, int* slot) {
    lbfsi::TraceRange trace_("lbfsi_batch_add");
    if (!b || !d || !slot) return lbfsi::set_error(LBFSI_EINVAL, "null argument");
    auto acquire = [&](int* mk) {
        return acquire_mesh(
            b, [&](const lbfsi::HostMesh& h) { return same_mesh(h, *d); },
            [&](lbfsi::HostMesh& h) { return lbfsi::build_host_mesh(d->nr, d->ntheta, d->r, d->e, d->xc, d->yc, h); },
            mk);
    };
    return add_solve(b, d->body, d->flow, d->rho_u_T, d->steps, d->nr, d->ntheta, acquire, slot);
}

int lbfsi_batch_add_xy(lbfsi_batch b, const lbfsi_solve_xy_desc* d, int* slot) {
    lbfsi::TraceRange trace_("lbfsi_batch_add_xy");
    if (!b || !d || !slot) return lbfsi::set_error(LBFSI_EINVAL, "null argument");
    auto acquire = [&](int* mk) {
        return acquire_mesh(
            b, [&](const lbfsi::HostMesh& h) { return same_mesh_xy(h, *d); },
            [&](lbfsi::HostMesh& h) { return lbfsi::build_host_mesh_xy(d->nr, d->ntheta, d->X, d->xc, d->yc, h); },
            mk);
    };
    return add_solve(b, d->body, d->flow, d->rho_u_T, d->steps, d->nr, d->ntheta, acquire, slot);
}

int lbfsi_batch_add_cgrid(lbfsi_batch b, const lbfsi_solve_cgrid_desc* d, int* slot) {
    lbfsi::TraceRange trace_("lbfsi_batch_add_cgrid");
    if (!b || !d || !slot) return lbfsi::set_error(LBFSI_EINVAL, "null argument");
    auto acquire = [&](int* mk) {
        return acquire_mesh(
            b, [&](const lbfsi::HostMesh& h) { return same_mesh_c(h, *d); },
            [&](lbfsi::HostMesh& h) {
                const int walls[2] = {d->n_cut, d->ntheta - 1 - d->n_cut};
                return lbfsi::build_host_mesh_c(d->nr, d->ntheta, 1, walls, d->X, d->xc, d->yc, h);
            },
            mk);
    };
    return add_solve(b, d->body, d->flow, d->rho_u_T, d->steps, d->nr, d->ntheta, acquire, slot);
}

int lbfsi_batch_step(lbfsi_batch b, int nsteps, int* active_after) {
    lbfsi::TraceRange trace_("lbfsi_batch_step");
    if (!b) return lbfsi::set_error(LBFSI_EINVAL, "null batch");
    if (nsteps < 0) return lbfsi::set_error(LBFSI_EINVAL, "nsteps must be >= 0");
    int st = 0;
    while (st < nsteps) {
        if (b->dirty) {
            const int rc = rebuild_tiles(b);
            if (rc) return rc;
        }
        if (b->ntiles + b->ngtiles + b->nctiles == 0) break;
        // steps until the next solve finishes: the tile table is fixed over them
        int run = nsteps - st;
        for (auto& s : b->slots)
            if (s.used && !s.finished) run = std::min(run, s.steps_target - s.steps_done);
        int done = 0;
        if (b->graph_steps > 0 && run >= b->graph_steps) {
            if (!b->graph) {
                const int rc = capture_graph(b);
                if (rc) return rc;
            }
            for (; run - done >= b->graph_steps; done += b->graph_steps) {
                const cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
                if (e != cudaSuccess) return cuda_err(e, "batch graph launch");
            }
        }
        for (; done < run; ++done) {
            const cudaError_t e = launch_all(b, b->stream);
            if (e != cudaSuccess) return cuda_err(e, "batch step launch");
        }
        st += run;
        for (auto& s : b->slots) {
            if (!s.used || s.finished) continue;
            s.steps_done += run;
            if (s.steps_done >= s.steps_target) {
                s.finished = true;
                b->dirty = true;
            }
        }
    }
    if (active_after) {
        int n = 0;
        for (auto& s : b->slots) n += (s.used && !s.finished) ? 1 : 0;
        *active_after = n;
    }
    return LBFSI_OK;
}

int lbfsi_batch_set_schedule(lbfsi_batch b, int variant, int order) {
    if (!b) return lbfsi::set_error(LBFSI_EINVAL, "null batch");
    if (variant < 0 || variant >= lbfsi::step_variants(b->precision) || (order != 0 && order != 1))
        return lbfsi::set_error(LBFSI_EINVAL, "variant or order out of range");
    if (variant == b->variant && order == b->order) return LBFSI_OK;
    drop_graph(b);
    b->variant = variant;
    b->order = order;
    b->tile_rows = lbfsi::tile_rows(b->precision, variant);
    // the per-solve CTA count of the completion counter follows the tile shape
    for (size_t k = 0; k < b->slots.size(); ++k) {
        Slot& s = b->slots[k];
        if (!s.used || s.general) continue;   // general meshes keep their one tile shape
        const lbfsi::HostMesh& h = b->meshes[s.mesh].host;
        s.dev.ntiles = ((h.nr + b->tile_rows - 1) / b->tile_rows) * h.ntj;
        s.ntiles = s.dev.ntiles;
        const cudaError_t e = cudaMemcpyAsync(b->d_solves + k, &s.dev, sizeof(SolveDev), cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return cuda_err(e, "solve record upload");
    }
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_err(e, "schedule change");
    b->dirty = true;
    return LBFSI_OK;
}

int lbfsi_batch_get_schedule(lbfsi_batch b, int* variant, int* order) {
    if (!b) return lbfsi::set_error(LBFSI_EINVAL, "null batch");
    if (variant) *variant = b->variant;
    if (order) *order = b->order;
    return LBFSI_OK;
}

int lbfsi_batch_set_graph_steps(lbfsi_batch b, int graph_steps) {
    if (!b) return lbfsi::set_error(LBFSI_EINVAL, "null batch");
    if (graph_steps < 0) return lbfsi::set_error(LBFSI_EINVAL, "graph_steps must be >= 0");
    if (graph_steps != b->graph_steps) drop_graph(b);
    b->graph_steps = graph_steps;
    return LBFSI_OK;
}

int lbfsi_batch_autotune(lbfsi_batch b, int steps_per_trial, int* best_variant, int* best_order,
                         float* ns_per_node) {
    lbfsi::TraceRange trace_("lbfsi_batch_autotune");
    if (!b) return lbfsi::set_error(LBFSI_EINVAL, "null batch");
    if (steps_per_trial < 1) return lbfsi::set_error(LBFSI_EINVAL, "steps_per_trial must be >= 1");
    const int nv = lbfsi::step_variants(b->precision);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_err(e, "tuner events");
    const int graph_steps = b->graph_steps;   // trials use plain launches
    lbfsi_batch_set_graph_steps(b, 0);
    int bv = b->variant, bo = b->order, rc = LBFSI_OK;
    float best = -1.0f;
    for (int v = 0; v < nv && !rc; ++v)
        for (int o = 0; o < 2 && !rc; ++o) {
            rc = lbfsi_batch_set_schedule(b, v, o);
            if (rc) break;
            rc = lbfsi_batch_step(b, 1, nullptr);   // configures the shape, rebuilds the table
            if (rc) break;
            // node updates of the trial, from the steps each solve takes
            std::vector<int> before(b->slots.size());
            for (size_t k = 0; k < b->slots.size(); ++k) before[k] = b->slots[k].steps_done;
            cudaEventRecord(e0, b->stream);
            rc = lbfsi_batch_step(b, steps_per_trial, nullptr);
            cudaEventRecord(e1, b->stream);
            e = cudaEventSynchronize(e1);
            if (!rc && e != cudaSuccess) rc = cuda_err(e, "tuner trial");
            if (rc) break;
            double nodes = 0.0;
            for (size_t k = 0; k < b->slots.size(); ++k)
                if (b->slots[k].used)
                    nodes += (double)(b->slots[k].steps_done - before[k]) * b->meshes[b->slots[k].mesh].host.N;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            const float ns = nodes > 0.0 ? (float)(ms * 1e6 / nodes) : -1.0f;
            if (ns_per_node) ns_per_node[2 * v + o] = ns;
            if (ns > 0.0f && (best < 0.0f || ns < best)) {
                best = ns;
                bv = v;
                bo = o;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    lbfsi_batch_set_graph_steps(b, graph_steps);
    if (rc) return rc;
    rc = lbfsi_batch_set_schedule(b, bv, bo);
    if (rc) return rc;
    if (best_variant) *best_variant = bv;
    if (best_order) *best_order = bo;
    return check_status(b);
}

int lbfsi_batch_poll(lbfsi_batch b, int slot, int* steps_done, int* finished) {
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used)
        return lbfsi::set_error(LBFSI_EINVAL, "invalid slot");
    if (steps_done) *steps_done = b->slots[slot].steps_done;
    if (finished) *finished = b->slots[slot].finished ? 1 : 0;
    return LBFSI_OK;
}

int lbfsi_batch_get(lbfsi_batch b, int slot, double* rho_u_T, double* loads, lbfsi_body_state* state) {
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used)
        return lbfsi::set_error(LBFSI_EINVAL, "invalid slot");
    const Slot& s = b->slots[slot];
    const int cur = s.steps_done & 1;
    const size_t N = (size_t)b->meshes[s.mesh].host.N, Nx = (size_t)b->meshes[s.mesh].host.Nx;
    cudaError_t e = cudaSuccess;
    std::vector<unsigned char> raw;
    if (rho_u_T) {
        // rows 0 .. nr-1 of the four components (Nx slots apart)
        raw.resize(4 * N * b->esize);
        e = cudaMemcpy2DAsync(raw.data(), N * b->esize, s.dev.M[cur], Nx * b->esize, N * b->esize, 4,
                              cudaMemcpyDeviceToHost, b->stream);
    }
    StepMaps mp{};
    if (e == cudaSuccess && (loads || state))
        e = cudaMemcpyAsync(&mp, s.dev.maps[cur], sizeof(StepMaps), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_err(e, "batch results copy");
    if (rho_u_T) {
        if (b->precision == LBFSI_FP64) {
            std::memcpy(rho_u_T, raw.data(), raw.size());
        } else {
            const float* f = reinterpret_cast<const float*>(raw.data());
            for (size_t n = 0; n < 4 * N; ++n) rho_u_T[n] = (double)f[n];
        }
    }
    if (loads)
        for (int c = 0; c < 3; ++c) loads[c] = mp.loads[c];
    if (state) {
        state->h = mp.S_next.h;
        state->alpha = mp.S_next.alpha;
        state->hdot = mp.S_next.hdot;
        state->adot = mp.S_next.adot;
    }
    return check_status(b);
}

int lbfsi_batch_remove(lbfsi_batch b, int slot) {
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used)
        return lbfsi::set_error(LBFSI_EINVAL, "invalid slot");
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_err(e, "batch remove");
    Slot& s = b->slots[slot];
    release_slot_memory(b, s);
    drop_mesh(b, s.mesh);
    if (!s.finished) b->dirty = true;
    s = Slot{};
    return LBFSI_OK;
}

int lbfsi_batch_memory(lbfsi_batch b, size_t* free_bytes, size_t* largest_free) {
    if (!b) return lbfsi::set_error(LBFSI_EINVAL, "null batch");
    if (free_bytes) *free_bytes = b->pool.free_bytes();
    if (largest_free) *largest_free = b->pool.largest();
    return LBFSI_OK;
}

}  // extern "C"
