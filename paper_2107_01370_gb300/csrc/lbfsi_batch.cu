// Batch runtime (declared in include/lbfsi.h): solves on O-grids of different
// sizes admitted into a device memory pool and retired while others run, all
// active solves advanced together by one table launch of the step kernel per
// step.  Native pieces: a first-fit pool allocator over one cudaMalloc, a
// cache of device mesh geometry shared by solves on identical O-grids, slot
// bookkeeping and the tile table (the node-to-CTA schedule) of each launch.
#include <algorithm>
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
    int mesh = -1;
    int steps_target = 0, steps_done = 0;
    int ntiles = 0;
    SolveDev dev{};
    std::vector<void*> blocks;
};

}  // namespace

struct lbfsi_batch_s {
    Pool pool;
    int precision = LBFSI_FP32, variant = 3, tile_rows = 12;
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
    BodyStateDev* d_zero_state = nullptr;
    double* d_zero_loads = nullptr;
    int ntiles = 0;
    bool dirty = true;
};

namespace {

int cuda_err(cudaError_t e, const char* where) {
    return lbfsi::set_error(LBFSI_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool same_mesh(const lbfsi::HostMesh& h, const lbfsi_solve_desc& d) {
    return h.nr == d.nr && h.nt == d.ntheta && h.xm == d.xc && h.ym == d.yc &&
           std::memcmp(h.r.data(), d.r, sizeof(double) * d.nr) == 0 &&
           std::memcmp(h.e.data(), d.e, sizeof(double) * 2 * d.ntheta) == 0;
}

// Find or create the device geometry of an O-grid; returns the mesh index.
int acquire_mesh(lbfsi_batch b, const lbfsi_solve_desc& d, int* out) {
    for (size_t k = 0; k < b->meshes.size(); ++k)
        if (b->meshes[k].used && same_mesh(b->meshes[k].host, d)) {
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
    int rc = lbfsi::build_host_mesh(d.nr, d.ntheta, d.r, d.e, d.xc, d.yc, me.host);
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

// Tile table of the next launches: every tile of every active solve.
int rebuild_tiles(lbfsi_batch b) {
    std::vector<TileDev> tiles;
    for (size_t k = 0; k < b->slots.size(); ++k) {
        const Slot& s = b->slots[k];
        if (!s.used || s.finished) continue;
        const lbfsi::HostMesh& h = b->meshes[s.mesh].host;
        const int nti = (h.nr + b->tile_rows - 1) / b->tile_rows;
        for (int ti = 0; ti < nti; ++ti)
            for (int tj = 0; tj < h.ntj; ++tj) {
                TileDev t{};
                t.solve = (int)k;
                t.mesh = s.mesh;
                t.i0 = ti * b->tile_rows;
                t.j0 = tj * lbfsi::TILE_J;
                t.tj = tj;
                t.counter = s.dev.counter;
                t.maps[0] = s.dev.maps[0];
                t.maps[1] = s.dev.maps[1];
                tiles.push_back(t);
            }
    }
    cudaError_t e = cudaSuccess;
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
    b->ntiles = (int)tiles.size();
    b->dirty = false;
    return LBFSI_OK;
}

int check_status(lbfsi_batch b) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_err(e, "stream synchronize");
    unsigned st = 0;
    e = cudaMemcpy(&st, b->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e, "status read");
    if (st & (lbfsi::ST_DEPARTURE | lbfsi::ST_BPOINT))
        return lbfsi::set_error(LBFSI_EDEPARTURE, "departure point outside the cells adjacent to its node (CFL)");
    if (st & lbfsi::ST_NONPHYS) return lbfsi::set_error(LBFSI_ENONPHYS, "non-physical state (rho<=0, T<=0 or NaN)");
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
    b->tile_rows = lbfsi::tile_rows(precision, b->variant);
    int rc = b->pool.init(pool_bytes);
    if (rc) {
        delete b;
        return rc;
    }
    cudaError_t e = cudaMalloc(&b->d_meshes, b->max_meshes * sizeof(MeshDev));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_solves, b->max_slots * sizeof(SolveDev));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(unsigned));
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
                    b->d_zero_loads};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete b;   // the pool frees its block
    return LBFSI_OK;
}

int lbfsi_batch_add(lbfsi_batch b, const lbfsi_solve_desc* d, int* slot) {
    if (!b || !d || !slot) return lbfsi::set_error(LBFSI_EINVAL, "null argument");
    *slot = -1;
    if (d->steps <= 0) return lbfsi::set_error(LBFSI_EINVAL, "steps must be > 0");
    const long long Nll = (long long)d->nr * d->ntheta;
    if (d->nr < 5 || d->ntheta < 4 || Nll * 9 > (1ll << 31))
        return lbfsi::set_error(LBFSI_EINVAL, "invalid mesh size");
    SolveDev sd{};
    int rc = lbfsi::fill_flow(d->flow, sd);
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
    rc = acquire_mesh(b, *d, &mk);
    if (rc) return rc;
    const lbfsi::HostMesh& h = b->meshes[mk].host;
    rc = lbfsi::validate_bodies(h, &d->body, 1);
    if (rc) {
        drop_mesh(b, mk);
        return rc;
    }
    Slot s;
    const size_t N = (size_t)h.N, es = b->esize;
    auto take = [&](size_t bytes) -> void* {
        void* p = b->pool.alloc(bytes);
        if (p) s.blocks.push_back(p);
        return p;
    };
    bool ok = true;
    for (int p = 0; p < 2 && ok; ++p) {
        ok = ok && (sd.p[p] = take(18 * N * es)) != nullptr;
        ok = ok && (sd.M[p] = take(4 * N * es)) != nullptr;
        ok = ok && (sd.maps[p] = (StepMaps*)take(sizeof(StepMaps))) != nullptr;
    }
    ok = ok && (sd.part = (double*)take((size_t)h.ntj * 3 * sizeof(double))) != nullptr;
    ok = ok && (sd.counter = (unsigned*)take(2 * sizeof(unsigned))) != nullptr;
    BodyDev* body = nullptr;
    ok = ok && (body = (BodyDev*)take(sizeof(BodyDev))) != nullptr;
    double* stage = nullptr;
    ok = ok && (stage = (double*)take(4 * N * sizeof(double))) != nullptr;
    if (!ok) {
        release_slot_memory(b, s);
        drop_mesh(b, mk);
        return lbfsi::set_error(LBFSI_ENOMEM, "the pool has no room for this solve now");
    }
    sd.body = body;
    sd.mesh = mk;
    sd.ntiles = ((h.nr + b->tile_rows - 1) / b->tile_rows) * h.ntj;
    sd.ppost = nullptr;
    // initial state: equilibria of the initial field, bodies at rest
    std::vector<double> M(4 * N);
    if (d->rho_u_T) {
        std::memcpy(M.data(), d->rho_u_T, M.size() * sizeof(double));
    } else {
        for (size_t n = 0; n < N; ++n) {
            M[n] = sd.rho_inf;
            M[N + n] = sd.uinf_x;
            M[2 * N + n] = 0.0;
            M[3 * N + n] = sd.T_inf;
        }
    }
    const BodyDev bd = lbfsi::body_dev(d->body, sd.rho_inf, sd.uinf_x);
    cudaError_t e = cudaMemcpyAsync(stage, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(body, &bd, sizeof(BodyDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sd.counter, 0, 2 * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = lbfsi::launch_init(b->precision, stage, sd.p[0], sd.M[0], (int)N, 1, sd.Cv, b->stream);
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
    s.mesh = mk;
    s.steps_target = d->steps;
    s.steps_done = 0;
    s.ntiles = sd.ntiles;
    s.dev = sd;
    b->slots[k] = std::move(s);
    b->dirty = true;
    *slot = k;
    return LBFSI_OK;
}

int lbfsi_batch_step(lbfsi_batch b, int nsteps, int* active_after) {
    if (!b) return lbfsi::set_error(LBFSI_EINVAL, "null batch");
    if (nsteps < 0) return lbfsi::set_error(LBFSI_EINVAL, "nsteps must be >= 0");
    for (int st = 0; st < nsteps; ++st) {
        if (b->dirty) {
            const int rc = rebuild_tiles(b);
            if (rc) return rc;
        }
        if (b->ntiles == 0) break;
        lbfsi::StepArgs a{};
        a.meshes = b->d_meshes;
        a.solves = b->d_solves;
        a.tiles = b->d_tiles;
        a.ntiles = b->ntiles;
        a.collide_only = 0;
        a.ustep = -1;
        a.status = b->d_status;
        const cudaError_t e = lbfsi::launch_step(a, b->precision, b->variant, b->stream);
        if (e != cudaSuccess) return cuda_err(e, "batch step launch");
        for (auto& s : b->slots) {
            if (!s.used || s.finished) continue;
            if (++s.steps_done >= s.steps_target) {
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
    const size_t N = (size_t)b->meshes[s.mesh].host.N;
    cudaError_t e = cudaSuccess;
    std::vector<unsigned char> raw;
    if (rho_u_T) {
        raw.resize(4 * N * b->esize);
        e = cudaMemcpyAsync(raw.data(), s.dev.M[cur], raw.size(), cudaMemcpyDeviceToHost, b->stream);
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
