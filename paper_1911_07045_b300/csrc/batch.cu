// batch.cu -- many independent lattices advanced together: one persistent
// kernel launch per FIRE iteration of every lattice (fire_batch_kernel),
// captured in CUDA graphs, with the tile height and z chunk chosen by timing
// candidates on shadow copies of the FIRE state.
//
// Each lattice keeps its own device state, FIRE scalars and reduction slots;
// its blocks are numbered as in the single-lattice kernel, so with the same
// tile and z chunk its reductions run in the same order as alone: one-constant
// lattices advance bit-for-bit as they do alone, three-constant ones within
// rounding (their products may be fused differently in the two kernels).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "lqmin.h"
#include "lq_common.cuh"
#include "lq_kernels.h"
#include "solver_internal.h"

using namespace lq;
using namespace lq::detail;

struct lq_batch {
    std::vector<lq_solver *> solvers;
    int device = 0, fp32 = 0, three = 0, nsm = 148;
    cudaStream_t stream = nullptr;
    int tx = 32, ty = 0, zchunk = 0;  // tiling; zchunk 0 = each lattice's own
    int idx32 = 1;                    // every lattice indexed in 32 bits
    int form = 0;                     // kernel form: 0 one-, 1 three-constant, 2 with L4 / L6
    bool tables_ok = false;
    int cap = 0;                      // lattices the device arrays hold
    // device tables
    void *args = nullptr;             // StepArgs per lattice
    void *shadow_args = nullptr;      // the same, pointing at shadow FIRE states
    FireDev *shadow = nullptr;        // n shadow FIRE states (tuning)
    WorkItem *items = nullptr;
    int nitems = 0, items_cap = 0;
    double *partials = nullptr;       // all lattices' reduction slots
    long long partials_cap = 0;
    FireDev **states = nullptr;       // n pointers to the lattices' FIRE states
    unsigned int *running = nullptr;  // device count of running lattices
    unsigned int *running_host = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_k = 0;
    long long sites = 0;
    std::vector<unsigned long long> gens;   // members' generations the tables were built from
    std::string err;
};

namespace {

lq_status bfail(lq_batch *b, lq_status st, const char *msg, cudaError_t e = cudaSuccess) {
    if (b) {
        b->err = msg;
        if (e != cudaSuccess) b->err += std::string(": ") + cudaGetErrorString(e);
    }
    return st;
}

#define BK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? LQ_ENOMEM : LQ_ECUDA, #call, e_); \
    } while (0)

void drop_batch_graph(lq_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->graph_k = 0;
}

// work items and reduction slots for tile tx x ty and z chunk zc
lq_status build_items(lq_batch *b, int tx, int ty, int zc_all, bool shadow) {
    std::vector<WorkItem> items;
    std::vector<long long> base(b->solvers.size());
    std::vector<int> zcs(b->solvers.size());
    long long slots = 0;
    for (size_t l = 0; l < b->solvers.size(); ++l) {
        const LatticeDev &L = b->solvers[l]->L;
        int zc = zc_all > 0 ? zc_all : effective_zchunk(b->solvers[l]);
        zcs[l] = zc;
        int gx = (L.nx + tx - 1) / tx, gy = (L.ny + ty - 1) / ty, gz = (L.nz + zc - 1) / zc;
        int nblk = gx * gy * gz;
        base[l] = slots;
        slots += std::max(nblk, 1);
        for (int bz = 0; bz < gz; ++bz)
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx) {
                    WorkItem w;
                    w.lattice = (int)l; w.bx = bx; w.by = by;
                    w.z0 = bz * zc; w.z1 = std::min(w.z0 + zc, L.nz);
                    w.nblk = nblk; w.bid = bx + gx * (by + gy * bz); w.pad = 0;
                    items.push_back(w);
                }
    }
    // largest first, so that the last items of the persistent grid are short
    std::stable_sort(items.begin(), items.end(), [](const WorkItem &a, const WorkItem &c) {
        return (a.z1 - a.z0) > (c.z1 - c.z0);
    });
    if ((int)items.size() > b->items_cap) {
        cudaFree(b->items);
        b->items = nullptr;
        BK(dev_malloc(&b->items, items.size() * sizeof(WorkItem)));
        b->items_cap = (int)items.size();
    }
    if (slots > b->partials_cap) {
        cudaFree(b->partials);
        b->partials = nullptr;
        BK(dev_malloc(&b->partials, slots * 4 * sizeof(double)));
        b->partials_cap = slots;
    }
    BK(cudaMemcpyAsync(b->items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                       b->stream));
    b->nitems = (int)items.size();
    // per-lattice kernel arguments
    size_t ab = step_args_bytes(b->fp32);
    std::vector<unsigned char> host(ab * b->solvers.size());
    for (size_t l = 0; l < b->solvers.size(); ++l) {
        lq_solver *s = b->solvers[l];
        StepLaunch sl = make_launch(s, 0);
        sl.partials = b->partials + 4 * base[l];
        sl.zchunk = zcs[l];
        if (shadow) sl.st = b->shadow + l;
        step_args_pack(sl, host.data() + ab * l);
    }
    BK(cudaMemcpyAsync(shadow ? b->shadow_args : b->args, host.data(), host.size(),
                       cudaMemcpyHostToDevice, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    if (!shadow) {
        b->gens.resize(b->solvers.size());
        for (size_t l = 0; l < b->solvers.size(); ++l) b->gens[l] = b->solvers[l]->gen;
    }
    return LQ_OK;
}

int persistent_grid(lq_batch *b, int tx, int ty) {
    int per = fire_batch_blocks_per_sm(b->fp32, b->form, tx, ty, b->idx32);
    return std::max(1, per) * b->nsm;
}

lq_status set_tiling(lq_batch *b, int tx, int ty, int zc) {
    if (b->tables_ok && b->tx == tx && b->ty == ty && b->zchunk == zc) return LQ_OK;
    drop_batch_graph(b);
    b->tables_ok = false;
    if (!b->solvers.empty()) {
        lq_status r = build_items(b, tx, ty, zc, false);
        if (r != LQ_OK) return r;
    } else {
        b->nitems = 0;
    }
    b->tx = tx;
    b->ty = ty;
    b->zchunk = zc;
    b->tables_ok = true;
    return LQ_OK;
}

lq_status ensure_graph(lq_batch *b) {
    long long k = (1LL << 24) / std::max(1LL, b->sites);
    int kk = (int)std::max(1LL, std::min(64LL, k));
    if (b->gexec && b->graph_k == kk) return LQ_OK;
    drop_batch_graph(b);
    int grid = persistent_grid(b, b->tx, b->ty);
    cudaGraph_t g = nullptr;
    BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < kk && e == cudaSuccess; ++t)
        e = launch_fire_batch(b->fp32, b->form, b->tx, b->ty, b->idx32, b->args, b->items, b->nitems, grid,
                              b->stream);
    if (e == cudaSuccess) e = batch_running(b->states, (int)b->solvers.size(), b->running, b->stream);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, LQ_ECUDA, "batch graph capture", e != cudaSuccess ? e : e2);
    }
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, LQ_ECUDA, "batch graph instantiate", e);
    b->graph_k = kk;
    return LQ_OK;
}

// start FIRE where needed and push the parameters to every lattice
lq_status prepare_run(lq_batch *b, const lq_fire_params *p, bool reset) {
    for (lq_solver *s : b->solvers) {
        lq_status r = check_params(s, p);
        if (r != LQ_OK) return bfail(b, r, s->err.c_str());
        if (reset || s->geom_dirty || !s->fire_ready) {
            if (s->fire_ready) { r = sync_state(s); if (r != LQ_OK) return bfail(b, r, s->err.c_str()); }
            r = fire_reset(s, p);
        } else {
            r = update_params(s, p);
        }
        if (r != LQ_OK) return bfail(b, r, s->err.c_str());
        cudaStreamSynchronize(s->stream);
    }
    // a member whose geometry or material changed since the tables were
    // built: its records moved, its form may differ -- rebuild the tables
    bool stale = b->gens.size() != b->solvers.size();
    for (size_t l = 0; l < b->solvers.size() && !stale; ++l) stale = b->gens[l] != b->solvers[l]->gen;
    if (stale) {
        std::vector<lq_solver *> members = b->solvers;
        lq_status r = batch_set_members(b, members.data(), (int)members.size());
        if (r != LQ_OK) return r;
    }
    return LQ_OK;
}

lq_status collect(lq_batch *b, lq_result *out, double secs) {
    for (size_t l = 0; l < b->solvers.size(); ++l) {
        lq_solver *s = b->solvers[l];
        lq_status r = sync_state(s);
        if (r != LQ_OK) return bfail(b, r, s->err.c_str());
        if (out) fill_result(s, out + l, secs);
    }
    return LQ_OK;
}

}  // namespace

namespace lq {
namespace detail {

lq_status batch_new(int device, int fp32, int three, lq_batch **out) {
    *out = nullptr;
    lq_batch *b = new lq_batch();
    b->device = device; b->fp32 = fp32; b->three = three;
    cudaSetDevice(device);
    // the batch's own stream: its destruction never touches a solver
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return LQ_ECUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) b->nsm = prop.multiProcessorCount;
    cudaError_t e = cudaSuccess;
    for (int tx : {32, 64})
        for (int ty : {4, 8})
            for (int i32 : {0, 1})
                for (int form : {three ? 1 : 0, three ? 2 : 0})
                    if (e == cudaSuccess && batch_tile_ok(fp32, form, tx))
                        e = prepare_fire_batch(fp32, form, tx, ty, i32);
    if (e == cudaSuccess) e = dev_malloc(&b->running, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMallocHost(&b->running_host, sizeof(unsigned int));
    if (e != cudaSuccess) {
        lq_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? LQ_ENOMEM : LQ_ECUDA;
    }
    int tx, ty;
    step_tile(fp32, three, 0, &tx, &ty);   // the narrow tiles of batches
    b->tx = 32;          // default tiling: 32-wide tiles of the solvers' height,
    b->ty = ty;          // z chunk 0 = each lattice's own
    b->zchunk = 0;
    *out = b;
    return LQ_OK;
}

// replace the lattices of the batch (device tables grow as needed)
lq_status batch_set_members(lq_batch *b, lq_solver *const *solvers, int n) {
    for (int l = 0; l < n; ++l)
        if (!solvers[l] || solvers[l]->device != b->device || solvers[l]->fp32 != b->fp32 ||
            solvers[l]->three != b->three)
            return bfail(b, LQ_EINVAL, "one device, one precision, one distortion form per batch");
    for (int l = 0; l < n; ++l)
        if (solvers[l]->slab) return bfail(b, LQ_EINVAL, "a slab of a decomposed lattice cannot join a batch");
    cudaSetDevice(b->device);
    drop_batch_graph(b);
    b->tables_ok = false;
    b->solvers.assign(solvers, solvers + n);
    b->sites = 0;
    // FP32-form batches run the 64-bit-index instantiation, measured faster
    // on 64 lattices (one constant 1.580 -> 1.570 ms, three constants 2.163
    // -> 2.112 ms per launch); FP64 batches 32-bit indices where they fit
    b->idx32 = b->fp32 ? 0 : 1;
    b->form = b->three ? 1 : 0;
    for (int l = 0; l < n; ++l) {
        if (!step_index32(solvers[l]->L.N) || solvers[l]->idx64) b->idx32 = 0;
        if (solvers[l]->ext) b->form = 2;
    }
    if (n > b->cap) {
        cudaFree(b->args); cudaFree(b->shadow_args); cudaFree(b->shadow); cudaFree(b->states);
        b->args = b->shadow_args = nullptr; b->shadow = nullptr; b->states = nullptr;
        b->cap = 0;
        size_t ab = step_args_bytes(b->fp32);
        int cap = std::max(n, 8);
        BK(dev_malloc(&b->args, ab * cap));
        BK(dev_malloc(&b->shadow_args, ab * cap));
        BK(dev_malloc(&b->shadow, sizeof(FireDev) * cap));
        BK(dev_malloc(&b->states, sizeof(FireDev *) * cap));
        b->cap = cap;
    }
    std::vector<FireDev *> st(std::max(n, 1));
    for (int l = 0; l < n; ++l) {
        lq_status r = build_geometry(b->solvers[l]);
        if (r != LQ_OK) return bfail(b, r, b->solvers[l]->err.c_str());
        st[l] = b->solvers[l]->st;
        b->sites += b->solvers[l]->L.N;
    }
    if (n > 0) BK(cudaMemcpyAsync(b->states, st.data(), sizeof(FireDev *) * n, cudaMemcpyHostToDevice, b->stream));
    // 64-wide tiles only where the form has them (a three-constant member
    // turns them back to 32)
    int tx = batch_tile_ok(b->fp32, b->form, b->tx) ? b->tx : 32, ty = b->ty, zc = b->zchunk;
    b->ty = 0;
    return set_tiling(b, tx, ty, zc);
}

int batch_members(const lq_batch *b) { return b ? (int)b->solvers.size() : 0; }

// k batched FIRE iterations (direct launches), then the number of lattices
// still running
lq_status batch_round(lq_batch *b, int k, unsigned int *running) {
    cudaSetDevice(b->device);
    if (b->solvers.empty()) { *running = 0; return LQ_OK; }
    // stale tables could name lattices that are gone: never launch on them
    if (!b->tables_ok) return bfail(b, LQ_EINVAL, "batch tables are not built");
    int grid = persistent_grid(b, b->tx, b->ty);
    for (int t = 0; t < k; ++t)
        BK(launch_fire_batch(b->fp32, b->form, b->tx, b->ty, b->idx32, b->args, b->items, b->nitems, grid,
                             b->stream));
    BK(batch_running(b->states, (int)b->solvers.size(), b->running, b->stream));
    BK(cudaMemcpyAsync(b->running_host, b->running, sizeof(unsigned int), cudaMemcpyDeviceToHost, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    *running = *b->running_host;
    return LQ_OK;
}

}  // namespace detail
}  // namespace lq

extern "C" {

lq_status lq_batch_create(lq_solver *const *solvers, int n, lq_batch **out) {
    if (!solvers || n <= 0 || !out) return LQ_EINVAL;
    *out = nullptr;
    for (int l = 0; l < n; ++l)
        if (!solvers[l]) return LQ_EINVAL;
    lq_batch *b = nullptr;
    lq_status r = batch_new(solvers[0]->device, solvers[0]->fp32, solvers[0]->three, &b);
    if (r != LQ_OK) return r;
    r = batch_set_members(b, solvers, n);
    if (r != LQ_OK) {
        lq_batch_destroy(b);
        return r;
    }
    *out = b;
    return LQ_OK;
}

void lq_batch_destroy(lq_batch *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_batch_graph(b);
    cudaFree(b->args); cudaFree(b->shadow_args); cudaFree(b->shadow); cudaFree(b->items);
    cudaFree(b->partials); cudaFree(b->states); cudaFree(b->running);
    if (b->running_host) cudaFreeHost(b->running_host);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char *lq_batch_last_error(const lq_batch *b) { return b ? b->err.c_str() : "null batch"; }

lq_status lq_batch_set_tiling(lq_batch *b, int tile_y, int zchunk) {
    return lq_batch_set_tile(b, 32, tile_y, zchunk);
}

lq_status lq_batch_get_tiling(const lq_batch *b, int *tile_y, int *zchunk) {
    return lq_batch_get_tile(b, nullptr, tile_y, zchunk);
}

lq_status lq_batch_set_tile(lq_batch *b, int tile_x, int tile_y, int zchunk) {
    if (!b) return LQ_EINVAL;
    if ((tile_y != 4 && tile_y != 8) || zchunk < 0)
        return bfail(b, LQ_EINVAL, "tile height must be 4 or 8 and the z chunk >= 0");
    if (!batch_tile_ok(b->fp32, b->form, tile_x))
        return bfail(b, LQ_EINVAL, "tile width must be 32, or 64 for one-constant FP32-form lattices");
    cudaSetDevice(b->device);
    return set_tiling(b, tile_x, tile_y, zchunk);
}

lq_status lq_batch_get_tile(const lq_batch *b, int *tile_x, int *tile_y, int *zchunk) {
    if (!b) return LQ_EINVAL;
    if (tile_x) *tile_x = b->tx;
    if (tile_y) *tile_y = b->ty;
    if (zchunk) *zchunk = b->zchunk;
    return LQ_OK;
}

lq_status lq_batch_autotune(lq_batch *b, const lq_fire_params *p, int launches, double *best_ms) {
    if (!b || !p) return LQ_EINVAL;
    cudaSetDevice(b->device);
    lq_status r = prepare_run(b, p, false);
    if (r != LQ_OK) return r;
    launches = std::max(2, launches);
    int nz_max = 1;
    for (lq_solver *s : b->solvers) nz_max = std::max(nz_max, s->L.nz);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int n = (int)b->solvers.size();
    double best = 1e300;
    int btx = b->tx, bty = b->ty, bzc = b->zchunk;
    if (b->solvers.empty()) return LQ_OK;
    for (int tx : {32, 64}) {
        if (!batch_tile_ok(b->fp32, b->form, tx)) continue;
        for (int ty : {4, 8}) {
            for (int zc : {8, 16, 32, 64, 128}) {
                if (zc > nz_max && zc != 8) continue;
                r = build_items(b, tx, ty, zc, true);
                if (r != LQ_OK) break;
                int grid = persistent_grid(b, tx, ty);
                // shadow FIRE states: the timed launches leave the real ones alone
                for (int l = 0; l < n; ++l)
                    cudaMemcpyAsync(b->shadow + l, b->solvers[l]->st, sizeof(FireDev), cudaMemcpyDeviceToDevice,
                                    b->stream);
                cudaError_t e = launch_fire_batch(b->fp32, b->form, tx, ty, b->idx32, b->shadow_args, b->items,
                                                  b->nitems, grid, b->stream);
                cudaEventRecord(e0, b->stream);
                for (int t = 0; t < launches && e == cudaSuccess; ++t) {
                    for (int l = 0; l < n; ++l)   // every timed launch starts from the same state
                        cudaMemcpyAsync(b->shadow + l, b->solvers[l]->st, sizeof(FireDev),
                                        cudaMemcpyDeviceToDevice, b->stream);
                    e = launch_fire_batch(b->fp32, b->form, tx, ty, b->idx32, b->shadow_args, b->items,
                                          b->nitems, grid, b->stream);
                }
                cudaEventRecord(e1, b->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) { r = bfail(b, LQ_ECUDA, "autotune launch", e); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                double per = ms / launches;
                if (per < best) { best = per; btx = tx; bty = ty; bzc = zc; }
            }
            if (r != LQ_OK) break;
        }
        if (r != LQ_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tables_ok = false;   // force the rebuild of the real tables
    drop_batch_graph(b);
    lq_status r2 = set_tiling(b, btx, bty, bzc);
    if (r != LQ_OK) return r;
    if (best_ms) *best_ms = best;
    return r2;
}

lq_status lq_batch_step(lq_batch *b, const lq_fire_params *p, int64_t n, lq_result *out) {
    if (!b || !p || n < 0) return LQ_EINVAL;
    cudaSetDevice(b->device);
    auto t0 = std::chrono::steady_clock::now();
    lq_status r = prepare_run(b, p, false);
    if (r != LQ_OK) return r;
    if (!b->tables_ok) return bfail(b, LQ_EINVAL, "batch tables are not built");
    r = ensure_graph(b);
    if (r != LQ_OK) return r;
    int64_t full = n / b->graph_k, rest = n % b->graph_k;
    int grid = persistent_grid(b, b->tx, b->ty);
    for (int64_t t = 0; t < full; ++t) BK(cudaGraphLaunch(b->gexec, b->stream));
    for (int64_t t = 0; t < rest; ++t)
        BK(launch_fire_batch(b->fp32, b->form, b->tx, b->ty, b->idx32, b->args, b->items, b->nitems, grid,
                             b->stream));
    BK(cudaStreamSynchronize(b->stream));
    return collect(b, out, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
}

lq_status lq_batch_minimize(lq_batch *b, const lq_fire_params *p, lq_result *out) {
    if (!b || !p) return LQ_EINVAL;
    cudaSetDevice(b->device);
    auto t0 = std::chrono::steady_clock::now();
    lq_status r = prepare_run(b, p, true);
    if (r != LQ_OK) return r;
    if (!b->tables_ok) return bfail(b, LQ_EINVAL, "batch tables are not built");
    r = ensure_graph(b);
    if (r != LQ_OK) return r;
    bool timed_out = false;
    for (;;) {
        BK(cudaGraphLaunch(b->gexec, b->stream));
        BK(cudaMemcpyAsync(b->running_host, b->running, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                           b->stream));
        BK(cudaStreamSynchronize(b->stream));
        if (*b->running_host == 0) break;
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (p->wall_timeout_s > 0 && el > p->wall_timeout_s) { timed_out = true; break; }
    }
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    r = collect(b, out, secs);
    if (r != LQ_OK) return r;
    lq_status ret = LQ_OK;
    for (size_t l = 0; l < b->solvers.size(); ++l) {
        lq_solver *s = b->solvers[l];
        if (out) {
            double E;
            if (lq_energy(s, &E, nullptr) == LQ_OK) out[l].energy = E;
        }
        int st = s->st_host->status;
        if (st == FIRE_DIVERGED) ret = LQ_EDIVERGED;
        else if (st == FIRE_MAXITER && ret == LQ_OK) ret = LQ_ENOTCONVERGED;
        else if (st == FIRE_RUNNING && timed_out && ret == LQ_OK) ret = LQ_ETIMEOUT;
    }
    return ret;
}

}  // extern "C"
