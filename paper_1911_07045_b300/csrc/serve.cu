// serve.cu -- continuous batching of minimisation requests.
//
// A worker thread owns the GPU.  Requests wait in a queue until the HBM
// budget and the slot limit admit them; an admitted request becomes a solver
// (geometry, initial Q, FIRE started) and joins the active set, which is
// advanced in rounds of k iterations of the persistent batch kernel -- one
// batch per distortion form.  Between rounds, finished solves (converged,
// max_iter, diverged, timed out) are retired: their result, energy and,
// on request, order field are kept for polling, their device memory is freed
// and the queue is admitted again.  So requests that arrive while others are
// on the GPU join them as memory frees up, and their work shares each launch.
// Each solve runs with its own tiling and z chunk, so a one-constant solve
// follows the same trajectory as it would alone.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "lqmin.h"
#include "lq_common.cuh"
#include "lq_kernels.h"
#include "solver_internal.h"

using namespace lq;
using namespace lq::detail;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    lq_lattice lat{};
    lq_material mat{};
    std::vector<lq_object> objs;
    std::vector<std::vector<int32_t>> xyz;          // owned copies of the site lists
    std::vector<std::vector<lq_anchoring>> per_site;
    std::vector<double> q0;
    uint64_t seed = 0;
    double S = 0.0;
    lq_fire_params params{};
    int want_S = 0;
    size_t bytes = 0;
    Clock::time_point t_submit;
};

struct Active {
    Request req;
    lq_solver *s = nullptr;
    Clock::time_point t_start;
};

struct Done {
    lq_status status = LQ_OK;
    lq_result res{};
    std::vector<double> S;
};

// device bytes of one solve: two (q, v, F) buffers, the transfer buffer, the
// mask, geometry scratch and anchoring tables (upper estimate)
size_t estimate_bytes(const lq_lattice &L, int fp32) {
    double N = (double)L.nx * L.ny * L.nz;
    double esize = fp32 ? 4.0 : 8.0;
    double per_site = 6 * 5 * esize + 5 * 8 + 1 + 16;
    return (size_t)(N * per_site + 4.0 * L.ny * L.nz + (1 << 20));
}

}  // namespace

struct lq_server {
    int device = 0, fp32 = 1, max_active = 64;
    size_t budget = 0, used = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::map<uint64_t, Done> done;
    std::map<uint64_t, int> state;   // 0 queued, 1 active, 2 done
    uint64_t next_ticket = 1;
    int64_t n_active = 0, completed = 0;
    double site_updates = 0.0;
    double site_updates_issued = 0.0;
    bool stop = false;
    std::thread worker;
    std::vector<Active> active;      // worker thread only
    lq_batch *batch[2] = {nullptr, nullptr};
};

namespace {

lq_status start_solve(lq_server *sv, Active &a) {
    const Request &r = a.req;
    lq_status st = lq_create(&r.lat, &r.mat, sv->fp32 ? LQ_FP32_BULK_FP64_RED : LQ_FP64, nullptr, &a.s);
    if (st != LQ_OK) return st;
    for (const lq_object &o : r.objs) {
        switch (o.type) {
        case LQ_OBJ_WALL: st = lq_add_wall(a.s, o.axis, o.plane, &o.anch); break;
        case LQ_OBJ_SPHERE: st = lq_add_sphere(a.s, o.c, o.R, &o.anch); break;
        case LQ_OBJ_DROPLET: st = lq_add_droplet(a.s, o.c, o.R, &o.anch); break;
        case LQ_OBJ_SPHEROCYLINDER: st = lq_add_spherocylinder(a.s, o.c, o.c2, o.R, &o.anch); break;
        case LQ_OBJ_SITES: st = lq_add_object_sites(a.s, o.n, o.xyz, &o.anch); break;
        case LQ_OBJ_ANCHORED: st = lq_add_anchored_sites(a.s, o.n, o.xyz, o.per_site); break;
        default: st = LQ_EINVAL;
        }
        if (st != LQ_OK) return st;
    }
    if (!r.q0.empty()) st = lq_set_q(a.s, r.q0.data());
    else st = lq_init_random_uniaxial(a.s, r.seed, r.S);
    if (st != LQ_OK) return st;
    return fire_reset(a.s, &r.params);
}

void finish(lq_server *sv, Active &a, lq_status st, bool have_result) {
    Done d;
    d.status = st;
    if (have_result && a.s) {
        if (sync_state(a.s) == LQ_OK) fill_result(a.s, &d.res, 0.0);
        double E;
        if (lq_energy(a.s, &E, nullptr) == LQ_OK) d.res.energy = E;
        if (a.req.want_S) {
            d.S.resize((size_t)a.s->L.N);
            if (lq_order_field(a.s, d.S.data()) != LQ_OK) d.S.clear();
        }
    }
    d.res.seconds = std::chrono::duration<double>(Clock::now() - a.req.t_submit).count();
    double nsites = a.s ? (double)a.s->L.N : 0.0;
    if (a.s) lq_destroy(a.s);
    a.s = nullptr;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->used -= a.req.bytes;
    sv->n_active -= 1;
    sv->completed += 1;
    sv->site_updates += nsites * (double)d.res.iterations;
    sv->state[a.req.ticket] = 2;
    sv->done[a.req.ticket] = std::move(d);
    sv->cv.notify_all();
}

// false when a batch could not be built (retried on the next round)
bool rebuild_batches(lq_server *sv) {
    std::vector<lq_solver *> group[2];
    for (Active &a : sv->active) group[a.s->three ? 1 : 0].push_back(a.s);
    bool ok = true;
    for (int g = 0; g < 2; ++g) {
        if (!sv->batch[g]) {
            if (group[g].empty()) continue;
            if (batch_new(sv->device, sv->fp32, g, &sv->batch[g]) != LQ_OK) { ok = false; continue; }
        }
        if (batch_set_members(sv->batch[g], group[g].data(), (int)group[g].size()) != LQ_OK) ok = false;
    }
    return ok;
}

void worker_loop(lq_server *sv) {
    cudaSetDevice(sv->device);
    bool changed = false;
    int failed_rounds = 0;   // consecutive rounds without a batch or with a failed launch
    for (;;) {
        // admit what the budget and the slot limit allow
        std::vector<Request> admit;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            if (sv->active.empty() && sv->queue.empty())
                sv->cv.wait_for(lk, std::chrono::milliseconds(50));
            if (sv->stop) break;
            while (!sv->queue.empty() && (int)(sv->active.size() + admit.size()) < sv->max_active &&
                   sv->used + sv->queue.front().bytes <= sv->budget) {
                sv->used += sv->queue.front().bytes;
                sv->n_active += 1;
                sv->state[sv->queue.front().ticket] = 1;
                admit.push_back(std::move(sv->queue.front()));
                sv->queue.pop_front();
            }
        }
        for (Request &r : admit) {
            Active a;
            a.req = std::move(r);
            a.t_start = Clock::now();
            lq_status st = start_solve(sv, a);
            if (st != LQ_OK) {
                finish(sv, a, st, false);
                continue;
            }
            sync_state(a.s);
            if (a.s->st_host->status != FIRE_RUNNING) {   // converged at the start
                finish(sv, a, a.s->st_host->status == FIRE_CONVERGED ? LQ_OK : LQ_EDIVERGED, true);
                continue;
            }
            sv->active.push_back(std::move(a));
            changed = true;
        }
        if (sv->active.empty()) continue;
        if (changed) changed = !rebuild_batches(sv);   // a failed build is retried
        if (changed) {
            // no batch for this round: fail everything after repeated failures
            if (++failed_rounds >= 3) {
                for (Active &a : sv->active) finish(sv, a, LQ_ENOMEM, false);
                sv->active.clear();
                failed_rounds = 0;
                changed = true;    // the batches still name the finished solves
            }
            continue;
        }
        // one round of the persistent kernel over every active solve
        long long sites = 0;
        for (Active &a : sv->active) sites += a.s->L.N;
        int k = (int)std::max(1LL, std::min(64LL, (1LL << 27) / std::max(1LL, sites)));
        unsigned int running_total = 0;
        lq_status round_err = LQ_OK;
        for (int g = 0; g < 2; ++g) {
            if (batch_members(sv->batch[g]) == 0) continue;
            unsigned int running = 0;
            lq_status st = batch_round(sv->batch[g], k, &running);
            if (st == LQ_OK) running_total += running;
            else round_err = st;
        }
        if (round_err != LQ_OK) {
            // a round that failed (its lattices stay resident): rebuild and
            // retry; after three failures in a row its solves fail with it
            changed = true;
            if (++failed_rounds >= 3) {
                for (Active &a : sv->active) finish(sv, a, round_err, false);
                sv->active.clear();
                failed_rounds = 0;
            }
            continue;   // changed is set: the next round rebuilds the batches
        }
        failed_rounds = 0;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->site_updates_issued += (double)sites * k;
        }
        // retire the finished and the timed-out
        auto now = Clock::now();
        bool any_done = running_total < sv->active.size();
        std::vector<Active> keep;
        for (Active &a : sv->active) {
            int st = FIRE_RUNNING;
            if (any_done) {
                sync_state(a.s);
                st = a.s->st_host->status;
            }
            double age = std::chrono::duration<double>(now - a.t_start).count();
            if (st == FIRE_CONVERGED) finish(sv, a, LQ_OK, true);
            else if (st == FIRE_MAXITER) finish(sv, a, LQ_ENOTCONVERGED, true);
            else if (st == FIRE_DIVERGED) finish(sv, a, LQ_EDIVERGED, true);
            else if (a.req.params.wall_timeout_s > 0 && age > a.req.params.wall_timeout_s)
                finish(sv, a, LQ_ETIMEOUT, true);
            else keep.push_back(std::move(a));
        }
        if (keep.size() != sv->active.size()) changed = true;
        sv->active = std::move(keep);
    }
    for (Active &a : sv->active)
        if (a.s) lq_destroy(a.s);
    sv->active.clear();
}

lq_status copy_done(lq_server *sv, std::map<uint64_t, Done>::iterator it, lq_result *out,
                    double *S_out) {
    lq_status st = it->second.status;
    if (out) *out = it->second.res;
    if (S_out && !it->second.S.empty())
        std::memcpy(S_out, it->second.S.data(), it->second.S.size() * sizeof(double));
    sv->state.erase(it->first);
    sv->done.erase(it);
    return st;
}

}  // namespace

extern "C" {

lq_status lq_server_create(size_t hbm_budget_bytes, int precision, int max_active, lq_server **out) {
    if (!out || hbm_budget_bytes == 0 || max_active <= 0 ||
        (precision != LQ_FP64 && precision != LQ_FP32_BULK_FP64_RED))
        return LQ_EINVAL;
    lq_server *sv = new lq_server();
    cudaGetDevice(&sv->device);
    sv->fp32 = precision == LQ_FP32_BULK_FP64_RED;
    sv->budget = hbm_budget_bytes;
    sv->max_active = max_active;
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return LQ_OK;
}

void lq_server_destroy(lq_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->device);
    for (int g = 0; g < 2; ++g) lq_batch_destroy(sv->batch[g]);
    delete sv;
}

lq_status lq_server_submit(lq_server *sv, const lq_request *rq, uint64_t *ticket) {
    if (!sv || !rq || !ticket) return LQ_EINVAL;
    const lq_lattice &L = rq->lattice;
    if (L.nx <= 0 || L.ny <= 0 || L.nz <= 0 || rq->n_objects < 0 || (rq->n_objects > 0 && !rq->objects))
        return LQ_EINVAL;
    Request r;
    r.lat = L;
    r.mat = rq->material;
    r.seed = rq->seed;
    r.S = rq->S;
    r.params = rq->params;
    r.want_S = rq->want_order_field;
    long long N = (long long)L.nx * L.ny * L.nz;
    if (rq->q0) r.q0.assign(rq->q0, rq->q0 + 5 * N);
    for (int t = 0; t < rq->n_objects; ++t) {
        lq_object o = rq->objects[t];
        if (o.n < 0 || ((o.type == LQ_OBJ_SITES || o.type == LQ_OBJ_ANCHORED) && o.n > 0 && !o.xyz) ||
            (o.type == LQ_OBJ_ANCHORED && o.n > 0 && !o.per_site))
            return LQ_EINVAL;
        r.xyz.emplace_back();
        r.per_site.emplace_back();
        if (o.xyz) r.xyz.back().assign(o.xyz, o.xyz + 3 * o.n);
        if (o.per_site) r.per_site.back().assign(o.per_site, o.per_site + o.n);
        r.objs.push_back(o);
    }
    for (size_t t = 0; t < r.objs.size(); ++t) {   // point at the owned copies
        r.objs[t].xyz = r.xyz[t].empty() ? nullptr : r.xyz[t].data();
        r.objs[t].per_site = r.per_site[t].empty() ? nullptr : r.per_site[t].data();
    }
    r.bytes = estimate_bytes(L, sv->fp32);
    if (r.bytes > sv->budget) return LQ_ENOMEM;   // could never be admitted
    r.t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    r.ticket = sv->next_ticket++;
    *ticket = r.ticket;
    sv->state[r.ticket] = 0;
    sv->queue.push_back(std::move(r));
    sv->cv.notify_all();
    return LQ_OK;
}

lq_status lq_server_poll(lq_server *sv, uint64_t ticket, lq_result *out, double *S_out) {
    if (!sv) return LQ_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto st = sv->state.find(ticket);
    if (st == sv->state.end()) return LQ_EINVAL;
    if (st->second != 2) return LQ_EBUSY;
    return copy_done(sv, sv->done.find(ticket), out, S_out);
}

lq_status lq_server_wait(lq_server *sv, uint64_t ticket, double timeout_s, lq_result *out,
                         double *S_out) {
    if (!sv) return LQ_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                       std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9));
    for (;;) {
        auto st = sv->state.find(ticket);
        if (st == sv->state.end()) return LQ_EINVAL;
        if (st->second == 2) return copy_done(sv, sv->done.find(ticket), out, S_out);
        if (sv->cv.wait_until(lk, deadline) == std::cv_status::timeout) return LQ_EBUSY;
    }
}

lq_status lq_server_stats_get(lq_server *sv, lq_server_stats *out) {
    if (!sv || !out) return LQ_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    out->queued = (int64_t)sv->queue.size();
    out->active = sv->n_active;
    out->completed = sv->completed;
    out->bytes_in_use = sv->used;
    out->budget = sv->budget;
    out->site_updates = sv->site_updates;
    out->site_updates_issued = sv->site_updates_issued;
    return LQ_OK;
}

}  // extern "C"
