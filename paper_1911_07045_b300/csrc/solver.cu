// solver.cu -- the C interface of include/lqmin.h: solver lifetime, object
// geometry, state transfer, the FIRE driver (CUDA graphs of fused steps with
// device-side convergence flags) and readback.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lqmin.h"
#include "lq_common.cuh"
#include "lq_kernels.h"
#include "solver_internal.h"

using namespace lq;

namespace {

thread_local std::string g_create_error;



}  // namespace



namespace lq {
namespace detail {

lq_status fail(lq_solver *s, lq_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    else g_create_error = buf;
    return st;
}

#define CK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return fail(s, e_ == cudaErrorMemoryAllocation ? LQ_ENOMEM : LQ_ECUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

int auto_zchunk(const lq_solver *s) {
    int tx, ty;
    step_tile(s->fp32, s->three, s->L.nx, &tx, &ty);
    long long tiles = (long long)((s->L.nx + tx - 1) / tx) * ((s->L.ny + ty - 1) / ty);
    // enough blocks for several waves on 148 SMs, marches of at most 128
    // planes (measured best at 512^3), at least 8 planes to amortise the halo
    long long want = 148LL * 16;
    long long chunks = std::max(1LL, (want + tiles - 1) / tiles);
    int zc = (int)((s->L.nz + chunks - 1) / chunks);
    zc = std::min(zc, 128);
    return std::max(zc, std::min(8, s->L.nz));
}

int effective_zchunk(const lq_solver *s) { return s->zchunk > 0 ? s->zchunk : auto_zchunk(s); }

// the force of the external fields, the same at every site: f_ext =
// -(1/3) K:Q with K = mu0_dchi H H^T + eps0_deps E E^T, so F = (1/3) J^T K
void field_tensor(const lq_material &m, double K[3][3]) {
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) K[a][b] = m.mu0_dchi * m.H[a] * m.H[b] + m.eps0_deps * m.E[a] * m.E[b];
}
void field_force(const lq_material &m, double f[5]) {
    double K[3][3];
    field_tensor(m, K);
    f[0] = (K[0][0] - K[2][2]) / 3.0;
    f[1] = 2.0 * K[0][1] / 3.0;
    f[2] = 2.0 * K[0][2] / 3.0;
    f[3] = (K[1][1] - K[2][2]) / 3.0;
    f[4] = 2.0 * K[1][2] / 3.0;
}

StepLaunch make_launch(lq_solver *s, int force_only) {
    StepLaunch sl;
    for (int b = 0; b < 2; ++b) { sl.q[b] = s->q[b]; sl.v[b] = s->v[b]; sl.F[b] = s->F[b]; }
    sl.Fonly = s->F[s->cur ^ 1];
    sl.qonly = s->q[s->cur];
    sl.g.mask = s->mask;
    sl.g.row_start = s->row_start;
    sl.g.rec_x = s->rec_x;
    sl.g.recs = s->recs;
    sl.L = s->L;
    sl.A = s->mat.A; sl.B = s->mat.B; sl.C = s->mat.C;
    sl.L1 = s->mat.L1; sl.L2 = s->mat.L2; sl.L3 = s->mat.L3; sl.S0 = s->S0;
    sl.L4 = s->mat.L4; sl.L6 = s->mat.L6;
    field_force(s->mat, sl.fext);
    sl.st = s->st;
    sl.partials = s->partials;
    sl.zchunk = effective_zchunk(s);
    sl.force_only = force_only;
    sl.fp32 = s->fp32;
    sl.three = s->three;
    sl.ext = s->ext;
    sl.idx64 = s->idx64;
    sl.wide = wide_tiles(s->fp32, s->three, s->L.nx);
    sl.tma = s->staging == 2 && s->fp32 && s->three && !s->ext && tma_staging_fits(s->L) &&
             tma_staging_available();
    if (s->slab) {            // own planes only; the FIRE update waits for every slab's sums
        sl.zbeg = 1;
        sl.zend = s->L.nz - 1;
        sl.reduce_only = 1;
    }
    return sl;
}

void drop_graph(lq_solver *s);

lq_status ensure_partials(lq_solver *s) {
    int tx, ty;
    step_tile(s->fp32, s->three, s->L.nx, &tx, &ty);
    dim3 g = step_grid(s->L, effective_zchunk(s), tx, ty);
    int need = std::max<int>(g.x * g.y * g.z, 148 * 64);
    if (need > s->partials_cap) {
        drop_graph(s);  // captured launches hold the old pointer
        if (s->partials) cudaFree(s->partials);
        s->partials = nullptr;
        CK(dev_malloc(&s->partials, sizeof(double) * 4 * (size_t)need));
        s->partials_cap = need;
    }
    return LQ_OK;
}

void drop_graph(lq_solver *s) {
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    s->gexec = nullptr;
    s->graph_k = 0;
}

lq_status build_geometry(lq_solver *s) {
    if (!s->geom_dirty) return LQ_OK;
    drop_graph(s);   // captured launches hold the record tables freed below
    ++s->gen;
    const LatticeDev &L = s->L;
    cudaStream_t st = s->stream;
    int nobj = (int)s->objects.size();

    std::vector<GeoObjDev> hobj(std::max(1, nobj));
    std::vector<void *> temps;
    auto cleanup = [&]() {
        for (void *p : temps) cudaFree(p);
    };
    bool any_anch = false;
    for (int o = 0; o < nobj; ++o) {
        const HostObject &h = s->objects[o];
        GeoObjDev &d = hobj[o];
        memset(&d, 0, sizeof d);
        d.type = h.type; d.axis = h.axis; d.plane = h.plane;
        for (int k = 0; k < 3; ++k) { d.c[k] = h.c[k]; d.c2[k] = h.c2[k]; }
        d.R = h.R;
        d.spec.kind = h.anch.kind; d.spec.W = h.anch.W;
        for (int k = 0; k < 3; ++k) d.spec.dir[k] = h.anch.dir[k];
        d.n = (long long)h.xyz.size() / 3;
        if (d.n > 0) {
            int32_t *dx = nullptr;
            cudaError_t e = dev_malloc(&dx, h.xyz.size() * sizeof(int32_t));
            if (e != cudaSuccess) { cleanup(); return fail(s, LQ_ENOMEM, "geometry: %s", cudaGetErrorString(e)); }
            temps.push_back(dx);
            cudaMemcpyAsync(dx, h.xyz.data(), h.xyz.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
            d.xyz = dx;
        }
        if (h.type == 3) {
            any_anch = true;
            std::vector<AnchorSpecDev> ps(h.per_site.size());
            for (size_t t = 0; t < ps.size(); ++t) {
                ps[t].kind = h.per_site[t].kind; ps[t].W = h.per_site[t].W;
                for (int k = 0; k < 3; ++k) ps[t].dir[k] = h.per_site[t].dir[k];
            }
            AnchorSpecDev *dp = nullptr;
            cudaError_t e = dev_malloc(&dp, std::max<size_t>(1, ps.size()) * sizeof(AnchorSpecDev));
            if (e != cudaSuccess) { cleanup(); return fail(s, LQ_ENOMEM, "geometry: %s", cudaGetErrorString(e)); }
            temps.push_back(dp);
            cudaMemcpyAsync(dp, ps.data(), ps.size() * sizeof(AnchorSpecDev), cudaMemcpyHostToDevice, st);
            // the host vector must outlive the copy
            cudaStreamSynchronize(st);
            d.per_site = dp;
        }
    }
    GeoObjDev *dobj = nullptr;
    int *owner = nullptr;
    unsigned long long *xclaim = nullptr;
    int *counts = nullptr;
    cudaError_t e;
#define GK(call)                                                                          \
    do {                                                                                  \
        e = (call);                                                                       \
        if (e != cudaSuccess) {                                                           \
            cleanup();                                                                    \
            return fail(s, e == cudaErrorMemoryAllocation ? LQ_ENOMEM : LQ_ECUDA,         \
                        "geometry: %s: %s", #call, cudaGetErrorString(e));                \
        }                                                                                 \
    } while (0)
    GK(dev_malloc(&dobj, sizeof(GeoObjDev) * hobj.size()));
    temps.push_back(dobj);
    GK(cudaMemcpyAsync(dobj, hobj.data(), sizeof(GeoObjDev) * hobj.size(), cudaMemcpyHostToDevice, st));
    GK(dev_malloc(&owner, sizeof(int) * L.N));
    temps.push_back(owner);
    if (any_anch) {
        GK(dev_malloc(&xclaim, sizeof(unsigned long long) * L.N));
        temps.push_back(xclaim);
        GK(cudaMemsetAsync(xclaim, 0xff, sizeof(unsigned long long) * L.N, st));
    }
    GK(geo_owner(L, dobj, nobj, owner, st));
    for (int o = 0; o < nobj; ++o) {
        if (hobj[o].type == 2) GK(geo_scatter_sites(L, hobj[o].xyz, hobj[o].n, o, owner, st));
        if (hobj[o].type == 3) GK(geo_scatter_anchored(L, hobj[o].xyz, hobj[o].n, o, xclaim, st));
    }
    GK(geo_mask(L, owner, xclaim, s->mask, st));
    long long rows = (long long)L.ny * L.nz;
    GK(dev_malloc(&counts, sizeof(int) * rows));
    temps.push_back(counts);
    GK(geo_row_count(L, s->mask, counts, st));
    std::vector<int> hc(rows), hstart(rows + 1);
    GK(cudaMemcpyAsync(hc.data(), counts, sizeof(int) * rows, cudaMemcpyDeviceToHost, st));
    GK(cudaStreamSynchronize(st));
    long long acc = 0;
    for (long long r = 0; r < rows; ++r) { hstart[r] = (int)acc; acc += hc[r]; }
    hstart[rows] = (int)acc;
    if (acc > 0x7fffffffLL) { cleanup(); return fail(s, LQ_EINVAL, "too many anchored sites"); }
    if (s->row_start) cudaFree(s->row_start);
    if (s->rec_x) cudaFree(s->rec_x);
    if (s->recs) cudaFree(s->recs);
    s->row_start = nullptr; s->rec_x = nullptr; s->recs = nullptr;
    size_t rsize = s->fp32 ? sizeof(AnchorRec<float>) : sizeof(AnchorRec<double>);
    GK(dev_malloc(&s->row_start, sizeof(int) * (rows + 1)));
    GK(dev_malloc(&s->rec_x, sizeof(int) * std::max<long long>(1, acc)));
    GK(dev_malloc(&s->recs, rsize * std::max<long long>(1, acc)));
    GK(cudaMemcpyAsync(s->row_start, hstart.data(), sizeof(int) * (rows + 1), cudaMemcpyHostToDevice, st));
    GK(geo_fill(L, s->mask, owner, xclaim, dobj, s->S0, s->row_start, s->rec_x, s->recs, s->fp32, st));
    s->nrec = acc;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(s->out3);
    GK(count_simulated(L, s->mask, cnt, st));
    unsigned long long hn = 0;
    GK(cudaMemcpyAsync(&hn, cnt, sizeof hn, cudaMemcpyDeviceToHost, st));
    GK(cudaStreamSynchronize(st));
    s->nsim = (long long)hn;
    void *arrays[6] = {s->q[0], s->v[0], s->F[0], s->q[1], s->v[1], s->F[1]};
    GK(zero_object_sites(L, s->mask, arrays, 6, s->fp32, st));
    GK(cudaStreamSynchronize(st));
#undef GK
    cleanup();
    s->geom_dirty = false;
    s->fire_ready = false;
    return LQ_OK;
}

lq_status check_params(lq_solver *s, const lq_fire_params *p) {
    if (!p) return fail(s, LQ_EINVAL, "null minimiser parameters");
    if (p->method < LQ_MIN_FIRE || p->method > LQ_MIN_NESTEROV)
        return fail(s, LQ_EINVAL, "unknown minimiser %d", p->method);
    if (!(p->dt0 > 0) || !std::isfinite(p->dt0) || p->max_iter < 0 || !(p->force_tol >= 0))
        return fail(s, LQ_EINVAL, "invalid minimiser parameters");
    if (p->method == LQ_MIN_FIRE &&
        (!(p->dt_max >= p->dt0) || !(p->alpha0 >= 0 && p->alpha0 <= 1) ||
         !(p->f_alpha > 0 && p->f_alpha <= 1) || !(p->f_inc >= 1) || !(p->f_dec > 0 && p->f_dec <= 1) ||
         p->n_min < 0))
        return fail(s, LQ_EINVAL, "invalid FIRE parameters");
    if (p->method == LQ_MIN_NESTEROV && !(p->momentum >= 0 && p->momentum < 1))
        return fail(s, LQ_EINVAL, "Nesterov momentum must be in [0, 1)");
    return LQ_OK;
}

void fill_params(FireDev &f, const lq_fire_params *p) {
    f.dt0 = p->dt0; f.dt_max = p->dt_max; f.alpha0 = p->alpha0; f.f_alpha = p->f_alpha;
    f.f_inc = p->f_inc; f.f_dec = p->f_dec; f.tol = p->force_tol;
    f.n_min = p->n_min; f.max_iter = p->max_iter;
    f.method = p->method;
    f.eta = p->dt0;
    f.mu = p->method == LQ_MIN_NESTEROV ? p->momentum : 0.0;
}

lq_status sync_state(lq_solver *s) {
    CK(cudaMemcpyAsync(s->st_host, s->st, sizeof(FireDev), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->cur = s->st_host->cur;
    return LQ_OK;
}

void fill_result(lq_solver *s, lq_result *out, double seconds) {
    if (!out) return;
    const FireDev &f = *s->st_host;
    memset(out, 0, sizeof *out);
    out->iterations = f.iter;
    out->max_force = std::sqrt(f.r2);
    out->norm_force = std::sqrt(f.F2);
    out->norm_velocity = std::sqrt(f.v2);
    out->rms_force = s->nsim > 0 ? std::sqrt(f.F2 / (double)s->nsim) : 0.0;
    out->power = f.P;
    out->dt = f.method == LQ_MIN_FIRE ? f.dt : f.eta;
    out->alpha = f.alpha;
    out->npos = f.npos;
    out->fire_status = f.status;
    out->energy = NAN;
    out->seconds = seconds;
}

lq_status launch_steps(lq_solver *s, int64_t n);

lq_status fire_reset(lq_solver *s, const lq_fire_params *p) {
    lq_status r = check_params(s, p);
    if (r != LQ_OK) return r;
    r = build_geometry(s);
    if (r != LQ_OK) return r;
    r = ensure_partials(s);
    if (r != LQ_OK) return r;
    FireDev &f = *s->st_host;
    memset(&f, 0, sizeof f);
    fill_params(f, p);
    f.dt = p->dt0;
    f.alpha = p->alpha0;
    f.status = FIRE_RUNNING;
    f.cur = s->cur;
    f.cv = 0.0; f.cF = 0.0; f.dt_step = 0.0;
    f.nsim = s->nsim;
    CK(cudaMemcpyAsync(s->st, &f, sizeof f, cudaMemcpyHostToDevice, s->stream));
    size_t bytes = 5 * (size_t)s->L.N * s->esize;
    CK(cudaMemsetAsync(s->v[s->cur], 0, bytes, s->stream));
    CK(cudaMemsetAsync(s->F[s->cur], 0, bytes, s->stream));
    StepLaunch sl = make_launch(s, 0);
    CK(launch_fire_step(sl, s->stream));   // F(q0)
    CK(cudaStreamSynchronize(s->stream));  // the pinned mirror is reused below
    s->fire_ready = true;
    return LQ_OK;
}

int graph_len(const lq_solver *s) {
    long long k = (1LL << 24) / std::max<long long>(1, s->L.N);
    return (int)std::max(1LL, std::min(128LL, k));
}

lq_status ensure_graph(lq_solver *s) {
    int k = graph_len(s);
    if (s->gexec && s->graph_k == k) return LQ_OK;
    drop_graph(s);
    StepLaunch sl = make_launch(s, 0);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < k && e == cudaSuccess; ++t) e = launch_fire_step(sl, s->stream);
    cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(s, LQ_ECUDA, "graph capture: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&s->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(s, LQ_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    s->graph_k = k;
    return LQ_OK;
}

lq_status launch_steps(lq_solver *s, int64_t n) {
    if (n <= 0) return LQ_OK;
    lq_status r = ensure_graph(s);
    if (r != LQ_OK) return r;
    int64_t full = n / s->graph_k, rest = n % s->graph_k;
    for (int64_t t = 0; t < full; ++t) CK(cudaGraphLaunch(s->gexec, s->stream));
    StepLaunch sl = make_launch(s, 0);
    for (int64_t t = 0; t < rest; ++t) CK(launch_fire_step(sl, s->stream));
    return LQ_OK;
}

lq_status update_params(lq_solver *s, const lq_fire_params *p) {
    lq_status r = sync_state(s);
    if (r != LQ_OK) return r;
    // another minimiser restarts from the current Q
    if (s->st_host->method != p->method) return fire_reset(s, p);
    FireDev f = *s->st_host;
    fill_params(f, p);
    if (f.method != LQ_MIN_FIRE && f.kcount >= 1) {
        // a new step or momentum applies from the next step on
        f.cv = f.mu; f.cF = f.eta; f.dt_step = f.eta;
        f.c_alpha = f.mu * f.mu;
        f.c_beta = f.eta * (1.0 + f.mu);
        f.c_kick = 0.0;
    }
    if (f.status == FIRE_MAXITER && f.iter < f.max_iter) f.status = FIRE_RUNNING;
    if (f.status == FIRE_CONVERGED && std::sqrt(f.r2) >= f.tol) f.status = FIRE_RUNNING;
    *s->st_host = f;
    CK(cudaMemcpyAsync(s->st, s->st_host, sizeof(FireDev), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LQ_OK;
}

lq_status check_solver(lq_solver *s) {
    if (!s) return LQ_EINVAL;
    cudaSetDevice(s->device);
    return LQ_OK;
}

const char *validate_material(const lq_material *m, double *S0) {
    if (m->n_constants != 1 && m->n_constants != 3) return "n_constants must be 1 or 3";
    if (m->n_constants == 1 && (m->L2 != 0.0 || m->L3 != 0.0 || m->L4 != 0.0 || m->L6 != 0.0))
        return "one-constant form needs L2 = L3 = L4 = L6 = 0";
    double disc = m->B * m->B - 24.0 * m->A * m->C;
    double s0 = m->S0;
    if (!(s0 > 0)) {
        if (!(m->C > 0) || disc < 0) return "no nematic minimum for these A, B, C";
        s0 = (-m->B + std::sqrt(disc)) / (6.0 * m->C);  // Eq. (S0def)
    }
    *S0 = s0;
    return nullptr;
}

lq_status add_object(lq_solver *s, HostObject &&o) {
    if (s->slab) return fail(s, LQ_EINVAL, "a slab takes its geometry from the whole lattice");
    if (o.type != 3) {
        const lq_anchoring &a = o.anch;
        if (a.kind < 0 || a.kind > 2 || !(a.W >= 0)) return fail(s, LQ_EINVAL, "bad anchoring");
    }
    if (s->objects.size() >= 0x7ffffff0u) return fail(s, LQ_EINVAL, "too many objects");
    s->objects.push_back(std::move(o));
    s->geom_dirty = true;
    s->fire_ready = false;
    return LQ_OK;
}

lq_status copy_out_state(lq_solver *s, const void *src, double *out, bool is_q = false) {
    size_t n = 5 * (size_t)s->L.N;
    if (s->fp32) {
        if (is_q) CK(q_export(src, s->xfer, (long long)n, 1, s->stream));
        else CK(state_to_f64(src, s->xfer, (long long)n, 1, s->stream));
        CK(cudaMemcpyAsync(out, s->xfer, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    } else {
        CK(cudaMemcpyAsync(out, src, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    }
    CK(cudaStreamSynchronize(s->stream));
    return LQ_OK;
}

}  // namespace detail
}  // namespace lq

using namespace lq::detail;

// ---- C interface ---------------------------------------------------------------

extern "C" {

const char *lq_create_error(void) { return g_create_error.c_str(); }

const char *lq_last_error(const lq_solver *s) { return s ? s->err.c_str() : "null solver"; }

lq_status lq_create(const lq_lattice *lat, const lq_material *mat, int precision,
                    void *cuda_stream, lq_solver **out) {
    lq_solver *s = nullptr;
    if (!lat || !mat || !out) return fail(s, LQ_EINVAL, "null argument");
    *out = nullptr;
    if (lat->nx <= 0 || lat->ny <= 0 || lat->nz <= 0) return fail(s, LQ_EINVAL, "lattice sizes must be positive");
    if (lat->spacing != 1.0) return fail(s, LQ_EINVAL, "spacing must be 1 (lattice units)");
    double S0 = 0;
    if (const char *why = validate_material(mat, &S0)) return fail(s, LQ_EINVAL, "%s", why);
    if (precision != LQ_FP64 && precision != LQ_FP32_BULK_FP64_RED) return fail(s, LQ_EINVAL, "bad precision");
    long long N = (long long)lat->nx * lat->ny * lat->nz;
    if ((long long)lat->ny * lat->nz + 1 > 0x7fffffffLL) return fail(s, LQ_EINVAL, "lattice too large");

    s = new lq_solver();
    cudaGetDevice(&s->device);
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    if (!s->stream) {
        // CUDA graphs cannot capture the legacy default stream: own a stream
        cudaError_t es = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (es != cudaSuccess) {
            g_create_error = std::string("lq_create: ") + cudaGetErrorString(es);
            delete s;
            return LQ_ECUDA;
        }
        s->own_stream = true;
    }
    s->fp32 = precision == LQ_FP32_BULK_FP64_RED;
    s->three = mat->n_constants == 3;
    s->ext = s->three && (mat->L4 != 0.0 || mat->L6 != 0.0);
    s->esize = s->fp32 ? sizeof(float) : sizeof(double);
    s->L.nx = lat->nx; s->L.ny = lat->ny; s->L.nz = lat->nz;
    s->L.px = lat->periodic[0] ? 1 : 0; s->L.py = lat->periodic[1] ? 1 : 0;
    s->L.pz = lat->periodic[2] ? 1 : 0;
    s->L.N = N;
    s->mat = *mat;
    s->S0 = S0;

    auto bad = [&](cudaError_t e) {
        g_create_error = std::string("lq_create: ") + cudaGetErrorString(e);
        lq_destroy(s);
        return e == cudaErrorMemoryAllocation ? LQ_ENOMEM : LQ_ECUDA;
    };
    size_t sb = 5 * (size_t)N * s->esize;
    cudaError_t e;
    for (int b = 0; b < 2; ++b) {
        if ((e = dev_malloc(&s->q[b], sb)) != cudaSuccess) return bad(e);
        if ((e = dev_malloc(&s->v[b], sb)) != cudaSuccess) return bad(e);
        if ((e = dev_malloc(&s->F[b], sb)) != cudaSuccess) return bad(e);
        if ((e = cudaMemsetAsync(s->q[b], 0, sb, s->stream)) != cudaSuccess) return bad(e);
        if ((e = cudaMemsetAsync(s->v[b], 0, sb, s->stream)) != cudaSuccess) return bad(e);
        if ((e = cudaMemsetAsync(s->F[b], 0, sb, s->stream)) != cudaSuccess) return bad(e);
    }
    if ((e = dev_malloc(&s->mask, (size_t)N)) != cudaSuccess) return bad(e);
    if ((e = dev_malloc(&s->xfer, 5 * (size_t)N * sizeof(double))) != cudaSuccess) return bad(e);
    if ((e = dev_malloc(&s->st, sizeof(FireDev))) != cudaSuccess) return bad(e);
    if ((e = cudaMemsetAsync(s->st, 0, sizeof(FireDev), s->stream)) != cudaSuccess) return bad(e);
    if ((e = dev_malloc(&s->out3, 4 * sizeof(double))) != cudaSuccess) return bad(e);
    if ((e = cudaMallocHost(&s->st_host, sizeof(FireDev))) != cudaSuccess) return bad(e);
    memset(s->st_host, 0, sizeof(FireDev));
    if ((e = prepare_fire_step(s->fp32, s->three)) != cudaSuccess) return bad(e);
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return bad(e);
    s->bytes = 6 * sb + (size_t)N + 5 * (size_t)N * sizeof(double);
    *out = s;
    return LQ_OK;
}

void lq_destroy(lq_solver *s) {
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    drop_graph(s);
    for (int b = 0; b < 2; ++b) { cudaFree(s->q[b]); cudaFree(s->v[b]); cudaFree(s->F[b]); }
    cudaFree(s->mask); cudaFree(s->row_start); cudaFree(s->rec_x); cudaFree(s->recs);
    cudaFree(s->xfer); cudaFree(s->st); cudaFree(s->partials); cudaFree(s->out3);
    if (s->st_host) cudaFreeHost(s->st_host);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

lq_status lq_add_wall(lq_solver *s, int axis, int plane, const lq_anchoring *a) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!a || axis < 0 || axis > 2) return fail(s, LQ_EINVAL, "bad wall");
    HostObject o;
    o.type = 0; o.axis = axis; o.plane = plane; o.anch = *a;
    return add_object(s, std::move(o));
}

lq_status lq_add_sphere(lq_solver *s, const double c[3], double radius, const lq_anchoring *a) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!a || !c || !(radius >= 0)) return fail(s, LQ_EINVAL, "bad sphere");
    HostObject o;
    o.type = 1; o.R = radius; o.anch = *a;
    for (int k = 0; k < 3; ++k) o.c[k] = c[k];
    return add_object(s, std::move(o));
}

lq_status lq_add_droplet(lq_solver *s, const double c[3], double radius, const lq_anchoring *a) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!a || !c || !(radius > 0)) return fail(s, LQ_EINVAL, "bad droplet");
    HostObject o;
    o.type = 4; o.R = radius; o.anch = *a;
    for (int k = 0; k < 3; ++k) o.c[k] = c[k];
    return add_object(s, std::move(o));
}

lq_status lq_add_spherocylinder(lq_solver *s, const double p0[3], const double p1[3], double radius,
                                const lq_anchoring *a) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!a || !p0 || !p1 || !(radius >= 0)) return fail(s, LQ_EINVAL, "bad spherocylinder");
    HostObject o;
    o.type = 5; o.R = radius; o.anch = *a;
    for (int k = 0; k < 3; ++k) { o.c[k] = p0[k]; o.c2[k] = p1[k]; }
    return add_object(s, std::move(o));
}

lq_status lq_add_object_sites(lq_solver *s, int64_t n, const int32_t *xyz, const lq_anchoring *a) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!a || n < 0 || (n > 0 && !xyz) || n > 0x7fffffff) return fail(s, LQ_EINVAL, "bad site list");
    HostObject o;
    o.type = 2; o.anch = *a;
    o.xyz.assign(xyz, xyz + 3 * n);
    return add_object(s, std::move(o));
}

lq_status lq_add_anchored_sites(lq_solver *s, int64_t n, const int32_t *xyz, const lq_anchoring *per) {
    if (check_solver(s)) return LQ_EINVAL;
    if (n < 0 || (n > 0 && (!xyz || !per)) || n > 0x7fffffff) return fail(s, LQ_EINVAL, "bad anchored list");
    HostObject o;
    o.type = 3;
    o.xyz.assign(xyz, xyz + 3 * n);
    o.per_site.assign(per, per + n);
    for (const lq_anchoring &a : o.per_site)
        if (a.kind < 0 || a.kind > 2 || !(a.W >= 0)) return fail(s, LQ_EINVAL, "bad anchoring in list");
    return add_object(s, std::move(o));
}

lq_status lq_geometry_info(lq_solver *s, int64_t *n_sim, int64_t *n_anch) {
    if (check_solver(s)) return LQ_EINVAL;
    lq_status r = build_geometry(s);
    if (r != LQ_OK) return r;
    if (n_sim) *n_sim = s->nsim;
    if (n_anch) *n_anch = s->nrec;
    return LQ_OK;
}

lq_status lq_get_mask(lq_solver *s, uint8_t *out) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!out) return fail(s, LQ_EINVAL, "null output");
    lq_status r = build_geometry(s);
    if (r != LQ_OK) return r;
    CK(cudaMemcpyAsync(out, s->mask, (size_t)s->L.N, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LQ_OK;
}

static lq_status after_set_q(lq_solver *s, bool check_range) {
    if (check_range) {
        unsigned int bad = 0;
        CK(cudaMemcpyAsync(&bad, s->out3, sizeof bad, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        if (bad)
            return fail(s, LQ_EINVAL, "%u Q components outside |q| < %g (FP32 form fixed-point range)",
                        bad, QFIX_LIMIT);
    }
    void *arrays[1] = {s->q[s->cur]};
    CK(zero_object_sites(s->L, s->mask, arrays, 1, s->fp32, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->fire_ready = false;
    return LQ_OK;
}

lq_status lq_set_q(lq_solver *s, const double *qh) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!qh) return fail(s, LQ_EINVAL, "null input");
    lq_status r = build_geometry(s);
    if (r != LQ_OK) return r;
    if (s->fire_ready) { r = sync_state(s); if (r != LQ_OK) return r; }
    size_t n = 5 * (size_t)s->L.N;
    unsigned int *err = reinterpret_cast<unsigned int *>(s->out3);
    if (s->fp32) {
        CK(cudaMemcpyAsync(s->xfer, qh, n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        CK(q_import(s->xfer, 0, s->q[s->cur], (long long)n, 1, err, s->stream));
    } else {
        CK(cudaMemcpyAsync(s->q[s->cur], qh, n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    }
    return after_set_q(s, s->fp32 != 0);
}

lq_status lq_set_q_device(lq_solver *s, const void *dptr, int dtype) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!dptr || (dtype != 0 && dtype != 1)) return fail(s, LQ_EINVAL, "bad device input");
    lq_status r = build_geometry(s);
    if (r != LQ_OK) return r;
    if (s->fire_ready) { r = sync_state(s); if (r != LQ_OK) return r; }
    long long n = 5 * s->L.N;
    unsigned int *err = reinterpret_cast<unsigned int *>(s->out3);
    CK(q_import(dptr, dtype, s->q[s->cur], n, s->fp32, err, s->stream));
    return after_set_q(s, s->fp32 != 0);
}

lq_status lq_init_random_uniaxial(lq_solver *s, uint64_t seed, double S) {
    if (check_solver(s)) return LQ_EINVAL;
    lq_status r = build_geometry(s);
    if (r != LQ_OK) return r;
    if (s->fire_ready) { r = sync_state(s); if (r != LQ_OK) return r; }
    double Sv = S > 0 ? S : s->S0;
    if (s->fp32 && !(1.5 * Sv < QFIX_LIMIT)) return fail(s, LQ_EINVAL, "S outside the FP32 form's range");
    CK(init_random_uniaxial(s->L, s->mask, seed, Sv, s->q[s->cur], s->fp32, s->stream));
    return after_set_q(s, false);
}

lq_status lq_get_q(lq_solver *s, double *out) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!out) return fail(s, LQ_EINVAL, "null output");
    lq_status r = build_geometry(s);
    if (r != LQ_OK) return r;
    if (s->fire_ready) { r = sync_state(s); if (r != LQ_OK) return r; }
    return copy_out_state(s, s->q[s->cur], out, true);
}

lq_status lq_get_force(lq_solver *s, double *out) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!out) return fail(s, LQ_EINVAL, "null output");
    if (!s->fire_ready) return fail(s, LQ_EINVAL, "FIRE has not started");
    lq_status r = sync_state(s);
    if (r != LQ_OK) return r;
    return copy_out_state(s, s->F[s->cur], out);
}

lq_status lq_get_velocity(lq_solver *s, double *out) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!out) return fail(s, LQ_EINVAL, "null output");
    if (!s->fire_ready) return fail(s, LQ_EINVAL, "FIRE has not started");
    lq_status r = sync_state(s);
    if (r != LQ_OK) return r;
    size_t n = 5 * (size_t)s->L.N;
    CK(mixed_velocity(s->v[s->cur], s->F[s->cur], s->st, s->xfer, (long long)n, s->fp32, s->stream));
    CK(cudaMemcpyAsync(out, s->xfer, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LQ_OK;
}

lq_status lq_force(lq_solver *s, double *out) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!out) return fail(s, LQ_EINVAL, "null output");
    lq_status r = build_geometry(s);
    if (r != LQ_OK) return r;
    if (s->fire_ready) { r = sync_state(s); if (r != LQ_OK) return r; }
    // the inactive buffer's F is free between steps; the next step rewrites it
    StepLaunch sl = make_launch(s, 1);
    CK(cudaMemsetAsync(sl.Fonly, 0, 5 * (size_t)s->L.N * s->esize, s->stream));
    CK(launch_fire_step(sl, s->stream));
    return copy_out_state(s, sl.Fonly, out);
}

lq_status lq_energy(lq_solver *s, double *total, double parts[3]) {
    if (check_solver(s)) return LQ_EINVAL;
    lq_status r = build_geometry(s);
    if (r != LQ_OK) return r;
    if (s->fire_ready) { r = sync_state(s); if (r != LQ_OK) return r; }
    r = ensure_partials(s);
    if (r != LQ_OK) return r;
    Geometry g{s->mask, s->row_start, s->rec_x, s->recs};
    double Kf[3][3];
    field_tensor(s->mat, Kf);
    EnergyExtra ex{s->mat.L4, s->mat.L6, {Kf[0][0], Kf[0][1], Kf[0][2], Kf[1][1], Kf[1][2], Kf[2][2]}};
    CK(energy_parts(s->L, g, s->q[s->cur], s->fp32, s->mat.A, s->mat.B, s->mat.C, s->mat.L1,
                    s->mat.L2, s->mat.L3, s->S0, ex, s->partials, s->partials_cap, s->out3, s->stream));
    double h[3];
    CK(cudaMemcpyAsync(h, s->out3, sizeof h, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (parts) { parts[0] = h[0]; parts[1] = h[1]; parts[2] = h[2]; }
    if (total) *total = (h[0] + h[1]) + h[2];
    return LQ_OK;
}

lq_status lq_order_field(lq_solver *s, double *S_out) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!S_out) return fail(s, LQ_EINVAL, "null output");
    lq_status r = build_geometry(s);
    if (r != LQ_OK) return r;
    if (s->fire_ready) { r = sync_state(s); if (r != LQ_OK) return r; }
    CK(order_field(s->L, s->mask, s->q[s->cur], s->fp32, s->xfer, s->stream));
    CK(cudaMemcpyAsync(S_out, s->xfer, (size_t)s->L.N * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LQ_OK;
}

lq_status lq_fire_reset(lq_solver *s, const lq_fire_params *p) {
    if (check_solver(s)) return LQ_EINVAL;
    if (s->slab) return fail(s, LQ_EINVAL, "a slab starts FIRE through lq_slab_start");
    if (s->fire_ready) { lq_status r = sync_state(s); if (r != LQ_OK) return r; }
    return fire_reset(s, p);
}

lq_status lq_step(lq_solver *s, const lq_fire_params *p, int64_t n, lq_result *out) {
    if (check_solver(s)) return LQ_EINVAL;
    if (s->slab) return fail(s, LQ_EINVAL, "a slab steps through lq_slab_step and lq_slab_finish");
    if (n < 0) return fail(s, LQ_EINVAL, "negative step count");
    auto t0 = std::chrono::steady_clock::now();
    lq_status r = check_params(s, p);
    if (r != LQ_OK) return r;
    if (s->geom_dirty || !s->fire_ready) {
        r = fire_reset(s, p);
    } else {
        r = update_params(s, p);
    }
    if (r != LQ_OK) return r;
    r = launch_steps(s, n);
    if (r != LQ_OK) return r;
    r = sync_state(s);
    if (r != LQ_OK) return r;
    fill_result(s, out, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    if (s->st_host->status == FIRE_STALLED)
        return fail(s, LQ_ECUDA, "a tensor copy of the step did not complete (FIRE stopped)");
    return LQ_OK;
}

lq_status lq_fire_result(lq_solver *s, lq_result *out) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!out) return fail(s, LQ_EINVAL, "null output");
    lq_status r = sync_state(s);
    if (r != LQ_OK) return r;
    fill_result(s, out, 0.0);
    return LQ_OK;
}

lq_status lq_minimize(lq_solver *s, const lq_fire_params *p, lq_result *out) {
    if (check_solver(s)) return LQ_EINVAL;
    if (s->slab) return fail(s, LQ_EINVAL, "a slab steps through lq_slab_step and lq_slab_finish");
    auto t0 = std::chrono::steady_clock::now();
    if (s->fire_ready) { lq_status r = sync_state(s); if (r != LQ_OK) return r; }
    lq_status r = fire_reset(s, p);
    if (r != LQ_OK) return r;
    r = ensure_graph(s);
    if (r != LQ_OK) return r;
    // two graphs in flight; each poll reads the status of the older one
    FireDev *ring = nullptr;
    CK(cudaMallocHost(&ring, 2 * sizeof(FireDev)));
    cudaEvent_t ev[2];
    cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
    lq_status ret = LQ_OK;
    auto issue = [&](int slot) -> cudaError_t {
        cudaError_t e = cudaGraphLaunch(s->gexec, s->stream);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(&ring[slot], s->st, sizeof(FireDev), cudaMemcpyDeviceToHost, s->stream);
        if (e != cudaSuccess) return e;
        return cudaEventRecord(ev[slot], s->stream);
    };
    int slot = 0;
    cudaError_t e = issue(0);
    bool timed_out = false;
    while (e == cudaSuccess) {
        e = issue(slot ^ 1);
        if (e != cudaSuccess) break;
        e = cudaEventSynchronize(ev[slot]);
        if (e != cudaSuccess) break;
        if (ring[slot].status != FIRE_RUNNING) break;
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (p->wall_timeout_s > 0 && el > p->wall_timeout_s) { timed_out = true; break; }
        slot ^= 1;
    }
    cudaError_t es = cudaStreamSynchronize(s->stream);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    cudaFreeHost(ring);
    if (e != cudaSuccess || es != cudaSuccess)
        return fail(s, LQ_ECUDA, "minimize: %s", cudaGetErrorString(e != cudaSuccess ? e : es));
    r = sync_state(s);
    if (r != LQ_OK) return r;
    if (timed_out && s->st_host->status == FIRE_RUNNING) ret = LQ_ETIMEOUT;
    else if (s->st_host->status == FIRE_MAXITER) ret = LQ_ENOTCONVERGED;
    else if (s->st_host->status == FIRE_DIVERGED) ret = LQ_EDIVERGED;
    else if (s->st_host->status == FIRE_STALLED) ret = LQ_ECUDA;
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    fill_result(s, out, secs);
    if (out) {
        double E;
        if (lq_energy(s, &E, nullptr) == LQ_OK) out->energy = E;
    }
    if (ret == LQ_ETIMEOUT) fail(s, ret, "wall-clock limit reached");
    if (ret == LQ_ENOTCONVERGED) fail(s, ret, "max_iter reached");
    if (ret == LQ_EDIVERGED) fail(s, ret, "FIRE diverged (non-finite reduction)");
    if (ret == LQ_ECUDA) fail(s, ret, "a tensor copy of the step did not complete (FIRE stopped)");
    return ret;
}

// checkpoint: header + q, v, F of the current buffer in the storage type
struct StateHeader {
    uint64_t magic;
    int64_t nx, ny, nz;
    int32_t fp32, fire_ready;
    FireDev fire;
};
static const uint64_t STATE_MAGIC = 0x4c514d494e535432ull;  // "LQMINST2"

lq_status lq_get_state(lq_solver *s, void *buf, size_t *bytes) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!bytes) return fail(s, LQ_EINVAL, "null size");
    size_t arr = 5 * (size_t)s->L.N * s->esize;
    size_t need = sizeof(StateHeader) + 3 * arr;
    if (!buf) { *bytes = need; return LQ_OK; }
    if (*bytes < need) return fail(s, LQ_EINVAL, "buffer too small (%zu < %zu)", *bytes, need);
    lq_status r = build_geometry(s);
    if (r != LQ_OK) return r;
    if (s->fire_ready) { r = sync_state(s); if (r != LQ_OK) return r; }
    StateHeader h;
    memset(&h, 0, sizeof h);
    h.magic = STATE_MAGIC;
    h.nx = s->L.nx; h.ny = s->L.ny; h.nz = s->L.nz;
    h.fp32 = s->fp32;
    h.fire_ready = s->fire_ready;
    h.fire = *s->st_host;
    char *p = static_cast<char *>(buf);
    memcpy(p, &h, sizeof h);
    CK(cudaMemcpyAsync(p + sizeof h, s->q[s->cur], arr, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(p + sizeof h + arr, s->v[s->cur], arr, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(p + sizeof h + 2 * arr, s->F[s->cur], arr, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    *bytes = need;
    return LQ_OK;
}

lq_status lq_set_state(lq_solver *s, const void *buf, size_t bytes) {
    if (check_solver(s)) return LQ_EINVAL;
    size_t arr = 5 * (size_t)s->L.N * s->esize;
    if (!buf || bytes < sizeof(StateHeader) + 3 * arr) return fail(s, LQ_EINVAL, "state too small");
    StateHeader h;
    memcpy(&h, buf, sizeof h);
    if (h.magic != STATE_MAGIC || h.nx != s->L.nx || h.ny != s->L.ny || h.nz != s->L.nz || h.fp32 != s->fp32)
        return fail(s, LQ_EINVAL, "state does not match this solver");
    lq_status r = build_geometry(s);
    if (r != LQ_OK) return r;
    r = ensure_partials(s);
    if (r != LQ_OK) return r;
    if (s->fire_ready) { r = sync_state(s); if (r != LQ_OK) return r; }
    const char *p = static_cast<const char *>(buf);
    CK(cudaMemcpyAsync(s->q[s->cur], p + sizeof h, arr, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->v[s->cur], p + sizeof h + arr, arr, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->F[s->cur], p + sizeof h + 2 * arr, arr, cudaMemcpyHostToDevice, s->stream));
    FireDev f = h.fire;
    f.cur = s->cur;
    f.counter = 0;
    f.nsim = s->nsim;
    *s->st_host = f;
    CK(cudaMemcpyAsync(s->st, s->st_host, sizeof f, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->fire_ready = h.fire_ready != 0;
    return LQ_OK;
}

lq_status lq_set_zchunk(lq_solver *s, int zchunk) {
    if (check_solver(s)) return LQ_EINVAL;
    if (zchunk < 0) return fail(s, LQ_EINVAL, "zchunk must be >= 0");
    if (s->fire_ready) { lq_status r = sync_state(s); if (r != LQ_OK) return r; }
    s->zchunk = zchunk;
    drop_graph(s);
    return ensure_partials(s);
}

lq_status lq_set_index_width(lq_solver *s, int bits) {
    if (check_solver(s)) return LQ_EINVAL;
    if (bits != 0 && bits != 64) return fail(s, LQ_EINVAL, "index width must be 0 (automatic) or 64");
    if (s->fire_ready) { lq_status r = sync_state(s); if (r != LQ_OK) return r; }
    s->idx64 = bits == 64;
    ++s->gen;          // batches pick their kernel instantiation again
    drop_graph(s);
    return LQ_OK;
}

lq_status lq_set_staging(lq_solver *s, int mode) {
    if (check_solver(s)) return LQ_EINVAL;
    if (mode < 0 || mode > 2) return fail(s, LQ_EINVAL, "staging mode must be 0, 1 or 2");
    if (mode == 2 && !(s->fp32 && s->three && !s->ext && tma_staging_fits(s->L) && tma_staging_available()))
        return fail(s, LQ_EINVAL,
                    "tensor-copy staging needs the FP32 form, three constants without the chiral or cubic "
                    "terms, an x extent that is a multiple of 32 and a driver with the tensor-map encoder");
    if (mode != s->staging) {
        s->staging = mode;
        drop_graph(s);       // captured launches name the kernel of the old mode
    }
    return LQ_OK;
}

lq_status lq_get_staging(lq_solver *s, int *uses_tensor_copies) {
    if (check_solver(s) || !uses_tensor_copies) return LQ_EINVAL;
    *uses_tensor_copies = make_launch(s, 0).tma;
    return LQ_OK;
}

size_t lq_device_bytes(const lq_solver *s) { return s ? s->bytes : 0; }

}  // extern "C"
