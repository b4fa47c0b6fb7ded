// slab.cu -- one lattice decomposed into z slabs, one per GPU (section
// III.B: the lattice is split into sub-domains with halos, and FIRE's global
// power and norms are sums over every sub-domain).
//
// A slab solver holds planes [z_lo, z_hi) of a lattice and one halo plane
// below and one above (local planes 0 and n + 1, n = z_hi - z_lo), taken
// with the lattice's own periodicity.  Its masks and anchoring records are
// copied from a solver of the whole lattice (whose geometry decides every
// neighbour bit, halo planes included), so a slab evaluates exactly the
// force the whole lattice would at its planes.  One FIRE iteration of the
// decomposed lattice is, on every slab:
//   lq_slab_step    the fused step over the slab's own planes; its last block
//                   leaves the slab's sums (P, |F|^2, |v|^2, largest site
//                   |F|^2) instead of running the FIRE scalar update;
//   (the caller sums the first three over every slab and takes the largest
//   fourth, in FP64)
//   lq_slab_finish  the FIRE scalar update from those totals -- the same on
//                   every slab, so every slab keeps the same dt, alpha, N_pos;
//   lq_slab_get_planes / lq_slab_set_halos  the first and last own planes of
//                   q, v, F go to the neighbouring slabs' halos.
#include <algorithm>
#include <cstring>
#include <vector>

#include "lqmin.h"
#include "lq_common.cuh"
#include "lq_kernels.h"
#include "solver_internal.h"

using namespace lq;
using namespace lq::detail;

#define SK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(s, e_ == cudaErrorMemoryAllocation ? LQ_ENOMEM : LQ_ECUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                    \
    } while (0)

namespace {

long long plane_sites(const lq_solver *s) { return (long long)s->L.nx * s->L.ny; }

// copy the slab's geometry out of the whole lattice's
lq_status copy_geometry(lq_solver *g, lq_solver *s, int z_lo, int z_hi) {
    const long long nxy = plane_sites(g);
    const int n = z_hi - z_lo, ny = g->L.ny, nzg = g->L.nz;
    cudaStream_t st = s->stream;
    // masks of the own and halo planes (a halo beyond an open z edge: no sites)
    for (int zl = 0; zl < n + 2; ++zl) {
        int Z = z_lo - 1 + zl;
        if (Z < 0 || Z >= nzg) Z = g->L.pz ? (Z + nzg) % nzg : -1;
        if (Z < 0) SK(cudaMemsetAsync(s->mask + zl * nxy, 0, (size_t)nxy, st));
        else SK(cudaMemcpyAsync(s->mask + zl * nxy, g->mask + Z * nxy, (size_t)nxy, cudaMemcpyDeviceToDevice, st));
    }
    // anchoring records of the own planes (records are sorted by (z, y) row)
    const long long rows_g = (long long)ny * nzg;
    std::vector<int> start_g(rows_g + 1);
    SK(cudaMemcpyAsync(start_g.data(), g->row_start, sizeof(int) * (rows_g + 1), cudaMemcpyDeviceToHost,
                       g->stream));
    SK(cudaStreamSynchronize(g->stream));
    const int first = start_g[(long long)z_lo * ny], last = start_g[(long long)z_hi * ny];
    const long long rows_s = (long long)ny * (n + 2);
    std::vector<int> start_s(rows_s + 1);
    for (long long r = 0; r < ny; ++r) start_s[r] = 0;                        // lower halo
    for (int zl = 1; zl <= n; ++zl)
        for (int y = 0; y < ny; ++y)
            start_s[(long long)zl * ny + y] = start_g[(long long)(z_lo + zl - 1) * ny + y] - first;
    for (long long r = (long long)(n + 1) * ny; r <= rows_s; ++r) start_s[r] = last - first;   // upper halo
    const size_t rsize = g->fp32 ? sizeof(AnchorRec<float>) : sizeof(AnchorRec<double>);
    const long long cnt = last - first;
    if (s->row_start) cudaFree(s->row_start);
    if (s->rec_x) cudaFree(s->rec_x);
    if (s->recs) cudaFree(s->recs);
    s->row_start = nullptr; s->rec_x = nullptr; s->recs = nullptr;
    SK(dev_malloc(&s->row_start, sizeof(int) * (rows_s + 1)));
    SK(dev_malloc(&s->rec_x, sizeof(int) * std::max<long long>(1, cnt)));
    SK(dev_malloc(&s->recs, rsize * std::max<long long>(1, cnt)));
    SK(cudaMemcpyAsync(s->row_start, start_s.data(), sizeof(int) * (rows_s + 1), cudaMemcpyHostToDevice, st));
    if (cnt > 0) {
        SK(cudaMemcpyAsync(s->rec_x, g->rec_x + first, sizeof(int) * cnt, cudaMemcpyDeviceToDevice, st));
        SK(cudaMemcpyAsync(s->recs, static_cast<const char *>(g->recs) + rsize * first, rsize * cnt,
                           cudaMemcpyDeviceToDevice, st));
    }
    s->nrec = cnt;
    // simulated sites of the own planes
    LatticeDev own = s->L;
    own.nz = n;
    own.N = nxy * n;
    unsigned long long *dcnt = reinterpret_cast<unsigned long long *>(s->out3);
    SK(count_simulated(own, s->mask + nxy, dcnt, st));
    unsigned long long hn = 0;
    SK(cudaMemcpyAsync(&hn, dcnt, sizeof hn, cudaMemcpyDeviceToHost, st));
    void *arrays[6] = {s->q[0], s->v[0], s->F[0], s->q[1], s->v[1], s->F[1]};
    SK(zero_object_sites(s->L, s->mask, arrays, 6, s->fp32, st));
    SK(cudaStreamSynchronize(st));
    s->nsim = (long long)hn;
    s->geom_dirty = false;
    s->fire_ready = false;
    ++s->gen;
    return LQ_OK;
}

lq_status slab_sums(lq_solver *s, double local[4]) {
    lq_status r = sync_state(s);
    if (r != LQ_OK) return r;
    const FireDev &f = *s->st_host;
    local[0] = f.P; local[1] = f.F2; local[2] = f.v2; local[3] = f.r2;
    return LQ_OK;
}

// copy plane zl of (q, v, F) of the current buffer to / from a host buffer
// laid out [array q, v, F][component][site of the plane]
lq_status plane_copy(lq_solver *s, int zl, void *host, bool to_host) {
    const long long nxy = plane_sites(s), N = s->L.N;
    const size_t pb = (size_t)nxy * s->esize;
    void *arr[3] = {s->q[s->cur], s->v[s->cur], s->F[s->cur]};
    char *h = static_cast<char *>(host);
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 5; ++c) {
            char *dev = static_cast<char *>(arr[a]) + ((size_t)c * N + (size_t)zl * nxy) * s->esize;
            char *hp = h + (size_t)(a * 5 + c) * pb;
            if (to_host) SK(cudaMemcpyAsync(hp, dev, pb, cudaMemcpyDeviceToHost, s->stream));
            else SK(cudaMemcpyAsync(dev, hp, pb, cudaMemcpyHostToDevice, s->stream));
        }
    return LQ_OK;
}

}  // namespace

extern "C" {

lq_status lq_slab_create(lq_solver *whole, int z_lo, int z_hi, lq_solver **out) {
    if (!whole || !out) return LQ_EINVAL;
    *out = nullptr;
    lq_solver *g = whole;
    if (check_solver(g)) return LQ_EINVAL;
    if (g->slab) return fail(g, LQ_EINVAL, "a slab is cut from the whole lattice, not from a slab");
    if (z_lo < 0 || z_hi > g->L.nz || z_hi - z_lo < 1)
        return fail(g, LQ_EINVAL, "slab planes [%d, %d) outside [0, %d)", z_lo, z_hi, g->L.nz);
    lq_status r = build_geometry(g);
    if (r != LQ_OK) return r;
    lq_lattice lat{};
    lat.nx = g->L.nx; lat.ny = g->L.ny; lat.nz = z_hi - z_lo + 2;
    lat.spacing = 1.0;
    lat.periodic[0] = g->L.px; lat.periodic[1] = g->L.py; lat.periodic[2] = 0;
    lq_solver *s = nullptr;
    r = lq_create(&lat, &g->mat, g->fp32 ? LQ_FP32_BULK_FP64_RED : LQ_FP64, nullptr, &s);
    if (r != LQ_OK) return fail(g, r, "slab: %s", lq_create_error());
    s->slab = 1;
    s->zchunk = g->zchunk;
    s->idx64 = g->idx64;
    r = copy_geometry(g, s, z_lo, z_hi);
    if (r != LQ_OK) {
        fail(g, r, "slab geometry: %s", s->err.c_str());
        lq_destroy(s);
        return r;
    }
    *out = s;
    return LQ_OK;
}

lq_status lq_slab_start(lq_solver *s, const lq_fire_params *p, double local[4]) {
    if (check_solver(s) || !local) return LQ_EINVAL;
    if (!s->slab) return fail(s, LQ_EINVAL, "not a slab (lq_slab_create)");
    if (s->fire_ready) { lq_status r = sync_state(s); if (r != LQ_OK) return r; }
    lq_status r = fire_reset(s, p);   // F(q0) over the own planes, sums left in the state
    if (r != LQ_OK) return r;
    return slab_sums(s, local);
}

lq_status lq_slab_step(lq_solver *s, double local[4]) {
    if (check_solver(s) || !local) return LQ_EINVAL;
    if (!s->slab) return fail(s, LQ_EINVAL, "not a slab (lq_slab_create)");
    if (!s->fire_ready) return fail(s, LQ_EINVAL, "lq_slab_start has not run");
    StepLaunch sl = make_launch(s, 0);
    SK(launch_fire_step(sl, s->stream));
    return slab_sums(s, local);
}

lq_status lq_slab_finish(lq_solver *s, const double total[4], lq_result *out) {
    if (check_solver(s) || !total) return LQ_EINVAL;
    if (!s->slab) return fail(s, LQ_EINVAL, "not a slab (lq_slab_create)");
    if (!s->fire_ready) return fail(s, LQ_EINVAL, "lq_slab_start has not run");
    SK(fire_apply(s->st, total, s->stream));
    lq_status r = sync_state(s);
    if (r != LQ_OK) return r;
    fill_result(s, out, 0.0);
    return LQ_OK;
}

lq_status lq_slab_plane_bytes(const lq_solver *s, size_t *bytes) {
    if (!s || !bytes) return LQ_EINVAL;
    *bytes = 15 * (size_t)s->L.nx * s->L.ny * s->esize;
    return LQ_OK;
}

lq_status lq_slab_get_planes(lq_solver *s, void *lower, void *upper) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!s->slab) return fail(s, LQ_EINVAL, "not a slab (lq_slab_create)");
    if (lower) { lq_status r = plane_copy(s, 1, lower, true); if (r != LQ_OK) return r; }
    if (upper) { lq_status r = plane_copy(s, s->L.nz - 2, upper, true); if (r != LQ_OK) return r; }
    SK(cudaStreamSynchronize(s->stream));
    return LQ_OK;
}

lq_status lq_slab_set_halos(lq_solver *s, const void *below, const void *above) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!s->slab) return fail(s, LQ_EINVAL, "not a slab (lq_slab_create)");
    if (below) { lq_status r = plane_copy(s, 0, const_cast<void *>(below), false); if (r != LQ_OK) return r; }
    if (above) {
        lq_status r = plane_copy(s, s->L.nz - 1, const_cast<void *>(above), false);
        if (r != LQ_OK) return r;
    }
    SK(cudaStreamSynchronize(s->stream));
    return LQ_OK;
}

}  // extern "C"
