// objects.cu -- object manipulation after creation (section VI: objects
// are moved and the liquid crystal re-minimised, repeated to map a
// potential of mean force; energy terms changed between minimisations),
// solver clones, potential-of-mean-force sweeps run as one batch, the
// custom boundary text format (section VI, custom boundary files) and the
// dipolar initial condition about a colloid (section IV.A).
#include <algorithm>
#include <atomic>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lqmin.h"
#include "lq_common.cuh"
#include "lq_kernels.h"
#include "solver_internal.h"

using namespace lq;
using namespace lq::detail;

namespace lq {

// injected failures: kind and the number of operations of that kind that
// still succeed before the one that fails
static std::atomic<int> g_fault_kind{0};
static std::atomic<long long> g_fault_after{0};

bool fault_due(int kind) {
    if (g_fault_kind.load(std::memory_order_acquire) != kind) return false;
    long long left = g_fault_after.load(std::memory_order_acquire);
    for (;;) {
        if (g_fault_kind.load(std::memory_order_acquire) != kind) return false;
        if (left > 0) {
            if (g_fault_after.compare_exchange_weak(left, left - 1)) return false;
            continue;
        }
        int k = kind;
        return g_fault_kind.compare_exchange_strong(k, 0);   // one-shot
    }
}

}  // namespace lq

namespace {

bool is_integral(double v) { return std::isfinite(v) && v == std::floor(v) && std::fabs(v) < 1e9; }

// ---- boundary text format ---------------------------------------------------

struct Parsed {
    std::vector<HostObject> objects;
    long long sites = 0;
    std::string err;
};

bool parse_kind(const std::string &t, int *kind) {
    if (t == "homeotropic" || t == "0") *kind = LQ_ANCHOR_ND_HOMEOTROPIC;
    else if (t == "oriented" || t == "1") *kind = LQ_ANCHOR_ND_ORIENTED;
    else if (t == "planar" || t == "2") *kind = LQ_ANCHOR_FG_PLANAR;
    else return false;
    return true;
}

bool parse_double(const std::string &t, double *v) {
    if (t.empty()) return false;
    char *end = nullptr;
    *v = std::strtod(t.c_str(), &end);
    return end && *end == '\0' && std::isfinite(*v);
}

bool parse_int(const std::string &t, int32_t *v) {
    if (t.empty()) return false;
    char *end = nullptr;
    long long x = std::strtoll(t.c_str(), &end, 10);
    if (!end || *end != '\0' || x < INT32_MIN || x > INT32_MAX) return false;
    *v = (int32_t)x;
    return true;
}

// tokens of one line, '#' starts a comment
std::vector<std::string> tokens(const std::string &line) {
    std::vector<std::string> out;
    size_t i = 0, n = line.find('#');
    if (n == std::string::npos) n = line.size();
    while (i < n) {
        while (i < n && std::isspace((unsigned char)line[i])) ++i;
        size_t j = i;
        while (j < n && !std::isspace((unsigned char)line[j])) ++j;
        if (j > i) out.push_back(line.substr(i, j - i));
        i = j;
    }
    return out;
}

bool anchoring_ok(const lq_anchoring &a) { return a.W >= 0 && std::isfinite(a.W); }

// the whole text is checked before anything is added
bool parse_boundary(const char *text, Parsed *P) {
    std::string all(text);
    size_t pos = 0;
    int lineno = 0;
    enum { NONE, OBJECT, BOUNDARY } mode = NONE;
    int block_line = 0;
    auto bad = [&](const char *what) {
        char buf[160];
        snprintf(buf, sizeof buf, "line %d: %s", lineno, what);
        P->err = buf;
        return false;
    };
    while (pos <= all.size()) {
        size_t nl = all.find('\n', pos);
        if (nl == std::string::npos) nl = all.size();
        std::string line = all.substr(pos, nl - pos);
        pos = nl + 1;
        ++lineno;
        std::vector<std::string> t = tokens(line);
        if (t.empty()) continue;
        if (mode == NONE) {
            if (t[0] == "object") {
                if (t.size() != 3 && t.size() != 6) return bad("object takes <anchoring> <W> [dx dy dz]");
                HostObject o;
                o.type = 2;
                o.anch.dir[0] = 0; o.anch.dir[1] = 0; o.anch.dir[2] = 1;
                if (!parse_kind(t[1], &o.anch.kind)) return bad("unknown anchoring");
                if (!parse_double(t[2], &o.anch.W) || !anchoring_ok(o.anch)) return bad("bad anchoring strength");
                if (t.size() == 6)
                    for (int k = 0; k < 3; ++k)
                        if (!parse_double(t[3 + k], &o.anch.dir[k])) return bad("bad direction");
                P->objects.push_back(std::move(o));
                mode = OBJECT;
            } else if (t[0] == "boundary") {
                if (t.size() != 1) return bad("boundary takes no arguments");
                HostObject o;
                o.type = 3;
                P->objects.push_back(std::move(o));
                mode = BOUNDARY;
            } else {
                return bad("expected 'object' or 'boundary'");
            }
            block_line = lineno;
            continue;
        }
        if (t[0] == "object" || t[0] == "boundary") return bad("previous block not closed by 'end'");
        if (t[0] == "end") {
            if (t.size() != 1) return bad("end takes no arguments");
            mode = NONE;
            continue;
        }
        HostObject &o = P->objects.back();
        int32_t xyz[3];
        if (mode == OBJECT) {
            if (t.size() != 3) return bad("object site takes x y z");
        } else if (t.size() != 8) {
            return bad("boundary site takes x y z <anchoring> <W> dx dy dz");
        }
        for (int k = 0; k < 3; ++k)
            if (!parse_int(t[k], &xyz[k])) return bad("bad site coordinate");
        o.xyz.insert(o.xyz.end(), xyz, xyz + 3);
        if (mode == BOUNDARY) {
            lq_anchoring a{};
            if (!parse_kind(t[3], &a.kind)) return bad("unknown anchoring");
            if (!parse_double(t[4], &a.W) || !anchoring_ok(a)) return bad("bad anchoring strength");
            for (int k = 0; k < 3; ++k)
                if (!parse_double(t[5 + k], &a.dir[k])) return bad("bad direction");
            o.per_site.push_back(a);
        }
        if (o.xyz.size() / 3 > 0x7fffffffu) return bad("too many sites in one block");
        ++P->sites;
    }
    if (mode != NONE) {
        lineno = block_line;
        return bad("block not closed by 'end'");
    }
    return true;
}

}  // namespace

extern "C" {

lq_status lq_bounds_check_hits(uint32_t *hits) {
    if (!hits) return LQ_EINVAL;
    unsigned int h = 0;
    int r = bounds_hits(&h);
    *hits = h;
    return r == 1 ? LQ_OK : (r == 0 ? LQ_EINVAL : LQ_ECUDA);
}

lq_status lq_inject_fault(int kind, int64_t after) {
    if (kind < LQ_FAULT_NONE || kind > LQ_FAULT_COPY_WAIT || after < 0) return LQ_EINVAL;
    g_fault_kind.store(LQ_FAULT_NONE, std::memory_order_release);
    g_fault_after.store(after, std::memory_order_release);
    g_fault_kind.store(kind, std::memory_order_release);
    return LQ_OK;
}

lq_status lq_frank_to_landau(double K1, double K2, double K3, double K24, double q0, double S,
                             double L[5]) {
    if (!L || !(S > 0) || !std::isfinite(S) || !std::isfinite(K1) || !std::isfinite(K2) ||
        !std::isfinite(K3) || !std::isfinite(K24) || !std::isfinite(q0))
        return LQ_EINVAL;
    double s2 = S * S;
    L[0] = 2.0 * (K3 - K1 + 3.0 * K2) / (27.0 * s2);
    L[1] = 4.0 * (K1 - K24) / (9.0 * s2);
    L[2] = 4.0 * (K24 - K2) / (9.0 * s2);
    L[3] = -8.0 * q0 * K2 / (9.0 * s2);
    L[4] = 4.0 * (K3 - K1) / (27.0 * s2 * S);
    return LQ_OK;
}

lq_status lq_set_material(lq_solver *s, const lq_material *mat) {
    if (check_solver(s)) return LQ_EINVAL;
    if (s->slab) return fail(s, LQ_EINVAL, "a slab takes its geometry and material from the whole lattice");
    if (!mat) return fail(s, LQ_EINVAL, "null material");
    double S0 = 0;
    if (const char *why = validate_material(mat, &S0)) return fail(s, LQ_EINVAL, "%s", why);
    if (s->fire_ready) {
        lq_status r = sync_state(s);
        if (r != LQ_OK) return r;
    }
    int three = mat->n_constants == 3;
    if (three != s->three) {
        cudaError_t e = prepare_fire_step(s->fp32, three);
        if (e != cudaSuccess) return fail(s, LQ_ECUDA, "lq_set_material: %s", cudaGetErrorString(e));
    }
    s->mat = *mat;
    s->S0 = S0;
    s->three = three;
    s->ext = three && (mat->L4 != 0.0 || mat->L6 != 0.0);
    drop_graph(s);
    // anchoring records hold Q0 = 3/2 S0 (nu nu - I/3): rebuilt on next use
    s->geom_dirty = true;
    s->fire_ready = false;
    ++s->gen;
    return ensure_partials(s);
}

lq_status lq_object_count(lq_solver *s, int *n) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!n) return fail(s, LQ_EINVAL, "null output");
    *n = (int)s->objects.size();
    return LQ_OK;
}

lq_status lq_move_object(lq_solver *s, int index, const double shift[3]) {
    if (check_solver(s)) return LQ_EINVAL;
    if (s->slab) return fail(s, LQ_EINVAL, "a slab takes its geometry and material from the whole lattice");
    if (!shift || index < 0 || index >= (int)s->objects.size()) return fail(s, LQ_EINVAL, "no object %d", index);
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(shift[k])) return fail(s, LQ_EINVAL, "shift must be finite");
    HostObject &o = s->objects[index];
    int n[3] = {s->L.nx, s->L.ny, s->L.nz}, per[3] = {s->L.px, s->L.py, s->L.pz};
    switch (o.type) {
    case 0:
        if (!is_integral(shift[o.axis])) return fail(s, LQ_EINVAL, "a wall moves by whole lattice planes");
        o.plane += (int)shift[o.axis];
        if (per[o.axis]) o.plane = ((o.plane % n[o.axis]) + n[o.axis]) % n[o.axis];
        break;
    case 1: case 4: case 5:
        for (int k = 0; k < 3; ++k) { o.c[k] += shift[k]; o.c2[k] += shift[k]; }
        break;
    default: {   // site lists move by whole lattice vectors, wrapping periodic axes
        for (int k = 0; k < 3; ++k)
            if (!is_integral(shift[k])) return fail(s, LQ_EINVAL, "site lists move by whole lattice vectors");
        for (size_t t = 0; t < o.xyz.size(); ++t) {
            int k = (int)(t % 3);
            long long v = (long long)o.xyz[t] + (long long)shift[k];
            if (per[k]) v = ((v % n[k]) + n[k]) % n[k];
            if (v < INT32_MIN || v > INT32_MAX) return fail(s, LQ_EINVAL, "site moved out of range");
            o.xyz[t] = (int32_t)v;
        }
    }
    }
    s->geom_dirty = true;
    s->fire_ready = false;
    return LQ_OK;
}

lq_status lq_clear_objects(lq_solver *s) {
    if (check_solver(s)) return LQ_EINVAL;
    if (s->slab) return fail(s, LQ_EINVAL, "a slab takes its geometry and material from the whole lattice");
    s->objects.clear();
    s->geom_dirty = true;
    s->fire_ready = false;
    return LQ_OK;
}

lq_status lq_clone(lq_solver *src, void *cuda_stream, lq_solver **out) {
    if (check_solver(src) || !out) return LQ_EINVAL;
    *out = nullptr;
    if (src->slab) return fail(src, LQ_EINVAL, "a slab is cut from the whole lattice (lq_slab_create)");
    lq_status r = build_geometry(src);
    if (r != LQ_OK) return r;
    if (src->fire_ready) {
        r = sync_state(src);
        if (r != LQ_OK) return r;
    }
    lq_lattice lat{};
    lat.nx = src->L.nx; lat.ny = src->L.ny; lat.nz = src->L.nz;
    lat.spacing = 1.0;
    lat.periodic[0] = src->L.px; lat.periodic[1] = src->L.py; lat.periodic[2] = src->L.pz;
    lq_solver *d = nullptr;
    r = lq_create(&lat, &src->mat, src->fp32 ? LQ_FP32_BULK_FP64_RED : LQ_FP64, cuda_stream, &d);
    if (r != LQ_OK) return fail(src, r, "clone: %s", lq_create_error());
    d->objects = src->objects;
    d->zchunk = src->zchunk;
    d->geom_dirty = true;
    r = build_geometry(d);
    if (r == LQ_OK) {
        // the source's state is complete once its stream is idle
        cudaError_t e = cudaStreamSynchronize(src->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d->q[d->cur], src->q[src->cur], 5 * (size_t)src->L.N * src->esize,
                                cudaMemcpyDeviceToDevice, d->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
        if (e != cudaSuccess) r = fail(src, LQ_ECUDA, "clone: %s", cudaGetErrorString(e));
    } else {
        fail(src, r, "clone: %s", d->err.c_str());
    }
    if (r != LQ_OK) {
        lq_destroy(d);
        return r;
    }
    d->fire_ready = false;
    *out = d;
    return LQ_OK;
}

lq_status lq_pmf_sweep(lq_solver *base, int index, int n, const double *shifts, const lq_fire_params *p,
                       lq_result *out) {
    if (check_solver(base)) return LQ_EINVAL;
    if (n <= 0 || !shifts || !p) return fail(base, LQ_EINVAL, "bad sweep arguments");
    if (index < 0 || index >= (int)base->objects.size()) return fail(base, LQ_EINVAL, "no object %d", index);
    lq_status r = check_params(base, p);
    if (r != LQ_OK) return r;
    std::vector<lq_solver *> members;
    auto cleanup = [&]() {
        for (lq_solver *m : members) lq_destroy(m);
    };
    for (int k = 0; k < n; ++k) {
        lq_solver *m = nullptr;
        r = lq_clone(base, nullptr, &m);
        if (r != LQ_OK) { cleanup(); return r; }
        members.push_back(m);
        r = lq_move_object(m, index, shifts + 3 * k);
        if (r == LQ_OK) r = build_geometry(m);
        if (r != LQ_OK) {
            fail(base, r, "sweep position %d: %s", k, m->err.c_str());
            cleanup();
            return r;
        }
    }
    lq_batch *b = nullptr;
    r = lq_batch_create(members.data(), n, &b);
    if (r != LQ_OK) {
        fail(base, r, "sweep batch: could not create");
        cleanup();
        return r;
    }
    r = lq_batch_minimize(b, p, out);
    if (r != LQ_OK && r != LQ_ENOTCONVERGED && r != LQ_ETIMEOUT && r != LQ_EDIVERGED)
        fail(base, r, "sweep batch: %s", lq_batch_last_error(b));
    lq_batch_destroy(b);
    cleanup();
    return r;
}

lq_status lq_boundary_check(const char *text, int64_t *n_blocks, int64_t *n_sites, char *err, size_t errlen) {
    if (err && errlen) err[0] = '\0';
    if (!text) return LQ_EINVAL;
    Parsed P;
    bool ok = parse_boundary(text, &P);
    if (!ok) {
        if (err && errlen) snprintf(err, errlen, "%s", P.err.c_str());
        return LQ_EINVAL;
    }
    if (n_blocks) *n_blocks = (int64_t)P.objects.size();
    if (n_sites) *n_sites = P.sites;
    return LQ_OK;
}

lq_status lq_add_boundary_text(lq_solver *s, const char *text) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!text) return fail(s, LQ_EINVAL, "null text");
    Parsed P;
    if (!parse_boundary(text, &P)) return fail(s, LQ_EINVAL, "boundary text: %s", P.err.c_str());
    size_t before = s->objects.size();
    for (HostObject &o : P.objects) {
        lq_status r = add_object(s, std::move(o));
        if (r != LQ_OK) {
            s->objects.resize(before);
            return r;
        }
    }
    return LQ_OK;
}

lq_status lq_load_boundary_file(lq_solver *s, const char *path) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!path) return fail(s, LQ_EINVAL, "null path");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(s, LQ_EINVAL, "cannot open %s", path);
    std::string text;
    char buf[1 << 16];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    if (text.find('\0') != std::string::npos) return fail(s, LQ_EINVAL, "%s: not a text file", path);
    return lq_add_boundary_text(s, text.c_str());
}

lq_status lq_init_dipolar(lq_solver *s, const double c[3], const double axis[3], double rd, double S) {
    if (check_solver(s)) return LQ_EINVAL;
    if (!c || !axis) return fail(s, LQ_EINVAL, "null argument");
    double an = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
    if (!(an > 0) || !std::isfinite(an) || !(rd > 0) || !std::isfinite(rd))
        return fail(s, LQ_EINVAL, "dipolar start needs a non-zero axis and rd > 0");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(c[k])) return fail(s, LQ_EINVAL, "centre must be finite");
    lq_status r = build_geometry(s);
    if (r != LQ_OK) return r;
    if (s->fire_ready) {
        r = sync_state(s);
        if (r != LQ_OK) return r;
    }
    double Sv = S > 0 ? S : s->S0;
    if (s->fp32 && !(1.5 * Sv < QFIX_LIMIT)) return fail(s, LQ_EINVAL, "S outside the FP32 form's range");
    double a[3] = {axis[0] / an, axis[1] / an, axis[2] / an};
    cudaError_t e = init_dipolar(s->L, s->mask, c, a, rd, Sv, s->q[s->cur], s->fp32, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return fail(s, LQ_ECUDA, "init_dipolar: %s", cudaGetErrorString(e));
    s->fire_ready = false;
    return LQ_OK;
}

}  // extern "C"
