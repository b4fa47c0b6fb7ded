// solver_internal.h -- the solver object and host helpers shared by the C
// interface files (solver.cu, batch.cu).  Not part of the public interface.
#pragma once

#include <string>
#include <vector>

#include "lqmin.h"
#include "lq_common.cuh"
#include "lq_kernels.h"

namespace lq {
namespace detail {

struct HostObject {
    int type;                       // 0 wall, 1 sphere, 2 object sites, 3 anchored sites,
                                    // 4 droplet, 5 spherocylinder
    int axis = 0, plane = 0;
    double c[3] = {0, 0, 0}, R = 0;
    double c2[3] = {0, 0, 0};       // spherocylinder: second end of the axis
    lq_anchoring anch{};
    std::vector<int32_t> xyz;
    std::vector<lq_anchoring> per_site;
};

}  // namespace detail
}  // namespace lq

struct lq_solver {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;        // created by lq_create when given NULL
    int fp32 = 0, three = 0;
    int ext = 0;                    // chiral / cubic terms on (three-constant form)
    lq::LatticeDev L{};
    lq_material mat{};
    double S0 = 0;
    size_t esize = 8;

    std::vector<lq::detail::HostObject> objects;
    bool geom_dirty = true;
    unsigned long long gen = 0;     // bumped when device geometry or material change
                                    // (batches rebuild their kernel arguments)

    uint8_t *mask = nullptr;
    int *row_start = nullptr, *rec_x = nullptr;
    void *recs = nullptr;
    long long nrec = 0, nsim = 0;

    void *q[2] = {nullptr, nullptr}, *v[2] = {nullptr, nullptr}, *F[2] = {nullptr, nullptr};
    double *xfer = nullptr;         // 5 N doubles for conversions and readback
    lq::FireDev *st = nullptr;
    lq::FireDev *st_host = nullptr;     // pinned mirror
    double *partials = nullptr;
    int partials_cap = 0;
    double *out3 = nullptr;

    int cur = 0;                    // buffer holding the state (host view)
    bool fire_ready = false;
    int zchunk = 0;                 // 0 = automatic
    int idx64 = 0;                  // 64-bit element indices forced (lq_set_index_width)
    int staging = 0;                // lq_set_staging: 0 automatic, 1 loads, 2 tensor copies
    int slab = 0;                   // a z slab of a decomposed lattice (lq_slab_create): its own
                                    // planes are 1 .. nz-2, planes 0 and nz-1 are halos

    cudaGraphExec_t gexec = nullptr;
    int graph_k = 0;
    size_t bytes = 0;
    std::string err;
};

namespace lq {
namespace detail {

lq_status fail(lq_solver *s, lq_status st, const char *fmt, ...);
lq_status check_solver(lq_solver *s);
// material checks shared by lq_create and lq_set_material; S0 from Eq. (S0def)
// unless given; returns a message or nullptr
const char *validate_material(const lq_material *m, double *S0);
lq_status add_object(lq_solver *s, HostObject &&o);
void drop_graph(lq_solver *s);
lq_status ensure_partials(lq_solver *s);
int effective_zchunk(const lq_solver *s);
StepLaunch make_launch(lq_solver *s, int force_only);
lq_status build_geometry(lq_solver *s);
lq_status check_params(lq_solver *s, const lq_fire_params *p);
void fill_params(FireDev &f, const lq_fire_params *p);
lq_status sync_state(lq_solver *s);
void fill_result(lq_solver *s, lq_result *out, double seconds);
lq_status fire_reset(lq_solver *s, const lq_fire_params *p);
lq_status update_params(lq_solver *s, const lq_fire_params *p);

// batches (batch.cu): an empty batch for one device / precision / form, its
// lattices replaced in place, and k persistent-kernel iterations
lq_status batch_new(int device, int fp32, int three, lq_batch **out);
lq_status batch_set_members(lq_batch *b, lq_solver *const *solvers, int n);
lq_status batch_round(lq_batch *b, int k, unsigned int *running);
int batch_members(const lq_batch *b);

}  // namespace detail
}  // namespace lq
