// lq_kernels.h -- host-side entry points of the kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lq_common.cuh"

namespace lq {

struct StepLaunch {
    void *q[2], *v[2], *F[2];
    void *Fonly;
    const void *qonly;
    Geometry g;
    LatticeDev L;
    double A, B, C, L1, L2, L3, S0;
    double L4, L6, fext[5];
    int ext;                  // the chiral / cubic terms are on (three-constant form)
    FireDev *st;
    double *partials;
    int zchunk, force_only, fp32, three;
    int idx64;                // 64-bit element indices even where 32 bits would do
    int wide;                 // 64-wide tiles (wide_tiles)
    int tma;                  // FP32 form: plane rows staged by tensor copies
    int zbeg = 0, zend = 0;   // planes updated (zend 0: all); a slab owns [zbeg, zend)
    int reduce_only = 0;      // slab: the sums stay in the FIRE state (fire_apply)
};

// one block's share of a batched step: lattice, tile, z range, and its
// number among that lattice's nblk blocks (the single-lattice numbering)
struct WorkItem {
    int lattice, bx, by, z0, z1, nblk, bid, pad;
};

dim3 step_grid(const LatticeDev &L, int zchunk, int tx, int ty);
bool wide_tiles(int fp32, int three, int nx);
// tensor-copy staging of the FP32 form: the driver offers the tensor-map
// encoder; the lattice's x extent is a multiple of 32
bool tma_staging_available();
bool tma_staging_fits(const LatticeDev &L);
void step_tile(int fp32, int three, int nx, int *tx, int *ty);
cudaError_t prepare_fire_step(int fp32, int three);
cudaError_t launch_fire_step(const StepLaunch &sl, cudaStream_t stream);
// the FIRE scalar update with sums taken over every slab of a lattice
cudaError_t fire_apply(FireDev *st, const double sums[4], cudaStream_t stream);

// true when the state arrays of a lattice of N sites are indexed in 32 bits
bool step_index32(long long N);

// host-side fault injection (lq_inject_fault): true once when an injected
// failure of this kind (1 device allocation, 2 step-kernel launch) is due
bool fault_due(int kind);
// bounds-checked build: index checks of the step kernels that failed since
// load (returns 1; 0 and *out = 0 in the release build; -1 on a CUDA error)
int bounds_hits(unsigned int *out);
// cudaMalloc, or cudaErrorMemoryAllocation without allocating when an
// injected allocation failure is due
template <typename P>
inline cudaError_t dev_malloc(P **p, size_t bytes) {
    if (fault_due(1)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}

// batched steps (tile 32 x ty, ty in {4, 8}; form 0 one-constant, 1
// three-constant, 2 with the chiral / cubic terms; idx32: every lattice of
// the batch indexed in 32 bits)
size_t step_args_bytes(int fp32);
void step_args_pack(const StepLaunch &sl, void *out);   // host memory, step_args_bytes()
// batch tiles tx x ty: tx 32 in every form, 64 for one-constant FP32 lattices
bool batch_tile_ok(int fp32, int form, int tx);
cudaError_t prepare_fire_batch(int fp32, int form, int tx, int ty, int idx32);
int fire_batch_blocks_per_sm(int fp32, int form, int tx, int ty, int idx32);
cudaError_t launch_fire_batch(int fp32, int form, int tx, int ty, int idx32, const void *dev_args,
                              const WorkItem *items, int nitems, int grid, cudaStream_t stream);
// running[0] = number of lattices whose FIRE status is still running
cudaError_t batch_running(FireDev *const *states, int n, unsigned int *running, cudaStream_t s);

// geometry construction (device)
struct AnchorSpecDev {
    int kind;
    double W;
    double dir[3];
};
struct GeoObjDev {
    int type;                 // 0 wall, 1 sphere, 2 object sites, 3 anchored sites,
                              // 4 droplet (outside a ball), 5 spherocylinder
    int axis, plane;
    double c[3], R;
    double c2[3];             // spherocylinder: second end of the axis segment
    AnchorSpecDev spec;
    const int32_t *xyz;       // device copy of a site list
    long long n;
    const AnchorSpecDev *per_site;
};
cudaError_t geo_owner(const LatticeDev &L, const GeoObjDev *objs_dev, int nobj, int *owner,
                      cudaStream_t s);
cudaError_t geo_scatter_sites(const LatticeDev &L, const int32_t *xyz, long long n, int id,
                              int *owner, cudaStream_t s);
cudaError_t geo_scatter_anchored(const LatticeDev &L, const int32_t *xyz, long long n, int id,
                                 unsigned long long *xclaim, cudaStream_t s);
cudaError_t geo_mask(const LatticeDev &L, const int *owner, const unsigned long long *xclaim,
                     uint8_t *mask, cudaStream_t s);
cudaError_t geo_row_count(const LatticeDev &L, const uint8_t *mask, int *counts, cudaStream_t s);
cudaError_t geo_fill(const LatticeDev &L, const uint8_t *mask, const int *owner,
                     const unsigned long long *xclaim, const GeoObjDev *objs_dev, double S0,
                     const int *row_start, int *rec_x, void *recs, int fp32, cudaStream_t s);

// state helpers
cudaError_t zero_object_sites(const LatticeDev &L, const uint8_t *mask, void *const *arrays,
                              int narrays, int fp32, cudaStream_t s);
// Q into / out of the state format (FP32 form: fixed point, range errors
// counted in *err); v and F out as doubles
cudaError_t q_import(const void *src, int src_f32, void *dst, long long n, int fp32,
                     unsigned int *err, cudaStream_t s);
cudaError_t q_export(const void *src, double *dst, long long n, int fp32, cudaStream_t s);
cudaError_t state_to_f64(const void *src, double *dst, long long n, int fp32, cudaStream_t s);
// out = cv v + cF F (the velocity after the pending FIRE mixing), as doubles
cudaError_t mixed_velocity(const void *v, const void *F, const FireDev *st, double *out,
                           long long n, int fp32, cudaStream_t s);
cudaError_t init_random_uniaxial(const LatticeDev &L, const uint8_t *mask, unsigned long long seed,
                                 double S, void *q, int fp32, cudaStream_t s);
// dipolar start about a colloid (centre c, unit far-field axis a, hyperbolic
// hedgehog at c + rd a), Q = 3/2 S (n n - I/3) on simulated sites
cudaError_t init_dipolar(const LatticeDev &L, const uint8_t *mask, const double c[3], const double a[3],
                         double rd, double S, void *q, int fp32, cudaStream_t s);
cudaError_t count_simulated(const LatticeDev &L, const uint8_t *mask, unsigned long long *out,
                            cudaStream_t s);

// readback
// chiral and cubic constants and the field tensor K (xx, xy, xz, yy, yz, zz)
// of the energy readback
struct EnergyExtra {
    double L4, L6;
    double K[6];
};
cudaError_t energy_parts(const LatticeDev &L, const Geometry &g, const void *q, int fp32,
                         double A, double B, double C, double L1, double L2, double L3, double S0,
                         const EnergyExtra &ex, double *partials, int max_blocks, double *out3,
                         cudaStream_t s);
cudaError_t order_field(const LatticeDev &L, const uint8_t *mask, const void *q, int fp32,
                        double *S_out, cudaStream_t s);

}  // namespace lq
