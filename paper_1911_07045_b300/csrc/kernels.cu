// kernels.cu -- geometry construction, state conversion and readback kernels
// (off the per-iteration path).
//
// Geometry (section III.B: an integer type per site; section V: walls,
// spheres and custom site lists).  Object sites are the union of all objects.
// A simulated site with an object site as face neighbour, or named by an
// explicit anchoring list, is a boundary site; its anchoring comes from the
// first object added among those that touch or name it.  Object ids are the
// order of addition, so "first added" is the minimum id.
#include <cmath>

#include "lq_common.cuh"
#include "lq_kernels.h"

namespace lq {

constexpr int NO_OWNER = 0x7fffffff;
constexpr unsigned long long NO_CLAIM = ~0ull;

static inline int blocks_for(long long n, int nt) {
    long long b = (n + nt - 1) / nt;
    return (int)(b > 148LL * 64 ? 148LL * 64 : (b < 1 ? 1 : b));
}

__device__ __forceinline__ void site_xyz(const LatticeDev &L, long long i, int &x, int &y, int &z) {
    x = (int)(i % L.nx);
    long long r = i / L.nx;
    y = (int)(r % L.ny);
    z = (int)(r / L.ny);
}

// neighbour one step along axis k (dir +1/-1), -1 beyond a non-periodic edge
__device__ __forceinline__ long long nbr(const LatticeDev &L, int x, int y, int z, int k, int dir) {
    int c[3] = {x, y, z};
    int n[3] = {L.nx, L.ny, L.nz};
    int p[3] = {L.px, L.py, L.pz};
    c[k] += dir;
    if (c[k] < 0 || c[k] >= n[k]) {
        if (!p[k]) return -1;
        c[k] = (c[k] + n[k]) % n[k];
    }
    return ((long long)c[2] * L.ny + c[1]) * L.nx + c[0];
}

__device__ __forceinline__ double min_image(double d, int n, int periodic) {
    if (periodic) d -= n * floor(d / n + 0.5);
    return d;
}

// |d|^2 summed in x, y, z order with every product rounded (no contraction),
// so that sites on an object's surface are classified like the host geometry
__device__ __forceinline__ double norm2_rn(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// offset of site (x, y, z) from the nearest point of the segment o.c .. o.c2:
// d = site - midpoint (minimum image), a = c2 - c, nearest point at
// midpoint + t a with t = clamp(d.a / a.a, -1/2, 1/2)
__device__ void capsule_offset(const LatticeDev &L, const GeoObjDev &o, int x, int y, int z, double r[3]) {
    double m[3];
    for (int k = 0; k < 3; ++k) m[k] = __dmul_rn(__dadd_rn(o.c[k], o.c2[k]), 0.5);
    double d[3] = {min_image(x - m[0], L.nx, L.px), min_image(y - m[1], L.ny, L.py),
                   min_image(z - m[2], L.nz, L.pz)};
    double a[3] = {o.c2[0] - o.c[0], o.c2[1] - o.c[1], o.c2[2] - o.c[2]};
    double aa = norm2_rn(a[0], a[1], a[2]);
    double da = __dadd_rn(__dadd_rn(__dmul_rn(d[0], a[0]), __dmul_rn(d[1], a[1])), __dmul_rn(d[2], a[2]));
    double t = aa > 0.0 ? __ddiv_rn(da, aa) : 0.0;
    t = fmin(fmax(t, -0.5), 0.5);
    for (int k = 0; k < 3; ++k) r[k] = __dadd_rn(d[k], -__dmul_rn(t, a[k]));
}

__device__ bool obj_contains(const LatticeDev &L, const GeoObjDev &o, int x, int y, int z) {
    if (o.type == 0) {
        int c = o.axis == 0 ? x : (o.axis == 1 ? y : z);
        return c == o.plane;
    }
    if (o.type == 1 || o.type == 4) {   // sphere; droplet = everything outside the ball
        double r2 = norm2_rn(min_image(x - o.c[0], L.nx, L.px), min_image(y - o.c[1], L.ny, L.py),
                             min_image(z - o.c[2], L.nz, L.pz));
        return o.type == 1 ? r2 <= o.R * o.R : r2 > o.R * o.R;
    }
    if (o.type == 5) {   // spherocylinder: within R of its axis segment
        double r[3];
        capsule_offset(L, o, x, y, z, r);
        return norm2_rn(r[0], r[1], r[2]) <= o.R * o.R;
    }
    return false;
}

__global__ void k_owner(LatticeDev L, const GeoObjDev *objs, int nobj, int *owner) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.N;
         i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        site_xyz(L, i, x, y, z);
        int o = NO_OWNER;
        for (int t = 0; t < nobj; ++t)
            if ((objs[t].type <= 1 || objs[t].type >= 4) && obj_contains(L, objs[t], x, y, z)) {
                o = t;
                break;
            }
        owner[i] = o;
    }
}

__global__ void k_scatter_sites(LatticeDev L, const int32_t *xyz, long long n, int id, int *owner) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        int x = xyz[3 * t], y = xyz[3 * t + 1], z = xyz[3 * t + 2];
        if (x < 0 || x >= L.nx || y < 0 || y >= L.ny || z < 0 || z >= L.nz) continue;
        atomicMin(owner + ((long long)z * L.ny + y) * L.nx + x, id);
    }
}

__global__ void k_scatter_anch(LatticeDev L, const int32_t *xyz, long long n, int id,
                               unsigned long long *xclaim) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        int x = xyz[3 * t], y = xyz[3 * t + 1], z = xyz[3 * t + 2];
        if (x < 0 || x >= L.nx || y < 0 || y >= L.ny || z < 0 || z >= L.nz) continue;
        unsigned long long key = ((unsigned long long)(unsigned)id << 32) | (unsigned long long)t;
        atomicMin(xclaim + ((long long)z * L.ny + y) * L.nx + x, key);
    }
}

// winning claim of a simulated site: returns object id (NO_OWNER if none)
// and, for an explicit list, the list position
__device__ __forceinline__ int site_claim(const LatticeDev &L, const int *owner,
                                          const unsigned long long *xclaim, long long i, int x,
                                          int y, int z, long long *pos) {
    int w = NO_OWNER;
    for (int k = 0; k < 3; ++k)
        for (int d = -1; d <= 1; d += 2) {
            long long j = nbr(L, x, y, z, k, d);
            if (j >= 0) w = min(w, owner[j]);
        }
    *pos = -1;
    if (xclaim) {
        unsigned long long c = xclaim[i];
        if (c != NO_CLAIM) {
            int e = (int)(c >> 32);
            if (e < w) { w = e; *pos = (long long)(c & 0xffffffffull); }
        }
    }
    return w;
}

__global__ void k_mask(LatticeDev L, const int *owner, const unsigned long long *xclaim,
                       uint8_t *mask) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.N;
         i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        site_xyz(L, i, x, y, z);
        uint8_t m = 0;
        if (owner[i] == NO_OWNER) {
            m = M_SIM;
            for (int k = 0; k < 3; ++k) {
                long long jf = nbr(L, x, y, z, k, +1), jb = nbr(L, x, y, z, k, -1);
                if (jf >= 0 && owner[jf] == NO_OWNER) m |= m_fwd(k);
                if (jb >= 0 && owner[jb] == NO_OWNER) m |= m_bwd(k);
            }
            long long pos;
            if (site_claim(L, owner, xclaim, i, x, y, z, &pos) != NO_OWNER) m |= M_ANCH;
        }
        mask[i] = m;
    }
}

__global__ void k_row_count(LatticeDev L, const uint8_t *mask, int *counts) {
    long long rows = (long long)L.ny * L.nz;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        int c = 0;
        const uint8_t *m = mask + r * L.nx;
        for (int x = 0; x < L.nx; ++x) c += (m[x] & M_ANCH) ? 1 : 0;
        counts[r] = c;
    }
}

template <typename T>
__global__ void k_fill(LatticeDev L, const uint8_t *mask, const int *owner,
                       const unsigned long long *xclaim, const GeoObjDev *objs, double S0,
                       const int *row_start, int *rec_x, AnchorRec<T> *recs) {
    long long rows = (long long)L.ny * L.nz;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        int out = row_start[r];
        int y = (int)(r % L.ny), z = (int)(r / L.ny);
        for (int x = 0; x < L.nx; ++x) {
            long long i = r * L.nx + x;
            if (!(mask[i] & M_ANCH)) continue;
            long long pos;
            int id = site_claim(L, owner, xclaim, i, x, y, z, &pos);
            const GeoObjDev &o = objs[id];
            AnchorSpecDev sp = o.spec;
            double nrm[3] = {0.0, 0.0, 0.0};
            if (o.type == 0) {
                nrm[o.axis] = 1.0;
            } else if (o.type == 1 || o.type == 4) {
                nrm[0] = min_image(x - o.c[0], L.nx, L.px);
                nrm[1] = min_image(y - o.c[1], L.ny, L.py);
                nrm[2] = min_image(z - o.c[2], L.nz, L.pz);
            } else if (o.type == 5) {
                capsule_offset(L, o, x, y, z, nrm);
            } else {
                if (o.type == 3) sp = o.per_site[pos];
                nrm[0] = sp.dir[0]; nrm[1] = sp.dir[1]; nrm[2] = sp.dir[2];
            }
            AnchorRec<T> rec;
            rec.W = T(sp.W);
            const double *n = (sp.kind == 1) ? sp.dir : nrm;
            double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            double u[3] = {n[0] / len, n[1] / len, n[2] / len};
            if (sp.kind == 2) {
                rec.kind = 2;
                rec.a[0] = T(u[0]); rec.a[1] = T(u[1]); rec.a[2] = T(u[2]);
                rec.a[3] = T(0); rec.a[4] = T(0);
            } else {
                // Q0 = 3/2 S0 (n n - I/3), Eq. (Qtensor) in the uniaxial limit
                rec.kind = 1;
                rec.a[0] = T(1.5 * S0 * (u[0] * u[0] - 1.0 / 3.0));
                rec.a[1] = T(1.5 * S0 * u[0] * u[1]);
                rec.a[2] = T(1.5 * S0 * u[0] * u[2]);
                rec.a[3] = T(1.5 * S0 * (u[1] * u[1] - 1.0 / 3.0));
                rec.a[4] = T(1.5 * S0 * u[1] * u[2]);
            }
            // the FP32 form compares against the target on its fixed-point Q grid
            for (int c = 0; c < 5; ++c) rec.qi[c] = 0;
            if (rec.kind == 1) {
                double q0[5] = {1.5 * S0 * (u[0] * u[0] - 1.0 / 3.0), 1.5 * S0 * u[0] * u[1],
                                1.5 * S0 * u[0] * u[2], 1.5 * S0 * (u[1] * u[1] - 1.0 / 3.0),
                                1.5 * S0 * u[1] * u[2]};
                for (int c = 0; c < 5; ++c) rec.qi[c] = (int)llrint(q0[c] * QFIX_SCALE);
            }
            rec_x[out] = x;
            recs[out] = rec;
            ++out;
        }
    }
}

cudaError_t geo_owner(const LatticeDev &L, const GeoObjDev *objs, int nobj, int *owner,
                      cudaStream_t s) {
    k_owner<<<blocks_for(L.N, 256), 256, 0, s>>>(L, objs, nobj, owner);
    return cudaGetLastError();
}
cudaError_t geo_scatter_sites(const LatticeDev &L, const int32_t *xyz, long long n, int id,
                              int *owner, cudaStream_t s) {
    if (n > 0) k_scatter_sites<<<blocks_for(n, 256), 256, 0, s>>>(L, xyz, n, id, owner);
    return cudaGetLastError();
}
cudaError_t geo_scatter_anchored(const LatticeDev &L, const int32_t *xyz, long long n, int id,
                                 unsigned long long *xclaim, cudaStream_t s) {
    if (n > 0) k_scatter_anch<<<blocks_for(n, 256), 256, 0, s>>>(L, xyz, n, id, xclaim);
    return cudaGetLastError();
}
cudaError_t geo_mask(const LatticeDev &L, const int *owner, const unsigned long long *xclaim,
                     uint8_t *mask, cudaStream_t s) {
    k_mask<<<blocks_for(L.N, 256), 256, 0, s>>>(L, owner, xclaim, mask);
    return cudaGetLastError();
}
cudaError_t geo_row_count(const LatticeDev &L, const uint8_t *mask, int *counts, cudaStream_t s) {
    k_row_count<<<blocks_for((long long)L.ny * L.nz, 128), 128, 0, s>>>(L, mask, counts);
    return cudaGetLastError();
}
cudaError_t geo_fill(const LatticeDev &L, const uint8_t *mask, const int *owner,
                     const unsigned long long *xclaim, const GeoObjDev *objs, double S0,
                     const int *row_start, int *rec_x, void *recs, int fp32, cudaStream_t s) {
    int nb = blocks_for((long long)L.ny * L.nz, 128);
    if (fp32)
        k_fill<float><<<nb, 128, 0, s>>>(L, mask, owner, xclaim, objs, S0, row_start, rec_x,
                                         static_cast<AnchorRec<float> *>(recs));
    else
        k_fill<double><<<nb, 128, 0, s>>>(L, mask, owner, xclaim, objs, S0, row_start, rec_x,
                                          static_cast<AnchorRec<double> *>(recs));
    return cudaGetLastError();
}

// ---- state helpers ------------------------------------------------------------

template <typename T>
__global__ void k_zero_objects(LatticeDev L, const uint8_t *mask, T *a0, T *a1, T *a2, T *a3,
                               T *a4, T *a5, int narr) {
    T *arr[6] = {a0, a1, a2, a3, a4, a5};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.N;
         i += (long long)gridDim.x * blockDim.x) {
        if (mask[i] & M_SIM) continue;
        for (int a = 0; a < narr; ++a)
            for (int c = 0; c < 5; ++c) arr[a][c * L.N + i] = T(0);
    }
}

cudaError_t zero_object_sites(const LatticeDev &L, const uint8_t *mask, void *const *arrays,
                              int narrays, int fp32, cudaStream_t s) {
    void *a[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int t = 0; t < narrays && t < 6; ++t) a[t] = arrays[t];
    if (fp32)
        k_zero_objects<float><<<blocks_for(L.N, 256), 256, 0, s>>>(
            L, mask, (float *)a[0], (float *)a[1], (float *)a[2], (float *)a[3], (float *)a[4],
            (float *)a[5], narrays);
    else
        k_zero_objects<double><<<blocks_for(L.N, 256), 256, 0, s>>>(
            L, mask, (double *)a[0], (double *)a[1], (double *)a[2], (double *)a[3],
            (double *)a[4], (double *)a[5], narrays);
    return cudaGetLastError();
}

template <typename S, typename D>
__global__ void k_convert(const S *src, D *dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = D(src[i]);
}

// Q into the fixed-point grid of the FP32 form; values with |q| >= 4 are
// counted in *err and clamped
template <typename S>
__global__ void k_q_to_fixed(const S *src, int *dst, long long n, unsigned int *err) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double v = (double)src[i];
        if (!(fabs(v) < QFIX_LIMIT)) {
            atomicAdd(err, 1u);
            v = 0.0;
        }
        dst[i] = (int)llrint(v * QFIX_SCALE);
    }
}

__global__ void k_fixed_to_f64(const int *src, double *dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (double)src[i] * QFIX_INV;
}

cudaError_t q_import(const void *src, int src_f32, void *dst, long long n, int fp32,
                     unsigned int *err, cudaStream_t s) {
    int nb = blocks_for(n, 256);
    if (fp32) {
        cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
        if (src_f32) k_q_to_fixed<float><<<nb, 256, 0, s>>>((const float *)src, (int *)dst, n, err);
        else k_q_to_fixed<double><<<nb, 256, 0, s>>>((const double *)src, (int *)dst, n, err);
    } else {
        if (src_f32) k_convert<float, double><<<nb, 256, 0, s>>>((const float *)src, (double *)dst, n);
        else k_convert<double, double><<<nb, 256, 0, s>>>((const double *)src, (double *)dst, n);
    }
    return cudaGetLastError();
}

cudaError_t q_export(const void *src, double *dst, long long n, int fp32, cudaStream_t s) {
    int nb = blocks_for(n, 256);
    if (fp32) k_fixed_to_f64<<<nb, 256, 0, s>>>((const int *)src, dst, n);
    else k_convert<double, double><<<nb, 256, 0, s>>>((const double *)src, dst, n);
    return cudaGetLastError();
}

cudaError_t state_to_f64(const void *src, double *dst, long long n, int fp32, cudaStream_t s) {
    if (fp32) k_convert<float, double><<<blocks_for(n, 256), 256, 0, s>>>((const float *)src, dst, n);
    else k_convert<double, double><<<blocks_for(n, 256), 256, 0, s>>>((const double *)src, dst, n);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_mixed_velocity(const T *v, const T *F, const FireDev *st, double *out,
                                 long long n) {
    T cv = T(st->cv), cF = T(st->cF);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = double(cv * v[i] + cF * F[i]);
}

cudaError_t mixed_velocity(const void *v, const void *F, const FireDev *st, double *out,
                           long long n, int fp32, cudaStream_t s) {
    if (fp32)
        k_mixed_velocity<float><<<blocks_for(n, 256), 256, 0, s>>>((const float *)v,
                                                                   (const float *)F, st, out, n);
    else
        k_mixed_velocity<double><<<blocks_for(n, 256), 256, 0, s>>>((const double *)v,
                                                                    (const double *)F, st, out, n);
    return cudaGetLastError();
}

// SplitMix64 (Steele, Lea & Flood 2014): output k of the stream started at seed
__device__ __forceinline__ unsigned long long splitmix(unsigned long long seed,
                                                       unsigned long long k) {
    unsigned long long z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ void store_q(double *q, long long i, double v) { q[i] = v; }
__device__ __forceinline__ void store_q(int *q, long long i, double v) { q[i] = (int)llrint(v * QFIX_SCALE); }
__device__ __forceinline__ double load_q(const double *q, long long i) { return q[i]; }
__device__ __forceinline__ double load_q(const int *q, long long i) { return (double)q[i] * QFIX_INV; }

template <typename T>
__global__ void k_random_uniaxial(LatticeDev L, const uint8_t *mask, unsigned long long seed,
                                  double S, T *q) {
    const double two53 = 1.0 / 9007199254740992.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.N;
         i += (long long)gridDim.x * blockDim.x) {
        double qq[5] = {0, 0, 0, 0, 0};
        if (mask[i] & M_SIM) {
            double u1 = (double)(splitmix(seed, 2ull * i + 1) >> 11) * two53;
            double u2 = (double)(splitmix(seed, 2ull * i + 2) >> 11) * two53;
            double z = 2.0 * u1 - 1.0, phi = 2.0 * 3.141592653589793 * u2;
            double r = sqrt(fmax(0.0, 1.0 - z * z));
            double n0 = r * cos(phi), n1 = r * sin(phi), n2 = z;
            qq[0] = 1.5 * S * (n0 * n0 - 1.0 / 3.0);
            qq[1] = 1.5 * S * n0 * n1;
            qq[2] = 1.5 * S * n0 * n2;
            qq[3] = 1.5 * S * (n1 * n1 - 1.0 / 3.0);
            qq[4] = 1.5 * S * n1 * n2;
        }
        for (int c = 0; c < 5; ++c) store_q(q, c * L.N + i, qq[c]);
    }
}

cudaError_t init_random_uniaxial(const LatticeDev &L, const uint8_t *mask, unsigned long long seed,
                                 double S, void *q, int fp32, cudaStream_t s) {
    if (fp32) k_random_uniaxial<int><<<blocks_for(L.N, 256), 256, 0, s>>>(L, mask, seed, S, (int *)q);
    else k_random_uniaxial<double><<<blocks_for(L.N, 256), 256, 0, s>>>(L, mask, seed, S, (double *)q);
    return cudaGetLastError();
}

// Dipolar start about a colloid at c with far-field director a (unit): a
// radial hedgehog at c superposed on a hyperbolic hedgehog at h = c + rd a,
// director tilt psi = theta_c - theta_h from a (polar angles of the site
// seen from c and from h).  With u = x - c, u_a = u.a, w_a = u_a - rd and
// u_perp = u - u_a a, the angle difference expands to
//   n = ((u_a w_a + |u_perp|^2) a - rd u_perp) / (|u| |w|),
// a unit vector; at c and at h, where it is undefined, n = a.
template <typename T>
__global__ void k_dipolar(LatticeDev L, const uint8_t *mask, double3 c, double3 a, double rd, double S,
                          T *q) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.N;
         i += (long long)gridDim.x * blockDim.x) {
        double qq[5] = {0, 0, 0, 0, 0};
        if (mask[i] & M_SIM) {
            int x, y, z;
            site_xyz(L, i, x, y, z);
            double u0 = min_image(x - c.x, L.nx, L.px), u1 = min_image(y - c.y, L.ny, L.py),
                   u2 = min_image(z - c.z, L.nz, L.pz);
            double ua = u0 * a.x + u1 * a.y + u2 * a.z;
            double p0 = u0 - ua * a.x, p1 = u1 - ua * a.y, p2 = u2 - ua * a.z;
            double rho2 = p0 * p0 + p1 * p1 + p2 * p2;
            double wa = ua - rd;
            double den = sqrt((ua * ua + rho2) * (wa * wa + rho2));
            double n0 = a.x, n1 = a.y, n2 = a.z;
            if (den > 0.0) {
                double ca = (ua * wa + rho2) / den, cp = -rd / den;
                n0 = ca * a.x + cp * p0;
                n1 = ca * a.y + cp * p1;
                n2 = ca * a.z + cp * p2;
            }
            qq[0] = 1.5 * S * (n0 * n0 - 1.0 / 3.0);
            qq[1] = 1.5 * S * n0 * n1;
            qq[2] = 1.5 * S * n0 * n2;
            qq[3] = 1.5 * S * (n1 * n1 - 1.0 / 3.0);
            qq[4] = 1.5 * S * n1 * n2;
        }
        for (int k = 0; k < 5; ++k) store_q(q, k * L.N + i, qq[k]);
    }
}

cudaError_t init_dipolar(const LatticeDev &L, const uint8_t *mask, const double c[3], const double a[3],
                         double rd, double S, void *q, int fp32, cudaStream_t s) {
    double3 cc = make_double3(c[0], c[1], c[2]), aa = make_double3(a[0], a[1], a[2]);
    if (fp32) k_dipolar<int><<<blocks_for(L.N, 256), 256, 0, s>>>(L, mask, cc, aa, rd, S, (int *)q);
    else k_dipolar<double><<<blocks_for(L.N, 256), 256, 0, s>>>(L, mask, cc, aa, rd, S, (double *)q);
    return cudaGetLastError();
}

__global__ void k_count_sim(LatticeDev L, const uint8_t *mask, unsigned long long *out) {
    unsigned long long c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.N;
         i += (long long)gridDim.x * blockDim.x)
        c += (mask[i] & M_SIM) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

cudaError_t count_simulated(const LatticeDev &L, const uint8_t *mask, unsigned long long *out,
                            cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_count_sim<<<blocks_for(L.N, 256), 256, 0, s>>>(L, mask, out);
    return cudaGetLastError();
}

// ---- energy readback (FP64 arithmetic for both storage types) -------------------

__device__ __forceinline__ double frob2(const double *d) {
    double zz = -d[0] - d[3];
    return d[0] * d[0] + d[3] * d[3] + zz * zz + 2.0 * (d[1] * d[1] + d[2] * d[2] + d[4] * d[4]);
}

template <typename QS>
__device__ __forceinline__ void load5(const QS *q, long long N, long long i, double *o) {
    for (int c = 0; c < 5; ++c) o[c] = load_q(q, c * N + i);
}

// T: arithmetic type of the form (selects the record layout); QS: Q storage
template <typename T, typename QS>
__global__ void k_energy(LatticeDev L, Geometry g, const QS *q, double A, double B, double C,
                         double L1, double L2, double L3, double S0, EnergyExtra ex,
                         double *partials) {
    double eb = 0.0, ed = 0.0, ea = 0.0;
    const long long N = L.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        uint8_t m = g.mask[i];
        if (!(m & M_SIM)) continue;
        int x, y, z;
        site_xyz(L, i, x, y, z);
        double q0[5];
        load5(q, N, i, q0);
        // bulk, Eq. (fphase)
        {
            double a = q0[0], b = q0[1], c = q0[2], d = q0[3], e = q0[4], f = -a - d;
            double tr2 = a * a + d * d + f * f + 2.0 * (b * b + c * c + e * e);
            double det = a * (d * f - e * e) - b * (b * f - e * c) + c * (b * e - d * c);
            // tr Q^3 = 3 det Q for a traceless Q
            eb += A / 2.0 * tr2 + B / 3.0 * (3.0 * det) + C / 4.0 * tr2 * tr2;
            // external fields: -(1/3) K:Q
            const double *K = ex.K;
            eb -= (K[0] * a + K[3] * d + K[5] * f + 2.0 * (K[1] * b + K[2] * c + K[4] * e)) / 3.0;
        }
        // distortion: factorised average over allowed differences
        double mk[3][5], sqF[3], squ[3];
        for (int k = 0; k < 3; ++k) {
            int fo = (m & m_fwd(k)) ? 1 : 0, bo = (m & m_bwd(k)) ? 1 : 0;
            int n = fo + bo;
            for (int c = 0; c < 5; ++c) mk[k][c] = 0.0;
            sqF[k] = squ[k] = 0.0;
            if (!n) continue;
            double w = 1.0 / n;
            for (int s = 0; s < 2; ++s) {
                if (s == 0 && !fo) continue;
                if (s == 1 && !bo) continue;
                long long j = nbr(L, x, y, z, k, s == 0 ? +1 : -1);
                double qn[5], d[5];
                load5(q, N, j, qn);
                for (int c = 0; c < 5; ++c) d[c] = (s == 0) ? qn[c] - q0[c] : q0[c] - qn[c];
                for (int c = 0; c < 5; ++c) mk[k][c] += w * d[c];
                sqF[k] += w * frob2(d);
                double col = 0.0;
                for (int r = 0; r < 3; ++r) {
                    double e = sym(d, r, k);
                    col += e * e;
                }
                squ[k] += w * col;
            }
        }
        double f = 0.0;
        for (int k = 0; k < 3; ++k) f += L1 / 2.0 * sqF[k] + (L2 + L3) / 2.0 * squ[k];
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                if (j == k) continue;
                double t2 = 0.0, t3 = 0.0;
                for (int r = 0; r < 3; ++r) {
                    t2 += sym(mk[j], r, j) * sym(mk[k], r, k);
                    t3 += sym(mk[j], r, k) * sym(mk[k], r, j);
                }
                f += L2 / 2.0 * t2 + L3 / 2.0 * t3;
            }
        if (ex.L4 != 0.0 || ex.L6 != 0.0) {
            // chiral: L4/2 eps_lik Q_lj m_k[ij]; cubic: L6/2 (Q_kk <|D_k|^2>
            // + sum_{l != k} Q_lk m_l . m_k)
            double f4 = 0.0, f6 = 0.0;
            for (int l = 0; l < 3; ++l)
                for (int i2 = 0; i2 < 3; ++i2)
                    for (int k = 0; k < 3; ++k) {
                        int e3 = (l - i2) * (i2 - k) * (k - l) / 2;
                        if (!e3) continue;
                        for (int j = 0; j < 3; ++j) f4 += e3 * sym(q0, l, j) * sym(mk[k], i2, j);
                    }
            for (int k = 0; k < 3; ++k) {
                f6 += sym(q0, k, k) * sqF[k];
                for (int l = 0; l < 3; ++l) {
                    if (l == k) continue;
                    double dot = 0.0;
                    for (int a2 = 0; a2 < 3; ++a2)
                        for (int b2 = 0; b2 < 3; ++b2) dot += sym(mk[l], a2, b2) * sym(mk[k], a2, b2);
                    f6 += sym(q0, l, k) * dot;
                }
            }
            f += ex.L4 / 2.0 * f4 + ex.L6 / 2.0 * f6;
        }
        ed += f;
        // anchoring
        if (m & M_ANCH) {
            long long row = (long long)z * L.ny + y;
            int lo = g.row_start[row], hi = g.row_start[row + 1] - 1;
            const AnchorRec<T> *rec = nullptr;
            while (lo <= hi) {
                int mid = (lo + hi) >> 1;
                if (g.rec_x[mid] == x) { rec = reinterpret_cast<const AnchorRec<T> *>(g.recs) + mid; break; }
                if (g.rec_x[mid] < x) lo = mid + 1; else hi = mid - 1;
            }
            if (rec) {
                double W = (double)rec->W;
                if (rec->kind == 1) {
                    double d[5];
                    for (int c = 0; c < 5; ++c)
                        d[c] = q0[c] - (sizeof(T) == 4 ? (double)rec->qi[c] * QFIX_INV : (double)rec->a[c]);
                    ea += W * frob2(d);
                } else {
                    double nu[3] = {(double)rec->a[0], (double)rec->a[1], (double)rec->a[2]};
                    double w[3];
                    for (int r = 0; r < 3; ++r) {
                        w[r] = S0 / 2.0 * nu[r];
                        for (int c = 0; c < 3; ++c) w[r] += sym(q0, r, c) * nu[c];
                    }
                    double nw = nu[0] * w[0] + nu[1] * w[1] + nu[2] * w[2];
                    double R2 = 0.0;
                    for (int r = 0; r < 3; ++r)
                        for (int c = 0; c < 3; ++c) {
                            double R = nu[r] * w[c] + w[r] * nu[c] - nw * nu[r] * nu[c];
                            R2 += R * R;
                        }
                    ea += W * R2;
                }
            }
        }
    }
    // block sums in a fixed order
    __shared__ double sh[3][256];
    sh[0][threadIdx.x] = eb; sh[1][threadIdx.x] = ed; sh[2][threadIdx.x] = ea;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int t = 0; t < 3; ++t) sh[t][threadIdx.x] += sh[t][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int t = 0; t < 3; ++t) partials[3 * blockIdx.x + t] = sh[t][0];
}

__global__ void k_sum_partials3(const double *partials, int n, double *out3) {
    __shared__ double sh[3][256];
    double a[3] = {0, 0, 0};
    for (int b = threadIdx.x; b < n; b += blockDim.x)
        for (int t = 0; t < 3; ++t) a[t] += partials[3 * b + t];
    for (int t = 0; t < 3; ++t) sh[t][threadIdx.x] = a[t];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int t = 0; t < 3; ++t) sh[t][threadIdx.x] += sh[t][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int t = 0; t < 3; ++t) out3[t] = sh[t][0];
}

cudaError_t energy_parts(const LatticeDev &L, const Geometry &g, const void *q, int fp32,
                         double A, double B, double C, double L1, double L2, double L3, double S0,
                         const EnergyExtra &ex, double *partials, int max_blocks, double *out3,
                         cudaStream_t s) {
    int nb = blocks_for(L.N, 256);
    if (nb > max_blocks) nb = max_blocks;
    if (fp32)
        k_energy<float, int><<<nb, 256, 0, s>>>(L, g, (const int *)q, A, B, C, L1, L2, L3, S0, ex,
                                                 partials);
    else
        k_energy<double, double><<<nb, 256, 0, s>>>(L, g, (const double *)q, A, B, C, L1, L2, L3, S0,
                                                    ex, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_partials3<<<1, 256, 0, s>>>(partials, nb, out3);
    return cudaGetLastError();
}

// largest eigenvalue of a symmetric traceless 3x3 by the trigonometric
// solution of its characteristic cubic (Smith 1961)
template <typename T>
__global__ void k_order(LatticeDev L, const uint8_t *mask, const T *q, double *S) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.N;
         i += (long long)gridDim.x * blockDim.x) {
        if (!(mask[i] & M_SIM)) { S[i] = 0.0; continue; }
        double a, b, c, d, e;
        a = load_q(q, i); b = load_q(q, L.N + i); c = load_q(q, 2 * L.N + i);
        d = load_q(q, 3 * L.N + i); e = load_q(q, 4 * L.N + i);
        double f = -a - d;
        double p2 = (a * a + d * d + f * f + 2.0 * (b * b + c * c + e * e)) / 6.0;
        if (p2 <= 0.0) { S[i] = 0.0; continue; }
        double p = sqrt(p2);
        double ia = a / p, ib = b / p, ic = c / p, id = d / p, ie = e / p, iff = f / p;
        double det = ia * (id * iff - ie * ie) - ib * (ib * iff - ie * ic) + ic * (ib * ie - id * ic);
        double r = fmin(1.0, fmax(-1.0, det / 2.0));
        double phi = acos(r) / 3.0;
        S[i] = 2.0 * p * cos(phi);
    }
}

cudaError_t order_field(const LatticeDev &L, const uint8_t *mask, const void *q, int fp32,
                        double *S_out, cudaStream_t s) {
    if (fp32) k_order<int><<<blocks_for(L.N, 256), 256, 0, s>>>(L, mask, (const int *)q, S_out);
    else k_order<double><<<blocks_for(L.N, 256), 256, 0, s>>>(L, mask, (const double *)q, S_out);
    return cudaGetLastError();
}

}  // namespace lq
