// noalloc.cu -- lq_energy_noalloc: the bulk and distortion energy of a
// caller-owned device Q field, computed without allocating any memory.
//
// Who needs it: callers that cannot let a library call cudaMalloc -- a
// process whose device memory is fully reserved up front by its own
// allocator or budget (a serving loop that admits work by an HBM budget, a
// framework whose caching allocator owns the device), or a latency-bound
// loop that cannot afford the device-wide synchronisation that cudaMalloc
// and cudaFree imply.  The caller passes every input and output buffer; the
// only scratch is the file-scope array below, one slot of three doubles per
// z plane, held by every GPU that loads the library until the process exits.
//
// The per-plane sums are written (not accumulated), so nothing needs
// clearing between calls; calls that overlap on the GPU (on different
// streams, or from different threads) share the array and race.
#include <cstdint>
#include <mutex>

#include "lqmin.h"
#include "lq_common.cuh"
#include "solver_internal.h"

namespace lq {
namespace {

struct double6 {
    double v[6];   // symmetric tensor: xx, xy, xz, yy, yz, zz
};

constexpr int NOALLOC_MAX_NZ = 4096;
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

// per-plane (bulk, distortion, 0) sums of the last call
static __device__ __align__(256) double g_plane_sums[3 * NOALLOC_MAX_NZ];

// device addresses of g_plane_sums, set up once per device
std::mutex g_setup_mutex;
double *g_scratch_addr[NOALLOC_MAX_DEVICES] = {nullptr};

__device__ __forceinline__ double sq_frob(const double *d) {
    double zz = -d[0] - d[3];
    return d[0] * d[0] + d[3] * d[3] + zz * zz + 2.0 * (d[1] * d[1] + d[2] * d[2] + d[4] * d[4]);
}

__device__ __forceinline__ long long step_site(int nx, int ny, int nz, const int per[3], int x,
                                               int y, int z, int k, int dir) {
    int c[3] = {x, y, z}, n[3] = {nx, ny, nz};
    c[k] += dir;
    if (c[k] < 0 || c[k] >= n[k]) {
        if (!per[k]) return -1;
        c[k] = (c[k] + n[k]) % n[k];
    }
    return ((long long)c[2] * ny + c[1]) * nx + c[0];
}

// one block per z plane: fixed-order sum of the bulk (Eq. fphase) and the
// averaged-difference distortion density (Eq. fdistortionFull) of its sites
__global__ void __launch_bounds__(NOALLOC_THREADS)
k_plane_energy(int nx, int ny, int nz, int px, int py, int pz, double A, double B, double C,
               double L1, double L2, double L3, double L4, double L6, double6 K, const double *q,
               const uint8_t *mask, double *plane_sums) {
    const int z = blockIdx.x;
    const long long N = (long long)nx * ny * nz;
    const int per[3] = {px, py, pz};
    double eb = 0.0, ed = 0.0;
    for (int t = threadIdx.x; t < nx * ny; t += blockDim.x) {
        int x = t % nx, y = t / nx;
        long long i = (long long)z * nx * ny + t;
        uint8_t m = mask[i];
        if (!(m & M_SIM)) continue;
        double q0[5];
        for (int c = 0; c < 5; ++c) q0[c] = q[c * N + i];
        double a = q0[0], b = q0[1], c3 = q0[2], d = q0[3], e = q0[4], f = -a - d;
        double tr2 = a * a + d * d + f * f + 2.0 * (b * b + c3 * c3 + e * e);
        double det = a * (d * f - e * e) - b * (b * f - e * c3) + c3 * (b * e - d * c3);
        eb += A / 2.0 * tr2 + B * det + C / 4.0 * tr2 * tr2;   // tr Q^3 = 3 det Q
        // external fields, -(1/3) K:Q
        eb -= (K.v[0] * a + K.v[3] * d + K.v[5] * f + 2.0 * (K.v[1] * b + K.v[2] * c3 + K.v[4] * e)) / 3.0;
        double mk[3][5], sqF[3], squ[3];
        for (int k = 0; k < 3; ++k) {
            // a mask bit that names a neighbour outside a non-periodic edge
            // (a mask built for other periodic flags) counts as absent, so
            // that no site outside the lattice is ever read
            const long long jn[2] = {step_site(nx, ny, nz, per, x, y, z, k, 1),
                                     step_site(nx, ny, nz, per, x, y, z, k, -1)};
            int fo = ((m & m_fwd(k)) && jn[0] >= 0) ? 1 : 0, bo = ((m & m_bwd(k)) && jn[1] >= 0) ? 1 : 0;
            for (int c = 0; c < 5; ++c) mk[k][c] = 0.0;
            sqF[k] = squ[k] = 0.0;
            if (fo + bo == 0) continue;
            double w = 1.0 / (fo + bo);
            for (int s = 0; s < 2; ++s) {
                if ((s == 0 && !fo) || (s == 1 && !bo)) continue;
                const long long j = jn[s];
                double dd[5];
                for (int c = 0; c < 5; ++c) dd[c] = s == 0 ? q[c * N + j] - q0[c] : q0[c] - q[c * N + j];
                for (int c = 0; c < 5; ++c) mk[k][c] += w * dd[c];
                sqF[k] += w * sq_frob(dd);
                double col = 0.0;
                for (int r = 0; r < 3; ++r) {
                    double v = sym(dd, r, k);
                    col += v * v;
                }
                squ[k] += w * col;
            }
        }
        double fd = 0.0;
        for (int k = 0; k < 3; ++k) fd += L1 / 2.0 * sqF[k] + (L2 + L3) / 2.0 * squ[k];
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                if (j == k) continue;
                double t2 = 0.0, t3 = 0.0;
                for (int r = 0; r < 3; ++r) {
                    t2 += sym(mk[j], r, j) * sym(mk[k], r, k);
                    t3 += sym(mk[j], r, k) * sym(mk[k], r, j);
                }
                fd += L2 / 2.0 * t2 + L3 / 2.0 * t3;
            }
        if (L4 != 0.0 || L6 != 0.0) {
            // chiral L4/2 eps_lik Q_lj m_k[ij], cubic L6/2 (Q_kk <|D_k|^2>
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
            fd += L4 / 2.0 * f4 + L6 / 2.0 * f6;
        }
        ed += fd;
    }
    __shared__ double sh[2][NOALLOC_THREADS];
    sh[0][threadIdx.x] = eb;
    sh[1][threadIdx.x] = ed;
    __syncthreads();
    for (int s = NOALLOC_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        plane_sums[3 * z] = sh[0][0];
        plane_sums[3 * z + 1] = sh[1][0];
        plane_sums[3 * z + 2] = 0.0;
    }
}

// sum the per-plane values in a fixed order into the caller's output
__global__ void __launch_bounds__(NOALLOC_THREADS)
k_sum_planes(const double *plane_sums, int nz, double *out3) {
    __shared__ double sh[2][NOALLOC_THREADS];
    double a = 0.0, b = 0.0;
    for (int z = threadIdx.x; z < nz; z += blockDim.x) {
        a += plane_sums[3 * z];
        b += plane_sums[3 * z + 1];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = NOALLOC_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out3[0] = sh[0][0];
        out3[1] = sh[1][0];
        out3[2] = 0.0;
    }
}

// device address of the static scratch for the current device (set up on
// the first call made with that device current)
double *scratch_for_current_device(lq_status *st) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        *st = LQ_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        double *p = nullptr;
        if (cudaGetSymbolAddress((void **)&p, g_plane_sums) != cudaSuccess || !p) {
            *st = LQ_ECUDA;
            return nullptr;
        }
        g_scratch_addr[dev] = p;
    }
    *st = LQ_OK;
    return g_scratch_addr[dev];
}

}  // namespace
}  // namespace lq

extern "C" lq_status lq_energy_noalloc(const lq_lattice *lat, const lq_material *mat,
                                       const double *q_dev, const uint8_t *mask_dev,
                                       double *parts_dev, void *cuda_stream) {
    using namespace lq;
    if (!lat || !mat || !q_dev || !mask_dev || !parts_dev) return LQ_EINVAL;
    if (lat->nx <= 0 || lat->ny <= 0 || lat->nz <= 0) return LQ_EINVAL;
    if (lat->nz > NOALLOC_MAX_NZ) return LQ_EINVAL;
    // the same lattice and material checks as lq_create (host arithmetic only)
    if (lat->spacing != 1.0) return LQ_EINVAL;
    double S0 = 0.0;
    if (detail::validate_material(mat, &S0)) return LQ_EINVAL;
    lq_status st;
    double *scratch = scratch_for_current_device(&st);
    if (!scratch) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double6 K;
    {
        double Kf[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                Kf[a][b] = mat->mu0_dchi * mat->H[a] * mat->H[b] + mat->eps0_deps * mat->E[a] * mat->E[b];
        const double v[6] = {Kf[0][0], Kf[0][1], Kf[0][2], Kf[1][1], Kf[1][2], Kf[2][2]};
        for (int t = 0; t < 6; ++t) K.v[t] = v[t];
    }
    k_plane_energy<<<lat->nz, NOALLOC_THREADS, 0, s>>>(
        lat->nx, lat->ny, lat->nz, lat->periodic[0] ? 1 : 0, lat->periodic[1] ? 1 : 0,
        lat->periodic[2] ? 1 : 0, mat->A, mat->B, mat->C, mat->L1, mat->L2, mat->L3, mat->L4,
        mat->L6, K, q_dev, mask_dev, scratch);
    if (cudaGetLastError() != cudaSuccess) return LQ_ECUDA;
    k_sum_planes<<<1, NOALLOC_THREADS, 0, s>>>(scratch, lat->nz, parts_dev);
    if (cudaGetLastError() != cudaSuccess) return LQ_ECUDA;
    return LQ_OK;
}
