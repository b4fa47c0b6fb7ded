// lq_common.cuh -- device data layout and small algebra shared by the kernels.
//
// Layout in HBM (one solver):
//   q, v, F      structure of arrays, component c of site i at [c*N + i],
//                two copies (ping-pong) because a FIRE step reads the
//                neighbours' old state while it writes the new one;
//   mask         one byte per site (bits below);
//   anchoring    records of the anchored sites, sorted by site index, found
//                through a per-(z, y)-row offset table and the x coordinate;
//   FireDev      the FIRE scalars, the coefficients of the next step and the
//                last reductions, written only by the last block of a step.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lq {

// mask bits
constexpr uint8_t M_SIM = 1u << 0;   // simulated (bulk or boundary) site
constexpr uint8_t M_ANCH = 1u << 1;  // carries an anchoring record
// neighbour simulated along +x, -x, +y, -y, +z, -z: bit 2 + 2k (+), 3 + 2k (-)
__host__ __device__ constexpr uint8_t m_fwd(int k) { return (uint8_t)(1u << (2 + 2 * k)); }
__host__ __device__ constexpr uint8_t m_bwd(int k) { return (uint8_t)(1u << (3 + 2 * k)); }

// FIRE_STALLED: a tensor copy of the step did not complete within its time
// limit; the step kernel stopped (the entry point returns LQ_ECUDA)
enum : int { FIRE_RUNNING = 0, FIRE_CONVERGED = 1, FIRE_MAXITER = 2, FIRE_DIVERGED = 3, FIRE_STALLED = 4 };

// Anchoring record of one boundary site.  kind 1: Nobili-Durand, a = q0 (5
// components of Q0), qi = the same in the fixed-point Q format of the FP32
// form; kind 2: Fournier-Galatola, a[0..2] = unit normal nu.
template <typename T>
struct AnchorRec {
    T a[5];
    T W;
    int kind;
    int qi[5];
};

// FP32 form: Q is stored as 32-bit fixed point, q = n * 2^-28.  An FP32 Q
// resolves only ~3e-8 at |Q| ~ 0.4, which is the size of the last FIRE
// updates before max|F| < 1e-6, and the minimisation stalls there; the fixed
// grid resolves 3.7e-9 everywhere with the same 4 bytes, and the stencil's
// differences are exact integer arithmetic.  Components are kept in
// |q| < 2 (Q entries of a physical state are bounded by |S| <= 1), so that
// second differences a + b - 2c and mixed differences a - b - c + d stay
// inside int32.
constexpr double QFIX_SCALE = 268435456.0;          // 2^28
constexpr double QFIX_INV = 1.0 / 268435456.0;
constexpr double QFIX_LIMIT = 2.0;                  // |q| must stay below

struct FireDev {
    // parameters
    double dt0, dt_max, alpha0, f_alpha, f_inc, f_dec, tol;
    long long n_min, max_iter;
    // scalars of Algorithm 1
    double dt, alpha;
    long long npos, iter, kcount;
    int status, cur;          // cur: which ping-pong buffer holds the state
    // coefficients of the next step: v_mix = cv v + cF F, drift
    // q + c_alpha v + c_beta F, kick v_mix + c_kick (F_old + F_new); dt_step
    // is FIRE's dt of that step
    double cv, cF, dt_step;
    double c_alpha, c_beta, c_kick;
    // minimiser (lq_minimizer), Nesterov momentum, descent step
    long long method;
    double mu, eta;
    // reductions of the last evaluated state
    double P, F2, v2, r2;
    long long nsim;
    unsigned int counter;     // last-block-done ticket
    unsigned int pad;
};

struct Geometry {
    const uint8_t *mask;
    const int *row_start;     // nz*ny + 1 offsets into the record arrays
    const int *rec_x;         // x coordinate of each record
    const void *recs;         // AnchorRec<T>
};

struct LatticeDev {
    int nx, ny, nz;
    int px, py, pz;           // periodic flags
    long long N;
};

// ---- 5-component algebra --------------------------------------------------
// A symmetric traceless 3x3 stored as q = (xx, xy, xz, yy, yz).

template <typename T>
__device__ __forceinline__ T sym(const T *q, int i, int j) {
    // entry (i, j) of the full tensor
    if (i > j) { int t = i; i = j; j = t; }
    if (i == 0) return q[j];                 // xx, xy, xz
    if (i == 1) return j == 1 ? q[3] : q[4]; // yy, yz
    return -q[0] - q[3];                     // zz
}

// J^T of a symmetric traceless tensor: the derivative with respect to the
// five components of <G, Q(q)> when G = that tensor.
template <typename T>
__device__ __forceinline__ void jt_sym(const T *d, T *out) {
    out[0] = T(2) * d[0] + d[3];
    out[1] = T(2) * d[1];
    out[2] = T(2) * d[2];
    out[3] = d[0] + T(2) * d[3];
    out[4] = T(2) * d[4];
}

}  // namespace lq
