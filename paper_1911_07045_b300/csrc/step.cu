// step.cu -- one FIRE iteration as one kernel: velocity mixing of the
// previous iteration, Verlet drift, the Landau-de Gennes force, the Verlet
// kick, and the FIRE reductions with the scalar update done by the last block.
//
// Force (section III.B).  The discrete energy is the sum over simulated
// sites of f_bulk (Eq. fphase) + the distortion density (Eq.
// fdistortionFull) averaged over every allowed forward/backward difference
// combination (Eq. onesidedderivatives) + the anchoring terms (section II).
// The force is minus its derivative with respect to every q_i(x_j).
//
// Factorised form used here (exact rearrangement of that average).  For a
// site i and axis k let n_k(i) be the number of allowed one-sided
// differences, D_k^s the difference tensor for choice s, m_k = the mean of
// the allowed D_k^s.  Since the choices along different axes are independent
// and equally weighted, the combination average of Eq. (fdistortionFull) is
//   sum_k [ L1/2 <|D_k|^2> + (L2+L3)/2 <|D_k[:,k]|^2> ]
//   + L2/2 sum_{j!=k} m_j[:,j].m_k[:,k] + L3/2 sum_{j!=k} m_j[:,k].m_k[:,j].
// Each link (i, i+e_k) carries one difference Delta; the energy derivative
// with respect to it ("flux") is
//   Phi = (w_f(i) + w_b(i+e_k)) [L1 Delta + (L2+L3) col_k(Delta[:,k])]
//         + w_f(i) X_k(i) + w_b(i+e_k) X_k(i+e_k),   w = 1/n_k,
// where X_k(i) holds the cross terms: column k = L2 (m_a[:,a] + m_b[:,b]),
// column a = L3 m_a[:,k], column b = L3 m_b[:,k] ({a, b} = the other axes).
// The distortion gradient at j is sum_k (Phi_k(j - e_k) - Phi_k(j)), mapped
// to the five components by J^T.  One-constant: Phi = (w_f + w_b) L1 Delta.
//
// Schedule.  A block owns a TX x TY column of sites and marches along z
// through zchunk planes.  Each plane of drifted Q (tile + 1-site ring incl.
// corners) is staged once in shared memory (4-slot ring over z); the z-link
// flux and the z cross terms are carried in registers from plane to plane.
// Three-constant: the in-plane cross terms X_x, X_y of the tile and its ring
// are computed once per plane into shared memory (two slots).
//
// FIRE (Algorithm 1).  Iteration n of the paper is: drift q += dt v +
// dt^2/2 F, new force F', kick v += dt/2 (F + F'), reductions P = F.v, |F|,
// |v|, then mixing v <- (1-alpha) v + alpha |v| F/|F| and the P test.  The
// mixing needs the global reductions, so it is applied at the start of the
// NEXT kernel: v_mix = cv v + cF F with (cv, cF, dt) written by the last
// block of the previous kernel.  The first kernel after a reset (dt = 0,
// cv = cF = 0) only evaluates F(q0).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cfloat>
#include <cstdio>

#include "lq_common.cuh"
#include "lq_kernels.h"

namespace lq {

// Index checks of the bounds-checked build (-DLQ_BOUNDS_CHECK): an index
// outside [0, n) is counted and replaced by 0, so that nothing is ever read
// or written out of range; the release build compiles them away.
#ifdef LQ_BOUNDS_CHECK
__device__ unsigned int bounds_hits_dev;
__device__ __forceinline__ int bchk(int i, int n) {
    if (i < 0 || i >= n) { atomicAdd(&bounds_hits_dev, 1u); return 0; }
    return i;
}
template <typename I>
__device__ __forceinline__ I bchk_idx(I i, I n) {
    if (i >= n) { atomicAdd(&bounds_hits_dev, 1u); return I(0); }
    return i;
}
#define LQ_CHK(i, n) bchk((i), (n))
#define LQ_CHK_IDX(i, n) bchk_idx((i), (n))
#else
#define LQ_CHK(i, n) (i)
#define LQ_CHK_IDX(i, n) (i)
#endif

int bounds_hits(unsigned int *out) {
#ifdef LQ_BOUNDS_CHECK
    return cudaMemcpyFromSymbol(out, bounds_hits_dev, sizeof(unsigned int)) == cudaSuccess ? 1 : -1;
#else
    *out = 0;
    return 0;
#endif
}

template <typename T>
struct Prec;

// explicitly rounded products and fused multiply-adds: the FIRE update of a
// site is then the same operation sequence in every kernel that inlines it
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
struct StepArgs {
    typename Prec<T>::Q *q[2];
    T *v[2], *F[2];
    T *Fonly;                 // force-only output (5 N)
    const typename Prec<T>::Q *qonly;  // force-only input (5 N)
    Geometry g;
    LatticeDev L;
    T A, B, C, L1, L2, L3, S0;
    T L4, L6;                 // chiral and cubic distortion terms (three-constant form)
    T fext[5];                // force of the external fields (the same at every site)
    int fields;               // fext is not zero
    FireDev *st;
    double *partials;         // 4 doubles per block
    int zchunk;
    int force_only;
    unsigned tma_extra;       // testing: bytes a plane's barrier expects beyond its copies
                              // (lq_inject_fault LQ_FAULT_COPY_WAIT); 0 otherwise
    int zbeg, zend;           // the planes the step updates (a slab owns [zbeg, zend))
    int reduce_only;          // slab of a decomposed lattice: the last block leaves the
                              // slab's sums (P, |F|^2, |v|^2, max) in the FIRE state and
                              // the scalar update waits for the sums of every slab
};

__device__ __forceinline__ int wrap_coord(int g, int n, int periodic) {
    if (g >= 0 && g < n) return g;
    if (periodic) {
        if (g == -1) return n - 1;
        if (g == n) return 0;
    }
    return -1;
}

// Storage and arithmetic of the two forms.  FP64: Q, v, F in double.  FP32
// form: Q in 32-bit fixed point (exact integer differences), v and F in
// float, every stencil and bulk operation in float.
template <>
struct Prec<double> {
    using Q = double;
    static constexpr double scale = 1.0;   // storage unit of Q
    __device__ static __forceinline__ double val(double q) { return q; }
    __device__ static __forceinline__ double diff(double a, double b) { return b - a; }
    // q + alpha v + beta F as two fused multiply-adds; never out of range in FP64
    __device__ static __forceinline__ double drift(double q, double v, double f, double alpha,
                                                   double beta, bool &bad) {
        return __fma_rn(alpha, v, __fma_rn(beta, f, q));
    }
};
template <>
struct Prec<float> {
    using Q = int;
    static constexpr double scale = QFIX_SCALE;
    __device__ static __forceinline__ float val(int q) { return __int2float_rn(q) * float(QFIX_INV); }
    __device__ static __forceinline__ float diff(int a, int b) {
        return __int2float_rn(b - a) * float(QFIX_INV);
    }
    // q + alpha v + beta F with alpha, beta in fixed-point units.  A step
    // that would leave |q| < 2 (or is not finite) keeps q and raises the
    // divergence flag.  |u| < 2^29 and |q| < 2^29 keep q + u inside int32;
    // the conversion saturates (NaN -> 0), and the sum is formed unsigned so
    // that a rejected step never overflows.
    __device__ static __forceinline__ int drift(int q, float v, float f, float alpha, float beta,
                                                bool &bad) {
        const float lim = float(QFIX_LIMIT * QFIX_SCALE);
        const unsigned ilim = (unsigned)(QFIX_LIMIT * QFIX_SCALE);
        const float u = __fmaf_rn(alpha, v, __fmul_rn(beta, f));
        const int qn = (int)((unsigned)q + (unsigned)__float2int_rn(u));
        const bool ok = fabsf(u) < lim && (unsigned)qn + ilim < 2u * ilim;
        bad |= !ok;
        return ok ? qn : q;
    }
};

// ---- the FIRE update of a site, five components at a time -------------------
// FP64: scalar.  FP32 form: components (0,1) and (2,3) as pairs through the
// packed two-lane FP32 instructions (FFMA2 / FADD2 / FMUL2 of sm_100 and
// later), component 4 alone; each lane rounds exactly as the scalar
// instruction would.
template <typename T>
struct Site5;
template <>
struct Site5<double> {
    // q + alpha v + beta F; never out of range in FP64
    __device__ static __forceinline__ void drift(const double *q, const double *v, const double *f,
                                                 double alpha, double beta, double *out, bool &bad,
                                                 bool checked) {
#pragma unroll
        for (int c = 0; c < 5; ++c) out[c] = Prec<double>::drift(q[c], v[c], f[c], alpha, beta, bad);
    }
    // v_new = v_mix + dt/2 (F_old + F_new) = cv v + (cF + dt/2) F_old + dt/2 F_new
    // (cFh = cF + dt/2)
    __device__ static __forceinline__ void kick(const double *vold, const double *fold, const double *fn,
                                                double cv, double cFh, double hdt, double *vn) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            double vx = fma_rn(cFh, fold[c], mul_rn(cv, vold[c]));
            vn[c] = fma_rn(hdt, fn[c], vx);
        }
    }
};
template <>
struct Site5<float> {
    // fixed-point drift; a staged ring site (checked = false) is also the
    // own site of the block that stores it, which checks its range
    __device__ static __forceinline__ void drift(const int *q, const float *v, const float *f,
                                                 float alpha, float beta, int *out, bool &bad,
                                                 bool checked) {
        const float2 A = make_float2(alpha, alpha), B = make_float2(beta, beta);
        float u[5];
#pragma unroll
        for (int c = 0; c < 4; c += 2) {
            float2 w = __ffma2_rn(A, make_float2(v[c], v[c + 1]),
                                  __fmul2_rn(B, make_float2(f[c], f[c + 1])));
            u[c] = w.x; u[c + 1] = w.y;
        }
        u[4] = __fmaf_rn(alpha, v[4], __fmul_rn(beta, f[4]));
        const float lim = float(QFIX_LIMIT * QFIX_SCALE);
        const unsigned ilim = (unsigned)(QFIX_LIMIT * QFIX_SCALE);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const int qn = (int)((unsigned)q[c] + (unsigned)__float2int_rn(u[c]));
            if (checked) {
                const bool ok = fabsf(u[c]) < lim && (unsigned)qn + ilim < 2u * ilim;
                bad |= !ok;
                out[c] = ok ? qn : q[c];
            } else {
                out[c] = qn;
            }
        }
    }
    // the old-state part of the kick, cv v + cFh F (the same operations as
    // in kick)
    __device__ static __forceinline__ void mix_old(const float *vold, const float *fold, float cv,
                                                   float cFh, float *w) {
        const float2 CV = make_float2(cv, cv), CF = make_float2(cFh, cFh);
#pragma unroll
        for (int c = 0; c < 4; c += 2) {
            const float2 vo = make_float2(vold[c], vold[c + 1]), fo = make_float2(fold[c], fold[c + 1]);
            const float2 vx = __ffma2_rn(CF, fo, __fmul2_rn(CV, vo));
            w[c] = vx.x; w[c + 1] = vx.y;
        }
        w[4] = __fmaf_rn(cFh, fold[4], __fmul_rn(cv, vold[4]));
    }
    // kick from the kept old-state part: v_new = w + dt/2 F_new
    __device__ static __forceinline__ void kick_w(const float *w, const float *fn, float hdt, float *vn) {
        const float2 H = make_float2(hdt, hdt);
#pragma unroll
        for (int c = 0; c < 4; c += 2) {
            const float2 wv = __ffma2_rn(H, make_float2(fn[c], fn[c + 1]), make_float2(w[c], w[c + 1]));
            vn[c] = wv.x; vn[c + 1] = wv.y;
        }
        vn[4] = __fmaf_rn(hdt, fn[4], w[4]);
    }
    __device__ static __forceinline__ void kick(const float *vold, const float *fold, const float *fn,
                                                float cv, float cFh, float hdt, float *vn) {
        const float2 CV = make_float2(cv, cv), CF = make_float2(cFh, cFh), H = make_float2(hdt, hdt);
#pragma unroll
        for (int c = 0; c < 4; c += 2) {
            const float2 vo = make_float2(vold[c], vold[c + 1]), fo = make_float2(fold[c], fold[c + 1]);
            const float2 vx = __ffma2_rn(CF, fo, __fmul2_rn(CV, vo));
            const float2 w = __ffma2_rn(H, make_float2(fn[c], fn[c + 1]), vx);
            vn[c] = w.x; vn[c + 1] = w.y;
        }
        const float vx4 = __fmaf_rn(cFh, fold[4], __fmul_rn(cv, vold[4]));
        vn[4] = __fmaf_rn(hdt, fn[4], vx4);
    }
};

// five-component sums: FP32 pairs (0,1), (2,3) through FADD2, then 4
__device__ __forceinline__ void add5(const double *a, const double *b, double *o) {
#pragma unroll
    for (int c = 0; c < 5; ++c) o[c] = a[c] + b[c];
}
__device__ __forceinline__ void add5(const float *a, const float *b, float *o) {
#pragma unroll
    for (int c = 0; c < 4; c += 2) {
        float2 w = __fadd2_rn(make_float2(a[c], a[c + 1]), make_float2(b[c], b[c + 1]));
        o[c] = w.x; o[c + 1] = w.y;
    }
    o[4] = __fadd_rn(a[4], b[4]);
}
// FP32 form: Q in its storage unit (fixed point) to float
__device__ __forceinline__ void q_values(const double *q, double *o) {
#pragma unroll
    for (int c = 0; c < 5; ++c) o[c] = q[c];
}
__device__ __forceinline__ void q_values(const int *q, float *o) {
    const float2 s = make_float2(float(QFIX_INV), float(QFIX_INV));
#pragma unroll
    for (int c = 0; c < 4; c += 2) {
        float2 w = __fmul2_rn(make_float2(__int2float_rn(q[c]), __int2float_rn(q[c + 1])), s);
        o[c] = w.x; o[c + 1] = w.y;
    }
    o[4] = __fmul_rn(__int2float_rn(q[4]), float(QFIX_INV));
}

// Per-thread FIRE contributions of the sites a thread owns: P = sum F.v,
// |F|^2, |v|^2 and the largest site |F|^2 (Algorithm 1's power, norms and the
// convergence residual).  FP64 form: FP64 products and sums.  FP32 form: the
// same quantities without FP64 work per site, to FP64 accuracy.  Every
// product of two floats is split without error into p = fl(a b) and
// e = fma(a, b, -p) (the error-free product of Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005); the p are
// summed with Knuth's two-sum, which returns the rounding error of each
// addition exactly, and the small parts (the e and the two-sum errors) are
// added in plain float, where their own rounding is of order 2^-48 of the
// result.  A site's P and |F|^2 are formed this way as float-float pairs,
// the largest |F|^2 is kept as a normalised pair, and each site's pair is
// added into the thread's float-float sums; from there on the sums are FP64.
template <typename T>
struct FireSums;
template <>
struct FireSums<double> {
    double p = 0.0, f = 0.0, v = 0.0, r = 0.0;
    __device__ __forceinline__ void site(const double *fn, const double *vn) {
        double pv = 0.0, ff = 0.0, vv = 0.0;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            pv = fma_rn(fn[c], vn[c], pv);
            ff = fma_rn(fn[c], fn[c], ff);
            vv = fma_rn(vn[c], vn[c], vv);
        }
        p += pv; f += ff; v += vv;
        r = fmax(r, ff);
    }
    __device__ __forceinline__ void get(double &P, double &F2, double &V2, double &R2) const {
        P = p; F2 = f; V2 = v; R2 = r;
    }
};
// two-sum on two lanes: s + e = a + b exactly, s = fl(a + b) (a - b is
// written fma(-1, b, a): an exact product and one rounding, as the subtraction)
__device__ __forceinline__ float2 two_sum2(float2 a, float2 b, float2 &e) {
    const float2 M1 = make_float2(-1.f, -1.f);
    const float2 s = __fadd2_rn(a, b);
    const float2 bp = __ffma2_rn(M1, a, s);
    e = __fadd2_rn(__ffma2_rn(M1, __ffma2_rn(M1, bp, s), a), __ffma2_rn(M1, bp, b));
    return s;
}
// error-free product on two lanes: p + e = a b exactly
__device__ __forceinline__ float2 two_prod2(float2 a, float2 b, float2 &e) {
    const float2 p = __fmul2_rn(a, b);
    e = __ffma2_rn(a, b, make_float2(-p.x, -p.y));
    return p;
}
template <>
struct FireSums<float> {
    float2 pf_hi = make_float2(0.f, 0.f), pf_lo = pf_hi;   // lanes (P, |F|^2)
    float2 vv_hi = make_float2(0.f, 0.f), vv_lo = vv_hi;   // |v|^2 in two lanes
    float r_hi = 0.f, r_lo = 0.f;                           // largest site |F|^2
    __device__ __forceinline__ void site(const float *fn, const float *vn) {
        // the site's (F.v, |F|^2) as float-float pairs (s, lo), summed as a
        // tree ((0 + 1) + (2 + 3)) + 4 to shorten the dependent chain
        float2 p[5], e[5], t0, t1, t2, t3, t;
#pragma unroll
        for (int c = 0; c < 5; ++c)
            p[c] = two_prod2(make_float2(fn[c], fn[c]), make_float2(vn[c], fn[c]), e[c]);
        const float2 s01 = two_sum2(p[0], p[1], t0);
        const float2 s23 = two_sum2(p[2], p[3], t1);
        const float2 s03 = two_sum2(s01, s23, t2);
        const float2 s = two_sum2(s03, p[4], t3);
        const float2 lo = __fadd2_rn(__fadd2_rn(__fadd2_rn(e[0], e[1]), __fadd2_rn(e[2], e[3])),
                                     __fadd2_rn(__fadd2_rn(e[4], t0), __fadd2_rn(__fadd2_rn(t1, t2), t3)));
        // largest site |F|^2: normalise the pair (fast two-sum, |s| >= |lo|),
        // compare high parts first
        {
            const float h = __fadd_rn(s.y, lo.y);
            const float l = __fsub_rn(lo.y, __fsub_rn(h, s.y));
            if (h > r_hi || (h == r_hi && l > r_lo)) { r_hi = h; r_lo = l; }
        }
        pf_hi = two_sum2(pf_hi, s, t);
        pf_lo = __fadd2_rn(pf_lo, __fadd2_rn(t, lo));
        // |v|^2: components (0, 1), (2, 3), (4, -) summed within the site,
        // then one two-sum into the thread's pair
        {
            float2 ea, eb, ec, ta, tb, tc;
            const float2 va = make_float2(vn[0], vn[1]), vb = make_float2(vn[2], vn[3]),
                         vc = make_float2(vn[4], 0.f);
            const float2 pa = two_prod2(va, va, ea), pb = two_prod2(vb, vb, eb), pcc = two_prod2(vc, vc, ec);
            const float2 sv = two_sum2(two_sum2(pa, pb, ta), pcc, tb);
            vv_hi = two_sum2(vv_hi, sv, tc);
            vv_lo = __fadd2_rn(vv_lo, __fadd2_rn(__fadd2_rn(__fadd2_rn(ea, eb), __fadd2_rn(ec, ta)),
                                                 __fadd2_rn(tb, tc)));
        }
    }
    __device__ __forceinline__ void get(double &P, double &F2, double &V2, double &R2) const {
        P = (double)pf_hi.x + (double)pf_lo.x;
        F2 = (double)pf_hi.y + (double)pf_lo.y;
        V2 = ((double)vv_hi.x + (double)vv_lo.x) + ((double)vv_hi.y + (double)vv_lo.y);
        R2 = (double)r_hi + (double)r_lo;
    }
};

template <typename T>
__device__ __forceinline__ T inv_count(uint8_t m, int k) {
    int n = ((m & m_fwd(k)) ? 1 : 0) + ((m & m_bwd(k)) ? 1 : 0);
    return n == 2 ? T(0.5) : T(1);
}

// J^T of the matrix whose column k is Delta[:, k] (all else 0)
template <int K, typename T>
__device__ __forceinline__ void jt_col(const T *d, T *o) {
    if (K == 0) { o[0] = d[0]; o[1] = d[1]; o[2] = d[2]; o[3] = T(0); o[4] = T(0); }
    if (K == 1) { o[0] = T(0); o[1] = d[1]; o[2] = T(0); o[3] = d[3]; o[4] = d[4]; }
    if (K == 2) { o[0] = d[0] + d[3]; o[1] = T(0); o[2] = d[2]; o[3] = d[0] + d[3]; o[4] = d[4]; }
}

// J^T X_k for the cross terms, from the means m_a, m_b of the other axes
template <int K, typename T>
__device__ __forceinline__ void jt_cross(const T *ma, const T *mb, T L2, T L3, T *o) {
    constexpr int a = K == 0 ? 1 : 0;
    constexpr int b = K == 2 ? 1 : 2;
    T X[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        X[i][K] = L2 * (sym(ma, i, a) + sym(mb, i, b));
        X[i][a] = L3 * sym(ma, i, K);
        X[i][b] = L3 * sym(mb, i, K);
    }
    o[0] = X[0][0] - X[2][2];
    o[1] = X[0][1] + X[1][0];
    o[2] = X[0][2] + X[2][0];
    o[3] = X[1][1] - X[2][2];
    o[4] = X[1][2] + X[2][1];
}

// ---- chiral (L4) and cubic (L6) terms of Eq. (fdistortionFull) -------------
// Averaged over the allowed differences like the other terms, the density
// of a site adds  L4/2 eps_lik Q_lj m_k[ij]  +  L6/2 [ sum_k Q_kk <|D_k|^2>
// + sum_{l != k} Q_lk m_l . m_k ]  (Q the site's tensor, m_k the mean of its
// allowed differences along k, <|D_k|^2> the mean of their squared norms).
// Its derivative enters the link flux through X_K (dE/dm_K, below), a
// diagonal coefficient L6 Q_KK on the squared differences (link_flux), and
// a local term through the site's own Q (jt_extra_local).

__host__ __device__ constexpr int levi3(int i, int j, int k) {
    return (i - j) * (j - k) * (k - i) / 2;
}
template <int K, typename T>
__device__ __forceinline__ T qdiag(const T *q) {
    return K == 0 ? q[0] : (K == 1 ? q[3] : -q[0] - q[3]);
}
// Frobenius product of two symmetric traceless tensors given as 5 components
template <typename T>
__device__ __forceinline__ T dot5(const T *a, const T *b) {
    return a[0] * b[0] + a[3] * b[3] + (a[0] + a[3]) * (b[0] + b[3]) +
           T(2) * (a[1] * b[1] + a[2] * b[2] + a[4] * b[4]);
}
// J^T of a general 3x3 matrix
template <typename T>
__device__ __forceinline__ void jt_mat(T X[3][3], T *o) {
    o[0] = X[0][0] - X[2][2];
    o[1] = X[0][1] + X[1][0];
    o[2] = X[0][2] + X[2][0];
    o[3] = X[1][1] - X[2][2];
    o[4] = X[1][2] + X[2][1];
}
// J^T of dE/dm_K from the L4 and L6 terms at a site with tensor q and means
// ma, mb along the other two axes:  L4/2 eps_{l i K} Q_{l j}
// + L6 (Q_{a K} m_a[ij] + Q_{b K} m_b[ij])
template <int K, typename T>
__device__ __forceinline__ void jt_extra_x(const T *q, const T *ma, const T *mb, T L4, T L6, T *o) {
    constexpr int a = K == 0 ? 1 : 0;
    constexpr int b = K == 2 ? 1 : 2;
    const T qa = sym(q, a, K), qb = sym(q, b, K);
    T X[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T chi = T(0);
#pragma unroll
            for (int l = 0; l < 3; ++l)
                if (levi3(l, i, K) != 0) chi += T(levi3(l, i, K)) * sym(q, l, j);
            X[i][j] = T(0.5) * L4 * chi + L6 * (qa * sym(ma, i, j) + qb * sym(mb, i, j));
        }
    jt_mat(X, o);
}
// J^T of dE/dQ through the site's own tensor: L4/2 sum_{i,k} eps_{a i k}
// m_k[i b]; L6/2 <|D_k|^2> on (k, k) and L6/2 m_l . m_k on (l, k), l != k
template <typename T>
__device__ __forceinline__ void jt_extra_local(const T *mx, const T *my, const T *mz, const T *sq,
                                               T L4, T L6, T *o) {
    const T *mk[3] = {mx, my, mz};
    T G[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            T chi = T(0);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (levi3(a, i, k) != 0) chi += T(levi3(a, i, k)) * sym(mk[k], i, b);
            G[a][b] = T(0.5) * L4 * chi;
        }
#pragma unroll
    for (int k = 0; k < 3; ++k) G[k][k] += T(0.5) * L6 * sq[k];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (l != k) G[l][k] += T(0.5) * L6 * dot5(mk[l], mk[k]);
    jt_mat(G, o);
}

// Shared-memory staging of one block.  A plane slot keeps the drifted Q of
// the tile and its ring with the five components of a site packed so that a
// site loads in 2 (fixed point: int4 + int) or 3 (FP64: 2 double2 + double)
// conflict-free instructions: [c0..c3 | c4] or [c0 c1 | c2 c3 | c4] arrays.
// FP32 form: each own site's old-state part of the kick, cv v + cFh F, is
// kept in shared memory from its drift to its kick (three planes), instead
// of re-reading v, F; not in the L1/L2/L3 form, where at 128 registers it
// causes spills and runs slower
template <typename T, int FORM>
__host__ __device__ constexpr bool keeps_w() { return sizeof(T) == 4 && FORM != 1; }

template <typename T, int TX, int TY>
struct Smem {
    using QS = typename Prec<T>::Q;
    static constexpr int SX = TX + 2, SY = TY + 2;
    static constexpr int PL = ((SX * SY + 3) / 4) * 4;          // sites per plane slot
    static constexpr int SLOT_BYTES = 5 * sizeof(QS) * PL;      // multiple of 16
    unsigned char *Q;  // [slots] x SLOT_BYTES
    T *X;              // [2][5][PL] cross terms of one plane (general path):
                       // the plane barrier orders the last reads of a plane
                       // before the first writes of the next
    T *D;              // [2][2][5][PL] FP64 three-constant form: the central
                       // differences D_y, D_z of a plane (regular path)
    T *W;              // [3][5][TX*TY] FP32 form: each own site's mixed old
                       // velocity cv v + (cF + dt/2) F, kept from its drift
    uint8_t *M;        // [slots][PL]
    __device__ __forceinline__ T &w(int slot, int c) {
        return W[(LQ_CHK(slot, 3) * 5 + LQ_CHK(c, 5)) * (TX * TY) + threadIdx.x];
    }
    __device__ __forceinline__ int idx(int lx, int ly) const { return LQ_CHK(ly, SY) * SX + LQ_CHK(lx, SX); }
    __device__ __forceinline__ QS &q(int slot, int c, int lx, int ly) {
        unsigned char *b = Q + LQ_CHK(slot, 5) * SLOT_BYTES;
        int i = idx(lx, ly);
        if (sizeof(QS) == 4) {
            if (c < 4) return reinterpret_cast<QS *>(b)[4 * i + c];
            return reinterpret_cast<QS *>(b + 16 * PL)[i];
        }
        if (c < 2) return reinterpret_cast<QS *>(b)[2 * i + c];
        if (c < 4) return reinterpret_cast<QS *>(b + 16 * PL)[2 * i + c - 2];
        return reinterpret_cast<QS *>(b + 32 * PL)[i];
    }
    __device__ __forceinline__ void load5(int slot, int lx, int ly, QS *o) const {
        const unsigned char *b = Q + LQ_CHK(slot, 5) * SLOT_BYTES;
        int i = idx(lx, ly);
        if constexpr (sizeof(QS) == 4) {
            int4 a = reinterpret_cast<const int4 *>(b)[i];
            o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
            o[4] = reinterpret_cast<const QS *>(b + 16 * PL)[i];
        } else {
            double2 a = reinterpret_cast<const double2 *>(b)[i];
            double2 c = reinterpret_cast<const double2 *>(b + 16 * PL)[i];
            o[0] = a.x; o[1] = a.y; o[2] = c.x; o[3] = c.y;
            o[4] = reinterpret_cast<const QS *>(b + 32 * PL)[i];
        }
    }
    __device__ __forceinline__ void store5(int slot, int lx, int ly, const QS *v) {
        unsigned char *b = Q + LQ_CHK(slot, 5) * SLOT_BYTES;
        int i = idx(lx, ly);
        if constexpr (sizeof(QS) == 4) {
            reinterpret_cast<int4 *>(b)[i] = make_int4(v[0], v[1], v[2], v[3]);
            reinterpret_cast<QS *>(b + 16 * PL)[i] = v[4];
        } else {
            reinterpret_cast<double2 *>(b)[i] = make_double2(v[0], v[1]);
            reinterpret_cast<double2 *>(b + 16 * PL)[i] = make_double2(v[2], v[3]);
            reinterpret_cast<QS *>(b + 32 * PL)[i] = v[4];
        }
    }
    __device__ __forceinline__ uint8_t &m(int slot, int lx, int ly) {
        return M[LQ_CHK(slot, 5) * PL + idx(lx, ly)];
    }

    __device__ __forceinline__ T &x(int ax, int c, int lx, int ly) {
        return X[(LQ_CHK(ax, 2) * 5 + LQ_CHK(c, 5)) * PL + idx(lx, ly)];
    }
    __device__ __forceinline__ T &d(int slot, int ax, int c, int lx, int ly) {
        return D[((LQ_CHK(slot, 2) * 2 + LQ_CHK(ax, 2)) * 5 + LQ_CHK(c, 5)) * PL + idx(lx, ly)];
    }
};

// the FP64 three-constant form shares the central differences of a plane
// between the mixed differences of neighbouring sites (FP64 operations are
// that form's limit): D_y(s) = q(s + y) - q(s - y) and D_z(s) = q(s + z) -
// q(s - z), so that E_xy(j) = D_y(j + x) - D_y(j - x), E_xz(j) = D_z(j + x) -
// D_z(j - x) and E_yz(j) = D_z(j + y) - D_z(j - y) -- the same operations in
// the same order as (a - b) - (c - d) on the four diagonal neighbours
template <typename T, int FORM>
constexpr bool shared_diffs() { return sizeof(T) == 8 && FORM >= 1; }

// mean of the allowed one-sided differences along axis K at (lx, ly) of
// plane slot sc; splus / sminus are the slots of the planes above / below
template <int K, typename T, int TX, int TY>
__device__ __forceinline__ void mean_diff(Smem<T, TX, TY> &S, int lx, int ly, int sc, int splus,
                                          int sminus, T *out) {
    uint8_t m = S.m(sc, lx, ly);
    T f = (m & m_fwd(K)) ? T(1) : T(0);
    T b = (m & m_bwd(K)) ? T(1) : T(0);
    T w = (f + b == T(2)) ? T(0.5) : T(1);
    using P = Prec<T>;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        typename P::Q q0 = S.q(sc, c, lx, ly), qf, qb;
        if (K == 0) { qf = S.q(sc, c, lx + 1, ly); qb = S.q(sc, c, lx - 1, ly); }
        if (K == 1) { qf = S.q(sc, c, lx, ly + 1); qb = S.q(sc, c, lx, ly - 1); }
        if (K == 2) { qf = S.q(splus, c, lx, ly); qb = S.q(sminus, c, lx, ly); }
        out[c] = w * (f * P::diff(q0, qf) + b * P::diff(qb, q0));
    }
}

// mean over the allowed one-sided differences along axis K of their squared
// norm |D|^2 (the L6 term's <|D_K|^2>)
template <int K, typename T, int TX, int TY>
__device__ __forceinline__ T mean_sq(Smem<T, TX, TY> &S, int lx, int ly, int sc, int splus,
                                     int sminus) {
    uint8_t m = S.m(sc, lx, ly);
    const bool f = (m & m_fwd(K)) != 0, b = (m & m_bwd(K)) != 0;
    using P = Prec<T>;
    T df[5], db[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        typename P::Q q0 = S.q(sc, c, lx, ly), qf, qb;
        if (K == 0) { qf = S.q(sc, c, lx + 1, ly); qb = S.q(sc, c, lx - 1, ly); }
        if (K == 1) { qf = S.q(sc, c, lx, ly + 1); qb = S.q(sc, c, lx, ly - 1); }
        if (K == 2) { qf = S.q(splus, c, lx, ly); qb = S.q(sminus, c, lx, ly); }
        df[c] = P::diff(q0, qf);
        db[c] = P::diff(qb, q0);
    }
    T sum = (f ? dot5(df, df) : T(0)) + (b ? dot5(db, db) : T(0));
    return (f && b) ? T(0.5) * sum : sum;
}

// the five components of a staged site as values
template <typename T, int TX, int TY>
__device__ __forceinline__ void q_at(Smem<T, TX, TY> &S, int slot, int lx, int ly, T *o) {
#pragma unroll
    for (int c = 0; c < 5; ++c) o[c] = Prec<T>::val(S.q(slot, c, lx, ly));
}

// flux through the link (a, a + e_K); ma/mb masks, qa/qb drifted Q,
// xa/xb the J^T X_K cross terms at both ends (three-constant only)
template <int K, bool THREE, bool EXT = false, typename T>
__device__ __forceinline__ void link_flux(uint8_t ma, uint8_t mb, const typename Prec<T>::Q *qa,
                                          const typename Prec<T>::Q *qb, const T *xa, const T *xb,
                                          T L1, T L23, T *phi, T L6 = T(0)) {
    if (!(ma & M_SIM) || !(ma & m_fwd(K))) {
#pragma unroll
        for (int c = 0; c < 5; ++c) phi[c] = T(0);
        return;
    }
    T wa = inv_count<T>(ma, K), wb = inv_count<T>(mb, K);
    T d[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) d[c] = Prec<T>::diff(qa[c], qb[c]);
    if (!THREE) {
        T w = wa + wb;
#pragma unroll
        for (int c = 0; c < 5; ++c) phi[c] = w * d[c];
    } else {
        T j1[5], j2[5];
        jt_sym(d, j1);
        jt_col<K>(d, j2);
        T w = wa + wb;
#pragma unroll
        for (int c = 0; c < 5; ++c)
            phi[c] = w * (L1 * j1[c] + L23 * j2[c]) + wa * xa[c] + wb * xb[c];
        if (EXT) {
            // L6: the squared differences of each end weighted by its Q_KK
            T va[5], vb[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) { va[c] = Prec<T>::val(qa[c]); vb[c] = Prec<T>::val(qb[c]); }
            const T l6 = L6 * (wa * qdiag<K>(va) + wb * qdiag<K>(vb));
#pragma unroll
            for (int c = 0; c < 5; ++c) phi[c] += l6 * j1[c];
        }
    }
}

template <typename T>
__device__ __forceinline__ void bulk_force(const T *q, T A, T B, T C, T *out) {
    // -(A + C tr Q^2) J^T q - B d/dq tr Q^3 / 3 with f = Qzz = -(a + d): J^T q =
    // (2a + d, 2b, 2c, a + 2d, 2e) = j, tr Q^2 = q . j, and the cubic term
    // needs (Q^2)_xx - (Q^2)_zz = b^2 - e^2 - d (2a + d), (Q^2)_yy - (Q^2)_zz =
    // b^2 - c^2 - a (a + 2d), (Q^2)_xy = ce - bf, (Q^2)_xz = be - cd,
    // (Q^2)_yz = bc - ae (the squares of Qzz folded into j)
    const T a = q[0], b = q[1], c = q[2], d = q[3], e = q[4];
    const T j0 = T(2) * a + d, j3 = T(2) * d + a, j1 = T(2) * b, j2 = T(2) * c, j4 = T(2) * e;
    const T tr2 = a * j0 + b * j1 + c * j2 + d * j3 + e * j4;
    const T bb = b * b;
    const T dxz = (bb - e * e) - d * j0;
    const T dyz = (bb - c * c) - a * j3;
    const T sxy = c * e + b * (a + d);
    const T sxz = b * e - c * d;
    const T syz = b * c - a * e;
    const T ng = -(A + C * tr2);
    const T nB = -B, n2B = T(-2) * B;
    out[0] = ng * j0 + nB * dxz;
    out[1] = ng * j1 + n2B * sxy;
    out[2] = ng * j2 + n2B * sxz;
    out[3] = ng * j3 + nB * dyz;
    out[4] = ng * j4 + n2B * syz;
}

// anchoring force of one record (Nobili-Durand or Fournier-Galatola)
template <typename T>
__device__ __forceinline__ T nd_target_diff(const typename Prec<T>::Q q, const AnchorRec<T> &r, int c);
template <>
__device__ __forceinline__ double nd_target_diff<double>(double q, const AnchorRec<double> &r, int c) {
    return q - r.a[c];
}
template <>
__device__ __forceinline__ float nd_target_diff<float>(int q, const AnchorRec<float> &r, int c) {
    return Prec<float>::diff(r.qi[c], q);   // exact fixed-point difference
}

template <typename T>
__device__ __forceinline__ void anchor_force(const T *q, const typename Prec<T>::Q *qraw,
                                             const AnchorRec<T> &r, T S0, T *out) {
    if (r.kind == 1) {
        T d[5], j[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) d[c] = nd_target_diff<T>(qraw[c], r, c);
        jt_sym(d, j);
#pragma unroll
        for (int c = 0; c < 5; ++c) out[c] = -T(2) * r.W * j[c];
    } else {
        // G = 2 W R, R = Qt - P Qt P = nu w^T + w nu^T - (nu.w) nu nu^T, w = Qt nu
        const T nx = r.a[0], ny = r.a[1], nz = r.a[2];
        T hs = T(0.5) * S0;
        T wx = q[0] * nx + q[1] * ny + q[2] * nz + hs * nx;
        T wy = q[1] * nx + q[3] * ny + q[4] * nz + hs * ny;
        T wz = q[2] * nx + q[4] * ny + (-q[0] - q[3]) * nz + hs * nz;
        T nw = nx * wx + ny * wy + nz * wz;
        T Rxx = T(2) * nx * wx - nw * nx * nx;
        T Ryy = T(2) * ny * wy - nw * ny * ny;
        T Rzz = T(2) * nz * wz - nw * nz * nz;
        T Rxy = nx * wy + wx * ny - nw * nx * ny;
        T Rxz = nx * wz + wx * nz - nw * nx * nz;
        T Ryz = ny * wz + wy * nz - nw * ny * nz;
        T w2 = T(2) * r.W;
        out[0] = -w2 * (Rxx - Rzz);
        out[1] = -w2 * T(2) * Rxy;
        out[2] = -w2 * T(2) * Rxz;
        out[3] = -w2 * (Ryy - Rzz);
        out[4] = -w2 * T(2) * Ryz;
    }
}

template <typename T>
__device__ __forceinline__ const AnchorRec<T> *find_record(const Geometry &g, const LatticeDev &L,
                                                           int x, int y, int z) {
    long long row = (long long)z * L.ny + y;
    int lo = g.row_start[row], hi = g.row_start[row + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int xm = g.rec_x[mid];
        if (xm == x) return reinterpret_cast<const AnchorRec<T> *>(g.recs) + mid;
        if (xm < x) lo = mid + 1; else hi = mid - 1;
    }
    return nullptr;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// block-wide fixed-order reduction of 4 values into thread 0
template <int NT>
__device__ __forceinline__ void block_reduce4(double &p, double &f, double &w, double &r,
                                              double *red) {
    constexpr int NW = NT / 32;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    p = warp_sum(p); f = warp_sum(f); w = warp_sum(w); r = warp_max(r);
    if (lane == 0) { red[wid] = p; red[NW + wid] = f; red[2 * NW + wid] = w; red[3 * NW + wid] = r; }
    __syncthreads();
    if (wid == 0) {
        p = lane < NW ? red[lane] : 0.0;
        f = lane < NW ? red[NW + lane] : 0.0;
        w = lane < NW ? red[2 * NW + lane] : 0.0;
        r = lane < NW ? red[3 * NW + lane] : 0.0;
        p = warp_sum(p); f = warp_sum(f); w = warp_sum(w); r = warp_max(r);
    }
    __syncthreads();
}

// coefficients of the next step from (cv, cF, dt_step) for FIRE, fixed for
// the descent methods: GD drifts x + eta F; Nesterov keeps y = x + mu v and
// advances it by y' = y + mu^2 v + eta (1 + mu) F(y), v' = mu v + eta F(y)
__device__ __forceinline__ void set_coefficients(FireDev *st) {
    if (st->method == 0) {
        st->c_alpha = st->dt_step * st->cv;
        st->c_beta = st->dt_step * st->cF + 0.5 * st->dt_step * st->dt_step;
        st->c_kick = 0.5 * st->dt_step;
    } else {
        const double mu = st->method == 2 ? st->mu : 0.0;
        st->cv = mu; st->cF = st->eta; st->dt_step = st->eta;
        st->c_alpha = mu * mu;
        st->c_beta = st->eta * (1.0 + mu);
        st->c_kick = 0.0;
    }
}

// FIRE scalar machine (Algorithm 1), run by one thread after the reductions;
// the descent methods share its bookkeeping (iterations, convergence,
// divergence, max_iter) with fixed coefficients
__device__ void fire_update(FireDev *st, double P, double F2, double v2, double r2) {
    st->P = P; st->F2 = F2; st->v2 = v2; st->r2 = r2;
    st->cur ^= 1;
    st->kcount += 1;
    bool bad = !isfinite(P) || !isfinite(F2) || !isfinite(v2) || !isfinite(r2);
    double rmax = sqrt(r2);
    st->cv = 1.0; st->cF = 0.0;
    if (st->kcount == 1) {           // the evaluation of F(q0)
        if (bad) st->status = FIRE_DIVERGED;
        else if (rmax < st->tol) st->status = FIRE_CONVERGED;
        st->dt_step = st->dt;
        set_coefficients(st);
        return;
    }
    st->iter += 1;
    if (bad) { st->status = FIRE_DIVERGED; return; }
    if (rmax < st->tol) { st->status = FIRE_CONVERGED; return; }
    if (st->iter >= st->max_iter) { st->status = FIRE_MAXITER; return; }
    if (st->method != 0) { set_coefficients(st); return; }
    double a = 1.0, b = 0.0;
    double nF = sqrt(F2), nv = sqrt(v2);
    if (nF > 0.0) { a = 1.0 - st->alpha; b = st->alpha * nv / nF; }
    if (P > 0.0) {
        st->npos += 1;
        if (st->npos > st->n_min) {
            st->dt = fmin(st->dt * st->f_inc, st->dt_max);
            st->alpha *= st->f_alpha;
        }
    } else {
        st->npos = 0;
        st->dt *= st->f_dec;
        st->alpha = st->alpha0;
        a = 0.0; b = 0.0;
    }
    st->cv = a; st->cF = b; st->dt_step = st->dt;
    set_coefficients(st);
}

// second differences and mixed differences in the storage format: exact
// integer arithmetic for the fixed-point form, one conversion per value
template <typename T>
struct Stencil;
template <>
struct Stencil<double> {
    static constexpr double scale = 1.0;
    // a + b - 2c as one add and one fused multiply-add (two FP64 operations,
    // the FP64 form's limiting resource, instead of three)
    __device__ static __forceinline__ double sec(double a, double b, double c) { return __fma_rn(-2.0, c, a + b); }
    __device__ static __forceinline__ double mix(double a, double b, double c, double d) {
        return (a - b) - (c - d);
    }
    __device__ static __forceinline__ double dif(double a, double b) { return a - b; }
};
template <>
struct Stencil<float> {
    static constexpr double scale = QFIX_INV;
    __device__ static __forceinline__ float sec(int a, int b, int c) { return __int2float_rn(a + b - 2 * c); }
    __device__ static __forceinline__ float mix(int a, int b, int c, int d) {
        return __int2float_rn((a - b) - (c - d));
    }
    __device__ static __forceinline__ float dif(int a, int b) { return __int2float_rn(a - b); }
};

// The cubic term L6/2 Q_lk dQ_ij/dx_l dQ_ij/dx_k at a regular site.  Averaged
// over the allowed differences, a site's density is L6/2 [sum_k Q_kk
// (|f_k|^2 + |b_k|^2)/2 + sum_{l != k} Q_lk C_l . C_k / 4] with f_k, b_k the
// forward and backward differences and C_k = f_k + b_k (dots over the nine
// entries).  Differentiating the sum over the site and its six neighbours
// with respect to Q(j) gives L6/2 (G_A + G_B), with G_A the density's own
// Q factor -- (|f_k|^2 + |b_k|^2)/2 at (k,k), C_l . C_k / 4 at (l,k) -- and
// G_B = sum_k [-Q_kk(j) D2_k + Q_kk(j - e_k) b_k - Q_kk(j + e_k) f_k]
//     + 1/2 sum_k sum_{l != k} [Q_lk(j - e_k) C_l(j - e_k) - Q_lk(j + e_k) C_l(j + e_k)]
// (D2_k = f_k - b_k); the force is -J^T (L6/2)(G_A + G_B).  Differences are
// in storage units, s is the value of one unit.  Inlined in the FP64 form;
// a call in the FP32 form, whose 128 registers would spill (l6_regular_call).
template <typename T, int TX, int TY>
__device__ __forceinline__ void l6_regular(Smem<T, TX, TY> &S, int lx, int ly, int sc, int sp, int sm,
                                           T L6h, T s, T *F) {
    using ST = Stencil<T>;
    using QS = typename Prec<T>::Q;
    QS c0[5], a[5], b[5];
    S.load5(sc, lx, ly, c0);
    T qv[5];
    q_values(c0, qv);
    T GB[5] = {T(0), T(0), T(0), T(0), T(0)};
    T nrm[3], C[3][5];
    T qo[3][2][2];   // neighbours' off-diagonal components (see the pairs below)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k == 0) { S.load5(sc, lx + 1, ly, a); S.load5(sc, lx - 1, ly, b); }
        if (k == 1) { S.load5(sc, lx, ly + 1, a); S.load5(sc, lx, ly - 1, b); }
        if (k == 2) { S.load5(sp, lx, ly, a); S.load5(sm, lx, ly, b); }
        T f[5], bk[5], av[5], bv[5];
        q_values(a, av);
        q_values(b, bv);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            f[c] = ST::dif(a[c], c0[c]);
            bk[c] = ST::dif(c0[c], b[c]);
            C[k][c] = ST::dif(a[c], b[c]);
        }
        nrm[k] = dot5(f, f) + dot5(bk, bk);
        const T qkk_c = k == 0 ? qv[0] : (k == 1 ? qv[3] : -qv[0] - qv[3]);
        const T qkk_p = k == 0 ? av[0] : (k == 1 ? av[3] : -av[0] - av[3]);
        const T qkk_m = k == 0 ? bv[0] : (k == 1 ? bv[3] : -bv[0] - bv[3]);
#pragma unroll
        for (int c = 0; c < 5; ++c) GB[c] += qkk_m * bk[c] - qkk_p * f[c] - qkk_c * (f[c] - bk[c]);
        // Q_lk of the neighbours along k for the two l != k:
        // k = x: (Q_xy, Q_xz); k = y: (Q_xy, Q_yz); k = z: (Q_xz, Q_yz)
        const int c1 = k == 2 ? 2 : 1, c2 = k == 0 ? 2 : 4;
        qo[k][0][0] = av[c1]; qo[k][0][1] = av[c2];
        qo[k][1][0] = bv[c1]; qo[k][1][1] = bv[c2];
    }
    // G_B's cross part from the central differences of the twelve edge
    // neighbours, grouped by the plane they lie in
    auto cross = [&](T qm, const T *cm, T qp, const T *cp) {
#pragma unroll
        for (int c = 0; c < 5; ++c) GB[c] += T(0.5) * (qm * cm[c] - qp * cp[c]);
    };
    {   // xy corners: C_y(j +- x) for (k = x, l = y), C_x(j +- y) for (k = y, l = x)
        QS pp[5], pm[5], mp[5], mm[5];
        S.load5(sc, lx + 1, ly + 1, pp); S.load5(sc, lx + 1, ly - 1, pm);
        S.load5(sc, lx - 1, ly + 1, mp); S.load5(sc, lx - 1, ly - 1, mm);
        T u[5], w[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) { u[c] = ST::dif(mp[c], mm[c]); w[c] = ST::dif(pp[c], pm[c]); }
        cross(qo[0][1][0], u, qo[0][0][0], w);
#pragma unroll
        for (int c = 0; c < 5; ++c) { u[c] = ST::dif(pm[c], mm[c]); w[c] = ST::dif(pp[c], mp[c]); }
        cross(qo[1][1][0], u, qo[1][0][0], w);
    }
    {   // xz edges: C_z(j +- x) for (k = x, l = z), C_x(j +- z) for (k = z, l = x)
        QS pp[5], pm[5], mp[5], mm[5];   // (x+, z+), (x+, z-), (x-, z+), (x-, z-)
        S.load5(sp, lx + 1, ly, pp); S.load5(sm, lx + 1, ly, pm);
        S.load5(sp, lx - 1, ly, mp); S.load5(sm, lx - 1, ly, mm);
        T u[5], w[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) { u[c] = ST::dif(mp[c], mm[c]); w[c] = ST::dif(pp[c], pm[c]); }
        cross(qo[0][1][1], u, qo[0][0][1], w);
#pragma unroll
        for (int c = 0; c < 5; ++c) { u[c] = ST::dif(pm[c], mm[c]); w[c] = ST::dif(pp[c], mp[c]); }
        cross(qo[2][1][0], u, qo[2][0][0], w);
    }
    {   // yz edges: C_z(j +- y) for (k = y, l = z), C_y(j +- z) for (k = z, l = y)
        QS pp[5], pm[5], mp[5], mm[5];   // (y+, z+), (y+, z-), (y-, z+), (y-, z-)
        S.load5(sp, lx, ly + 1, pp); S.load5(sm, lx, ly + 1, pm);
        S.load5(sp, lx, ly - 1, mp); S.load5(sm, lx, ly - 1, mm);
        T u[5], w[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) { u[c] = ST::dif(mp[c], mm[c]); w[c] = ST::dif(pp[c], pm[c]); }
        cross(qo[1][1][1], u, qo[1][0][1], w);
#pragma unroll
        for (int c = 0; c < 5; ++c) { u[c] = ST::dif(pm[c], mm[c]); w[c] = ST::dif(pp[c], mp[c]); }
        cross(qo[2][1][1], u, qo[2][0][1], w);
    }
    T jb[5];
    jt_sym(GB, jb);
    const T s2 = s * s;
    const T h = T(0.5) * s2;
    F[0] = -L6h * (h * (nrm[0] - nrm[2]) + s * jb[0]);
    F[1] = -L6h * (h * dot5(C[0], C[1]) + s * jb[1]);
    F[2] = -L6h * (h * dot5(C[0], C[2]) + s * jb[2]);
    F[3] = -L6h * (h * (nrm[1] - nrm[2]) + s * jb[3]);
    F[4] = -L6h * (h * dot5(C[1], C[2]) + s * jb[4]);
}

template <typename T, int TX, int TY>
__device__ __noinline__ void l6_regular_call(Smem<T, TX, TY> &S, int lx, int ly, int sc, int sp, int sm,
                                             T L6h, T s, T *F) {
    l6_regular(S, lx, ly, sc, sp, sm, L6h, s, F);
}

// Distortion force at a regular site: every site within the 19-point
// stencil and at distance 2 along the axes is simulated, so every allowed
// difference count is 2 and every weight 1/2.  Then the per-site cross terms
// X_k(j) cancel between the links (j - e_k, j) and (j, j + e_k), and
//   F = sum_k [ L1 J^T(D2_k) + (L2+L3) Jcol_k(D2_k) + 1/4 J^T X_k(E_ka, E_kb) ]
// with D2_k = q(j+e_k) + q(j-e_k) - 2 q(j) and the mixed differences
// E_ab = q(j+e_a+e_b) - q(j+e_a-e_b) - q(j-e_a+e_b) + q(j-e_a-e_b); an exact
// rearrangement of the general link-flux form for such sites.  Expanded per
// component (x, y, z: D2 along x, y, z; a, b, c: E_xy, E_xz, E_yz; s = x+y+z)
// the L2 and L3 terms only enter as L2 + L3:
//   F0 = L1 (2 s0 + s3) + L23 (x0 + z0 + z3) + L23/4 (a1 - c4)
//   F1 = 2 L1 s1 + L23 (x1 + y1) + L23/4 (a0 + a3 + b4 + c2)
//   F2 = 2 L1 s2 + L23 (x2 + z2) + L23/4 (a4 - b3 + c1)
//   F3 = L1 (s0 + 2 s3) + L23 (y3 + z0 + z3) + L23/4 (a1 - b2)
//   F4 = 2 L1 s4 + L23 (y4 + z4) + L23/4 (a2 + b1 - c0)
// FP64: Fb (the site's bulk and field force) starts each component's chain
// of fused multiply-adds, so the sum costs no separate additions
//
// With the chiral term and L6 = 0 (EXT) the averaged one-sided differences
// of L4/2 eps_lik Q_lj dQ_ij/dx_k at regular sites are the central
// differences C_k = q(j + e_k) - q(j - e_k), and the gradient of the energy
// is (L4/2) eps_aik C_k Q_ib; in the five components
//   F0 = -L4/2 (Cz1 - 2 Cy2 + Cx4)          F1 = -L4/2 (Cz3 - Cy4 + Cx2 - Cz0)
//   F2 = -L4/2 (Cz4 + 2 Cy0 + Cy3 - Cx1)    F3 = -L4/2 (2 Cx4 - Cz1 - Cy2)
//   F4 = -L4/2 (Cy1 - Cx0 - 2 Cx3 - Cz2)    (k4 = -L4/2 in storage units)
template <bool THREE, bool EXT = false, typename T, int TX, int TY>
__device__ __forceinline__ void regular_force(Smem<T, TX, TY> &S, int lx, int ly, int sc, int sp,
                                              int sm, int dslot, T L1s, T L23s, T L2q, T L3q,
                                              const T *Fb, T *Fd, T k4 = T(0), T L6h = T(0)) {
    using ST = Stencil<T>;
    using QS = typename Prec<T>::Q;
    T dx[5], dy[5], dz[5];
    T cx[5], cy[5], cz[5];
    {
        QS c0[5], a[5], b[5];
        S.load5(sc, lx, ly, c0);
        S.load5(sc, lx + 1, ly, a);
        S.load5(sc, lx - 1, ly, b);
#pragma unroll
        for (int c = 0; c < 5; ++c) dx[c] = ST::sec(a[c], b[c], c0[c]);
        if (EXT) {
#pragma unroll
            for (int c = 0; c < 5; ++c) cx[c] = ST::dif(a[c], b[c]);
        }
        S.load5(sc, lx, ly + 1, a);
        S.load5(sc, lx, ly - 1, b);
#pragma unroll
        for (int c = 0; c < 5; ++c) dy[c] = ST::sec(a[c], b[c], c0[c]);
        if (EXT) {
#pragma unroll
            for (int c = 0; c < 5; ++c) cy[c] = ST::dif(a[c], b[c]);
        }
        S.load5(sp, lx, ly, a);
        S.load5(sm, lx, ly, b);
#pragma unroll
        for (int c = 0; c < 5; ++c) dz[c] = ST::sec(a[c], b[c], c0[c]);
        if (EXT) {
#pragma unroll
            for (int c = 0; c < 5; ++c) cz[c] = ST::dif(a[c], b[c]);
        }
    }
    const T L1s2 = T(2) * L1s;
    if constexpr (!THREE && sizeof(T) == 8) {
        T s0 = dx[0] + dy[0] + dz[0], s1 = dx[1] + dy[1] + dz[1], s2 = dx[2] + dy[2] + dz[2];
        T s3 = dx[3] + dy[3] + dz[3], s4 = dx[4] + dy[4] + dz[4];
        Fd[0] = L1s * (T(2) * s0 + s3) + Fb[0];
        Fd[1] = L1s2 * s1 + Fb[1];
        Fd[2] = L1s2 * s2 + Fb[2];
        Fd[3] = L1s * (s0 + T(2) * s3) + Fb[3];
        Fd[4] = L1s2 * s4 + Fb[4];
        return;
    }
    if (!THREE || sizeof(T) == 4) {
        T s0 = dx[0] + dy[0] + dz[0], s1 = dx[1] + dy[1] + dz[1], s2 = dx[2] + dy[2] + dz[2];
        T s3 = dx[3] + dy[3] + dz[3], s4 = dx[4] + dy[4] + dz[4];
        Fd[0] = L1s * (T(2) * s0 + s3);
        Fd[1] = L1s2 * s1;
        Fd[2] = L1s2 * s2;
        Fd[3] = L1s * (s0 + T(2) * s3);
        Fd[4] = L1s2 * s4;
        if (!THREE) return;
    }
    // FP64: the L1 sums s_c = x_c + y_c + z_c and the L2 + L3 sums (below)
    // share their partial sums (in the FP32 form this costs a register and
    // measured 13% slower, so that form keeps separate sums)
    const T p0 = dx[0] + dz[0], p3 = dy[3] + dz[3];
    const T t1 = dx[1] + dy[1], t2 = dx[2] + dz[2], t4 = dy[4] + dz[4];
    const T s0 = p0 + dy[0], s1 = t1 + dz[1], s2 = t2 + dy[2], s3 = p3 + dx[3], s4 = t4 + dx[4];
    const T t0 = p0 + dz[3], t3 = p3 + dz[0];
    T a[5], b[5], c[5];   // E_xy, E_xz, E_yz
    if constexpr (sizeof(T) == 8) {
        // from the plane's shared central differences (shared_diffs)
#pragma unroll
        for (int k = 0; k < 5; ++k) a[k] = S.d(dslot, 0, k, lx + 1, ly) - S.d(dslot, 0, k, lx - 1, ly);
#pragma unroll
        for (int k = 1; k < 5; ++k) b[k] = S.d(dslot, 1, k, lx + 1, ly) - S.d(dslot, 1, k, lx - 1, ly);
#pragma unroll
        for (int k = 0; k < 5; ++k)
            if (k != 3) c[k] = S.d(dslot, 1, k, lx, ly + 1) - S.d(dslot, 1, k, lx, ly - 1);
    } else {
        QS p0[5], p1[5], p2[5], p3[5];
        S.load5(sc, lx + 1, ly + 1, p0);
        S.load5(sc, lx + 1, ly - 1, p1);
        S.load5(sc, lx - 1, ly + 1, p2);
        S.load5(sc, lx - 1, ly - 1, p3);
#pragma unroll
        for (int k = 0; k < 5; ++k) a[k] = ST::mix(p0[k], p1[k], p2[k], p3[k]);
        S.load5(sp, lx + 1, ly, p0);
        S.load5(sm, lx + 1, ly, p1);
        S.load5(sp, lx - 1, ly, p2);
        S.load5(sm, lx - 1, ly, p3);
#pragma unroll
        for (int k = 1; k < 5; ++k) b[k] = ST::mix(p0[k], p1[k], p2[k], p3[k]);
        S.load5(sp, lx, ly + 1, p0);
        S.load5(sm, lx, ly + 1, p1);
        S.load5(sp, lx, ly - 1, p2);
        S.load5(sm, lx, ly - 1, p3);
#pragma unroll
        for (int k = 0; k < 5; ++k)
            if (k != 3) c[k] = ST::mix(p0[k], p1[k], p2[k], p3[k]);
    }
    const T kq = T(0.25) * L23s;
    if constexpr (sizeof(T) == 8) {
        Fd[0] = L1s * (T(2) * s0 + s3) + (L23s * t0 + (kq * (a[1] - c[4]) + Fb[0]));
        Fd[1] = L1s2 * s1 + (L23s * t1 + (kq * ((a[0] + a[3]) + (b[4] + c[2])) + Fb[1]));
        Fd[2] = L1s2 * s2 + (L23s * t2 + (kq * (a[4] - b[3] + c[1]) + Fb[2]));
        Fd[3] = L1s * (s0 + T(2) * s3) + (L23s * t3 + (kq * (a[1] - b[2]) + Fb[3]));
        Fd[4] = L1s2 * s4 + (L23s * t4 + (kq * (a[2] + b[1] - c[0]) + Fb[4]));
    } else {
        Fd[0] += L23s * (dx[0] + dz[0] + dz[3]) + kq * (a[1] - c[4]);
        Fd[1] += L23s * (dx[1] + dy[1]) + kq * ((a[0] + a[3]) + (b[4] + c[2]));
        Fd[2] += L23s * (dx[2] + dz[2]) + kq * (a[4] - b[3] + c[1]);
        Fd[3] += L23s * (dy[3] + dz[0] + dz[3]) + kq * (a[1] - b[2]);
        Fd[4] += L23s * (dy[4] + dz[4]) + kq * (a[2] + b[1] - c[0]);
    }
    if (EXT) {
        Fd[0] += k4 * (cz[1] - T(2) * cy[2] + cx[4]);
        Fd[1] += k4 * ((cz[3] - cz[0]) + (cx[2] - cy[4]));
        Fd[2] += k4 * (cz[4] + T(2) * cy[0] + cy[3] - cx[1]);
        Fd[3] += k4 * (T(2) * cx[4] - cz[1] - cy[2]);
        Fd[4] += k4 * (cy[1] - cx[0] - T(2) * cx[3] - cz[2]);
        if (L6h != T(0)) {
            T F6[5];
            if constexpr (sizeof(T) == 8)
                l6_regular(S, lx, ly, sc, sp, sm, L6h, T(Stencil<T>::scale), F6);
            else
                l6_regular_call(S, lx, ly, sc, sp, sm, L6h, T(Stencil<T>::scale), F6);
#pragma unroll
            for (int c = 0; c < 5; ++c) Fd[c] += F6[c];
        }
    }
    (void)L2q; (void)L3q;
}

// ---- tensor-memory-access (TMA) staging of the FP32 form --------------------
// The rows of a plane that a tile needs -- its own TY rows and the ring rows
// above and below, TX sites each -- arrive in shared memory by bulk tensor
// copies (one per row and state array, all five components at once),
// completing on an mbarrier per buffer; only the 2 TY + 4 ring sites left and
// right of the tile (whose x offset is not 16-byte aligned) use per-thread
// loads.  The copies name only this GPU's own arrays and are never multicast.

// tensor maps of one lattice's state: q, v, F of both ping-pong buffers as
// 4-D (x, y, z, component) tensors with a (TX, 1, 1, 5) box, the mask as a
// 3-D (x, y, z) tensor with a (TX, 1, 1) box
struct TmaMaps {
    CUtensorMap q[2], v[2], f[2];
    CUtensorMap m;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make the initialised barriers visible to the copy engine
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait for the phase of the given parity; gives up after about one second
// (a copy takes microseconds) and returns false
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}
// order this thread's earlier shared-memory accesses before later copies
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int c,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(c), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory layout of the raw plane buffers: RB buffers, each with the
// TY + 2 rows of q, v, F (five components of TX sites: a multiple of 128 bytes)
// and the TY + 2 mask rows (TX bytes each, in 128-byte slots)
template <int TX, int TY>
struct RawLayout {
    static constexpr int RB = 3;                                    // buffers
    static constexpr int ROWS = TY + 2;
    static constexpr int ROWB = 5 * TX * 4;                         // one row of one array
    static constexpr int MROWB = 128;
    static constexpr int BYTES = 3 * ROWS * ROWB + ROWS * MROWB;    // one buffer
    static constexpr unsigned TX_BYTES = 3 * ROWS * ROWB + ROWS * TX;   // delivered per plane
    static constexpr int TOTAL = 128 + RB * BYTES + RB * 8;         // with alignment slack and barriers
    static_assert(ROWB % 128 == 0, "row boxes on 128-byte boundaries");
};

// One block's work for one lattice: the tile with origin (bx*TX, by*TY),
// planes [z0, z1), block number bid of the nblk blocks of that lattice's
// step (its partial-sum slot).  Shared memory is the caller's.
// FORM: 0 one-constant, 1 three-constant (L1, L2, L3), 2 three-constant
// with the chiral L4 and cubic L6 terms
// TMA: the plane rows arrive by tensor copies (FP32 form, lattices whose x
// extent is a multiple of TX; tm holds the tensor maps) instead of per-thread
// loads; the arithmetic of every site is the same, so are the results.
template <typename T, int FORM, int TX, int TY, typename I, bool TMA = false>
__device__ __forceinline__ void step_tile(const StepArgs<T> &args, int bx, int by, int z0, int z1,
                                          int nblk, int bid, unsigned char *smem_raw, double *red,
                                          int *am_last_p, const TmaMaps *tm = nullptr) {
    constexpr int NT = TX * TY;
    constexpr int NSLOT = 5;
    constexpr bool THREE = FORM >= 1;
    using SM = Smem<T, TX, TY>;
    using P = Prec<T>;
    using QS = typename P::Q;
    int &am_last = *am_last_p;
    SM S;
    S.Q = smem_raw;
    S.X = reinterpret_cast<T *>(smem_raw + NSLOT * SM::SLOT_BYTES);
    S.D = S.X + (THREE ? 2 * 5 * SM::PL : 0);
    constexpr bool DIFFS = sizeof(T) == 8 && THREE;
    // the TMA form has the registers to keep the kick's old-state part in
    // every distortion form (no prefetch registers)
    constexpr bool WCACHE = keeps_w<T, FORM>() || TMA;
    S.W = S.D + (DIFFS ? 2 * 2 * 5 * SM::PL : 0);
    S.M = reinterpret_cast<uint8_t *>(S.W + (WCACHE ? 3 * 5 * NT : 0));
    using RL = RawLayout<TX, TY>;
    unsigned char *raw_base = nullptr;
    uint64_t *bars = nullptr;
    if constexpr (TMA) {
        static_assert(sizeof(T) == 4, "tensor-copy staging serves the FP32 form");
        const uintptr_t a = reinterpret_cast<uintptr_t>(S.M + NSLOT * SM::PL);
        raw_base = reinterpret_cast<unsigned char *>((a + 127) & ~uintptr_t(127));
        bars = reinterpret_cast<uint64_t *>(raw_base + RL::RB * RL::BYTES);
    }
    const LatticeDev L = args.L;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = bx * TX, y0 = by * TY;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool valid = gx < L.nx && gy < L.ny;
    const int lx = tx + 1, ly = ty + 1;
    // element indices: 32-bit when every index of the state arrays (< 5 N)
    // fits, else 64-bit
    const I N = (I)L.N;
    const I NXY = (I)L.nx * (I)L.ny;
    const bool fo_mode = args.force_only != 0;

    // FIRE coefficients for this step
    T cv = T(0), cF = T(0);
    const QS *qin;
    const T *vin = nullptr, *Fin = nullptr;
    QS *qout = nullptr;
    T *vout = nullptr, *Fout;
    if (fo_mode) {
        qin = args.qonly;
        Fout = args.Fonly;
    } else {
        if (args.st->status != FIRE_RUNNING) return;
        const int cur = args.st->cur;
        cv = T(args.st->cv); cF = T(args.st->cF);
        qin = args.q[cur]; vin = args.v[cur]; Fin = args.F[cur];
        qout = args.q[cur ^ 1]; vout = args.v[cur ^ 1]; Fout = args.F[cur ^ 1];
    }
    // drift q + alpha v + beta F (alpha, beta in the storage unit of Q) and
    // kick v_mix + hdt (F_old + F_new), as the last block of the previous
    // step left them
    T alpha = T(0), beta = T(0), hdt = T(0);
    if (!fo_mode) {
        alpha = T(args.st->c_alpha * P::scale);
        beta = T(args.st->c_beta * P::scale);
        hdt = T(args.st->c_kick);
    }
    // the old force's weight in the kick, cF + dt/2, rounded once
    const T cFh = fo_mode ? T(0) : T(args.st->cF + args.st->c_kick);

    // ring sites of a staged plane: top row, bottom row, left/right columns.
    // TMA: threads [0, 2 TX) take the row sites above and below the tile
    // (from the copied rows), threads [2 TX, 2 TX + 2 (TY + 2)) the columns
    // left and right of it, corners included (per-thread loads)
    constexpr int NRING = 2 * SM::SX + 2 * TY;
    static_assert(NRING <= NT, "one ring site per thread");
    int rx = -1, ry = -1;
    if constexpr (TMA) {
        const int r = threadIdx.x;
        if (r < TX) { rx = r + 1; ry = 0; }
        else if (r < 2 * TX) { rx = r - TX + 1; ry = SM::SY - 1; }
        else if (r < 2 * TX + 2 * SM::SY) { const int q = r - 2 * TX; rx = (q & 1) ? SM::SX - 1 : 0; ry = q >> 1; }
    } else if ((int)threadIdx.x < NRING) {
        int r = threadIdx.x;
        if (r < SM::SX) { rx = r; ry = 0; }
        else if (r < 2 * SM::SX) { rx = r - SM::SX; ry = SM::SY - 1; }
        else { r -= 2 * SM::SX; rx = (r & 1) ? SM::SX - 1 : 0; ry = 1 + (r >> 1); }
    }
    // TMA: row sites come from shared memory, column sites by loads
    const bool ring_row = TMA && (int)threadIdx.x < 2 * TX;
    const bool ring_col = rx >= 0 && !ring_row;
    // in-plane offsets of the own and ring sites (-1: outside the lattice)
    auto xy_of = [&](int sx, int sy) -> long long {
        int X = wrap_coord(x0 + sx - 1, L.nx, L.px);
        int Y = wrap_coord(y0 + sy - 1, L.ny, L.py);
        return (X >= 0 && Y >= 0) ? (long long)Y * L.nx + X : -1;
    };
    const long long xy_own_l = xy_of(lx, ly);
    const long long xy_ring_l = rx >= 0 ? xy_of(rx, ry) : -1;
    const bool in_own = xy_own_l >= 0, in_ring = xy_ring_l >= 0;
    const I xy_own = in_own ? (I)xy_own_l : 0, xy_ring = in_ring ? (I)xy_ring_l : 0;

    // one site of a plane in flight from global memory (registers)
    struct Raw {
        QS q[5];
        T v[5], f[5];
        uint8_t m;
    };
    // loads are unconditional for sites inside the lattice, so that the mask
    // load does not serialise them
    auto fetch = [&](bool in, I xy, int z, Raw &r) {
        int Z = wrap_coord(z, L.nz, L.pz);
        r.m = 0;
        if (in && Z >= 0) {
            I i = LQ_CHK_IDX((I)Z * NXY + xy, N);
            r.m = __ldg(args.g.mask + i);
#pragma unroll
            for (int c = 0; c < 5; ++c) r.q[c] = __ldg(qin + c * N + i);
            if (!fo_mode) {
#pragma unroll
                for (int c = 0; c < 5; ++c) { r.v[c] = __ldg(vin + c * N + i); r.f[c] = __ldg(Fin + c * N + i); }
            }
        }
    };
    bool bad = false;   // a drift left the fixed-point range (FP32 form)
    // drift (after the pending FIRE mixing) and store into a plane slot
    auto commit = [&](int slot, int sx, int sy, const Raw &r, bool checked) {
        QS qh[5] = {QS(0), QS(0), QS(0), QS(0), QS(0)};
        if (r.m & M_SIM) {
            if (fo_mode) {
#pragma unroll
                for (int c = 0; c < 5; ++c) qh[c] = r.q[c];
            } else {
                Site5<T>::drift(r.q, r.v, r.f, alpha, beta, qh, bad, checked);
            }
        }
        S.m(slot, sx, sy) = r.m;
        S.store5(slot, sx, sy, qh);
    };

    // FP32 form: the own site's part of the kick that needs only the old
    // state, cv v + cFh F, computed while v, F are in registers
    auto keep_w = [&](int z, const Raw &r) {
        if constexpr (WCACHE) {
            if (!fo_mode && (r.m & M_SIM)) {
                T w[5];
                Site5<T>::mix_old(r.v, r.f, cv, cFh, w);
                const int ws = ((z % 3) + 3) % 3;
#pragma unroll
                for (int c = 0; c < 5; ++c) S.w(ws, c) = w[c];
            }
        }
    };

    // plane z lives in slot z mod 5: at step z the slots of z-1, z, z+1 are
    // read, z+2 is written before the barrier; slot z+3 = z-2 is the one the
    // next step writes, which no thread of this step reads
    auto slot_of = [&](int z) { return ((z % NSLOT) + NSLOT) % NSLOT; };

    Raw pf_own, pf_ring;
    // TMA: plane p (z0 - 1 <= p <= z1) is the k-th of the block, k = p - z0 + 1,
    // delivered into buffer k mod RB; its barrier phase has parity (k / RB) & 1
    __shared__ int s_stall;
    int issued = z0 - 2;          // last plane whose copies were issued
    auto issue = [&](int p) {     // warp 0: the copies of plane p
        if constexpr (TMA) {
            if (threadIdx.x >= 32 || p > z1) return;
            const int k = p - (z0 - 1), b = k % RL::RB;
            const int lane = threadIdx.x;
            if (lane == 0) {
                fence_proxy_async();
                mbar_arrive_expect_tx(&bars[b], RL::TX_BYTES + args.tma_extra);
            }
            __syncwarp();
            if (lane < 4 * RL::ROWS) {
                const int r = lane % RL::ROWS, a = lane / RL::ROWS;   // a: q, v, F, mask
                // coordinates outside the lattice (open axes, rows past a
                // ragged edge) read zeros: mask 0, a site that is not there
                int Y = wrap_coord(y0 - 1 + r, L.ny, L.py);
                int Z = wrap_coord(p, L.nz, L.pz);
                if (Y < 0) Y = -1;
                if (Z < 0) Z = -1;
                unsigned char *dst = raw_base + b * RL::BYTES;
                const int cur = args.st->cur;
                if (a < 3) {
                    const CUtensorMap *map = a == 0 ? &tm->q[cur] : (a == 1 ? &tm->v[cur] : &tm->f[cur]);
                    tma_load_4d(dst + (a * RL::ROWS + r) * RL::ROWB, map, x0, Y, Z, 0, &bars[b]);
                } else {
                    tma_load_3d(dst + 3 * RL::ROWS * RL::ROWB + r * RL::MROWB, &tm->m, x0, Y, Z, &bars[b]);
                }
            }
        }
        (void)p;
    };
    // TMA: the site at (row, x) of the copied rows of plane p
    auto raw_site = [&](int p, int row, int x, Raw &r) {
        if constexpr (TMA) {
            const int k = p - (z0 - 1);
            const unsigned char *b = raw_base + (k % RL::RB) * RL::BYTES;
            const QS *q = reinterpret_cast<const QS *>(b + row * RL::ROWB);
            const T *v = reinterpret_cast<const T *>(b + (RL::ROWS + row) * RL::ROWB);
            const T *f = reinterpret_cast<const T *>(b + (2 * RL::ROWS + row) * RL::ROWB);
#pragma unroll
            for (int c = 0; c < 5; ++c) { r.q[c] = q[c * TX + x]; r.v[c] = v[c * TX + x]; r.f[c] = f[c * TX + x]; }
            r.m = b[3 * RL::ROWS * RL::ROWB + row * RL::MROWB + x];
        }
        (void)p; (void)row; (void)x; (void)r;
    };
    // TMA: wait for plane p; a wait that gives up marks the block stalled
    auto wait_plane = [&](int p) {
        if constexpr (TMA) {
            const int k = p - (z0 - 1);
            if (!mbar_wait_bounded(&bars[k % RL::RB], (k / RL::RB) & 1)) s_stall = 1;
        }
        (void)p;
    };
    // TMA: stage plane p into its slot from the copied rows (own site and the
    // row ring sites) and, for the column ring sites, from registers
    auto stage_plane = [&](int p, const Raw &col, bool own_w) {
        Raw r;
        raw_site(p, ly, tx, r);
        commit(slot_of(p), lx, ly, r, true);
        if (own_w) keep_w(p, r);
        if (ring_row) {
            raw_site(p, ry, rx - 1, r);
            commit(slot_of(p), rx, ry, r, false);
        } else if (ring_col) {
            commit(slot_of(p), rx, ry, col, false);
        }
    };
    // after a barrier: give up the whole block if any wait gave up; the
    // copies in flight are awaited (bounded) before the block leaves
    auto stalled = [&]() -> bool {
        if constexpr (TMA) {
            if (!s_stall) return false;
            for (int p = issued; p > issued - RL::RB && p >= z0 - 1; --p) {
                const int k = p - (z0 - 1);
                mbar_wait_bounded(&bars[k % RL::RB], (k / RL::RB) & 1);
            }
            if (threadIdx.x == 0 && !fo_mode) args.st->status = FIRE_STALLED;
            return true;
        }
        return false;
    };

    if constexpr (TMA) {
        if (threadIdx.x == 0) {
            s_stall = 0;
            for (int b = 0; b < RL::RB; ++b) mbar_init(&bars[b], 1);
            mbar_init_fence();
        }
        __syncthreads();
        for (int p = z0 - 1; p < z0 - 1 + RL::RB; ++p) issue(p);
        issued = min(z0 - 2 + RL::RB, z1);
        for (int p = z0 - 1; p <= z0 + 1; ++p) {
            Raw col;
            if (ring_col) fetch(in_ring, xy_ring, p, col);
            wait_plane(p);
            stage_plane(p, col, p >= z0);
            __syncthreads();     // every thread is done with the buffer of plane p
            if (stalled()) return;
            if (p + RL::RB <= z1) { issue(p + RL::RB); issued = p + RL::RB; }
        }
        if (ring_col) fetch(in_ring, xy_ring, z0 + 2, pf_ring);
    } else {
        Raw r;
        for (int p = -1; p <= 1; ++p) {
            fetch(in_own, xy_own, z0 + p, r);
            commit(slot_of(z0 + p), lx, ly, r, true);
            if (p >= 0) keep_w(z0 + p, r);
            if (rx >= 0) {
                fetch(in_ring, xy_ring, z0 + p, r);
                commit(slot_of(z0 + p), rx, ry, r, false);
            }
        }
        fetch(in_own, xy_own, z0 + 2, pf_own);
        if (rx >= 0) fetch(in_ring, xy_ring, z0 + 2, pf_ring);
        __syncthreads();   // the first regularity check reads neighbours' masks
    }

    // central differences of plane `pz` (slot s_pl, the planes below and
    // above in s_dn, s_up) into the difference slot pz & 1: D_z at the tile,
    // the ring columns and rows, D_y at the tile and the ring columns
    auto plane_diffs = [&](int pz, int s_pl, int s_dn, int s_up) {
        const int ds = pz & 1;
        auto one = [&](int sx, int sy, bool with_y) {
            QS u[5], w[5];
            S.load5(s_up, sx, sy, u);
            S.load5(s_dn, sx, sy, w);
#pragma unroll
            for (int c = 0; c < 5; ++c) S.d(ds, 1, c, sx, sy) = T(u[c]) - T(w[c]);
            if (with_y) {
                S.load5(s_pl, sx, sy + 1, u);
                S.load5(s_pl, sx, sy - 1, w);
#pragma unroll
                for (int c = 0; c < 5; ++c) S.d(ds, 0, c, sx, sy) = T(u[c]) - T(w[c]);
            }
        };
        one(lx, ly, true);
        if (rx >= 0) {
            const bool col = (rx == 0 || rx == SM::SX - 1) && ry >= 1 && ry <= TY;
            const bool row = (ry == 0 || ry == SM::SY - 1) && rx >= 1 && rx <= TX;
            if (col || row) one(rx, ry, col);
        }
    };
    if constexpr (shared_diffs<T, FORM>()) plane_diffs(z0, slot_of(z0), slot_of(z0 - 1), slot_of(z0 + 1));

    const T L1 = args.L1, L23 = args.L2 + args.L3;
    // chiral / cubic terms: both have a regular-site path (central
    // differences; l6_regular) besides the general link-flux path
    constexpr bool ext = FORM == 2;
    const T L4 = args.L4, L6 = ext ? args.L6 : T(0);
    const T sc_ = T(Stencil<T>::scale);
    const T L1s = L1 * sc_, L23s = L23 * sc_;
    const T L2q = T(0.25) * args.L2 * sc_, L3q = T(0.25) * args.L3 * sc_;

    FireSums<T> sums;
    const uint8_t FULL = M_SIM | 0xFC;

    int sm = slot_of(z0 - 1), sc = slot_of(z0), sp = slot_of(z0 + 1), s2 = slot_of(z0 + 2);
    for (int z = z0; z < z1; ++z) {
        // pipeline: plane z+2 into its slot, plane z+3 in flight
        if constexpr (TMA) {
            if (z + 2 <= z1) {
                wait_plane(z + 2);
                stage_plane(z + 2, pf_ring, z + 2 < z1);
            }
            if (z + 3 <= z1 && ring_col) fetch(in_ring, xy_ring, z + 3, pf_ring);
        } else {
            if (z + 2 <= z1) {
                commit(s2, lx, ly, pf_own, true);
                if (z + 2 < z1) keep_w(z + 2, pf_own);
                if (rx >= 0) commit(s2, rx, ry, pf_ring, false);
            }
            if (z + 3 <= z1) {
                fetch(in_own, xy_own, z + 3, pf_own);
                if (rx >= 0) fetch(in_ring, xy_ring, z + 3, pf_ring);
            }
        }
        const uint8_t m0 = S.m(sc, lx, ly);
        const bool own = valid && (m0 & M_SIM);
        // regular own site: it and its six face neighbours have every neighbour
        bool reg = true;
        if (own) {
            uint8_t a = S.m(sc, lx - 1, ly) & S.m(sc, lx + 1, ly) & S.m(sc, lx, ly - 1) &
                        S.m(sc, lx, ly + 1) & S.m(sp, lx, ly) & S.m(sm, lx, ly) & m0;
            reg = (m0 & FULL) == FULL && (a & 0xFC) == 0xFC;
        }
        const I i = own ? LQ_CHK_IDX((I)z * NXY + (I)gy * (I)L.nx + (I)gx, N)
                        : (I)z * NXY + (I)gy * (I)L.nx + (I)gx;
        // the own site's v, F for the kick: FP32 form read here, ahead of the
        // barrier, to hide the load latency; the FP64 form, bound by its
        // arithmetic pipe, reads them at the kick and keeps the registers
        // free through the force (fewer registers, 2% faster)
        T vold[5], fold[5];
        if constexpr (!WCACHE && sizeof(T) == 4) {
            if (own && !fo_mode) {
#pragma unroll
                for (int c = 0; c < 5; ++c) { vold[c] = __ldg(vin + c * N + i); fold[c] = __ldg(Fin + c * N + i); }
            }
        }
        // the barrier publishes plane z+2.  The path of this plane: with one
        // constant the general path has no block-wide step, so each warp
        // takes the regular path when its own sites allow it; with three
        // constants the general path's cross terms need the whole block
        bool all_reg;
        if constexpr (THREE) {
            all_reg = __syncthreads_and(reg) != 0;
        } else {
            __syncthreads();
            all_reg = __all_sync(0xffffffffu, reg);
        }
        if constexpr (TMA) {
            // every thread is done with the buffer of plane z+2: refill it
            if (stalled()) return;
            if (z + 2 + RL::RB <= z1) { issue(z + 2 + RL::RB); issued = z + 2 + RL::RB; }
        }
        // the next plane's central differences: planes z .. z+2 are published,
        // and the slot (z+1) & 1 was last read by the previous plane's force
        if constexpr (shared_diffs<T, FORM>()) {
            if (z + 1 < z1) plane_diffs(z + 1, sp, sc, s2);
        }

        T Fd[5];
        // FP64 regular planes: Fd already holds the bulk and field force
        const bool fused_bulk = sizeof(T) == 8 && all_reg;
        if (all_reg) {
            if (own) {
                T fb0[5];
                if constexpr (sizeof(T) == 8) {
                    QS qc[5];
                    T qcv[5];
                    S.load5(sc, lx, ly, qc);
                    q_values(qc, qcv);
                    bulk_force(qcv, args.A, args.B, args.C, fb0);
                    if (args.fields) {
#pragma unroll
                        for (int c = 0; c < 5; ++c) fb0[c] += args.fext[c];
                    }
                }
                regular_force<THREE, ext>(S, lx, ly, sc, sp, sm, z & 1, L1s, L23s, L2q, L3q, fb0, Fd,
                                          T(-0.5) * args.L4 * sc_, T(0.5) * L6);
            }
        } else {
            // general path (planes touching objects or open edges): the z
            // link below and the in-plane means are rebuilt on every such plane
            T phi_zm[5], xz_cur[5], mx_cur[5], my_cur[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) { xz_cur[c] = T(0); mx_cur[c] = T(0); my_cur[c] = T(0); }
            {
                T xz_m[5];
#pragma unroll
                for (int c = 0; c < 5; ++c) xz_m[c] = T(0);
                if (THREE) {
                    T mx[5], my[5];
                    mean_diff<0>(S, lx, ly, sm, 0, 0, mx);
                    mean_diff<1>(S, lx, ly, sm, 0, 0, my);
                    jt_cross<2>(mx, my, args.L2, args.L3, xz_m);
                    mean_diff<0>(S, lx, ly, sc, 0, 0, mx_cur);
                    mean_diff<1>(S, lx, ly, sc, 0, 0, my_cur);
                    jt_cross<2>(mx_cur, my_cur, args.L2, args.L3, xz_cur);
                    if (ext) {
                        T qv[5], e[5];
                        q_at(S, sm, lx, ly, qv);
                        jt_extra_x<2>(qv, mx, my, L4, L6, e);
#pragma unroll
                        for (int c = 0; c < 5; ++c) xz_m[c] += e[c];
                        q_at(S, sc, lx, ly, qv);
                        jt_extra_x<2>(qv, mx_cur, my_cur, L4, L6, e);
#pragma unroll
                        for (int c = 0; c < 5; ++c) xz_cur[c] += e[c];
                    }
                }
                QS qa[5], qb[5];
#pragma unroll
                for (int c = 0; c < 5; ++c) { qa[c] = S.q(sm, c, lx, ly); qb[c] = S.q(sc, c, lx, ly); }
                link_flux<2, THREE, ext>(S.m(sm, lx, ly), m0, qa, qb, xz_m, xz_cur, L1, L23, phi_zm, L6);
            }
            T xz_nxt[5], mx_nxt[5], my_nxt[5];
            if (THREE) {
                // cross terms of the tile at plane z
                if (m0 & M_SIM) {
                    T o[5], e[5], qv[5], mz_cur[5];
                    mean_diff<2>(S, lx, ly, sc, sp, sm, mz_cur);
                    if (ext) q_at(S, sc, lx, ly, qv);
                    jt_cross<0>(my_cur, mz_cur, args.L2, args.L3, o);
                    if (ext) {
                        jt_extra_x<0>(qv, my_cur, mz_cur, L4, L6, e);
#pragma unroll
                        for (int c = 0; c < 5; ++c) o[c] += e[c];
                    }
#pragma unroll
                    for (int c = 0; c < 5; ++c) S.x(0, c, lx, ly) = o[c];
                    jt_cross<1>(mx_cur, mz_cur, args.L2, args.L3, o);
                    if (ext) {
                        jt_extra_x<1>(qv, mx_cur, mz_cur, L4, L6, e);
#pragma unroll
                        for (int c = 0; c < 5; ++c) o[c] += e[c];
                    }
#pragma unroll
                    for (int c = 0; c < 5; ++c) S.x(1, c, lx, ly) = o[c];
                }
                // ring: X_x on the left/right columns, X_y on the top/bottom rows
                if ((int)threadIdx.x < 2 * TY) {
                    int sx = (threadIdx.x & 1) ? SM::SX - 1 : 0, sy = 1 + (threadIdx.x >> 1);
                    if (S.m(sc, sx, sy) & M_SIM) {
                        T my[5], mz[5], o[5];
                        mean_diff<1>(S, sx, sy, sc, sp, sm, my);
                        mean_diff<2>(S, sx, sy, sc, sp, sm, mz);
                        jt_cross<0>(my, mz, args.L2, args.L3, o);
                        if (ext) {
                            T qv[5], e[5];
                            q_at(S, sc, sx, sy, qv);
                            jt_extra_x<0>(qv, my, mz, L4, L6, e);
#pragma unroll
                            for (int c = 0; c < 5; ++c) o[c] += e[c];
                        }
#pragma unroll
                        for (int c = 0; c < 5; ++c) S.x(0, c, sx, sy) = o[c];
                    }
                } else if ((int)threadIdx.x < 2 * TY + 2 * TX) {
                    int r = threadIdx.x - 2 * TY;
                    int sx = 1 + (r >> 1), sy = (r & 1) ? SM::SY - 1 : 0;
                    if (S.m(sc, sx, sy) & M_SIM) {
                        T mx[5], mz[5], o[5];
                        mean_diff<0>(S, sx, sy, sc, sp, sm, mx);
                        mean_diff<2>(S, sx, sy, sc, sp, sm, mz);
                        jt_cross<1>(mx, mz, args.L2, args.L3, o);
                        if (ext) {
                            T qv[5], e[5];
                            q_at(S, sc, sx, sy, qv);
                            jt_extra_x<1>(qv, mx, mz, L4, L6, e);
#pragma unroll
                            for (int c = 0; c < 5; ++c) o[c] += e[c];
                        }
#pragma unroll
                        for (int c = 0; c < 5; ++c) S.x(1, c, sx, sy) = o[c];
                    }
                }
                // in-plane means and z cross term of the own column at plane z + 1
                mean_diff<0>(S, lx, ly, sp, 0, 0, mx_nxt);
                mean_diff<1>(S, lx, ly, sp, 0, 0, my_nxt);
                jt_cross<2>(mx_nxt, my_nxt, args.L2, args.L3, xz_nxt);
                if (ext) {
                    T qv[5], e[5];
                    q_at(S, sp, lx, ly, qv);
                    jt_extra_x<2>(qv, mx_nxt, my_nxt, L4, L6, e);
#pragma unroll
                    for (int c = 0; c < 5; ++c) xz_nxt[c] += e[c];
                }
                __syncthreads();
            }
            QS q0[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) q0[c] = S.q(sc, c, lx, ly);
            // z link (z, z+1) of the own column
            T phi_zp[5];
            {
                QS qb[5];
#pragma unroll
                for (int c = 0; c < 5; ++c) qb[c] = S.q(sp, c, lx, ly);
                link_flux<2, THREE, ext>(m0, S.m(sp, lx, ly), q0, qb, xz_cur, THREE ? xz_nxt : xz_cur, L1,
                                    L23, phi_zp, L6);
            }
            if (own) {
                T grad[5];
#pragma unroll
                for (int c = 0; c < 5; ++c) grad[c] = phi_zm[c] - phi_zp[c];
                QS qn[5];
                T xa[5], xb[5], phi[5];
                // (x-1, x)
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    qn[c] = S.q(sc, c, lx - 1, ly);
                    if (THREE) { xa[c] = S.x(0, c, lx - 1, ly); xb[c] = S.x(0, c, lx, ly); }
                }
                link_flux<0, THREE, ext>(S.m(sc, lx - 1, ly), m0, qn, q0, xa, xb, L1, L23, phi, L6);
#pragma unroll
                for (int c = 0; c < 5; ++c) grad[c] += phi[c];
                // (x, x+1)
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    qn[c] = S.q(sc, c, lx + 1, ly);
                    if (THREE) { xa[c] = xb[c]; xb[c] = S.x(0, c, lx + 1, ly); }
                }
                link_flux<0, THREE, ext>(m0, S.m(sc, lx + 1, ly), q0, qn, xa, xb, L1, L23, phi, L6);
#pragma unroll
                for (int c = 0; c < 5; ++c) grad[c] -= phi[c];
                // (y-1, y)
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    qn[c] = S.q(sc, c, lx, ly - 1);
                    if (THREE) { xa[c] = S.x(1, c, lx, ly - 1); xb[c] = S.x(1, c, lx, ly); }
                }
                link_flux<1, THREE, ext>(S.m(sc, lx, ly - 1), m0, qn, q0, xa, xb, L1, L23, phi, L6);
#pragma unroll
                for (int c = 0; c < 5; ++c) grad[c] += phi[c];
                // (y, y+1)
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    qn[c] = S.q(sc, c, lx, ly + 1);
                    if (THREE) { xa[c] = xb[c]; xb[c] = S.x(1, c, lx, ly + 1); }
                }
                link_flux<1, THREE, ext>(m0, S.m(sc, lx, ly + 1), q0, qn, xa, xb, L1, L23, phi, L6);
#pragma unroll
                for (int c = 0; c < 5; ++c) grad[c] -= phi[c];
                if (ext) {
                    // the site's own Q in the chiral and cubic terms
                    T sq[3] = {mean_sq<0>(S, lx, ly, sc, 0, 0), mean_sq<1>(S, lx, ly, sc, 0, 0),
                               mean_sq<2>(S, lx, ly, sc, sp, sm)};
                    T e[5], mz_cur[5];
                    mean_diff<2>(S, lx, ly, sc, sp, sm, mz_cur);
                    jt_extra_local(mx_cur, my_cur, mz_cur, sq, L4, L6, e);
#pragma unroll
                    for (int c = 0; c < 5; ++c) grad[c] += e[c];
                }
                if (!THREE) {
                    T j[5];
                    jt_sym(grad, j);
#pragma unroll
                    for (int c = 0; c < 5; ++c) Fd[c] = -L1 * j[c];
                } else {
#pragma unroll
                    for (int c = 0; c < 5; ++c) Fd[c] = -grad[c];
                }
            }
        }

        if (own) {
            QS q0[5];
            T qv[5], fb[5], Fn[5];
            S.load5(sc, lx, ly, q0);
            q_values(q0, qv);
            if (fused_bulk) {
#pragma unroll
                for (int c = 0; c < 5; ++c) Fn[c] = Fd[c];
            } else {
                bulk_force(qv, args.A, args.B, args.C, fb);
                if (args.fields) {
#pragma unroll
                    for (int c = 0; c < 5; ++c) fb[c] += args.fext[c];
                }
                add5(Fd, fb, Fn);
            }
            if (m0 & M_ANCH) {
                const AnchorRec<T> *r = find_record<T>(args.g, L, gx, gy, z);
                if (r) {
                    T fa[5];
                    anchor_force(qv, q0, *r, args.S0, fa);
#pragma unroll
                    for (int c = 0; c < 5; ++c) Fn[c] += fa[c];
                }
            }
            if (fo_mode) {
#pragma unroll
                for (int c = 0; c < 5; ++c) Fout[c * N + i] = Fn[c];
            } else {
                T vn[5];
                if constexpr (WCACHE) {
                    T w[5];
#pragma unroll
                    for (int c = 0; c < 5; ++c) w[c] = S.w(z % 3, c);
                    Site5<T>::kick_w(w, Fn, hdt, vn);
                } else {
                    if constexpr (sizeof(T) == 8) {
#pragma unroll
                        for (int c = 0; c < 5; ++c) {
                            vold[c] = __ldg(vin + c * N + i);
                            fold[c] = __ldg(Fin + c * N + i);
                        }
                    }
                    Site5<T>::kick(vold, fold, Fn, cv, cFh, hdt, vn);
                }
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    __stcs(qout + c * N + i, q0[c]);
                    __stcs(vout + c * N + i, vn[c]);
                    __stcs(Fout + c * N + i, Fn[c]);
                }
                sums.site(Fn, vn);
            }
        }
        // rotate the plane slots
        int t = sm;
        sm = sc; sc = sp; sp = s2; s2 = (t + 4) % NSLOT;   // plane z+3 = (z-1) + 4
    }

    if (args.force_only) return;

    // block reduction, then the last block reduces the partials in order; a
    // fixed-point range violation poisons the max with +inf (-> diverged)
    double sP, sF, sV, sR;
    sums.get(sP, sF, sV, sR);
    if (bad) sR = (double)INFINITY;
    block_reduce4<NT>(sP, sF, sV, sR, red);
    const int nblocks = nblk;
    if (threadIdx.x == 0) {
        double *p = args.partials + 4 * (long long)bid;
        p[0] = sP; p[1] = sF; p[2] = sV; p[3] = sR;
        __threadfence();
        unsigned int t = atomicAdd(&args.st->counter, 1u);
        am_last = (t == (unsigned)(nblocks - 1));
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double P2 = 0.0, F2 = 0.0, V2 = 0.0, R2 = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += NT) {
        const double *p = args.partials + 4 * (long long)b;
        P2 += __ldcg(p); F2 += __ldcg(p + 1); V2 += __ldcg(p + 2); R2 = fmax(R2, __ldcg(p + 3));
    }
    block_reduce4<NT>(P2, F2, V2, R2, red);
    if (threadIdx.x == 0) {
        if (args.reduce_only) {
            FireDev *st = args.st;
            st->P = P2; st->F2 = F2; st->v2 = V2; st->r2 = R2;
        } else {
            fire_update(args.st, P2, F2, V2, R2);
        }
        args.st->counter = 0;
    }
}

// the FIRE scalar update of a slab of a decomposed lattice from the sums over
// every slab (one thread; the same update on every slab)
__global__ void k_fire_apply(FireDev *st, double P, double F2, double v2, double r2) {
    if (st->status == FIRE_RUNNING) fire_update(st, P, F2, v2, r2);
}

cudaError_t fire_apply(FireDev *st, const double sums[4], cudaStream_t stream) {
    k_fire_apply<<<1, 1, 0, stream>>>(st, sums[0], sums[1], sums[2], sums[3]);
    return cudaGetLastError();
}


// one FIRE iteration of one lattice: one block per tile and z chunk
template <typename T, int FORM, int TX, int TY, typename I>
__global__ void __launch_bounds__(TX * TY, sizeof(T) == 4 ? (FORM == 2 ? 384 : 512) / (TX * TY) : 1)
fire_step_kernel(StepArgs<T> args) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4 * (TX * TY / 32)];
    __shared__ int am_last;
    const int z0 = args.zbeg + blockIdx.z * args.zchunk;
    const int z1 = min(z0 + args.zchunk, args.zend);
    const int nblk = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    step_tile<T, FORM, TX, TY, I>(args, blockIdx.x, blockIdx.y, z0, z1, nblk, bid, smem_raw, red,
                                  &am_last);
}

// one FIRE iteration of one lattice with the plane rows staged by tensor
// copies (FP32 form); three blocks per SM (the raw plane buffers take shared
// memory; the registers that prefetched planes in the other kernel are free)
template <typename T, int FORM, int TX, int TY, typename I>
__global__ void __launch_bounds__(TX * TY, 3)
fire_step_tma_kernel(const __grid_constant__ StepArgs<T> args, const __grid_constant__ TmaMaps maps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4 * (TX * TY / 32)];
    __shared__ int am_last;
    const int z0 = args.zbeg + blockIdx.z * args.zchunk;
    const int z1 = min(z0 + args.zchunk, args.zend);
    const int nblk = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    step_tile<T, FORM, TX, TY, I, true>(args, blockIdx.x, blockIdx.y, z0, z1, nblk, bid, smem_raw, red,
                                        &am_last, &maps);
}

// one FIRE iteration of every lattice of a batch: a persistent grid strides
// over the work items (lattice, tile, z chunk); each lattice keeps its own
// partial sums, last-block ticket and FIRE state, so a lattice advances
// exactly as it would alone with the same tile and z chunk
// FP32 form: three blocks of 128 threads per SM with three constants (168
// registers: at 128 the three-constant item loop spills 144 bytes a thread
// and runs 1.6 times slower), four with one constant
template <typename T, int FORM, int TX, int TY, typename I>
__global__ void __launch_bounds__(TX * TY, sizeof(T) == 4 ? (FORM == 2 || (FORM == 1 && TX * TY == 128) ? 384 : 512) /
                                                               (TX * TY)
                                                         : 1)
fire_batch_kernel(const StepArgs<T> *__restrict__ args, const WorkItem *__restrict__ items,
                  int nitems) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4 * (TX * TY / 32)];
    __shared__ int am_last;
    // the item's lattice arguments, copied into shared memory: read from
    // there, no field is reloaded from global memory after the step's stores
    // (which the compiler cannot tell apart from the argument array); 9%
    // faster than reading the array at 64 one-constant lattices
    __shared__ __align__(16) unsigned long long sa_raw[(sizeof(StepArgs<T>) + 7) / 8];
    const StepArgs<T> &sa = *reinterpret_cast<const StepArgs<T> *>(sa_raw);
    constexpr int NW = (int)((sizeof(StepArgs<T>) + 7) / 8);
    static_assert(sizeof(StepArgs<T>) % 8 == 0 && alignof(StepArgs<T>) <= 16, "whole 8-byte words");
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(args + w.lattice);
        for (int k = threadIdx.x; k < NW; k += TX * TY) sa_raw[k] = src[k];
        __syncthreads();
        step_tile<T, FORM, TX, TY, I>(sa, w.bx, w.by, w.z0, w.z1, w.nblk, w.bid, smem_raw, red, &am_last);
        __syncthreads();   // shared memory is reused by the next item
    }
}

// ---- host launchers ---------------------------------------------------------

template <typename T, int FORM, int TX, int TY, bool TMA = false>
static size_t step_smem_bytes() {
    constexpr bool THREE = FORM >= 1;
    using SM = Smem<T, TX, TY>;
    constexpr int PL = SM::PL;
    constexpr bool DIFFS = sizeof(T) == 8 && THREE;   // shared_diffs (form 1; unused by form 2)
    size_t b = 5 * (size_t)SM::SLOT_BYTES + sizeof(T) * (THREE ? 2 * 5 * PL : 0) +
               sizeof(T) * (DIFFS ? 2 * 2 * 5 * PL : 0) + 5 * PL +
               (keeps_w<T, FORM>() || TMA ? sizeof(T) * 3 * 5 * TX * TY : 0);
    if (TMA) b += RawLayout<TX, TY>::TOTAL;
    return (b + 15) & ~size_t(15);
}

// ---- tensor maps (host) ---------------------------------------------------------

// the driver's tensor-map encoder, found through the runtime (no link to the
// driver library); null where the driver has none
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool tma_staging_available() { return tensor_map_encoder() != nullptr; }

// lattices the tensor-copy staging serves: FP32 form, x extent a multiple of
// the 32-site tile (row boxes start on 16-byte boundaries and never cross the
// x edge; 16-byte mask rows)
bool tma_staging_fits(const LatticeDev &L) { return L.nx % 32 == 0 && L.nx >= 32; }

template <typename T, int TX>
static bool encode_maps(const StepLaunch &sl, TmaMaps &m) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const LatticeDev &L = sl.L;
    const cuuint64_t nx = L.nx, ny = L.ny, nz = L.nz;
    const cuuint64_t dims4[4] = {nx, ny, nz, 5};
    const cuuint64_t str4[3] = {nx * sizeof(T), nx * ny * sizeof(T), nx * ny * nz * sizeof(T)};
    const cuuint32_t box4[4] = {TX, 1, 1, 5};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    auto state = [&](CUtensorMap *out, void *base, CUtensorMapDataType dt) {
        return enc(out, dt, 4, base, dims4, str4, box4, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int b = 0; b < 2; ++b) {
        if (!state(&m.q[b], sl.q[b], CU_TENSOR_MAP_DATA_TYPE_INT32)) return false;
        if (!state(&m.v[b], sl.v[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32)) return false;
        if (!state(&m.f[b], sl.F[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32)) return false;
    }
    const cuuint64_t dims3[3] = {nx, ny, nz};
    const cuuint64_t str3[2] = {nx, nx * ny};
    const cuuint32_t box3[3] = {TX, 1, 1};
    return enc(&m.m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t *>(sl.g.mask), dims3, str3, box3, one,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T>
static void pack_args(const StepLaunch &sl, StepArgs<T> &a) {
    for (int b = 0; b < 2; ++b) {
        a.q[b] = static_cast<typename Prec<T>::Q *>(sl.q[b]);
        a.v[b] = static_cast<T *>(sl.v[b]);
        a.F[b] = static_cast<T *>(sl.F[b]);
    }
    a.Fonly = static_cast<T *>(sl.Fonly);
    a.qonly = static_cast<const typename Prec<T>::Q *>(sl.qonly);
    a.g = sl.g;
    a.L = sl.L;
    a.A = T(sl.A); a.B = T(sl.B); a.C = T(sl.C);
    a.L1 = T(sl.L1); a.L2 = T(sl.L2); a.L3 = T(sl.L3); a.S0 = T(sl.S0);
    a.L4 = T(sl.L4); a.L6 = T(sl.L6);
    a.fields = 0;
    for (int c = 0; c < 5; ++c) {
        a.fext[c] = T(sl.fext[c]);
        a.fields |= sl.fext[c] != 0.0;
    }
    a.st = sl.st;
    a.partials = sl.partials;
    a.zchunk = sl.zchunk;
    a.force_only = sl.force_only;
    a.tma_extra = 0;
    a.zbeg = sl.zbeg;
    a.zend = sl.zend > 0 ? sl.zend : sl.L.nz;
    a.reduce_only = sl.reduce_only;
}

// 32-bit element indices serve every lattice whose state arrays hold fewer
// than 2^32 elements (5 N < 2^32, N < 858,993,459 sites, about 950^3)
bool step_index32(long long N) { return 5 * N < (1LL << 32); }

template <typename T, int FORM, int TX, int TY, typename I>
static cudaError_t launch_impl(const StepLaunch &sl, cudaStream_t stream) {
    StepArgs<T> a;
    pack_args<T>(sl, a);
    dim3 grid = step_grid(sl.L, sl.zchunk, TX, TY);
    grid.z = (a.zend - a.zbeg + sl.zchunk - 1) / sl.zchunk;
    if constexpr (sizeof(T) == 4 && TX == 32) {
        if (sl.tma && !sl.force_only) {
            TmaMaps maps;
            if (!encode_maps<T, TX>(sl, maps)) return cudaErrorInvalidValue;
            // injected (direct launches only, never baked into a captured
            // graph): every plane's wait runs out
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            cudaStreamIsCapturing(stream, &cs);
            if (cs == cudaStreamCaptureStatusNone && fault_due(3)) a.tma_extra = 16;
            fire_step_tma_kernel<T, FORM, TX, TY, I>
                <<<grid, TX * TY, step_smem_bytes<T, FORM, TX, TY, true>(), stream>>>(a, maps);
            return cudaGetLastError();
        }
    }
    size_t smem = step_smem_bytes<T, FORM, TX, TY>();
    auto kern = fire_step_kernel<T, FORM, TX, TY, I>;
    kern<<<grid, TX * TY, smem, stream>>>(a);
    return cudaGetLastError();
}

dim3 step_grid(const LatticeDev &L, int zchunk, int tx, int ty) {
    return dim3((L.nx + tx - 1) / tx, (L.ny + ty - 1) / ty, (L.nz + zchunk - 1) / zchunk);
}

// tile of one block: the FP32 form runs 32x4 tiles at 4 blocks per SM (128
// registers per thread), the FP64 form 32x8 tiles at one block per SM with
// three constants and 32x4 tiles at 2 blocks per SM with one constant (4%
// faster there, 6% slower with three constants).  A one-constant FP32
// lattice at least 256 sites wide runs 64x4 tiles at 2 blocks per SM
// instead (half the ring columns per site: 8% faster at 512^3; 6% slower
// with three constants, and slower on narrow lattices, where a 64-wide tile
// is partly empty).  Batches always run 32-wide tiles.
bool wide_tiles(int fp32, int three, int nx) { return fp32 && !three && nx >= 256; }

void step_tile(int fp32, int three, int nx, int *tx, int *ty) {
    *tx = wide_tiles(fp32, three, nx) ? 64 : 32;
    *ty = fp32 || !three ? 4 : 8;
}

// calls F::template run<T, FORM, TY, I>() for the precision, distortion form
// (0 one-constant, 1 three-constant, 2 with chiral / cubic terms), tile
// height and index width of a launch
template <typename T, int TY, typename F>
static auto dispatch_form(int form, bool idx32, F &&f) {
    if (form == 2) return idx32 ? f.template run<T, 2, TY, unsigned>() : f.template run<T, 2, TY, long long>();
    if (form == 1) return idx32 ? f.template run<T, 1, TY, unsigned>() : f.template run<T, 1, TY, long long>();
    return idx32 ? f.template run<T, 0, TY, unsigned>() : f.template run<T, 0, TY, long long>();
}
template <typename F>
static auto dispatch(int fp32, int form, int ty, bool idx32, F &&f) {
    if (fp32) return ty == 4 ? dispatch_form<float, 4>(form, idx32, f) : dispatch_form<float, 8>(form, idx32, f);
    return ty == 4 ? dispatch_form<double, 4>(form, idx32, f) : dispatch_form<double, 8>(form, idx32, f);
}
// the single-lattice kernel: each precision at its own tile height (step_tile)
template <typename F>
static auto dispatch_single(int fp32, int form, bool idx32, F &&f) {
    if (fp32) return dispatch_form<float, 4>(form, idx32, f);
    if (form == 0) return dispatch_form<double, 4>(form, idx32, f);
    return dispatch_form<double, 8>(form, idx32, f);
}

struct PrepareStep {
    template <typename T, int FORM, int TY, typename I>
    cudaError_t run() {
        cudaError_t e = cudaFuncSetAttribute(fire_step_kernel<T, FORM, 32, TY, I>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)step_smem_bytes<T, FORM, 32, TY>());
        if constexpr (sizeof(T) == 4) {
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(fire_step_tma_kernel<T, FORM, 32, TY, I>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_smem_bytes<T, FORM, 32, TY, true>());
        }
        if constexpr (sizeof(T) == 4 && FORM == 0) {
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(fire_step_kernel<T, FORM, 64, TY, I>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_smem_bytes<T, 0, 64, TY>());
        }
        return e;
    }
};

cudaError_t prepare_fire_step(int fp32, int three) {
    cudaError_t e = cudaSuccess;
    const int forms[2] = {three ? 1 : 0, three ? 2 : 0};
    for (int form : forms)
        for (bool i32 : {true, false})
            if (e == cudaSuccess) e = dispatch_single(fp32, form, i32, PrepareStep{});
    return e;
}

struct LaunchStep {
    const StepLaunch &sl;
    cudaStream_t stream;
    template <typename T, int FORM, int TY, typename I>
    cudaError_t run() {
        if constexpr (sizeof(T) == 4 && FORM == 0) {
            if (sl.wide) return launch_impl<T, FORM, 64, TY, I>(sl, stream);
        }
        return launch_impl<T, FORM, 32, TY, I>(sl, stream);
    }
};

cudaError_t launch_fire_step(const StepLaunch &sl, cudaStream_t stream) {
    if (fault_due(2)) return cudaErrorLaunchFailure;   // injected: nothing is launched
    const int form = sl.three ? (sl.ext ? 2 : 1) : 0;
    // 32-bit element indices where they fit, except in the FP32-form
    // three-constant step with per-thread loads: its 64-bit instantiation
    // measured 2% faster at 512^3 (4.68 -> 4.58 ms), while the one-constant
    // and FP64 forms are as fast or faster with 32-bit indices
    const bool idx32 = step_index32(sl.L.N) && !sl.idx64 && !(sl.fp32 && form == 1 && !sl.tma);
    return dispatch_single(sl.fp32, form, idx32, LaunchStep{sl, stream});
}

// ---- batched launches ----------------------------------------------------------

size_t step_args_bytes(int fp32) { return fp32 ? sizeof(StepArgs<float>) : sizeof(StepArgs<double>); }

void step_args_pack(const StepLaunch &sl, void *out) {
    if (sl.fp32) pack_args<float>(sl, *static_cast<StepArgs<float> *>(out));
    else pack_args<double>(sl, *static_cast<StepArgs<double> *>(out));
}

// batch tiles: 32 x TY in every form; 64 x TY also for one-constant FP32
// lattices (the wide tiles of the single-lattice kernel)
bool batch_tile_ok(int fp32, int form, int tx) { return tx == 32 || (tx == 64 && fp32 && form == 0); }

struct PrepareBatch {
    int tx;
    template <typename T, int FORM, int TY, typename I>
    cudaError_t run() {
        if constexpr (sizeof(T) == 4 && FORM == 0) {
            if (tx == 64)
                return cudaFuncSetAttribute(fire_batch_kernel<T, FORM, 64, TY, I>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)step_smem_bytes<T, FORM, 64, TY>());
        }
        if (tx != 32) return cudaErrorInvalidValue;
        return cudaFuncSetAttribute(fire_batch_kernel<T, FORM, 32, TY, I>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)step_smem_bytes<T, FORM, 32, TY>());
    }
};

struct BlocksBatch {
    int tx;
    template <typename T, int FORM, int TY, typename I>
    int run() {
        int nb = 0;
        if constexpr (sizeof(T) == 4 && FORM == 0) {
            if (tx == 64) {
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fire_batch_kernel<T, FORM, 64, TY, I>,
                                                              64 * TY, step_smem_bytes<T, FORM, 64, TY>());
                return nb;
            }
        }
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fire_batch_kernel<T, FORM, 32, TY, I>,
                                                      32 * TY, step_smem_bytes<T, FORM, 32, TY>());
        return nb;
    }
};

struct LaunchBatch {
    const void *args;
    const WorkItem *items;
    int nitems, grid, tx;
    cudaStream_t stream;
    template <typename T, int FORM, int TY, typename I>
    cudaError_t run() {
        if constexpr (sizeof(T) == 4 && FORM == 0) {
            if (tx == 64) {
                fire_batch_kernel<T, FORM, 64, TY, I><<<grid, 64 * TY, step_smem_bytes<T, FORM, 64, TY>(),
                                                        stream>>>(static_cast<const StepArgs<T> *>(args),
                                                                  items, nitems);
                return cudaGetLastError();
            }
        }
        if (tx != 32) return cudaErrorInvalidValue;
        fire_batch_kernel<T, FORM, 32, TY, I><<<grid, 32 * TY, step_smem_bytes<T, FORM, 32, TY>(),
                                                stream>>>(static_cast<const StepArgs<T> *>(args), items,
                                                          nitems);
        return cudaGetLastError();
    }
};

cudaError_t prepare_fire_batch(int fp32, int form, int tx, int ty, int idx32) {
    if (!batch_tile_ok(fp32, form, tx)) return cudaErrorInvalidValue;
    return dispatch(fp32, form, ty, idx32 != 0, PrepareBatch{tx});
}

int fire_batch_blocks_per_sm(int fp32, int form, int tx, int ty, int idx32) {
    if (!batch_tile_ok(fp32, form, tx)) return 0;
    return dispatch(fp32, form, ty, idx32 != 0, BlocksBatch{tx});
}

cudaError_t launch_fire_batch(int fp32, int form, int tx, int ty, int idx32, const void *dev_args,
                              const WorkItem *items, int nitems, int grid, cudaStream_t stream) {
    if (fault_due(2)) return cudaErrorLaunchFailure;   // injected: nothing is launched
    if (!batch_tile_ok(fp32, form, tx)) return cudaErrorInvalidValue;
    return dispatch(fp32, form, ty, idx32 != 0, LaunchBatch{dev_args, items, nitems, grid, tx, stream});
}

__global__ void k_batch_running(FireDev *const *states, int n, unsigned int *running) {
    unsigned int c = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) c += (states[i]->status == FIRE_RUNNING) ? 1u : 0u;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    __shared__ unsigned int part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = 0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += part[w];
        *running = t;
    }
}

cudaError_t batch_running(FireDev *const *states, int n, unsigned int *running, cudaStream_t s) {
    k_batch_running<<<1, 256, 0, s>>>(states, n, running);
    return cudaGetLastError();
}

}  // namespace lq
