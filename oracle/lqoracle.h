/*
 * lqoracle.h -- plain FP64 CPU oracle for the lattice Landau-de Gennes
 * energy, its gradient and the FIRE minimiser.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes,
 * links or calls this code; only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark use it.  It shares no header, helper,
 * table or constant generator with the CUDA path.
 *
 * Conventions (paper section III.B):
 *   * cubic lattice, spacing 1, site (x,y,z) has linear index
 *     i = (z*ny + y)*nx + x;
 *   * five independent components per site, q = (Qxx, Qxy, Qxz, Qyy, Qyz),
 *     Qzz = -Qxx - Qyy;  arrays are structure-of-arrays: q[c*N + i];
 *   * only "simulated" sites (bulk or boundary) carry Q; object sites are
 *     ignored by every routine and receive force 0.
 */
#ifndef LQORACLE_H
#define LQORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    int periodic[3];          /* 1 = periodic along x / y / z */
    double A, B, C;           /* bulk constants, Eq. (fphase) */
    double L1, L2, L3;        /* distortion constants, Eq. (fdistortionFull) */
    double S0;                /* degree of order used by the anchoring terms */
    double L4, L6;            /* chiral and cubic terms of Eq. (fdistortionFull) */
    /* external fields (section II, external fields free energy):
       -(1/3) mu0_dchi H.Q.H - (1/3) eps0_deps E.Q.E, counted with the bulk */
    double H[3], mu0_dchi;
    double E[3], eps0_deps;
} orc_model;

/* anchoring kinds, boundary free energy of section II */
enum { ORC_ND_HOMEOTROPIC = 0, ORC_ND_ORIENTED = 1, ORC_FG_PLANAR = 2 };
/* object kinds */
enum { ORC_WALL = 0, ORC_SPHERE = 1, ORC_SITES = 2, ORC_ANCHORED = 3, ORC_DROPLET = 4,
       ORC_SPHEROCYLINDER = 5 };

typedef struct { int kind; double W; double dir[3]; } orc_anchor_spec;

typedef struct {
    int type;                 /* ORC_WALL / ORC_SPHERE / ORC_SITES / ORC_ANCHORED */
    int axis, plane;          /* wall: lattice plane coord[axis] == plane */
    double c[3], R;           /* sphere: centre, radius */
    int64_t n;                /* SITES / ANCHORED: number of listed sites */
    const int32_t *xyz;       /* SITES / ANCHORED: 3*n coordinates */
    const orc_anchor_spec *per_site; /* ANCHORED: n specs */
    orc_anchor_spec anch;     /* WALL / SPHERE / SITES: anchoring of the surface */
    double c2[3];             /* SPHEROCYLINDER: second end of the axis segment (c the first) */
} orc_object;
/* DROPLET: the nematic fills the ball |x - c| <= R (minimum image along
   periodic axes); every site outside is an object site; surface normal
   x - c.  SPHEROCYLINDER: object sites within R of the segment c..c2 (a
   capsule, Fig. 3); normal from the nearest point of the segment. */

/* resolved per-site anchoring record */
typedef struct {
    int kind;                 /* 1 = Nobili-Durand (uses q0), 2 = Fournier-Galatola (uses nu) */
    double W;
    double q0[5];             /* preferred Q^0 in the 5-component form */
    double nu[3];             /* surface normal for the planar-degenerate form */
} orc_anchor;

typedef struct {
    int64_t N;
    uint8_t *sim;             /* N entries, 1 = simulated */
    int32_t *rec_index;       /* N entries, -1 = no anchoring record */
    orc_anchor *recs;
    int64_t nrec;
} orc_geometry;

typedef struct {
    double dt0, dt_max, alpha0, f_alpha, f_inc, f_dec;
    int n_min;
    int64_t max_iter;
    double force_tol;         /* on max over sites of the 5-component force norm */
} orc_fire_params;

enum { ORC_RUNNING = 0, ORC_CONVERGED = 1, ORC_MAXITER = 2, ORC_DIVERGED = 3 };

typedef struct {
    double dt, alpha;
    int64_t npos, iter;       /* iter = completed FIRE iterations */
    int initialized, status;
    double P, normF, normv, rmax; /* reductions of the last evaluated state */
} orc_fire_state;

double orc_uniaxial_s0(double A, double B, double C);

int  orc_build_geometry(const orc_model *m, const orc_object *objs, int nobj,
                        orc_geometry *out);
void orc_free_geometry(orc_geometry *g);

/* Eq. (fdistortionFull) at one point: Q[3*i+j] = Q_ij, d[(3*i+j)*3+k] =
   dQ_ij/dx_k (the continuum density, before any lattice differencing) */
double orc_distortion_density(const orc_model *m, const double *Q9, const double *d27);
/* free energy density of one site, split as (bulk, distortion, anchoring) */
void   orc_site_energy(const orc_model *m, const orc_geometry *g,
                       const double *q, int64_t site, double parts[3]);
/* total free energy, parts[3] = (bulk, distortion, anchoring); returns the sum */
double orc_energy(const orc_model *m, const orc_geometry *g, const double *q,
                  double parts[3]);
/* force = -dF/dq at every site (5*N, SoA) */
void   orc_force(const orc_model *m, const orc_geometry *g, const double *q,
                 double *F);
/* force at a list of sites; F is 5*n, F[c*n + s] */
void   orc_force_sites(const orc_model *m, const orc_geometry *g,
                       const double *q, int64_t n, const int64_t *sites,
                       double *F);

/* one application of the FIRE scalar rules (mixing then the P test);
   returns the velocity-mixing pair (a, b): v <- a*v + b*F */
void orc_fire_scalars(const orc_fire_params *p, orc_fire_state *st,
                      double P, double normF, double normv,
                      double *a, double *b);
/* run up to max_steps FIRE iterations from the given state */
int  orc_fire_run(const orc_model *m, const orc_geometry *g,
                  const orc_fire_params *p, double *q, double *v, double *F,
                  orc_fire_state *st, int64_t max_steps);

/* Gradient descent and Nesterov's accelerated gradient, two of the
   minimisers section III.C names (Fig. 2 compares gradient descent with
   FIRE), in their textbook forms:
     method 1 (GD):        x_{k+1} = x_k + eta F(x_k)
     method 2 (Nesterov):  y_k = x_k + mu (x_k - x_{k-1}),
                           x_{k+1} = y_k + eta F(y_k)
   x is the iterate, xprev the previous one (equal to x at the start), y the
   point where the force is evaluated (GD: y = x) and F = F(y); residual and
   convergence test on F(y).  iter counts completed iterations after the
   initial evaluation, as for FIRE. */
typedef struct {
    int64_t iter;
    int initialized, status;
    double normF, rmax;
} orc_descent_state;
int  orc_descent_run(const orc_model *m, const orc_geometry *g, int method, double eta,
                     double mu, int64_t max_iter, double force_tol, double *x, double *xprev,
                     double *y, double *F, orc_descent_state *st, int64_t max_steps);

/* eigen-decomposition of one Q by cyclic Jacobi; values descending */
void orc_eig_sym3(const double q5[5], double evals[3], double evecs[9]);
/* largest eigenvalue per site (0 at object sites) */
void orc_order_field(const orc_geometry *g, const double *q, int64_t N,
                     double *S);

int orc_num_threads(void);
int orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
