/*
 * lqmin.h -- C interface of the B300 (sm_103a) lattice Landau-de Gennes
 * minimiser: force on the five-component Q-tensor lattice (bulk, averaged
 * one-sided-difference distortion, anchoring) fused with FIRE steps.
 *
 * Paper: D. M. Sussman and D. A. Beller, "Fast, scalable, and interactive
 * software for Landau-de Gennes numerical modeling of nematic topological
 * defects" (arXiv:1911.07045).  Each call names the passage that defines the
 * operation it performs.
 *
 * Conventions shared by every call
 *   * Lattice sites (x, y, z), 0 <= x < nx etc.; linear index
 *     i = (z*ny + y)*nx + x.  Spacing is 1 lattice unit (section III.B).
 *   * A Q field is five arrays of N = nx*ny*nz doubles, structure of arrays:
 *     q[c*N + i] for c = 0..4 = (Qxx, Qxy, Qxz, Qyy, Qyz); Qzz = -Qxx - Qyy
 *     (section III.B: five independent degrees of freedom per site).
 *   * Forces are -dF/dq over those five variables (section III.B, gradient
 *     by explicit differentiation of the discrete energy), 0 at object sites.
 *   * Host pointers are owned by the caller and only read or written during
 *     the call.  Device state is owned by the solver until lq_destroy.
 *   * Every call returns an lq_status; on failure lq_last_error() gives a
 *     message.  No call aborts or exits.  Calls on one solver must not
 *     overlap (the solver is not thread-safe); distinct solvers may be used
 *     from different threads.
 *   * All device work is issued on the CUDA stream given to lq_create (with
 *     NULL the solver creates and owns a non-blocking stream, since CUDA
 *     graphs cannot capture the legacy default stream); the calls that
 *     return host data synchronise that stream.  Device inputs handed to
 *     lq_set_q_device must be ready before the call (the caller orders its
 *     own stream against the solver's).
 */
#ifndef LQMIN_H
#define LQMIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lq_solver lq_solver;
typedef struct lq_server lq_server;

typedef enum {
    LQ_OK = 0,
    LQ_EINVAL = 1,          /* bad argument or state; nothing changed */
    LQ_ENOMEM = 2,          /* device or host allocation failed */
    LQ_ECUDA = 3,           /* a CUDA call failed; message has the CUDA error */
    LQ_ENOTCONVERGED = 4,   /* max_iter reached before the force tolerance */
    LQ_ETIMEOUT = 5,        /* wall-clock limit reached */
    LQ_EDIVERGED = 6,       /* a FIRE reduction became NaN or infinite */
    LQ_EBUSY = 7            /* work still running (server polling) */
} lq_status;

typedef enum {
    LQ_FP64 = 0,                 /* state, stencil and reductions in FP64 */
    LQ_FP32_BULK_FP64_RED = 1    /* state and stencil/bulk arithmetic in FP32,
                                    FIRE reductions, residual and energy in FP64 */
} lq_precision;

/* Lattice, section III.B.  spacing must be 1 (lattice units).
   periodic[k] != 0 wraps axis k; otherwise the lattice edge ends the
   one-sided differences along k (no neighbour beyond it). */
typedef struct {
    int nx, ny, nz;
    double spacing;
    int periodic[3];
} lq_lattice;

/* Material constants in lattice units.  Bulk A, B, C: Eq. (fphase).
   Distortion L1, L2, L3, the chiral L4 and the cubic L6 term:
   Eq. (fdistortionFull), each averaged over the allowed one-sided
   differences like the others.  n_constants = 1 uses the one-constant form
   Eq. (fd1) (L2 = L3 = L4 = L6 = 0 required), 3 the full form.  S0 <= 0
   selects Eq. (S0def) from A, B, C; it sets the preferred order of the
   anchoring terms.  External fields (section II): the density
   -(1/3) mu0_dchi H.Q.H - (1/3) eps0_deps E.Q.E (mu0 dchi and eps0 deps the
   anisotropic couplings, in lattice units), reported with the bulk energy;
   all zero for none. */
typedef struct {
    double A, B, C;
    double L1, L2, L3, L4, L6;
    int n_constants;
    double S0;
    double H[3], mu0_dchi;
    double E[3], eps0_deps;
} lq_material;

/* Anchoring of a surface, section II (boundary free energy):
   ND_HOMEOTROPIC  Nobili-Durand W tr((Q - Q0)^2), Q0 = 3/2 S0 (nu nu - I/3)
                   with nu the surface normal;
   ND_ORIENTED     the same with the preferred director dir instead of nu;
   FG_PLANAR       Fournier-Galatola planar-degenerate W |Qt - P Qt P|^2,
                   Qt = Q + S0 I/2, P = I - nu nu.
   For objects without a geometric normal (site lists) dir is used as nu. */
typedef enum {
    LQ_ANCHOR_ND_HOMEOTROPIC = 0,
    LQ_ANCHOR_ND_ORIENTED = 1,
    LQ_ANCHOR_FG_PLANAR = 2
} lq_anchor_kind;

typedef struct {
    int kind;       /* lq_anchor_kind */
    double W;       /* anchoring strength (lattice units) */
    double dir[3];  /* preferred director or normal, see above; need not be unit */
} lq_anchoring;

/* Minimiser parameters.  method LQ_MIN_FIRE (0): FIRE, Algorithm 1 (after
   Bitzek et al. 2006).  Velocity Verlet steps of size dt; alpha mixes v
   toward |v| F/|F|; after more than n_min consecutive steps with
   P = F.v > 0, dt <- min(dt f_inc, dt_max) and alpha <- alpha f_alpha; when
   P <= 0, dt <- dt f_dec, alpha <- alpha0, v <- 0.
   The paper's other minimisers (section III.C, which names gradient descent
   and Nesterov's accelerated gradient; Fig. 2 compares FIRE with gradient
   descent) use dt0 as the step eta and ignore the FIRE-only fields:
   LQ_MIN_GD (1): x <- x + eta F(x);
   LQ_MIN_NESTEROV (2): y = x_k + mu (x_k - x_{k-1}), x_{k+1} = y + eta F(y),
   momentum mu in [0, 1); the state (q, force, residual) is that of y, where
   the force is evaluated.
   All: converged when max over sites of the five-component force norm is
   below force_tol; wall_timeout_s <= 0 disables the wall-clock limit.  A
   zero-initialised method and momentum give FIRE. */
typedef enum { LQ_MIN_FIRE = 0, LQ_MIN_GD = 1, LQ_MIN_NESTEROV = 2 } lq_minimizer;

typedef struct {
    double dt0, dt_max, alpha0, f_alpha, f_inc, f_dec;
    int n_min;
    int64_t max_iter;
    double force_tol;
    double wall_timeout_s;
    int method;        /* lq_minimizer */
    double momentum;   /* LQ_MIN_NESTEROV: mu */
} lq_fire_params;

/* LQ_FIRE_STALLED: a tensor copy of the FP32 form's step did not complete
   within its time limit (about a second; copies take microseconds); the step
   kernel stopped and the entry point returned LQ_ECUDA.  lq_fire_reset (or a
   new lq_minimize) starts again. */
typedef enum { LQ_FIRE_RUNNING = 0, LQ_FIRE_CONVERGED = 1, LQ_FIRE_MAXITER = 2,
               LQ_FIRE_DIVERGED = 3, LQ_FIRE_STALLED = 4 } lq_fire_status;

/* State after the last completed FIRE iteration.  max_force is the largest
   site force norm, rms_force = |F| / sqrt(N simulated sites), power = F.v
   (section III.B, Fig. 2 measures); energy is filled by lq_minimize only. */
typedef struct {
    int64_t iterations;
    double max_force, rms_force, norm_force, norm_velocity, power;
    double dt, alpha;
    int64_t npos;
    double energy;
    int fire_status;        /* lq_fire_status */
    double seconds;         /* wall time of the call */
} lq_result;

/* Distortion constants from Frank constants (section II: Eq. (fdistortionFull)
   reproduces the Frank-Oseen density Eq. (FOfull) in the uniaxial limit):
   L[0..4] = L1, L2, L3, L4, L6 for splay K1, twist K2, bend K3, saddle-splay
   K24, chiral wavenumber q0 and order S (all in lattice units):
     L1 = 2 (K3 - K1 + 3 K2) / (27 S^2),  L2 = 4 (K1 - K24) / (9 S^2),
     L3 = 4 (K24 - K2) / (9 S^2),         L4 = -8 q0 K2 / (9 S^2),
     L6 = 4 (K3 - K1) / (27 S^3).
   K1 = K2 = K3 = K24 = K, q0 = 0 gives the one-constant L1 = 2K / (9 S^2)
   of Eq. (fd1).  Host arithmetic only.  LQ_EINVAL for S <= 0 or a
   non-finite input. */
lq_status lq_frank_to_landau(double K1, double K2, double K3, double K24, double q0, double S,
                             double L[5]);

/* ---- lifetime ------------------------------------------------------------- */

/* Create a solver for one lattice (section III.B).  cuda_stream is a
   cudaStream_t (NULL = a stream owned by the solver); precision is an
   lq_precision.
   Allocates the device state: 2 x (q, v, F) buffers, 1-byte site masks and
   the FIRE reduction scratch.  LQ_EINVAL for non-positive sizes, spacing
   != 1, n_constants not 1 or 3, L2..L6 != 0 with n_constants 1, or A, B, C
   without a nematic minimum (when S0 <= 0). */
lq_status lq_create(const lq_lattice *lattice, const lq_material *material,
                    int precision, void *cuda_stream, lq_solver **out);
/* Free all device and host memory of the solver (NULL is accepted). */
void lq_destroy(lq_solver *s);
/* Message of the last failed call on this solver (never NULL). */
const char *lq_last_error(const lq_solver *s);
/* Message of the last failed lq_create in this thread. */
const char *lq_create_error(void);

/* ---- geometry: objects and boundary sites (section III.B "type" per site;
        section V simple objects and custom boundary files) ----------------- */

/* Wall: every site with coord[axis] == plane becomes an object site; its
   simulated face neighbours are boundary sites with normal e_axis. */
lq_status lq_add_wall(lq_solver *s, int axis, int plane, const lq_anchoring *a);
/* Sphere: sites with |x - c|^2 <= R^2 (minimum image along periodic axes)
   are object sites; boundary normal (x - c)/|x - c|. */
lq_status lq_add_sphere(lq_solver *s, const double c[3], double radius,
                        const lq_anchoring *a);
/* Droplet (Fig. 3, the confining shell of a drop): every site with
   |x - c|^2 > R^2 (minimum image) is an object site, so the liquid crystal
   fills the ball; boundary normal (x - c)/|x - c|, pointing out of the drop.
   LQ_EINVAL for radius <= 0. */
lq_status lq_add_droplet(lq_solver *s, const double c[3], double radius,
                         const lq_anchoring *a);
/* Spherocylinder (Fig. 3): sites within distance R of the segment p0..p1
   are object sites; boundary normal x - p*, p* the nearest point of the
   segment.  Distances are taken from the segment's midpoint with the
   minimum image along periodic axes, so the object must fit in the box
   (|p1 - p0|/2 + R below half the period).  p0 == p1 is a sphere.
   LQ_EINVAL for radius < 0. */
lq_status lq_add_spherocylinder(lq_solver *s, const double p0[3], const double p1[3],
                                double radius, const lq_anchoring *a);
/* Custom object: the n listed sites (xyz[3*t..3*t+2]) become object sites;
   their simulated face neighbours take anchoring a (dir used as normal).
   Sites outside the lattice are ignored. */
lq_status lq_add_object_sites(lq_solver *s, int64_t n, const int32_t *xyz,
                              const lq_anchoring *a);
/* Custom boundary records: each listed simulated site gets its own
   anchoring per_site[t] (dir is the preferred director or normal).
   When several objects claim a boundary site, the first one added wins. */
lq_status lq_add_anchored_sites(lq_solver *s, int64_t n, const int32_t *xyz,
                                const lq_anchoring *per_site);
/* Custom boundary text (section VI: objects made of arbitrary site sets,
   each boundary site with its own homeotropic or planar anchoring, read
   from a prepared text file).  The format of this library:
     - '#' starts a comment; blank lines are skipped; tokens are separated
       by blanks;
     - a block "object <anchoring> <W> [dx dy dz]" ... "end" lists object
       sites, one "x y z" per line; their simulated face neighbours take the
       anchoring (as lq_add_object_sites, dir = (dx, dy, dz), default
       (0, 0, 1));
     - a block "boundary" ... "end" lists anchored sites, one
       "x y z <anchoring> <W> dx dy dz" per line (as lq_add_anchored_sites);
     - <anchoring> is homeotropic | oriented | planar (or 0 | 1 | 2, the
       lq_anchor_kind values); W >= 0.
   Blocks become objects in file order.  The whole text is checked before
   anything is added: on any error nothing changes and the message names
   the line.  lq_boundary_check parses without a solver (no device work)
   and reports the number of blocks and of site lines; err (errlen bytes,
   may be NULL) receives the message. */
lq_status lq_boundary_check(const char *text, int64_t *n_blocks, int64_t *n_sites,
                            char *err, size_t errlen);
lq_status lq_add_boundary_text(lq_solver *s, const char *text);
/* The same read from a file (LQ_EINVAL if it cannot be read). */
lq_status lq_load_boundary_file(lq_solver *s, const char *path);
/* Objects added so far (their index order is the order of addition). */
lq_status lq_object_count(lq_solver *s, int *n);
/* Move object `index` by shift (section VI: objects repositioned and the
   liquid crystal re-minimised).  Spheres, droplets and spherocylinders move
   by any shift; walls by whole planes along their axis (other components
   ignored); site lists by whole lattice vectors, wrapping periodic axes.
   Sites the object leaves become simulated with Q = 0; sites it covers
   become object sites.  The minimiser restarts at the next step. */
lq_status lq_move_object(lq_solver *s, int index, const double shift[3]);
/* Remove every object (Q on the freed sites is 0). */
lq_status lq_clear_objects(lq_solver *s);
/* Change the material constants of a live solver (section VI: energy terms
   changed between minimisations).  Same rules as lq_create; Q is kept, the
   anchoring targets follow the new S0 and the minimiser restarts at the
   next step. */
lq_status lq_set_material(lq_solver *s, const lq_material *material);
/* A new solver (on cuda_stream, NULL = its own) with the same lattice,
   material, precision, objects and current Q as src. */
lq_status lq_clone(lq_solver *src, void *cuda_stream, lq_solver **out);
/* Potential-of-mean-force sweep (section VI): for each k < n a clone of
   base with object `index` moved by shifts[3k..3k+2] starts from base's
   current Q (freed sites 0), and all n are minimised together in one batch
   (lq_batch_minimize; n results with the energy at the minimum).  base is
   not modified.  Returns what lq_batch_minimize returns. */
lq_status lq_pmf_sweep(lq_solver *base, int index, int n, const double *shifts,
                       const lq_fire_params *p, lq_result *out);
/* Dipolar start about a homeotropic colloid (section IV.A, the dipolar
   initial condition after Lubensky et al.): a radial hedgehog at c and a
   hyperbolic hedgehog at h = c + rd a (a = axis / |axis|, also the far-field
   director), n tilted from a by theta_c - theta_h, the polar angles of the
   site about a seen from c and from h (minimum image of x - c, w = u - rd a);
   Q = 3/2 S (n n - I/3) on simulated sites, S <= 0 selecting S0; n = a
   where the angles are undefined.  Resets the minimiser.  LQ_EINVAL for a
   zero axis or rd <= 0. */
lq_status lq_init_dipolar(lq_solver *s, const double c[3], const double axis[3], double rd,
                          double S);
/* Number of simulated sites and of sites carrying an anchoring record
   (builds the geometry if it changed). */
lq_status lq_geometry_info(lq_solver *s, int64_t *n_simulated, int64_t *n_anchored);
/* Per-site mask byte: bit0 simulated, bit1 anchored, bits 2..7 neighbour
   simulated along +x, -x, +y, -y, +z, -z.  out holds N bytes. */
lq_status lq_get_mask(lq_solver *s, uint8_t *out);

/* ---- state in and out ------------------------------------------------------ */

/* Set Q from a host array (5*N doubles, layout above).  Resets FIRE. */
lq_status lq_set_q(lq_solver *s, const double *q_host);
/* Set Q from a device array of 5*N elements, dtype 0 = double, 1 = float;
   the copy runs on the solver stream.  Resets FIRE. */
lq_status lq_set_q_device(lq_solver *s, const void *dptr, int dtype);
/* Random uniaxial start (section V: random initial Q, reproducible): site i
   gets 3/2 S (n n - I/3) with n uniform on the sphere from SplitMix64
   outputs 2i+1 (z = 2u-1) and 2i+2 (phi = 2 pi u) of the stream seed.
   S <= 0 selects S0.  Resets FIRE. */
lq_status lq_init_random_uniaxial(lq_solver *s, uint64_t seed, double S);
/* Copy the current Q / FIRE velocity / FIRE force to a host array (5*N). */
lq_status lq_get_q(lq_solver *s, double *out);
lq_status lq_get_velocity(lq_solver *s, double *out);
lq_status lq_get_force(lq_solver *s, double *out);
/* Evaluate F = -dF/dq at the current Q (section III.B) without touching the
   FIRE state; out = 5*N doubles. */
lq_status lq_force(lq_solver *s, double *out);
/* Total free energy of the current Q, summed in FP64: total and parts
   (bulk Eq. (fphase), distortion Eq. (fdistortionFull) averaged over allowed
   differences, anchoring).  Either pointer may be NULL. */
lq_status lq_energy(lq_solver *s, double *total, double parts[3]);
/* Largest eigenvalue of Q per site (the director's order, section II;
   defects are where it drops, section V); 0 at object sites.  N doubles. */
lq_status lq_order_field(lq_solver *s, double *S_out);

/* ---- FIRE (Algorithm 1) ------------------------------------------------------- */

/* Start FIRE from the current Q: v = 0, F = F(q), dt = dt0, alpha = alpha0. */
lq_status lq_fire_reset(lq_solver *s, const lq_fire_params *p);
/* Run up to n more FIRE iterations (starting FIRE first if needed); stops
   early at convergence, max_iter or divergence.  out may be NULL. */
lq_status lq_step(lq_solver *s, const lq_fire_params *p, int64_t n, lq_result *out);
/* Minimise from the current Q to force_tol (section V: until a force
   tolerance or the maximum number of iterations).  Returns LQ_OK when
   converged, LQ_ENOTCONVERGED at max_iter, LQ_EDIVERGED, LQ_ETIMEOUT. */
lq_status lq_minimize(lq_solver *s, const lq_fire_params *p, lq_result *out);
/* Read the FIRE counters without running anything. */
lq_status lq_fire_result(lq_solver *s, lq_result *out);

/* Checkpoint of Q, v, F and the FIRE scalars.  With buf == NULL, *bytes
   receives the size needed.  Resuming from a checkpoint continues the run
   bit-for-bit. */
lq_status lq_get_state(lq_solver *s, void *buf, size_t *bytes);
lq_status lq_set_state(lq_solver *s, const void *buf, size_t bytes);

/* ---- batches: many lattices, one persistent kernel per FIRE iteration ------------------ */

/* Independent minimisations advanced together (section III.B's per-site work
   is independent across lattices): each FIRE iteration of every lattice in
   the batch is one launch of a persistent kernel whose blocks stride over
   (lattice, tile, z chunk) work items; launches are captured in CUDA graphs.
   Every lattice keeps its own state, FIRE scalars (Algorithm 1) and
   reductions; with the solvers' own tiling (the default) a one-constant
   lattice advances bit-for-bit as it does alone, a three-constant one to
   within rounding (the two kernels may fuse its products differently).  All solvers must share device, precision and
   n_constants (LQ_EINVAL otherwise).  The batch runs on a stream of its own
   (ordered against the solvers' streams by synchronising them around each
   call) and borrows the solvers until lq_batch_destroy: destroy the batch
   before them.  Allocates its work-item and reduction tables. */
typedef struct lq_batch lq_batch;
lq_status lq_batch_create(lq_solver *const *solvers, int n, lq_batch **out);
void lq_batch_destroy(lq_batch *b);
const char *lq_batch_last_error(const lq_batch *b);
/* Tiling of the persistent kernel: tile 32 x tile_y (4 or 8) and z chunk
   (0 = each lattice's own z chunk, as lq_set_zchunk left it); LQ_EINVAL for
   other tile heights or a negative z chunk, the tiling unchanged.
   lq_batch_get_tiling reports the height and z chunk of the current tiling,
   whatever its width. */
lq_status lq_batch_set_tiling(lq_batch *b, int tile_y, int zchunk);
lq_status lq_batch_get_tiling(const lq_batch *b, int *tile_y, int *zchunk);
/* The same with the tile width: tile_x 32, or 64 when every lattice is a
   one-constant FP32-form lattice (the wide tiles of the single-lattice
   kernel: half the ring columns per site); LQ_EINVAL otherwise, the tiling
   unchanged.  A lattice advances bit-for-bit as it does alone when its own
   step runs the same tile (alone, 64-wide tiles serve one-constant FP32-form
   lattices at least 256 sites wide) and z chunk.  Any pointer of the getter
   may be NULL.  A change of members that brings a three-constant lattice
   into a batch with 64-wide tiles turns them back to 32. */
lq_status lq_batch_set_tile(lq_batch *b, int tile_x, int tile_y, int zchunk);
lq_status lq_batch_get_tile(const lq_batch *b, int *tile_x, int *tile_y, int *zchunk);
/* Autotuner: times every tile width the lattices allow (32, and 64 for
   one-constant FP32-form batches), tile_y in {4, 8} and z chunk in
   {8, ..., 128}, each over `launches` launches (CUDA events) on shadow copies
   of the FIRE states (the lattices' states do not advance), and keeps the
   fastest; *best_ms may be NULL.  Starts FIRE on lattices that have not
   started. */
lq_status lq_batch_autotune(lq_batch *b, const lq_fire_params *p, int launches, double *best_ms);
/* n more FIRE iterations of every lattice (converged ones stay put); out
   holds one lq_result per solver, or NULL. */
lq_status lq_batch_step(lq_batch *b, const lq_fire_params *p, int64_t n, lq_result *out);
/* Minimise every lattice from its current Q (FIRE restarted); returns LQ_OK
   when all converged, else the worst of LQ_EDIVERGED / LQ_ENOTCONVERGED /
   LQ_ETIMEOUT; out as above, energies filled. */
lq_status lq_batch_minimize(lq_batch *b, const lq_fire_params *p, lq_result *out);

/* ---- serving: continuous batching of minimisation requests -------------------------- */

/* An object of a request, the same objects lq_add_* take (section V). */
enum { LQ_OBJ_WALL = 0, LQ_OBJ_SPHERE = 1, LQ_OBJ_SITES = 2, LQ_OBJ_ANCHORED = 3,
       LQ_OBJ_DROPLET = 4, LQ_OBJ_SPHEROCYLINDER = 5 };
typedef struct {
    int type;                       /* LQ_OBJ_* */
    int axis, plane;                /* wall */
    double c[3], R;                 /* sphere, droplet (centre, radius); spherocylinder (end, radius) */
    lq_anchoring anch;              /* wall, sphere, droplet, spherocylinder, object sites */
    int64_t n;                      /* site lists: number of sites */
    const int32_t *xyz;             /* site lists: 3n coordinates */
    const lq_anchoring *per_site;   /* anchored sites: n records */
    double c2[3];                   /* spherocylinder: the other end of its axis */
} lq_object;

/* One minimisation (section V: set up a lattice and objects, start from a
   given or seeded random Q, minimise to a force tolerance). */
typedef struct {
    lq_lattice lattice;
    lq_material material;
    int n_objects;
    const lq_object *objects;
    const double *q0;               /* 5N host values, or NULL: seeded random start */
    uint64_t seed;                  /* random start (lq_init_random_uniaxial) */
    double S;                       /* its order, <= 0: S0 */
    lq_fire_params params;          /* wall_timeout_s counts from admission */
    int want_order_field;           /* keep lambda_max per site for the poll */
} lq_request;

typedef struct {
    int64_t queued, active, completed;
    size_t bytes_in_use, budget;    /* estimated device bytes of the active solves */
    double site_updates;            /* sum over finished solves of N x iterations */
    double site_updates_issued;     /* N x k over every active solve of every round of
                                       k launches so far (a solve that converges inside a
                                       round is counted to the round's end) */
} lq_server_stats;

/* A server on the current device: a worker thread admits queued requests
   while the estimated device memory of the active solves stays within
   hbm_budget_bytes and at most max_active run at once; every active solve
   is advanced by the same persistent-kernel launches (one batch per
   distortion form), and finished solves are retired between rounds of
   launches, so requests arriving while others run join them as memory frees
   up.  A one-constant solve follows the same trajectory as it would alone. */
lq_status lq_server_create(size_t hbm_budget_bytes, int precision, int max_active, lq_server **out);
/* Stops the worker (running solves are dropped) and frees everything. */
void lq_server_destroy(lq_server *sv);
/* Queue a request (its arrays are copied); LQ_ENOMEM if it could never fit
   the budget.  *ticket identifies it. */
lq_status lq_server_submit(lq_server *sv, const lq_request *rq, uint64_t *ticket);
/* LQ_EBUSY while queued or running; then the solve's status (LQ_OK when
   converged, LQ_ENOTCONVERGED, LQ_EDIVERGED, LQ_ETIMEOUT, or the error that
   stopped its set-up), *out with out->seconds = time from submission to
   completion and the final energy, S_out (N doubles, may be NULL) the order
   field if requested.  A finished ticket can be read once: LQ_EINVAL for a
   ticket the server never issued or has already handed back. */
lq_status lq_server_poll(lq_server *sv, uint64_t ticket, lq_result *out, double *S_out);
/* As lq_server_poll, waiting up to timeout_s (<= 0: no limit). */
lq_status lq_server_wait(lq_server *sv, uint64_t ticket, double timeout_s, lq_result *out,
                         double *S_out);
lq_status lq_server_stats_get(lq_server *sv, lq_server_stats *out);

/* ---- one lattice over several GPUs: z slabs ----------------------------------------- */

/* Section III.B decomposes the lattice into sub-domains with halos, and
   FIRE's power and norms (Algorithm 1) become sums over every sub-domain.
   Here the sub-domains are slabs of z planes, one per GPU (one rank each).
   lq_slab_create cuts planes [z_lo, z_hi) of a solver of the whole lattice
   (built on each rank; only its geometry is used -- its masks and anchoring
   records, so that every neighbour bit is the whole lattice's) into a new
   solver on the current device with one halo plane below and one above:
   its lattice is nx x ny x (z_hi - z_lo + 2), open in z, its own planes
   1 .. z_hi - z_lo.  Its Q is set with lq_set_q / lq_set_q_device on all
   its planes (halos included, taken from the whole lattice with its
   periodicity) and read with lq_get_q.  A slab refuses lq_step,
   lq_minimize, lq_fire_reset, objects, materials, clones and batches.
   LQ_EINVAL for planes outside [0, nz), an empty slab, or a slab of a slab.
   One FIRE iteration of the decomposed lattice, on every slab:
     lq_slab_step(s, local)       the fused step over the own planes; local =
                                  the slab's (P, |F|^2, |v|^2, largest site |F|^2);
     total = (sum, sum, sum, max) of local over every slab, in FP64;
     lq_slab_finish(s, total, out) the FIRE scalar update from total, the same
                                  on every slab; out as lq_step's (may be NULL;
                                  its rms_force uses the slab's own site count);
     lq_slab_get_planes / lq_slab_set_halos  the first and last own planes go to
                                  the neighbouring slabs' upper and lower halos.
   lq_slab_start(s, p, local) starts FIRE (v = 0, F = F(q0)) the same way, to be
   followed by lq_slab_finish and the halo exchange.  Plane buffers are host
   memory of lq_slab_plane_bytes bytes: q, v, F, each five components of the
   nx*ny sites of the plane, x fastest, in the solver's storage format (FP64
   form: doubles; FP32 form: q as 32-bit fixed point, q = n * 2^-28, v and F
   as floats).  NULL skips a plane (a halo beyond an open z edge, which holds
   no sites). */
lq_status lq_slab_create(lq_solver *whole, int z_lo, int z_hi, lq_solver **out);
lq_status lq_slab_start(lq_solver *s, const lq_fire_params *p, double local[4]);
lq_status lq_slab_step(lq_solver *s, double local[4]);
lq_status lq_slab_finish(lq_solver *s, const double total[4], lq_result *out);
lq_status lq_slab_plane_bytes(const lq_solver *s, size_t *bytes);
lq_status lq_slab_get_planes(lq_solver *s, void *lower_own, void *upper_own);
lq_status lq_slab_set_halos(lq_solver *s, const void *below, const void *above);

/* ---- without allocation ------------------------------------------------------------ */

/* The paper has no counterpart to this call; it exists for callers that cannot
   let a library call cudaMalloc: a process whose device memory is reserved
   up front by its own allocator or budget, or a latency-bound loop that
   cannot take the device-wide synchronisation of cudaMalloc/cudaFree.  It
   allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
   Computes two parts of the energy of a caller-owned device Q field, summed
   in FP64: the Landau bulk part (with the external-field term) and the
   elastic part from the averaged one-sided differences between
   neighbouring sites (with the chiral and cubic terms when L4, L6 are set);
   the surface anchoring part is not included.  Lattice and material are
   checked as lq_create checks them (spacing 1, n_constants 1 or 3, a
   one-constant material with L2 = L3 = L4 = L6 = 0, a nematic minimum):
   LQ_EINVAL otherwise.  q_dev = 5*N doubles (layout above), mask_dev = N
   mask bytes in the lq_get_mask layout, both on the device; a mask bit that
   names a neighbour beyond a non-periodic edge of this lattice (a mask
   built for other periodic flags) is treated as an absent neighbour, so
   nothing outside the arrays is read.  parts_dev = 3 device doubles
   receiving (bulk, elastic, 0).  Work runs on cuda_stream (NULL = legacy
   default stream) and is not synchronised.  Scratch is a static device
   array of 3 doubles per z plane, for at most 4096 planes (96 KB held on
   every GPU that loads the library until exit): nz > 4096 returns
   LQ_EINVAL, as do null pointers or non-positive sizes.  The first call on
   a device resolves that array's address with the device current; make
   that first call before any stream capture.  Every call shares the array
   (each call overwrites it), so calls that overlap on the GPU race.
   LQ_ECUDA if a launch or the address lookup fails. */
lq_status lq_energy_noalloc(const lq_lattice *lattice, const lq_material *material,
                            const double *q_dev, const uint8_t *mask_dev, double *parts_dev,
                            void *cuda_stream);

/* ---- testing: host-side fault injection ------------------------------------------
   After lq_inject_fault(kind, after), the (after + 1)-th device allocation
   (LQ_FAULT_DEVICE_ALLOC) or step-kernel launch (LQ_FAULT_STEP_LAUNCH, one
   launch of the single-lattice or the batched step kernel, direct or while
   a CUDA graph is captured) that the library makes fails as if CUDA had
   returned out-of-memory or a launch failure: nothing is allocated or
   launched for it, and the calling entry point returns LQ_ENOMEM or
   LQ_ECUDA.  LQ_FAULT_COPY_WAIT: the (after + 1)-th launch of the
   tensor-copy staging (lq_set_staging) makes its barriers expect more bytes
   than its copies deliver, so that every wait for a plane runs out (about a
   second each; copies take microseconds): the kernel stops with FIRE
   status LQ_FIRE_STALLED and the entry point returns LQ_ECUDA -- the path a
   copy that never completed would take.  No device fault is ever made.
   One-shot and process-wide; LQ_FAULT_NONE cancels.  LQ_EINVAL for an
   unknown kind or after < 0. */
enum { LQ_FAULT_NONE = 0, LQ_FAULT_DEVICE_ALLOC = 1, LQ_FAULT_STEP_LAUNCH = 2, LQ_FAULT_COPY_WAIT = 3 };
lq_status lq_inject_fault(int kind, int64_t after);
/* The bounds-checked build of the library (compiled with LQ_BOUNDS_CHECK)
   checks every shared-memory slot, tile and ring index and every global
   element index of the step kernels; an index out of range is counted and
   replaced by 0, so nothing is accessed out of range.  *hits: the count
   since the library was loaded.  The release build has no checks and
   returns LQ_EINVAL with *hits = 0. */
lq_status lq_bounds_check_hits(uint32_t *hits);

/* ---- tuning ---------------------------------------------------------------------- */

/* Number of z planes one thread block marches through (0 = automatic). */
lq_status lq_set_zchunk(lq_solver *s, int zchunk);
/* Element-index width of the step kernels: 0 = automatic (32-bit indices
   while 5 N < 2^32, i.e. below about 950^3 sites, 64-bit beyond; the FP32
   form's three-constant step always runs its 64-bit instantiation, which is
   faster), 64 = the 64-bit instantiation on any lattice (the code path of
   the largest lattices, for testing it on small ones; results are
   identical).  LQ_EINVAL for other values. */
lq_status lq_set_index_width(lq_solver *s, int bits);
/* Plane staging of the FP32 form's step kernel (three constants, no chiral
   or cubic term): 0 = automatic (the faster staging measured on B300:
   per-thread loads), 1 = per-thread loads, 2 = tensor copies, LQ_EINVAL
   where they cannot serve (they need the lattice's x extent a multiple of
   32 and a driver that encodes tensor maps).  In the tensor-copy staging the rows of each z plane that a
   32 x 4 tile and its ring need arrive in shared memory as bulk tensor
   copies completing on a barrier, instead of one load per thread and value;
   the arithmetic is the same and so are the results, bit for bit. */
lq_status lq_set_staging(lq_solver *s, int mode);
/* *uses_tensor_copies = 1 when the solver's next FIRE step runs the
   tensor-copy staging, else 0. */
lq_status lq_get_staging(lq_solver *s, int *uses_tensor_copies);
/* Bytes of device memory held by the solver. */
size_t lq_device_bytes(const lq_solver *s);

/* ---- measurement ------------------------------------------------------------------ */

/* Measured FP64 fused multiply-add rate of the current device, the ceiling
   of the FP64 form of the step (section III.B's force and Algorithm 1's
   update in double precision), which is bound by the FP64 pipe here rather
   than by memory.  Every resident thread runs 8 independent chains of iters
   dependent fused multiply-adds; one untimed launch first, then one launch
   timed with CUDA events on a stream of its own.  *fma_per_s receives the
   thread-level fused multiply-adds per second (each is one FP64 operation
   in the FP64 form's operation count; twice as many flops).  The call
   allocates and frees a small output buffer.  LQ_EINVAL for iters <= 0 or a
   null pointer, LQ_ENOMEM / LQ_ECUDA on a CUDA failure. */
lq_status lq_fp64_fma_rate(int64_t iters, double *fma_per_s);

#ifdef __cplusplus
}
#endif
#endif /* LQMIN_H */
