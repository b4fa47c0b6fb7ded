/*
 * lqoracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Slow and literal on purpose: every formula is written the way the paper
 * states it, so that a reader can check it against the text by eye.
 *   * bulk energy:        Eq. (fphase)                (section II.A)
 *   * distortion energy:  Eq. (fdistortionFull), L1/L2/L3 terms
 *   * finite differences: Eq. (onesidedderivatives), averaged over every
 *                         allowed forward/backward combination (sec. III.B)
 *   * anchoring:          Nobili-Durand and Fournier-Galatola forms
 *                         (section II, boundary free energy)
 *   * force:              minus the derivative of the discrete total energy
 *                         with respect to each q_i(x_j) (section III.B)
 *   * minimiser:          FIRE, Algorithm 1 (after Bitzek et al. 2006)
 * The distortion energy of a site is found by enumerating the allowed
 * difference combinations one by one; the force gathers, for each site j,
 * the derivative of the energy of every site whose energy involves q(j).
 * No blocking, no factorisation of the combination average.
 */
#include "lqoracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the parallel loops from now on (n >= 1); returns the count in
   effect, so that a timing can name the cores it used */
int orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ---- lattice helpers -------------------------------------------------- */

static int64_t idx3(const orc_model *m, int x, int y, int z) {
    return ((int64_t)z * m->ny + y) * m->nx + x;
}

static void coords(const orc_model *m, int64_t i, int c[3]) {
    c[0] = (int)(i % m->nx);
    c[1] = (int)((i / m->nx) % m->ny);
    c[2] = (int)(i / ((int64_t)m->nx * m->ny));
}

/* neighbour of site i one step along axis k in direction dir (+1 / -1);
   -1 when the step leaves a non-periodic lattice */
static int64_t neighbour(const orc_model *m, int64_t i, int k, int dir) {
    int c[3], n[3] = {m->nx, m->ny, m->nz};
    coords(m, i, c);
    c[k] += dir;
    if (c[k] < 0 || c[k] >= n[k]) {
        if (!m->periodic[k]) return -1;
        c[k] = (c[k] + n[k]) % n[k];
    }
    return idx3(m, c[0], c[1], c[2]);
}

/* Q as a full 3x3 matrix from the five independent components (sec. III.B) */
static void qmat(const double *q, int64_t N, int64_t i, double Q[3][3]) {
    double xx = q[0 * N + i], xy = q[1 * N + i], xz = q[2 * N + i];
    double yy = q[3 * N + i], yz = q[4 * N + i];
    Q[0][0] = xx; Q[0][1] = xy; Q[0][2] = xz;
    Q[1][0] = xy; Q[1][1] = yy; Q[1][2] = yz;
    Q[2][0] = xz; Q[2][1] = yz; Q[2][2] = -xx - yy;
}

static void qmat5(const double q5[5], double Q[3][3]) {
    Q[0][0] = q5[0]; Q[0][1] = q5[1]; Q[0][2] = q5[2];
    Q[1][0] = q5[1]; Q[1][1] = q5[3]; Q[1][2] = q5[4];
    Q[2][0] = q5[2]; Q[2][1] = q5[4]; Q[2][2] = -q5[0] - q5[3];
}

/* chain rule from a derivative with respect to the nine entries of Q
   (treated as independent) to the five independent components */
static void to_q5(double G[3][3], double out[5]) {
    out[0] = G[0][0] - G[2][2];
    out[1] = G[0][1] + G[1][0];
    out[2] = G[0][2] + G[2][0];
    out[3] = G[1][1] - G[2][2];
    out[4] = G[1][2] + G[2][1];
}

/* ---- bulk, Eq. (fphase) ------------------------------------------------ */

/* the external-field coupling tensor: f_ext = -(1/3) sum_ab K_ab Q_ab with
   K = mu0_dchi H H^T + eps0_deps E E^T */
static void field_tensor(const orc_model *m, double K[3][3]) {
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) K[a][b] = m->mu0_dchi * m->H[a] * m->H[b] + m->eps0_deps * m->E[a] * m->E[b];
}

static double bulk_energy(const orc_model *m, double Q[3][3]) {
    double trQ2 = 0.0, trQ3 = 0.0, ext = 0.0, K[3][3];
    field_tensor(m, K);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            trQ2 += Q[a][b] * Q[b][a];
            for (int c = 0; c < 3; ++c) trQ3 += Q[a][b] * Q[b][c] * Q[c][a];
            ext += K[a][b] * Q[a][b];
        }
    return m->A / 2.0 * trQ2 + m->B / 3.0 * trQ3 + m->C / 4.0 * trQ2 * trQ2 - ext / 3.0;
}

/* dF/dQ_ab of Eq. (fphase): A Q + B Q.Q + C tr(Q^2) Q */
static void bulk_grad(const orc_model *m, double Q[3][3], double G[3][3]) {
    double trQ2 = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) trQ2 += Q[a][b] * Q[b][a];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double QQ = 0.0;
            for (int c = 0; c < 3; ++c) QQ += Q[a][c] * Q[c][b];
            G[a][b] = m->A * Q[a][b] + m->B * QQ + m->C * trQ2 * Q[a][b];
        }
    double K[3][3];
    field_tensor(m, K);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[a][b] -= K[a][b] / 3.0;
}

/* ---- anchoring (boundary free energy) ---------------------------------- */

/* Nobili-Durand: W tr((Q - Q0)^2);  Fournier-Galatola: W |Qt - P Qt P|^2,
   Qt = Q + S0 I / 2, P = I - nu nu  (the projection is read as P.Qt.P) */
static double anchor_energy(const orc_model *m, const orc_anchor *r, double Q[3][3]) {
    double e = 0.0;
    if (r->kind == 1) {
        double Q0[3][3];
        qmat5(r->q0, Q0);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double d = Q[a][b] - Q0[a][b];
                e += d * d;
            }
        return r->W * e;
    }
    if (r->kind == 2) {
        double Qt[3][3], P[3][3], PQt[3][3], Qp[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                Qt[a][b] = Q[a][b] + (a == b ? m->S0 / 2.0 : 0.0);
                P[a][b] = (a == b ? 1.0 : 0.0) - r->nu[a] * r->nu[b];
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                PQt[a][b] = 0.0;
                for (int c = 0; c < 3; ++c) PQt[a][b] += P[a][c] * Qt[c][b];
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                Qp[a][b] = 0.0;
                for (int c = 0; c < 3; ++c) Qp[a][b] += PQt[a][c] * P[c][b];
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double d = Qt[a][b] - Qp[a][b];
                e += d * d;
            }
        return r->W * e;
    }
    return 0.0;
}

/* derivative of the anchoring energy with respect to the nine entries of Q:
   ND: 2 W (Q - Q0);  FG: 2 W (R - P R P) with R = Qt - P Qt P */
static void anchor_grad(const orc_model *m, const orc_anchor *r, double Q[3][3],
                        double G[3][3]) {
    memset(G, 0, 9 * sizeof(double));
    if (r->kind == 1) {
        double Q0[3][3];
        qmat5(r->q0, Q0);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a][b] = 2.0 * r->W * (Q[a][b] - Q0[a][b]);
    } else if (r->kind == 2) {
        double Qt[3][3], P[3][3], T[3][3], R[3][3], PRP[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                Qt[a][b] = Q[a][b] + (a == b ? m->S0 / 2.0 : 0.0);
                P[a][b] = (a == b ? 1.0 : 0.0) - r->nu[a] * r->nu[b];
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                T[a][b] = 0.0;
                for (int c = 0; c < 3; ++c)
                    for (int d = 0; d < 3; ++d) T[a][b] += P[a][c] * Qt[c][d] * P[d][b];
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) R[a][b] = Qt[a][b] - T[a][b];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                PRP[a][b] = 0.0;
                for (int c = 0; c < 3; ++c)
                    for (int d = 0; d < 3; ++d) PRP[a][b] += P[a][c] * R[c][d] * P[d][b];
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a][b] = 2.0 * r->W * (R[a][b] - PRP[a][b]);
    }
}

/* ---- distortion: averaged one-sided differences ------------------------ */

/* the allowed one-sided differences of site i along each axis:
   opt[k][.] = +1 forward (needs i+e_k simulated), -1 backward */
typedef struct {
    int nopt[3];
    int opt[3][2];
    int64_t fwd[3], bwd[3];
} fd_choices;

static void fd_allowed(const orc_model *m, const orc_geometry *g, int64_t i,
                       fd_choices *ch) {
    for (int k = 0; k < 3; ++k) {
        ch->nopt[k] = 0;
        ch->fwd[k] = neighbour(m, i, k, +1);
        ch->bwd[k] = neighbour(m, i, k, -1);
        if (ch->fwd[k] >= 0 && g->sim[ch->fwd[k]]) ch->opt[k][ch->nopt[k]++] = +1;
        if (ch->bwd[k] >= 0 && g->sim[ch->bwd[k]]) ch->opt[k][ch->nopt[k]++] = -1;
    }
}

/* d[a][b][k] = dQ_ab/dx_k for one combination s[k] in {+1,-1,0};
   0 marks an axis with no allowed difference, which then contributes none */
static void fd_tensor(const double *q, int64_t N, int64_t i, const fd_choices *ch,
                      const int s[3], double d[3][3][3]) {
    double Qi[3][3], Qn[3][3];
    qmat(q, N, i, Qi);
    for (int k = 0; k < 3; ++k) {
        if (s[k] == 0) {
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) d[a][b][k] = 0.0;
        } else if (s[k] > 0) {
            qmat(q, N, ch->fwd[k], Qn);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) d[a][b][k] = Qn[a][b] - Qi[a][b];
        } else {
            qmat(q, N, ch->bwd[k], Qn);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) d[a][b][k] = Qi[a][b] - Qn[a][b];
        }
    }
}

/* Levi-Civita symbol */
static double levi(int i, int j, int k) {
    return (double)((i - j) * (j - k) * (k - i)) / 2.0;
}

/* Eq. (fdistortionFull), Einstein summation written out, with Q the site's
   tensor (it multiplies the L4 and L6 terms):
   L1/2 d_ijk d_ijk + L2/2 d_ijj d_ikk + L3/2 d_ikj d_ijk
   + L4/2 eps_lik Q_lj d_ijk + L6/2 Q_lk d_ijl d_ijk,   d_ijk = dQ_ij/dx_k */
static double distortion_density(const orc_model *m, double Q[3][3], double d[3][3][3]) {
    double e1 = 0.0, e2 = 0.0, e3 = 0.0, e4 = 0.0, e6 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                e1 += d[i][j][k] * d[i][j][k];
                e2 += d[i][j][j] * d[i][k][k];
                e3 += d[i][k][j] * d[i][j][k];
                for (int l = 0; l < 3; ++l) {
                    e4 += levi(l, i, k) * Q[l][j] * d[i][j][k];
                    e6 += Q[l][k] * d[i][j][l] * d[i][j][k];
                }
            }
    return m->L1 / 2.0 * e1 + m->L2 / 2.0 * e2 + m->L3 / 2.0 * e3 + m->L4 / 2.0 * e4 +
           m->L6 / 2.0 * e6;
}

double orc_distortion_density(const orc_model *m, const double *Q9, const double *d27) {
    double Q[3][3], d[3][3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Q[i][j] = Q9[3 * i + j];
            for (int k = 0; k < 3; ++k) d[i][j][k] = d27[(3 * i + j) * 3 + k];
        }
    return distortion_density(m, Q, d);
}

/* derivative of the density above with respect to d[a][b][c] */
static void distortion_ddens(const orc_model *m, double Q[3][3], double d[3][3][3],
                             double g[3][3][3]) {
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) {
                double div = 0.0, chi = 0.0, cub = 0.0;
                for (int j = 0; j < 3; ++j) div += d[a][j][j];
                for (int l = 0; l < 3; ++l) {
                    chi += levi(l, a, c) * Q[l][b];
                    cub += Q[c][l] * d[a][b][l];
                }
                g[a][b][c] = m->L1 * d[a][b][c] + (b == c ? m->L2 * div : 0.0) +
                             m->L3 * d[a][c][b] + m->L4 / 2.0 * chi + m->L6 * cub;
            }
}

/* derivative of the density above with respect to the site's own Q_ab
   (through the L4 and L6 prefactors) */
static void distortion_dQ(const orc_model *m, double d[3][3][3], double gq[3][3]) {
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double chi = 0.0, cub = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int k = 0; k < 3; ++k) chi += levi(a, i, k) * d[i][b][k];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) cub += d[i][j][a] * d[i][j][b];
            gq[a][b] = m->L4 / 2.0 * chi + m->L6 / 2.0 * cub;
        }
}

/* list every combination (s_x, s_y, s_z) of allowed differences; an axis
   without an allowed difference takes the single value 0 (no derivative);
   returns the number of combinations (at most 8) */
static int list_combos(const fd_choices *ch, int s[8][3]) {
    int n = 0;
    for (int c0 = 0; c0 < (ch->nopt[0] ? ch->nopt[0] : 1); ++c0)
        for (int c1 = 0; c1 < (ch->nopt[1] ? ch->nopt[1] : 1); ++c1)
            for (int c2 = 0; c2 < (ch->nopt[2] ? ch->nopt[2] : 1); ++c2) {
                s[n][0] = ch->nopt[0] ? ch->opt[0][c0] : 0;
                s[n][1] = ch->nopt[1] ? ch->opt[1][c1] : 0;
                s[n][2] = ch->nopt[2] ? ch->opt[2][c2] : 0;
                ++n;
            }
    return n;
}

/* ---- site energy -------------------------------------------------------- */

void orc_site_energy(const orc_model *m, const orc_geometry *g, const double *q,
                     int64_t i, double parts[3]) {
    int64_t N = g->N;
    parts[0] = parts[1] = parts[2] = 0.0;
    if (!g->sim[i]) return;
    double Q[3][3];
    qmat(q, N, i, Q);
    parts[0] = bulk_energy(m, Q);

    fd_choices ch;
    fd_allowed(m, g, i, &ch);
    int s[8][3];
    int nc = list_combos(&ch, s);
    double sum = 0.0, d[3][3][3];
    for (int t = 0; t < nc; ++t) {
        fd_tensor(q, N, i, &ch, s[t], d);
        sum += distortion_density(m, Q, d);
    }
    parts[1] = sum / nc;

    if (g->rec_index[i] >= 0) parts[2] = anchor_energy(m, &g->recs[g->rec_index[i]], Q);
}

/* Kahan-compensated sum per z-plane, then over planes in order */
double orc_energy(const orc_model *m, const orc_geometry *g, const double *q,
                  double parts[3]) {
    int nz = m->nz;
    double *plane = (double *)calloc((size_t)nz * 3, sizeof(double));
    int64_t nxy = (int64_t)m->nx * m->ny;
#pragma omp parallel for schedule(dynamic, 1)
    for (int z = 0; z < nz; ++z) {
        double s[3] = {0, 0, 0}, c[3] = {0, 0, 0};
        for (int64_t j = 0; j < nxy; ++j) {
            double p[3];
            orc_site_energy(m, g, q, (int64_t)z * nxy + j, p);
            for (int t = 0; t < 3; ++t) {
                double y = p[t] - c[t], u = s[t] + y;
                c[t] = (u - s[t]) - y;
                s[t] = u;
            }
        }
        for (int t = 0; t < 3; ++t) plane[3 * z + t] = s[t];
    }
    double tot = 0.0, ct = 0.0;
    for (int t = 0; t < 3; ++t) {
        double s = 0.0, c = 0.0;
        for (int z = 0; z < nz; ++z) {
            double y = plane[3 * z + t] - c, u = s + y;
            c = (u - s) - y;
            s = u;
        }
        parts[t] = s;
        double y = s - ct, u = tot + y;
        ct = (u - tot) - y;
        tot = u;
    }
    free(plane);
    return tot;
}

/* ---- force: gather dE_i/dq(j) over every owner i of q(j) ---------------- */

static void site_force(const orc_model *m, const orc_geometry *g, const double *q,
                       int64_t j, double out[5]) {
    int64_t N = g->N;
    for (int c = 0; c < 5; ++c) out[c] = 0.0;
    if (!g->sim[j]) return;

    /* owners: j itself and its six face neighbours, without repeats */
    int64_t own[7];
    int nown = 0;
    own[nown++] = j;
    for (int k = 0; k < 3; ++k)
        for (int dir = -1; dir <= 1; dir += 2) {
            int64_t i = neighbour(m, j, k, dir);
            if (i < 0 || !g->sim[i]) continue;
            int dup = 0;
            for (int t = 0; t < nown; ++t) dup |= (own[t] == i);
            if (!dup) own[nown++] = i;
        }

    double G[3][3] = {{0}};
    for (int t = 0; t < nown; ++t) {
        int64_t i = own[t];
        fd_choices ch;
        fd_allowed(m, g, i, &ch);
        int s[8][3];
        int nc = list_combos(&ch, s);
        double inv = 1.0 / nc;
        double d[3][3][3], dd[3][3][3], Qi[3][3];
        qmat(q, N, i, Qi);
        for (int u = 0; u < nc; ++u) {
            /* coefficient of Q(j) in the difference along each axis */
            double coef[3];
            int any = 0;
            for (int k = 0; k < 3; ++k) {
                coef[k] = 0.0;
                if (s[u][k] > 0) {
                    if (ch.fwd[k] == j) coef[k] += 1.0;
                    if (i == j) coef[k] -= 1.0;
                } else if (s[u][k] < 0) {
                    if (i == j) coef[k] += 1.0;
                    if (ch.bwd[k] == j) coef[k] -= 1.0;
                }
                any |= (coef[k] != 0.0);
            }
            if (!any) continue;
            fd_tensor(q, N, i, &ch, s[u], d);
            distortion_ddens(m, Qi, d, dd);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    for (int k = 0; k < 3; ++k) G[a][b] += inv * coef[k] * dd[a][b][k];
            if (i == j) {
                /* the site's own Q multiplies the L4 and L6 terms */
                double gq[3][3];
                distortion_dQ(m, d, gq);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) G[a][b] += inv * gq[a][b];
            }
        }
    }

    double Q[3][3], Gb[3][3];
    qmat(q, N, j, Q);
    bulk_grad(m, Q, Gb);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[a][b] += Gb[a][b];
    if (g->rec_index[j] >= 0) {
        double Ga[3][3];
        anchor_grad(m, &g->recs[g->rec_index[j]], Q, Ga);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a][b] += Ga[a][b];
    }
    double dq[5];
    to_q5(G, dq);
    for (int c = 0; c < 5; ++c) out[c] = -dq[c];
}

void orc_force(const orc_model *m, const orc_geometry *g, const double *q, double *F) {
    int64_t N = g->N;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < N; ++j) {
        double f[5];
        site_force(m, g, q, j, f);
        for (int c = 0; c < 5; ++c) F[c * N + j] = f[c];
    }
}

void orc_force_sites(const orc_model *m, const orc_geometry *g, const double *q,
                     int64_t n, const int64_t *sites, double *F) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < n; ++t) {
        double f[5];
        site_force(m, g, q, sites[t], f);
        for (int c = 0; c < 5; ++c) F[c * n + t] = f[c];
    }
}

/* ---- geometry: objects, boundary sites and their anchoring -------------- */

double orc_uniaxial_s0(double A, double B, double C) {
    /* Eq. (S0def) */
    return (-B + sqrt(B * B - 24.0 * A * C)) / (6.0 * C);
}

/* displacement along axis k, minimum image on periodic axes */
static double disp(const orc_model *m, int k, double d) {
    int n[3] = {m->nx, m->ny, m->nz};
    if (m->periodic[k]) d -= n[k] * floor(d / n[k] + 0.5);
    return d;
}

typedef struct {
    int32_t *listed; /* SITES / ANCHORED: per-site list position, -1 if absent */
} obj_aux;

/* offset of site c from the nearest point of the segment o->c .. o->c2:
   d = site - midpoint (minimum image), a = c2 - c, nearest point at
   midpoint + t a with t = clamp(d.a / a.a, -1/2, 1/2) */
static void capsule_offset(const orc_model *m, const orc_object *o, const int c[3], double r[3]) {
    double d[3], a[3], aa = 0.0, da = 0.0;
    for (int k = 0; k < 3; ++k) {
        double mid = (o->c[k] + o->c2[k]) * 0.5;
        d[k] = disp(m, k, c[k] - mid);
        a[k] = o->c2[k] - o->c[k];
        aa += a[k] * a[k];
        da += d[k] * a[k];
    }
    double t = aa > 0.0 ? da / aa : 0.0;
    if (t < -0.5) t = -0.5;
    if (t > 0.5) t = 0.5;
    for (int k = 0; k < 3; ++k) r[k] = d[k] - t * a[k];
}

static int in_object(const orc_model *m, const orc_object *o, const obj_aux *ax,
                     int64_t i) {
    int c[3];
    coords(m, i, c);
    switch (o->type) {
    case ORC_WALL: return c[o->axis] == o->plane;
    case ORC_SPHERE: {
        double r2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            double d = disp(m, k, c[k] - o->c[k]);
            r2 += d * d;
        }
        return r2 <= o->R * o->R;
    }
    case ORC_SITES: return ax->listed[i] >= 0;
    case ORC_DROPLET: {
        double r2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            double d = disp(m, k, c[k] - o->c[k]);
            r2 += d * d;
        }
        return r2 > o->R * o->R;
    }
    case ORC_SPHEROCYLINDER: {
        double r[3];
        capsule_offset(m, o, c, r);
        return r[0] * r[0] + r[1] * r[1] + r[2] * r[2] <= o->R * o->R;
    }
    default: return 0;
    }
}

/* preferred Q of the uniaxial state 3/2 S0 (n n - I/3), Eq. (Qtensor) */
static void uniaxial_q5(double S, const double n_in[3], double q5[5]) {
    double nn = sqrt(n_in[0] * n_in[0] + n_in[1] * n_in[1] + n_in[2] * n_in[2]);
    double n[3] = {n_in[0] / nn, n_in[1] / nn, n_in[2] / nn};
    q5[0] = 1.5 * S * (n[0] * n[0] - 1.0 / 3.0);
    q5[1] = 1.5 * S * n[0] * n[1];
    q5[2] = 1.5 * S * n[0] * n[2];
    q5[3] = 1.5 * S * (n[1] * n[1] - 1.0 / 3.0);
    q5[4] = 1.5 * S * n[1] * n[2];
}

static void make_record(const orc_model *m, const orc_anchor_spec *sp,
                        const double normal[3], orc_anchor *r) {
    memset(r, 0, sizeof(*r));
    r->W = sp->W;
    double nn = sqrt(normal[0] * normal[0] + normal[1] * normal[1] + normal[2] * normal[2]);
    if (sp->kind == ORC_FG_PLANAR) {
        r->kind = 2;
        for (int k = 0; k < 3; ++k) r->nu[k] = normal[k] / nn;
    } else {
        r->kind = 1;
        uniaxial_q5(m->S0, sp->kind == ORC_ND_ORIENTED ? sp->dir : normal, r->q0);
    }
}

int orc_build_geometry(const orc_model *m, const orc_object *objs, int nobj,
                       orc_geometry *out) {
    int64_t N = (int64_t)m->nx * m->ny * m->nz;
    out->N = N;
    out->sim = (uint8_t *)malloc((size_t)N);
    out->rec_index = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    obj_aux *aux = (obj_aux *)calloc((size_t)(nobj > 0 ? nobj : 1), sizeof(obj_aux));
    if (!out->sim || !out->rec_index || !aux) return -1;

    for (int o = 0; o < nobj; ++o) {
        if (objs[o].type != ORC_SITES && objs[o].type != ORC_ANCHORED) continue;
        aux[o].listed = (int32_t *)malloc((size_t)N * sizeof(int32_t));
        for (int64_t i = 0; i < N; ++i) aux[o].listed[i] = -1;
        for (int64_t t = 0; t < objs[o].n; ++t) {
            const int32_t *p = objs[o].xyz + 3 * t;
            if (p[0] < 0 || p[0] >= m->nx || p[1] < 0 || p[1] >= m->ny || p[2] < 0 ||
                p[2] >= m->nz)
                continue;
            int64_t i = idx3(m, p[0], p[1], p[2]);
            if (aux[o].listed[i] < 0) aux[o].listed[i] = (int32_t)t;
        }
    }

    /* object sites: inside any wall, sphere or listed object */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        int inside = 0;
        for (int o = 0; o < nobj && !inside; ++o) inside = in_object(m, &objs[o], &aux[o], i);
        out->sim[i] = (uint8_t)!inside;
    }

    /* boundary records: the first object (in the order added) whose sites
       touch a simulated site through a face, or whose explicit list names it */
    int32_t *claim = (int32_t *)malloc((size_t)N * sizeof(int32_t));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        claim[i] = -1;
        if (!out->sim[i]) continue;
        for (int o = 0; o < nobj && claim[i] < 0; ++o) {
            if (objs[o].type == ORC_ANCHORED) {
                if (aux[o].listed[i] >= 0) claim[i] = o;
                continue;
            }
            for (int k = 0; k < 3 && claim[i] < 0; ++k)
                for (int dir = -1; dir <= 1; dir += 2) {
                    int64_t nb = neighbour(m, i, k, dir);
                    if (nb >= 0 && in_object(m, &objs[o], &aux[o], nb)) {
                        claim[i] = o;
                        break;
                    }
                }
        }
    }
    int64_t nrec = 0;
    for (int64_t i = 0; i < N; ++i) nrec += (claim[i] >= 0);
    out->nrec = nrec;
    out->recs = (orc_anchor *)malloc((size_t)(nrec > 0 ? nrec : 1) * sizeof(orc_anchor));
    int64_t r = 0;
    for (int64_t i = 0; i < N; ++i) {
        out->rec_index[i] = -1;
        int o = claim[i];
        if (o < 0) continue;
        const orc_object *ob = &objs[o];
        double normal[3] = {0, 0, 0};
        const orc_anchor_spec *sp = &ob->anch;
        int c[3];
        coords(m, i, c);
        if (ob->type == ORC_WALL) {
            normal[ob->axis] = 1.0;
        } else if (ob->type == ORC_SPHERE || ob->type == ORC_DROPLET) {
            for (int k = 0; k < 3; ++k) normal[k] = disp(m, k, c[k] - ob->c[k]);
        } else if (ob->type == ORC_SPHEROCYLINDER) {
            capsule_offset(m, ob, c, normal);
        } else if (ob->type == ORC_SITES) {
            for (int k = 0; k < 3; ++k) normal[k] = sp->dir[k];
        } else {
            sp = &ob->per_site[aux[o].listed[i]];
            for (int k = 0; k < 3; ++k) normal[k] = sp->dir[k];
        }
        make_record(m, sp, normal, &out->recs[r]);
        out->rec_index[i] = (int32_t)r;
        ++r;
    }
    free(claim);
    for (int o = 0; o < nobj; ++o) free(aux[o].listed);
    free(aux);
    return 0;
}

void orc_free_geometry(orc_geometry *g) {
    free(g->sim);
    free(g->rec_index);
    free(g->recs);
    g->sim = NULL;
    g->rec_index = NULL;
    g->recs = NULL;
}

/* ---- FIRE, Algorithm 1 --------------------------------------------------- */

/* velocity mixing ("rescale velocity by alpha") followed by the P test */
void orc_fire_scalars(const orc_fire_params *p, orc_fire_state *st, double P,
                      double normF, double normv, double *a, double *b) {
    *a = 1.0;
    *b = 0.0;
    if (normF > 0.0) {
        *a = 1.0 - st->alpha;
        *b = st->alpha * normv / normF;
    }
    if (P > 0.0) {
        st->npos += 1;
        if (st->npos > p->n_min) {
            st->dt = fmin(st->dt * p->f_inc, p->dt_max);
            st->alpha *= p->f_alpha;
        }
    } else {
        st->npos = 0;
        st->dt *= p->f_dec;
        st->alpha = p->alpha0;
        *a = 0.0;
        *b = 0.0;
    }
}

/* sums over simulated sites: P = F.v, |F|^2, |v|^2, max site |F|^2 */
static void fire_reduce(const orc_geometry *g, const double *v, const double *F,
                        int nz, double *P, double *F2, double *v2, double *r2) {
    int64_t N = g->N, per = N / nz;
    double *acc = (double *)calloc((size_t)nz * 4, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z) {
        double p = 0, f = 0, w = 0, r = 0;
        for (int64_t i = (int64_t)z * per; i < (int64_t)(z + 1) * per; ++i) {
            if (!g->sim[i]) continue;
            double fs = 0;
            for (int c = 0; c < 5; ++c) {
                p += F[c * N + i] * v[c * N + i];
                fs += F[c * N + i] * F[c * N + i];
                w += v[c * N + i] * v[c * N + i];
            }
            f += fs;
            if (fs > r) r = fs;
        }
        acc[4 * z] = p; acc[4 * z + 1] = f; acc[4 * z + 2] = w; acc[4 * z + 3] = r;
    }
    *P = *F2 = *v2 = *r2 = 0.0;
    for (int z = 0; z < nz; ++z) {
        *P += acc[4 * z]; *F2 += acc[4 * z + 1]; *v2 += acc[4 * z + 2];
        if (acc[4 * z + 3] > *r2) *r2 = acc[4 * z + 3];
    }
    free(acc);
}

int orc_fire_run(const orc_model *m, const orc_geometry *g, const orc_fire_params *p,
                 double *q, double *v, double *F, orc_fire_state *st, int64_t max_steps) {
    int64_t N = g->N;
    double P, F2, v2, r2;
    if (!st->initialized) {
        st->dt = p->dt0;
        st->alpha = p->alpha0;
        st->npos = 0;
        st->iter = 0;
        st->status = ORC_RUNNING;
        for (int64_t t = 0; t < 5 * N; ++t) v[t] = 0.0;
        orc_force(m, g, q, F);
        st->initialized = 1;
        fire_reduce(g, v, F, m->nz, &P, &F2, &v2, &r2);
        st->P = P; st->normF = sqrt(F2); st->normv = sqrt(v2); st->rmax = sqrt(r2);
        if (!isfinite(F2)) st->status = ORC_DIVERGED;
        else if (st->rmax < p->force_tol) st->status = ORC_CONVERGED;
    }
    double *Fn = (double *)malloc((size_t)5 * N * sizeof(double));
    for (int64_t step = 0; step < max_steps && st->status == ORC_RUNNING; ++step) {
        double dt = st->dt;
        /* velocity Verlet: drift, new force, kick */
        for (int64_t i = 0; i < N; ++i) {
            if (!g->sim[i]) continue;
            for (int c = 0; c < 5; ++c)
                q[c * N + i] += dt * v[c * N + i] + 0.5 * dt * dt * F[c * N + i];
        }
        orc_force(m, g, q, Fn);
        for (int64_t t = 0; t < 5 * N; ++t) {
            v[t] += 0.5 * dt * (F[t] + Fn[t]);
            F[t] = Fn[t];
        }
        st->iter += 1;
        fire_reduce(g, v, F, m->nz, &P, &F2, &v2, &r2);
        st->P = P; st->normF = sqrt(F2); st->normv = sqrt(v2); st->rmax = sqrt(r2);
        if (!isfinite(P) || !isfinite(F2) || !isfinite(v2)) {
            st->status = ORC_DIVERGED;
            break;
        }
        if (st->rmax < p->force_tol) {
            st->status = ORC_CONVERGED;
            break;
        }
        if (st->iter >= p->max_iter) {
            st->status = ORC_MAXITER;
            break;
        }
        double a, b;
        double nF = st->normF, nv = st->normv;
        orc_fire_scalars(p, st, P, nF, nv, &a, &b);
        /* v <- (1 - alpha) v + alpha |v| F/|F|, or 0 after an uphill step */
        for (int64_t t = 0; t < 5 * N; ++t) v[t] = a * v[t] + b * F[t];
    }
    free(Fn);
    return st->status;
}

/* ---- gradient descent and Nesterov's accelerated gradient ---------------- */

static void descent_norms(const orc_model *m, const orc_geometry *g, const double *F,
                          double *normF, double *rmax) {
    double P, F2, v2, r2;
    fire_reduce(g, F, F, m->nz, &P, &F2, &v2, &r2);   /* |F|^2 and max site |F|^2 */
    *normF = sqrt(F2);
    *rmax = sqrt(r2);
}

int orc_descent_run(const orc_model *m, const orc_geometry *g, int method, double eta,
                    double mu, int64_t max_iter, double force_tol, double *x, double *xprev,
                    double *y, double *F, orc_descent_state *st, int64_t max_steps) {
    int64_t N = g->N;
    if (method != 2) mu = 0.0;
    if (!st->initialized) {
        for (int64_t t = 0; t < 5 * N; ++t) { xprev[t] = x[t]; y[t] = x[t]; }
        orc_force(m, g, y, F);
        st->iter = 0;
        st->status = ORC_RUNNING;
        st->initialized = 1;
        descent_norms(m, g, F, &st->normF, &st->rmax);
        if (!isfinite(st->normF)) st->status = ORC_DIVERGED;
        else if (st->rmax < force_tol) st->status = ORC_CONVERGED;
    }
    for (int64_t step = 0; step < max_steps && st->status == ORC_RUNNING; ++step) {
        for (int64_t i = 0; i < N; ++i) {
            if (!g->sim[i]) continue;
            for (int c = 0; c < 5; ++c) {
                int64_t t = c * N + i;
                double xn = y[t] + eta * F[t];            /* x_{k+1} = y_k + eta F(y_k) */
                xprev[t] = x[t];
                x[t] = xn;
                y[t] = xn + mu * (xn - xprev[t]);        /* y_{k+1} */
            }
        }
        orc_force(m, g, y, F);
        st->iter += 1;
        descent_norms(m, g, F, &st->normF, &st->rmax);
        if (!isfinite(st->normF)) { st->status = ORC_DIVERGED; break; }
        if (st->rmax < force_tol) { st->status = ORC_CONVERGED; break; }
        if (st->iter >= max_iter) { st->status = ORC_MAXITER; break; }
    }
    return st->status;
}

/* ---- readback: largest eigenvalue (cyclic Jacobi, Golub & Van Loan 8.5) -- */

void orc_eig_sym3(const double q5[5], double evals[3], double evecs[9]) {
    double A[3][3], V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    qmat5(q5, A);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        if (off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int r = p + 1; r < 3; ++r) {
                if (A[p][r] == 0.0) continue;
                double tau = (A[r][r] - A[p][p]) / (2.0 * A[p][r]);
                double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < 3; ++k) { /* A <- A J */
                    double akp = A[k][p], akr = A[k][r];
                    A[k][p] = c * akp - s * akr;
                    A[k][r] = s * akp + c * akr;
                }
                for (int k = 0; k < 3; ++k) { /* A <- J^T A */
                    double apk = A[p][k], ark = A[r][k];
                    A[p][k] = c * apk - s * ark;
                    A[r][k] = s * apk + c * ark;
                }
                for (int k = 0; k < 3; ++k) {
                    double vkp = V[k][p], vkr = V[k][r];
                    V[k][p] = c * vkp - s * vkr;
                    V[k][r] = s * vkp + c * vkr;
                }
            }
    }
    int ord[3] = {0, 1, 2};
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (A[ord[b]][ord[b]] > A[ord[a]][ord[a]]) {
                int t = ord[a]; ord[a] = ord[b]; ord[b] = t;
            }
    for (int a = 0; a < 3; ++a) {
        evals[a] = A[ord[a]][ord[a]];
        for (int k = 0; k < 3; ++k) evecs[3 * a + k] = V[k][ord[a]];
    }
}

void orc_order_field(const orc_geometry *g, const double *q, int64_t N, double *S) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        if (!g->sim[i]) { S[i] = 0.0; continue; }
        double q5[5], ev[3], vec[9];
        for (int c = 0; c < 5; ++c) q5[c] = q[c * N + i];
        orc_eig_sym3(q5, ev, vec);
        S[i] = ev[0];
    }
}
