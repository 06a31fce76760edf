/*
 * Plain FP64 CPU oracle of one MPS time step (the method the paper compares
 * WCSPH against).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code with the CUDA library.
 *
 * It follows Section 2.3 of "A comparison between WCSPH and MPS methods for 3D
 * dam-break flows" (Amaro Jr., Cheng, Buruchenko) in the paper's order:
 *   Eq. 16  weight function (the second case printed "|r_ij| > 0" is read as
 *           |r_ij| > r_e)
 *   Eq. 17  particle number density
 *   Eq. 18  gradient operator, Eq. 19 Laplacian operator, Eq. 20 lambda0
 *   Eq. 21-22 explicit prediction of velocity (viscosity and gravity) and
 *           position
 *   Eq. 23  pressure Poisson equation with kappa_c and kappa_r, solved by the
 *           conjugate gradient method to a relative residual of 1e-6
 *   Eq. 24  first-order pressure gradient with the minimum neighbourhood
 *           pressure
 *   Eq. 25-26 velocity and position correction
 *   Eq. 28-30 free-surface detection (particle number density and centroid
 *           deviation, both criteria)
 * Parameters of Section 3: r_e = 2.1 l0, nu = 1e-6 m^2/s, kappa_c = 1e-8
 * m s^2/kg, kappa_r = 0.01, beta1 = 0.98, varrho1 = 0.2, a fixed time step
 * (Eq. 27), three layers of wall particles (the one touching the fluid is the
 * wall layer with a pressure, the two outer ones dummy particles without).
 * Every reading of a point the paper leaves open is written next to the line
 * that takes it.  All arithmetic is IEEE double (build with -ffp-contract=off).
 *
 * Particle types: 0 = fluid, 1 = wall (pressure solved), 2 = dummy (no
 * pressure).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MPS_FLUID 0
#define MPS_WALL 1
#define MPS_DUMMY 2

typedef struct {
    double tank[3];   /* tank length, width, height [m] */
    double column[3]; /* water column against the x = 0 wall [m] */
    double l0;        /* particle spacing [m] */
    double re;        /* effective radius r_e = k_MPS l0 [m] */
    double nu;        /* kinematic viscosity [m^2/s] */
    double rho;       /* density [kg/m^3] */
    double g;         /* gravity along -z [m/s^2] */
    double kappa_c;   /* artificial compressibility of Eq. 23 [m s^2/kg] */
    double kappa_r;   /* relaxation coefficient of Eq. 23 */
    double beta1;     /* free-surface threshold on n_i (Eq. 28) */
    double varrho1;   /* free-surface threshold on sigma_i / l0 (Eq. 29) */
    double dt;        /* fixed time step (Eq. 27) [s] */
    double cg_tol;    /* relative residual of the CG solve, 1e-6 */
    int32_t layers;   /* wall layers: 1 wall + (layers - 1) dummy, 3 */
    int32_t cg_max;   /* iteration cap of the CG solve */
} mps_case;

/* Eq. 16 with the second case read as |r| > r_e.  Coincident particles
 * (r = 0) have no finite weight; they are not neighbours of each other. */
double mps_weight(double r, double re)
{
    if (r <= 0.0 || r > re)
        return 0.0;
    return re / r - 1.0;
}

/* n0 and lambda0 (Eq. 20) of the fully filled initial lattice: sums over the
 * lattice points j != 0 of spacing l0 within r_e of the origin. */
void mps_lattice_constants(const mps_case *cs, double *n0, double *lambda0)
{
    int k = (int)ceil(cs->re / cs->l0);
    double sw = 0.0, sr2w = 0.0;
    for (int a = -k; a <= k; ++a)
        for (int b = -k; b <= k; ++b)
            for (int c = -k; c <= k; ++c) {
                if (a == 0 && b == 0 && c == 0)
                    continue;
                double r2 = (a * a + b * b + c * c) * cs->l0 * cs->l0;
                double w = mps_weight(sqrt(r2), cs->re);
                sw += w;
                sr2w += r2 * w;
            }
    *n0 = sw;
    *lambda0 = sr2w / sw;
}

/* ------------------------------------------------------------------------ */
/* Scene (the paper gives the geometry, Section 3, not the particle layout).  */
/* Reading: fluid on the lattice ((i+1/2) l0, (j+1/2) l0, (k+1/2) l0) from the */
/* inner tank corner, the column against x = 0; `layers` layers of wall       */
/* particles outside floor and walls up to the tank height, no lid; a wall     */
/* particle's layer is its largest distance, in lattice steps, from the fluid  */
/* side over the axes; layer 0 is the wall layer, the others dummy particles. */
/* Ids: fluid (x fastest), then the wall and dummy particles.                  */
/* ------------------------------------------------------------------------ */
static int64_t mps_nint(double x) { return (int64_t)floor(x + 0.5); }

int mps_scene_counts(const mps_case *cs, int64_t counts[3])
{
    int64_t ncx = mps_nint(cs->column[0] / cs->l0), ncy = mps_nint(cs->column[1] / cs->l0);
    int64_t ncz = mps_nint(cs->column[2] / cs->l0);
    int64_t ntx = mps_nint(cs->tank[0] / cs->l0), nty = mps_nint(cs->tank[1] / cs->l0);
    int64_t ntz = mps_nint(cs->tank[2] / cs->l0);
    int64_t L = cs->layers;
    if (cs->l0 <= 0 || ncx > ntx || ncy > nty || ncz > ntz || L < 1)
        return -1;
    counts[0] = ncx * ncy * ncz;
    counts[1] = counts[2] = 0;
    for (int64_t k = -L; k < ntz; ++k)
        for (int64_t j = -L; j < nty + L; ++j)
            for (int64_t i = -L; i < ntx + L; ++i) {
                int64_t dx = i < 0 ? -1 - i : (i >= ntx ? i - ntx : -1);
                int64_t dy = j < 0 ? -1 - j : (j >= nty ? j - nty : -1);
                int64_t dz = k < 0 ? -1 - k : -1;
                int64_t layer = dx > dy ? dx : dy;
                layer = layer > dz ? layer : dz;
                if (layer < 0)
                    continue;
                counts[layer == 0 ? 1 : 2] += 1;
            }
    return 0;
}

int mps_scene_build(const mps_case *cs, double *r, int32_t *type)
{
    int64_t counts[3];
    if (mps_scene_counts(cs, counts))
        return -1;
    double l0 = cs->l0;
    int64_t ncx = mps_nint(cs->column[0] / l0), ncy = mps_nint(cs->column[1] / l0), ncz = mps_nint(cs->column[2] / l0);
    int64_t ntx = mps_nint(cs->tank[0] / l0), nty = mps_nint(cs->tank[1] / l0), ntz = mps_nint(cs->tank[2] / l0);
    int64_t L = cs->layers, id = 0;
    for (int64_t k = 0; k < ncz; ++k)
        for (int64_t j = 0; j < ncy; ++j)
            for (int64_t i = 0; i < ncx; ++i) {
                r[3 * id] = (i + 0.5) * l0;
                r[3 * id + 1] = (j + 0.5) * l0;
                r[3 * id + 2] = (k + 0.5) * l0;
                type[id++] = MPS_FLUID;
            }
    for (int64_t k = -L; k < ntz; ++k)
        for (int64_t j = -L; j < nty + L; ++j)
            for (int64_t i = -L; i < ntx + L; ++i) {
                int64_t dx = i < 0 ? -1 - i : (i >= ntx ? i - ntx : -1);
                int64_t dy = j < 0 ? -1 - j : (j >= nty ? j - nty : -1);
                int64_t dz = k < 0 ? -1 - k : -1;
                int64_t layer = dx > dy ? dx : dy;
                layer = layer > dz ? layer : dz;
                if (layer < 0)
                    continue;
                r[3 * id] = (i + 0.5) * l0;
                r[3 * id + 1] = (j + 0.5) * l0;
                r[3 * id + 2] = (k + 0.5) * l0;
                type[id++] = layer == 0 ? MPS_WALL : MPS_DUMMY;
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Neighbours within r_e: cells of size r_e over the box                      */
/* [-L l0, Lt + L l0] x [-L l0, Wt + L l0] x [-L l0, Ht + 4 r_e]; a particle   */
/* outside the box is out of the domain (frozen, no neighbour of anyone).     */
/* ------------------------------------------------------------------------ */
typedef struct {
    double lo[3], size;
    int64_t n[3], ncells;
    int64_t *cell, *order, *start;
} mps_list;

static int mps_cell_coords(const mps_list *g, const double *x, int64_t c[3])
{
    for (int a = 0; a < 3; ++a) {
        double f = floor((x[a] - g->lo[a]) / g->size);
        if (!(f >= 0.0) || f >= (double)g->n[a])
            return 0;
        c[a] = (int64_t)f;
    }
    return 1;
}

static int mps_list_build(const mps_case *cs, int64_t n, const double *r, mps_list *g)
{
    double L = cs->layers * cs->l0;
    double hi[3] = {cs->tank[0] + L, cs->tank[1] + L, cs->tank[2] + 4.0 * cs->re};
    g->size = cs->re;
    for (int a = 0; a < 3; ++a) {
        g->lo[a] = -L;
        g->n[a] = (int64_t)ceil((hi[a] - g->lo[a]) / g->size);
    }
    g->ncells = g->n[0] * g->n[1] * g->n[2];
    g->cell = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    g->order = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    g->start = (int64_t *)calloc(g->ncells + 2, sizeof(int64_t));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (g->ncells + 1));
    if (!g->cell || !g->order || !g->start || !fill)
        return -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        g->cell[i] = mps_cell_coords(g, r + 3 * i, c) ? (c[2] * g->n[1] + c[1]) * g->n[0] + c[0] : g->ncells;
        g->start[g->cell[i] + 1] += 1;
    }
    for (int64_t c = 0; c <= g->ncells; ++c)
        g->start[c + 1] += g->start[c];
    for (int64_t c = 0; c <= g->ncells; ++c)
        fill[c] = g->start[c];
    for (int64_t i = 0; i < n; ++i)
        g->order[fill[g->cell[i]]++] = i;
    free(fill);
    return 0;
}

static void mps_list_free(mps_list *g)
{
    free(g->cell);
    free(g->order);
    free(g->start);
}

/* Neighbours j != i of particle i with 0 < |r_ij| <= r_e, in (cell, id)
 * order.  Returns their count; idx receives at most cap of them. */
static int64_t mps_neighbours(const mps_list *g, const mps_case *cs, const double *r, int64_t i, int64_t *idx,
                              int64_t cap)
{
    int64_t c[3], m = 0;
    if (g->cell[i] == g->ncells)
        return 0;
    mps_cell_coords(g, r + 3 * i, c);
    for (int64_t z = c[2] - 1; z <= c[2] + 1; ++z)
        for (int64_t y = c[1] - 1; y <= c[1] + 1; ++y)
            for (int64_t x = c[0] - 1; x <= c[0] + 1; ++x) {
                if (x < 0 || y < 0 || z < 0 || x >= g->n[0] || y >= g->n[1] || z >= g->n[2])
                    continue;
                int64_t cc = (z * g->n[1] + y) * g->n[0] + x;
                for (int64_t s = g->start[cc]; s < g->start[cc + 1]; ++s) {
                    int64_t j = g->order[s];
                    if (j == i)
                        continue;
                    double dx = r[3 * j] - r[3 * i], dy = r[3 * j + 1] - r[3 * i + 1], dz = r[3 * j + 2] - r[3 * i + 2];
                    double d = sqrt(dx * dx + dy * dy + dz * dz);
                    if (d > 0.0 && d <= cs->re) {
                        if (m < cap)
                            idx[m] = j;
                        ++m;
                    }
                }
            }
    return m;
}

#define MPS_NCAP 256

static double mps_dist(const double *r, int64_t i, int64_t j)
{
    double dx = r[3 * j] - r[3 * i], dy = r[3 * j + 1] - r[3 * i + 1], dz = r[3 * j + 2] - r[3 * i + 2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* Eq. 17 for every particle (out-of-domain particles get 0). */
int mps_pnd(const mps_case *cs, int64_t n, const double *r, double *nd)
{
    mps_list g;
    if (mps_list_build(cs, n, r, &g))
        return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t idx[MPS_NCAP];
        int64_t m = mps_neighbours(&g, cs, r, i, idx, MPS_NCAP);
        double s = 0.0;
        for (int64_t k = 0; k < m && k < MPS_NCAP; ++k)
            s += mps_weight(mps_dist(r, i, idx[k]), cs->re);
        nd[i] = s;
    }
    mps_list_free(&g);
    return 0;
}

/* Eq. 18 (gradient) and Eq. 19 (Laplacian) of a scalar field phi at every
 * particle, over all its neighbours. */
int mps_operators(const mps_case *cs, int64_t n, const double *r, const double *phi, double *grad, double *lap)
{
    double n0, lambda0;
    mps_lattice_constants(cs, &n0, &lambda0);
    mps_list g;
    if (mps_list_build(cs, n, r, &g))
        return -1;
    const double dim = 3.0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t idx[MPS_NCAP];
        int64_t m = mps_neighbours(&g, cs, r, i, idx, MPS_NCAP);
        double gx = 0.0, gy = 0.0, gz = 0.0, l = 0.0;
        for (int64_t k = 0; k < m && k < MPS_NCAP; ++k) {
            int64_t j = idx[k];
            double d = mps_dist(r, i, j), w = mps_weight(d, cs->re);
            double f = (phi[j] - phi[i]) / (d * d) * w;
            gx += f * (r[3 * j] - r[3 * i]);
            gy += f * (r[3 * j + 1] - r[3 * i + 1]);
            gz += f * (r[3 * j + 2] - r[3 * i + 2]);
            l += (phi[j] - phi[i]) * w;
        }
        grad[3 * i] = dim / n0 * gx;
        grad[3 * i + 1] = dim / n0 * gy;
        grad[3 * i + 2] = dim / n0 * gz;
        lap[i] = 2.0 * dim / (lambda0 * n0) * l;
    }
    mps_list_free(&g);
    return 0;
}

/* Eq. 28-30: free-surface flags of the fluid and wall particles (dummy and
 * out-of-domain particles: 0).  sigma receives sigma_i. */
static void mps_surface(const mps_case *cs, const mps_list *g, int64_t n, const double *r, const int32_t *type,
                        const double *nd, double n0, int32_t *surf, double *sigma)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t idx[MPS_NCAP];
        int64_t m = mps_neighbours(g, cs, r, i, idx, MPS_NCAP);
        double sx = 0.0, sy = 0.0, sz = 0.0, sw = 0.0;
        for (int64_t k = 0; k < m && k < MPS_NCAP; ++k) {
            int64_t j = idx[k];
            double w = mps_weight(mps_dist(r, i, j), cs->re);
            sx += (r[3 * j] - r[3 * i]) * w;
            sy += (r[3 * j + 1] - r[3 * i + 1]) * w;
            sz += (r[3 * j + 2] - r[3 * i + 2]) * w;
            sw += w;
        }
        double s = sw > 0.0 ? sqrt(sx * sx + sy * sy + sz * sz) / sw : 0.0;
        sigma[i] = s;
        surf[i] = (type[i] != MPS_DUMMY && g->cell[i] != g->ncells && nd[i] < cs->beta1 * n0 &&
                   s > cs->varrho1 * cs->l0)
                      ? 1
                      : 0;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 23.  Unknowns: the in-domain fluid and wall particles that are not on  */
/* the free surface.  Readings: a free-surface neighbour enters with its       */
/* Dirichlet pressure 0; dummy particles carry no pressure and are left out of */
/* the Laplacian sums (neither the diagonal nor an off-diagonal entry).  With  */
/* c = 2 dim / (lambda0 n0), row i of the system is                           */
/*   c sum_j (P_j - P_i) w_ij - (rho/dt^2) kappa_c P_i                         */
/*       = -kappa_r (rho/dt^2) (n*_i - n0) / n0,                               */
/* which times -1 is symmetric positive definite (w_ij = w_ji, kappa_c > 0).   */
/* The CG solve starts from P = 0 and stops when |r_k| <= tol |b|.            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t nrow;
    int64_t *row_of;   /* particle -> row or -1 */
    int64_t *part_of;  /* row -> particle */
    int64_t *rowptr, *col;
    double *val, *rhs;
} mps_system;

static int mps_assemble(const mps_case *cs, const mps_list *g, int64_t n, const double *r, const int32_t *type,
                        const double *nd, const int32_t *surf, double n0, double lambda0, mps_system *S)
{
    const double c = 2.0 * 3.0 / (lambda0 * n0), kc = cs->rho * cs->kappa_c / (cs->dt * cs->dt);
    S->row_of = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    S->part_of = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    if (!S->row_of || !S->part_of)
        return -1;
    S->nrow = 0;
    for (int64_t i = 0; i < n; ++i) {
        int unknown = type[i] != MPS_DUMMY && g->cell[i] != g->ncells && !surf[i];
        S->row_of[i] = unknown ? S->nrow : -1;
        if (unknown)
            S->part_of[S->nrow++] = i;
    }
    S->rowptr = (int64_t *)calloc(S->nrow + 1, sizeof(int64_t));
    S->rhs = (double *)malloc(sizeof(double) * (S->nrow > 0 ? S->nrow : 1));
    if (!S->rowptr || !S->rhs)
        return -1;
    for (int64_t q = 0; q < S->nrow; ++q) {
        int64_t idx[MPS_NCAP];
        int64_t i = S->part_of[q], m = mps_neighbours(g, cs, r, i, idx, MPS_NCAP), cnt = 1;
        for (int64_t k = 0; k < m && k < MPS_NCAP; ++k)
            if (S->row_of[idx[k]] >= 0)
                ++cnt;
        S->rowptr[q + 1] = S->rowptr[q] + cnt;
    }
    int64_t nnz = S->rowptr[S->nrow];
    S->col = (int64_t *)malloc(sizeof(int64_t) * (nnz > 0 ? nnz : 1));
    S->val = (double *)malloc(sizeof(double) * (nnz > 0 ? nnz : 1));
    if (!S->col || !S->val)
        return -1;
    for (int64_t q = 0; q < S->nrow; ++q) {
        int64_t idx[MPS_NCAP];
        int64_t i = S->part_of[q], m = mps_neighbours(g, cs, r, i, idx, MPS_NCAP), p = S->rowptr[q] + 1;
        double diag = kc;
        for (int64_t k = 0; k < m && k < MPS_NCAP; ++k) {
            int64_t j = idx[k];
            if (type[j] == MPS_DUMMY)
                continue;
            double w = mps_weight(mps_dist(r, i, j), cs->re);
            diag += c * w;
            if (S->row_of[j] >= 0) {
                S->col[p] = S->row_of[j];
                S->val[p] = -c * w;
                ++p;
            }
        }
        S->col[S->rowptr[q]] = q;
        S->val[S->rowptr[q]] = diag;
        S->rhs[q] = cs->kappa_r * cs->rho / (cs->dt * cs->dt) * (nd[i] - n0) / n0;
    }
    return 0;
}

static void mps_system_free(mps_system *S)
{
    free(S->row_of);
    free(S->part_of);
    free(S->rowptr);
    free(S->col);
    free(S->val);
    free(S->rhs);
}

static void mps_spmv(const mps_system *S, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < S->nrow; ++q) {
        double s = 0.0;
        for (int64_t p = S->rowptr[q]; p < S->rowptr[q + 1]; ++p)
            s += S->val[p] * x[S->col[p]];
        y[q] = s;
    }
}

static double mps_dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t q = 0; q < n; ++q)
        s += a[q] * b[q];
    return s;
}

/* Conjugate gradient method (Hestenes-Stiefel) on the SPD system. */
static int64_t mps_cg(const mps_system *S, double tol, int64_t maxit, double *x, double *res)
{
    int64_t n = S->nrow;
    double *rr = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *p = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *q = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int64_t k = 0; k < n; ++k) {
        x[k] = 0.0;
        rr[k] = S->rhs[k];
        p[k] = rr[k];
    }
    double bnorm = sqrt(mps_dot(n, S->rhs, S->rhs));
    double rho = mps_dot(n, rr, rr);
    int64_t it = 0;
    while (it < maxit && sqrt(rho) > tol * bnorm) {
        mps_spmv(S, p, q);
        double alpha = rho / mps_dot(n, p, q);
        for (int64_t k = 0; k < n; ++k) {
            x[k] += alpha * p[k];
            rr[k] -= alpha * q[k];
        }
        double rho_new = mps_dot(n, rr, rr);
        double beta = rho_new / rho;
        for (int64_t k = 0; k < n; ++k)
            p[k] = rr[k] + beta * p[k];
        rho = rho_new;
        ++it;
    }
    *res = bnorm > 0.0 ? sqrt(rho) / bnorm : 0.0;
    free(rr);
    free(p);
    free(q);
    return it;
}

/* ------------------------------------------------------------------------ */
/* One MPS step (Section 2.3 order).  State in id order: r (3n), u (3n);      */
/* outputs P (n), nd (n, n* of Eq. 23), surf (n), and cg[2] = iterations and  */
/* final relative residual.                                                    */
/*  1. Eq. 21-22 at time t: u* = u + dt (nu <lap u> + f), r* = r + dt u*,      */
/*     fluid only; walls and dummies keep u = 0 (no-slip), their zero velocity */
/*     entering the Laplacian.                                                 */
/*  2. at r*: n* (Eq. 17), free surface (Eq. 28-30), Eq. 23 solved by CG.      */
/*  3. Eq. 24 at r* for fluid particles: P_hat_i the minimum of P over i and   */
/*     its neighbours with a pressure (fluid and wall, free-surface ones at   */
/*     0); dummy particles left out of both sums; a moment matrix that cannot */
/*     be inverted (|det| <= 1e-12 of its scale) gives a zero gradient.       */
/*  4. Eq. 25-26: u = u* - dt/rho <grad P>, r = r* + dt (u - u*).              */
/* Out-of-domain fluid particles stay frozen.                                  */
/* ------------------------------------------------------------------------ */
int mps_step(const mps_case *cs, int64_t n, double *r, double *u, const int32_t *type, double *P, double *nd,
             int32_t *surf, double *cg)
{
    double n0, lambda0;
    mps_lattice_constants(cs, &n0, &lambda0);
    const double dim = 3.0, dt = cs->dt;
    double *ustar = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double *sigma = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    if (!ustar || !sigma)
        return -1;
    /* 1. prediction */
    mps_list g;
    if (mps_list_build(cs, n, r, &g))
        return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a)
            ustar[3 * i + a] = u[3 * i + a];
        if (type[i] != MPS_FLUID || g.cell[i] == g.ncells)
            continue;
        int64_t idx[MPS_NCAP];
        int64_t m = mps_neighbours(&g, cs, r, i, idx, MPS_NCAP);
        double l[3] = {0.0, 0.0, 0.0};
        for (int64_t k = 0; k < m && k < MPS_NCAP; ++k) {
            int64_t j = idx[k];
            double w = mps_weight(mps_dist(r, i, j), cs->re);
            for (int a = 0; a < 3; ++a)
                l[a] += (u[3 * j + a] - u[3 * i + a]) * w;
        }
        double f[3] = {0.0, 0.0, -cs->g};
        for (int a = 0; a < 3; ++a)
            ustar[3 * i + a] = u[3 * i + a] + dt * (cs->nu * 2.0 * dim / (lambda0 * n0) * l[a] + f[a]);
    }
    int64_t *frozen = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i)
        frozen[i] = g.cell[i] == g.ncells;
    for (int64_t i = 0; i < n; ++i)
        if (type[i] == MPS_FLUID && !frozen[i])
            for (int a = 0; a < 3; ++a)
                r[3 * i + a] = r[3 * i + a] + dt * ustar[3 * i + a];
    mps_list_free(&g);
    /* 2. pressure */
    if (mps_list_build(cs, n, r, &g))
        return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t idx[MPS_NCAP];
        int64_t m = mps_neighbours(&g, cs, r, i, idx, MPS_NCAP);
        double s = 0.0;
        for (int64_t k = 0; k < m && k < MPS_NCAP; ++k)
            s += mps_weight(mps_dist(r, i, idx[k]), cs->re);
        nd[i] = s;
    }
    mps_surface(cs, &g, n, r, type, nd, n0, surf, sigma);
    mps_system S;
    if (mps_assemble(cs, &g, n, r, type, nd, surf, n0, lambda0, &S))
        return -1;
    double *x = (double *)malloc(sizeof(double) * (S.nrow > 0 ? S.nrow : 1));
    double res = 0.0;
    int64_t it = mps_cg(&S, cs->cg_tol, cs->cg_max, x, &res);
    /* Reading (the paper is silent): a negative pressure from the solve is set
     * to zero.  The layer under the free-surface particles has a truncated
     * neighbourhood, n* < n0, whose source pulls its pressure below zero; left
     * in, it makes a still column unstable. */
    for (int64_t i = 0; i < n; ++i)
        P[i] = S.row_of[i] >= 0 ? (x[S.row_of[i]] > 0.0 ? x[S.row_of[i]] : 0.0) : 0.0;
    cg[0] = (double)it;
    cg[1] = res;
    /* 3-4. gradient and correction */
    double *unew = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a)
            unew[3 * i + a] = ustar[3 * i + a];
        if (type[i] != MPS_FLUID || g.cell[i] == g.ncells)
            continue;
        int64_t idx[MPS_NCAP];
        int64_t m = mps_neighbours(&g, cs, r, i, idx, MPS_NCAP);
        double phat = P[i];
        for (int64_t k = 0; k < m && k < MPS_NCAP; ++k)
            if (type[idx[k]] != MPS_DUMMY && P[idx[k]] < phat)
                phat = P[idx[k]];
        double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, v[3] = {0, 0, 0};
        for (int64_t k = 0; k < m && k < MPS_NCAP; ++k) {
            int64_t j = idx[k];
            if (type[j] == MPS_DUMMY)
                continue;
            double d = mps_dist(r, i, j), w = mps_weight(d, cs->re);
            double e[3] = {(r[3 * j] - r[3 * i]) / d, (r[3 * j + 1] - r[3 * i + 1]) / d,
                           (r[3 * j + 2] - r[3 * i + 2]) / d};
            for (int a = 0; a < 3; ++a) {
                for (int b = 0; b < 3; ++b)
                    M[a][b] += e[a] * e[b] * w;
                v[a] += (P[j] - phat) / (d * d) * (r[3 * j + a] - r[3 * i + a]) * w;
            }
        }
        /* M^{-1} v through the adjugate */
        double c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1], c01 = M[0][2] * M[2][1] - M[0][1] * M[2][2];
        double c02 = M[0][1] * M[1][2] - M[0][2] * M[1][1], c10 = M[1][2] * M[2][0] - M[1][0] * M[2][2];
        double c11 = M[0][0] * M[2][2] - M[0][2] * M[2][0], c12 = M[0][2] * M[1][0] - M[0][0] * M[1][2];
        double c20 = M[1][0] * M[2][1] - M[1][1] * M[2][0], c21 = M[0][1] * M[2][0] - M[0][0] * M[2][1];
        double c22 = M[0][0] * M[1][1] - M[0][1] * M[1][0];
        double det = M[0][0] * c00 + M[0][1] * c10 + M[0][2] * c20;
        double scale = (M[0][0] + M[1][1] + M[2][2]) / 3.0;
        double gp[3] = {0.0, 0.0, 0.0};
        if (fabs(det) > 1e-12 * scale * scale * scale) {
            gp[0] = (c00 * v[0] + c01 * v[1] + c02 * v[2]) / det;
            gp[1] = (c10 * v[0] + c11 * v[1] + c12 * v[2]) / det;
            gp[2] = (c20 * v[0] + c21 * v[1] + c22 * v[2]) / det;
        }
        for (int a = 0; a < 3; ++a)
            unew[3 * i + a] = ustar[3 * i + a] - dt / cs->rho * gp[a];
    }
    for (int64_t i = 0; i < n; ++i) {
        if (type[i] != MPS_FLUID || frozen[i])
            continue;
        for (int a = 0; a < 3; ++a) {
            r[3 * i + a] = r[3 * i + a] + dt * (unew[3 * i + a] - ustar[3 * i + a]);
            u[3 * i + a] = unew[3 * i + a];
        }
    }
    mps_system_free(&S);
    mps_list_free(&g);
    free(ustar);
    free(sigma);
    free(frozen);
    free(x);
    free(unew);
    return 0;
}

/* The PPE of a state, for the tests: n* of every particle, its free-surface
 * flags and the CG solution (P of the unknowns, 0 elsewhere, not clamped);
 * cg[2] as in mps_step; sigma receives the centroid deviations of Eq. 30. */
int mps_pressure(const mps_case *cs, int64_t n, const double *r, const int32_t *type, double *P, double *nd,
                 int32_t *surf, double *sigma, double *cg)
{
    double n0, lambda0;
    mps_lattice_constants(cs, &n0, &lambda0);
    mps_list g;
    if (mps_list_build(cs, n, r, &g))
        return -1;
    if (mps_pnd(cs, n, r, nd))
        return -1;
    mps_surface(cs, &g, n, r, type, nd, n0, surf, sigma);
    mps_system S;
    if (mps_assemble(cs, &g, n, r, type, nd, surf, n0, lambda0, &S))
        return -1;
    double *x = (double *)malloc(sizeof(double) * (S.nrow > 0 ? S.nrow : 1));
    double res = 0.0;
    int64_t it = mps_cg(&S, cs->cg_tol, cs->cg_max, x, &res);
    for (int64_t i = 0; i < n; ++i)
        P[i] = S.row_of[i] >= 0 ? x[S.row_of[i]] : 0.0;
    cg[0] = (double)it;
    cg[1] = res;
    free(x);
    mps_system_free(&S);
    mps_list_free(&g);
    return 0;
}
