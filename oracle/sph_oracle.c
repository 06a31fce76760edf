/*
 * Plain FP64 CPU oracle of the WCSPH particle-interaction pass.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; the two meet only through plain arrays.
 *
 * The code follows the method of "A comparison between WCSPH and MPS methods
 * for 3D dam-break flows" (Amaro Jr., Cheng, Buruchenko), Section 2.2, in the
 * order the paper states it, with no blocking, fusion or reordering:
 *   Eq. 3   momentum equation with the artificial viscosity term
 *   Eq. 4-5 Monaghan artificial viscosity, c_bar, rho_bar, mu_ij, eta^2
 *   Eq. 6   Wendland C2 kernel (3D normalisation read as 21/(16 pi h^3))
 *   Eq. 7   continuity equation with the delta-SPH diffusive term
 *   Eq. 8   Tait equation of state
 *   Eq. 9-14 Verlet scheme with a first-order step every Ns steps
 *   (or, as a switch, a symplectic predictor-corrector: the paper points to
 *   other time-integration schemes after Eq. 15 but prints none; the reading
 *   is stated at orc_step_symplectic)
 *   Eq. 15  adaptive time step
 *   Eq. 33  Shepard-averaged pressure at a point (Section 3.1)
 * Every reading of a point the paper leaves open is written next to the line
 * that takes it.  All arithmetic is IEEE double; build with
 * -ffp-contract=off so that no multiply-add is fused behind our back.
 *
 * Particle types: 0 = fluid, 1 = fixed wall/floor boundary, 2 = obstacle
 * boundary (also fixed; its particles carry the force probe), 3 = gate
 * boundary (moving at a prescribed constant velocity, Section 3.2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_FLUID 0
#define ORC_WALL 1
#define ORC_OBSTACLE 2
#define ORC_GATE 3

#define ORC_PI 3.14159265358979323846

/* One dam-break case: geometry, physical constants and method switches. */
typedef struct {
    double tank[3];      /* tank length, width, height (x, y, z) [m] */
    double column[3];    /* water column length, width, height [m] */
    int32_t has_obstacle;
    int32_t pad0;
    double obstacle[6];  /* lower corner x0,y0,z0 and size lx,ly,lz [m] */
    double dp;           /* initial particle spacing l0 [m] */
    double h;            /* smoothing length [m] */
    double c0;           /* artificial speed of sound [m/s] */
    double rho0;         /* reference density [kg/m^3] */
    double alpha;        /* artificial viscosity coefficient (Eq. 4) */
    double gamma;        /* Tait polytropic index (Eq. 8), 7 */
    double g;            /* gravity [m/s^2], acting along -z */
    double delta;        /* delta-SPH coefficient (Eq. 7), 0.1 */
    double cfl;          /* Courant number Cr (Eq. 15), 0.2 */
    int32_t ns;          /* first-order step every ns steps (Eqs. 12-14), 40 */
    int32_t layers;      /* boundary particle layers */
    int32_t init_mode;   /* 0 hydrostatic density, 1 uniform rho0 */
    int32_t csound_mode; /* 0 c_i from the EOS, 1 c_i = c0 */
    int32_t cell_div;    /* cells per support radius 2h */
    int32_t integrator;  /* 0 the Verlet scheme of Eqs. 9-14, 1 symplectic (see orc_step) */
    int32_t has_gate;
    int32_t delta_mode;  /* 0: delta term on every fluid particle (over fluid j);
                            1: off for a fluid particle with a boundary neighbour */
    double gate[6];      /* lower corner and size of the gate box [m] */
    double gate_v[3];    /* its constant velocity [m/s] */
} orc_case;

/* ------------------------------------------------------------------------ */
/* Eq. 6 and its derivative                                                   */
/* ------------------------------------------------------------------------ */

/* Wendland C2 kernel W(r) = wD (1 - q/2)^4 (2q + 1), q = r/h, 0 <= q <= 2.
 * The printed 3D constant reads "21/16 pi h^3"; the kernel only integrates to
 * one with wD = 21 / (16 pi h^3), which is the reading taken. */
double orc_kernel_w(double r, double h)
{
    double q = r / h;
    if (q >= 2.0)
        return 0.0;
    double wd = 21.0 / (16.0 * ORC_PI * h * h * h);
    double t = 1.0 - 0.5 * q;
    return wd * t * t * t * t * (2.0 * q + 1.0);
}

/* dW/dr differentiated from Eq. 6 by hand:
 *   dW/dq = wD (1 - q/2)^3 (-5 q),  dW/dr = dW/dq / h.                       */
double orc_kernel_dwdr(double r, double h)
{
    double q = r / h;
    if (q >= 2.0)
        return 0.0;
    double wd = 21.0 / (16.0 * ORC_PI * h * h * h);
    double t = 1.0 - 0.5 * q;
    return wd * t * t * t * (-5.0 * q) / h;
}

/* grad_i W_ij = dW/dr * (r_i - r_j) / |r_i - r_j|.  Written through the
 * factor F(r) = (dW/dr) / r = -5 wD (1 - q/2)^3 / h^2, which stays finite at
 * r = 0, so grad_i W_ij = F(r) (r_i - r_j). */
double orc_kernel_f(double r, double h)
{
    double q = r / h;
    if (q >= 2.0)
        return 0.0;
    double wd = 21.0 / (16.0 * ORC_PI * h * h * h);
    double t = 1.0 - 0.5 * q;
    return -5.0 * wd * t * t * t / (h * h);
}

/* ------------------------------------------------------------------------ */
/* Eq. 8 and the sound speed                                                  */
/* ------------------------------------------------------------------------ */

/* Tait equation of state, Eq. 8. */
double orc_tait(const orc_case *cs, double rho)
{
    double b = cs->rho0 * cs->c0 * cs->c0 / cs->gamma;
    return b * (pow(rho / cs->rho0, cs->gamma) - 1.0);
}

/* c_i: the paper defines c = sqrt(dP/drho) next to Eq. 8 but leaves the c_i
 * of Eq. 5 unstated.  Reading: c_i = sqrt(dP/drho) of Eq. 8 at rho_i, i.e.
 * c0 (rho_i/rho0)^((gamma-1)/2); csound_mode 1 takes c_i = c0 instead. */
double orc_sound(const orc_case *cs, double rho)
{
    if (cs->csound_mode == 1)
        return cs->c0;
    return cs->c0 * pow(rho / cs->rho0, 0.5 * (cs->gamma - 1.0));
}

/* Internal energy per unit mass with de/drho = P / rho^2 and e(rho0) = 0,
 * integrated by hand from Eq. 8 (used only by the diagnostics). */
static double orc_internal_energy(const orc_case *cs, double rho)
{
    double b = cs->rho0 * cs->c0 * cs->c0 / cs->gamma;
    double gm1 = cs->gamma - 1.0;
    return b / cs->rho0 * (pow(rho / cs->rho0, gm1) / gm1 + cs->rho0 / rho - cs->gamma / gm1);
}

/* Eq. 32: nu0 = alpha0 h c0 / (2 (dim + 2)). */
double orc_nu0(double alpha, double h, double c0, int dim)
{
    return alpha * h * c0 / (2.0 * (dim + 2.0));
}

/* ------------------------------------------------------------------------ */
/* Scene: the paper gives the tank, column and box sizes (Sections 3.1, 3.2)  */
/* but not the particle layout.  Reading: fluid on the lattice                */
/* ((i+1/2)dp, (j+1/2)dp, (k+1/2)dp) from the tank corner, the column against */
/* the x = 0 end wall; `layers` boundary layers outside floor and walls, up   */
/* to the tank height, no lid; the obstacle a filled lattice box.  Ids:       */
/* fluid (x fastest, then y, then z), then walls+floor (same loop order over  */
/* the enclosing box), then the obstacle, then the gate (a filled lattice box */
/* like the obstacle; the Case 2 column of Section 3.2 is held by a gate that */
/* is lifted at constant speed).  Every particle has m = rho0 dp^3.          */
/* ------------------------------------------------------------------------ */

static int64_t orc_nint(double x) { return (int64_t)floor(x + 0.5); }

/* counts[0] fluid, counts[1] walls+floor and gate, counts[2] obstacle. */
int orc_scene_counts(const orc_case *cs, int64_t counts[3])
{
    double dp = cs->dp;
    int64_t ncx = orc_nint(cs->column[0] / dp), ncy = orc_nint(cs->column[1] / dp);
    int64_t ncz = orc_nint(cs->column[2] / dp);
    int64_t ntx = orc_nint(cs->tank[0] / dp), nty = orc_nint(cs->tank[1] / dp);
    int64_t ntz = orc_nint(cs->tank[2] / dp);
    int64_t L = cs->layers;
    if (dp <= 0 || ncx < 0 || ncy < 0 || ncz < 0 || ncx > ntx || ncy > nty || ncz > ntz)
        return -1;
    counts[0] = ncx * ncy * ncz;
    counts[1] = (ntx + 2 * L) * (nty + 2 * L) * (ntz + L) - ntx * nty * ntz;
    counts[2] = 0;
    if (cs->has_obstacle)
        counts[2] = orc_nint(cs->obstacle[3] / dp) * orc_nint(cs->obstacle[4] / dp) *
                    orc_nint(cs->obstacle[5] / dp);
    if (cs->has_gate)
        counts[1] += orc_nint(cs->gate[3] / dp) * orc_nint(cs->gate[4] / dp) * orc_nint(cs->gate[5] / dp);
    return 0;
}

/* Fills r (3n), u (3n), rho (n), type (n) in id order.  Initial density
 * (the paper is silent): hydrostatic, inverting Eq. 8 for
 * P = rho0 g (Hc - z) in the fluid, rho0 on the boundary; init_mode 1 gives
 * rho0 everywhere.  Velocities start at zero, the gate's at its velocity. */
int orc_scene_build(const orc_case *cs, double *r, double *u, double *rho, int32_t *type)
{
    int64_t counts[3];
    if (orc_scene_counts(cs, counts))
        return -1;
    double dp = cs->dp;
    int64_t ncx = orc_nint(cs->column[0] / dp), ncy = orc_nint(cs->column[1] / dp);
    int64_t ncz = orc_nint(cs->column[2] / dp);
    int64_t ntx = orc_nint(cs->tank[0] / dp), nty = orc_nint(cs->tank[1] / dp);
    int64_t ntz = orc_nint(cs->tank[2] / dp);
    int64_t L = cs->layers;
    int64_t id = 0;
    for (int64_t k = 0; k < ncz; ++k)
        for (int64_t j = 0; j < ncy; ++j)
            for (int64_t i = 0; i < ncx; ++i) {
                double x = (i + 0.5) * dp, y = (j + 0.5) * dp, z = (k + 0.5) * dp;
                r[3 * id] = x;
                r[3 * id + 1] = y;
                r[3 * id + 2] = z;
                if (cs->init_mode == 0)
                    rho[id] = cs->rho0 * pow(1.0 + cs->gamma * cs->g * (cs->column[2] - z) / (cs->c0 * cs->c0),
                                             1.0 / cs->gamma);
                else
                    rho[id] = cs->rho0;
                type[id] = ORC_FLUID;
                ++id;
            }
    for (int64_t k = -L; k < ntz; ++k)
        for (int64_t j = -L; j < nty + L; ++j)
            for (int64_t i = -L; i < ntx + L; ++i) {
                int inside = i >= 0 && i < ntx && j >= 0 && j < nty && k >= 0;
                if (inside)
                    continue;
                r[3 * id] = (i + 0.5) * dp;
                r[3 * id + 1] = (j + 0.5) * dp;
                r[3 * id + 2] = (k + 0.5) * dp;
                rho[id] = cs->rho0;
                type[id] = ORC_WALL;
                ++id;
            }
    if (cs->has_obstacle) {
        int64_t i0 = orc_nint(cs->obstacle[0] / dp), j0 = orc_nint(cs->obstacle[1] / dp);
        int64_t k0 = orc_nint(cs->obstacle[2] / dp);
        int64_t nox = orc_nint(cs->obstacle[3] / dp), noy = orc_nint(cs->obstacle[4] / dp);
        int64_t noz = orc_nint(cs->obstacle[5] / dp);
        for (int64_t k = k0; k < k0 + noz; ++k)
            for (int64_t j = j0; j < j0 + noy; ++j)
                for (int64_t i = i0; i < i0 + nox; ++i) {
                    r[3 * id] = (i + 0.5) * dp;
                    r[3 * id + 1] = (j + 0.5) * dp;
                    r[3 * id + 2] = (k + 0.5) * dp;
                    rho[id] = cs->rho0;
                    type[id] = ORC_OBSTACLE;
                    ++id;
                }
    }
    for (int64_t p = 0; p < 3 * id; ++p)
        u[p] = 0.0;
    if (cs->has_gate) {
        int64_t i0 = orc_nint(cs->gate[0] / dp), j0 = orc_nint(cs->gate[1] / dp), k0 = orc_nint(cs->gate[2] / dp);
        int64_t ngx = orc_nint(cs->gate[3] / dp), ngy = orc_nint(cs->gate[4] / dp), ngz = orc_nint(cs->gate[5] / dp);
        for (int64_t k = k0; k < k0 + ngz; ++k)
            for (int64_t j = j0; j < j0 + ngy; ++j)
                for (int64_t i = i0; i < i0 + ngx; ++i) {
                    r[3 * id] = (i + 0.5) * dp;
                    r[3 * id + 1] = (j + 0.5) * dp;
                    r[3 * id + 2] = (k + 0.5) * dp;
                    for (int a = 0; a < 3; ++a)
                        u[3 * id + a] = cs->gate_v[a];
                    rho[id] = cs->rho0;
                    type[id] = ORC_GATE;
                    ++id;
                }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Neighbour structure.  The paper only says "all neighbouring particles"     */
/* within the kernel support 2h (Eq. 3, Eq. 6).  Cells of size 2h/cell_div    */
/* over the box [-L dp, Lt + L dp] x [-L dp, Wt + L dp] x [-L dp, Ht + 4h];   */
/* a particle whose cell falls outside the grid is out of the domain and      */
/* takes no further part in the computation.                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    double lo[3];
    double size;
    int64_t n[3];
    int64_t ncells;
} orc_grid;

static void orc_make_grid(const orc_case *cs, orc_grid *gr)
{
    double L = cs->layers * cs->dp;
    double hi[3] = {cs->tank[0] + L, cs->tank[1] + L, cs->tank[2] + 4.0 * cs->h};
    gr->size = 2.0 * cs->h / cs->cell_div;
    for (int a = 0; a < 3; ++a) {
        gr->lo[a] = -L;
        gr->n[a] = (int64_t)ceil((hi[a] - gr->lo[a]) / gr->size);
    }
    gr->ncells = gr->n[0] * gr->n[1] * gr->n[2];
}

/* Grid geometry for the tests: lo[3], size, and dims[3]. */
void orc_grid_info(const orc_case *cs, double lo[3], double *size, int64_t dims[3])
{
    orc_grid gr;
    orc_make_grid(cs, &gr);
    for (int a = 0; a < 3; ++a) {
        lo[a] = gr.lo[a];
        dims[a] = gr.n[a];
    }
    *size = gr.size;
}

/* Integer cell coordinates; returns 0 when the particle is out of the grid. */
static int orc_cell_coords(const orc_grid *gr, const double *x, int64_t c[3])
{
    for (int a = 0; a < 3; ++a) {
        double f = floor((x[a] - gr->lo[a]) / gr->size);
        if (!(f >= 0.0) || f >= (double)gr->n[a])
            return 0;
        c[a] = (int64_t)f;
    }
    return 1;
}

/* Linear cell id (cz ny + cy) nx + cx, or ncells when out of the domain. */
static int64_t orc_cell_id(const orc_grid *gr, const double *x)
{
    int64_t c[3];
    if (!orc_cell_coords(gr, x, c))
        return gr->ncells;
    return (c[2] * gr->n[1] + c[1]) * gr->n[0] + c[0];
}

/* Counting sort by cell, stable in particle id.  Outputs: cell[n],
 * order[n] (ids in ascending (cell, id)), start[ncells + 2] with the particles
 * of cell c at order[start[c] .. start[c+1]); the out-of-domain particles sit
 * in the extra bucket ncells. */
int orc_cells(const orc_case *cs, int64_t n, const double *r, int64_t *cell, int64_t *order, int64_t *start)
{
    orc_grid gr;
    orc_make_grid(cs, &gr);
    int64_t nb = gr.ncells + 1;
    for (int64_t c = 0; c <= nb; ++c)
        start[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        cell[i] = orc_cell_id(&gr, r + 3 * i);
        start[cell[i] + 1] += 1;
    }
    for (int64_t c = 0; c < nb; ++c)
        start[c + 1] += start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * nb);
    if (!fill)
        return -1;
    for (int64_t c = 0; c < nb; ++c)
        fill[c] = start[c];
    for (int64_t i = 0; i < n; ++i)
        order[fill[cell[i]]++] = i;
    free(fill);
    return 0;
}

int64_t orc_num_cells(const orc_case *cs)
{
    orc_grid gr;
    orc_make_grid(cs, &gr);
    return gr.ncells;
}

/* Squared distance |r_j - r_i|^2 evaluated as ((dx dx + dy dy) + dz dz). */
static double orc_dist2(const double *ri, const double *rj)
{
    double dx = rj[0] - ri[0], dy = rj[1] - ri[1], dz = rj[2] - ri[2];
    return dx * dx + dy * dy + dz * dz;
}

/* The cell list of a state. */
typedef struct {
    orc_grid gr;
    int64_t *cell, *order, *start;
} orc_list;

static int orc_list_build(const orc_case *cs, int64_t n, const double *r, orc_list *cl)
{
    orc_make_grid(cs, &cl->gr);
    cl->cell = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    cl->order = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    cl->start = (int64_t *)malloc(sizeof(int64_t) * (cl->gr.ncells + 2));
    if (!cl->cell || !cl->order || !cl->start)
        return -1;
    return orc_cells(cs, n, r, cl->cell, cl->order, cl->start);
}

static void orc_list_free(orc_list *cl)
{
    free(cl->cell);
    free(cl->order);
    free(cl->start);
}

/* Visit the candidates of particle i: every particle of the cells within
 * cell_div cells of i's cell along each axis, in (cell, id) order. */
#define ORC_FOR_CANDIDATES(cl, kdiv, r, i, jvar, BODY)                                    \
    do {                                                                                  \
        int64_t c_[3];                                                                    \
        if (orc_cell_coords(&(cl)->gr, (r) + 3 * (i), c_)) {                              \
            int64_t k_ = (kdiv);                                                          \
            for (int64_t z_ = c_[2] - k_; z_ <= c_[2] + k_; ++z_) {                       \
                if (z_ < 0 || z_ >= (cl)->gr.n[2])                                        \
                    continue;                                                             \
                for (int64_t y_ = c_[1] - k_; y_ <= c_[1] + k_; ++y_) {                   \
                    if (y_ < 0 || y_ >= (cl)->gr.n[1])                                    \
                        continue;                                                         \
                    for (int64_t x_ = c_[0] - k_; x_ <= c_[0] + k_; ++x_) {               \
                        if (x_ < 0 || x_ >= (cl)->gr.n[0])                                \
                            continue;                                                     \
                        int64_t cc_ = (z_ * (cl)->gr.n[1] + y_) * (cl)->gr.n[0] + x_;     \
                        for (int64_t s_ = (cl)->start[cc_]; s_ < (cl)->start[cc_ + 1]; ++s_) { \
                            int64_t jvar = (cl)->order[s_];                               \
                            BODY                                                          \
                        }                                                                 \
                    }                                                                     \
                }                                                                         \
            }                                                                             \
        }                                                                                 \
    } while (0)

/* Neighbour counts |P_i| = #{ j != i in the domain : |r_j - r_i| < 2h }.
 * mode 0 walks the cell list, mode 1 compares every pair (brute force);
 * out-of-domain particles get -1. */
int orc_neighbour_counts(const orc_case *cs, int64_t n, const double *r, int mode, int32_t *count)
{
    double sup2 = (2.0 * cs->h) * (2.0 * cs->h);
    orc_list cl;
    if (orc_list_build(cs, n, r, &cl))
        return -1;
    int64_t ncells = cl.gr.ncells;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        if (cl.cell[i] == ncells) {
            count[i] = -1;
            continue;
        }
        int32_t c = 0;
        if (mode == 1) {
            for (int64_t j = 0; j < n; ++j)
                if (j != i && cl.cell[j] != ncells && orc_dist2(r + 3 * i, r + 3 * j) < sup2)
                    ++c;
        } else {
            ORC_FOR_CANDIDATES(&cl, cs->cell_div, r, i, j, {
                if (j != i && orc_dist2(r + 3 * i, r + 3 * j) < sup2)
                    ++c;
            });
        }
        count[i] = c;
    }
    orc_list_free(&cl);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The pair pass: Eqs. 3-8 for one particle.                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    double drho;   /* D rho_i / Dt, Eq. 7 */
    double acc[3]; /* D u_i / Dt, Eq. 3, including f_i for fluid */
    double mumax;  /* max_j mu_ij of Eq. 15, at least 0 */
    int32_t nneigh;
    double delta_sum; /* the delta term of Eq. 7, added to drho by orc_particle */
    int32_t has_boundary; /* some neighbour j is a boundary particle */
} orc_deriv;

/* Contribution of neighbour j to particle i, Eqs. 3-7.
 *
 * Readings:
 *  - Eq. 7 as printed, with u_ij = u_j - u_i, makes compression lower the
 *    density; Eq. 1 drops the minus sign of -rho div u the same way.  The
 *    standard sign is taken: the first sum uses (u_i - u_j) . grad_i W_ij.
 *  - The delta term (r_ij . grad_i W_ij) / |r_ij|^2 with r_ij = r_j - r_i is
 *    kept as printed; for coincident distinct particles (|r_ij| = 0) its limit
 *    -F(0) is used.  It acts between fluid particles only (the paper does not
 *    say how it treats boundary particles).  With delta_mode 1 a fluid
 *    particle that has any boundary neighbour takes no delta term at all
 *    (orc_particle drops its sum): the kernel support of such a particle is
 *    cut by the wall, and a sum over fluid neighbours alone then does not
 *    vanish for a hydrostatic density field.
 *  - Boundary particles (dynamic boundary conditions, Section 2.2) sum over
 *    fluid neighbours only; with their zero velocity the density sum is the
 *    same as over all neighbours, and their acceleration (used only by the
 *    force probe, Section 3.2) then contains fluid forces alone. */
static void orc_pair(const orc_case *cs, double m, int32_t ti, const double *ri, const double *ui, double rhoi,
                     double Pi, double ci, int32_t tj, const double *rj, const double *uj, double rhoj,
                     orc_deriv *d)
{
    double h = cs->h;
    double rij[3] = {rj[0] - ri[0], rj[1] - ri[1], rj[2] - ri[2]};
    double uij[3] = {uj[0] - ui[0], uj[1] - ui[1], uj[2] - ui[2]};
    double r2 = rij[0] * rij[0] + rij[1] * rij[1] + rij[2] * rij[2];
    double r = sqrt(r2);
    double F = orc_kernel_f(r, h);
    /* grad_i W_ij = F (r_i - r_j) = -F r_ij */
    double gw[3] = {-F * rij[0], -F * rij[1], -F * rij[2]};

    double Pj = orc_tait(cs, rhoj);
    double cj = orc_sound(cs, rhoj);

    /* Eq. 7, first sum (standard sign). */
    d->drho += m * ((-uij[0]) * gw[0] + (-uij[1]) * gw[1] + (-uij[2]) * gw[2]);
    /* Eq. 7, delta-SPH diffusive term between fluid particles. */
    if (ti == ORC_FLUID && tj == ORC_FLUID && cs->delta != 0.0) {
        double rg = rij[0] * gw[0] + rij[1] * gw[1] + rij[2] * gw[2];
        double ratio = r2 > 0.0 ? rg / r2 : -F;
        double term = 2.0 * cs->delta * h * cs->c0 * (rhoj - rhoi) * ratio * m / rhoj;
        if (cs->delta_mode == 1)
            d->delta_sum += term; /* kept apart until the neighbour set is known */
        else
            d->drho += term;
    }
    /* Eqs. 4-5. */
    double eta2 = 0.01 * h * h;
    double udotr = uij[0] * rij[0] + uij[1] * rij[1] + uij[2] * rij[2];
    double mu = h * udotr / (r2 + eta2);
    double Pi_ij = 0.0;
    if (udotr < 0.0) {
        double cbar = 0.5 * (ci + cj);
        double rhobar = 0.5 * (rhoi + rhoj);
        Pi_ij = -cs->alpha * cbar * mu / rhobar;
    }
    /* Eq. 3. */
    double coef = m * ((Pi + Pj) / (rhoi * rhoj) + Pi_ij);
    d->acc[0] -= coef * gw[0];
    d->acc[1] -= coef * gw[1];
    d->acc[2] -= coef * gw[2];
    /* Eq. 15, inner max over j (signed, the running max starts at 0). */
    if (mu > d->mumax)
        d->mumax = mu;
}

/* Derivatives of particle i over its cell-list neighbours (Eqs. 3-8).
 * Fluid particles add the body force f_i = (0, 0, -g). */
static void orc_particle(const orc_case *cs, const orc_list *cl, int64_t i, const double *r, const double *u,
                         const double *rho, const int32_t *type, orc_deriv *d)
{
    double sup2 = (2.0 * cs->h) * (2.0 * cs->h);
    double m = cs->rho0 * cs->dp * cs->dp * cs->dp;
    int64_t ncells = cl->gr.ncells;
    memset(d, 0, sizeof(*d));
    if (cl->cell[i] == ncells) {
        d->nneigh = -1;
        return;
    }
    double Pi = orc_tait(cs, rho[i]);
    double ci = orc_sound(cs, rho[i]);
    int32_t ti = type[i];
    ORC_FOR_CANDIDATES(cl, cs->cell_div, r, i, j, {
        if (j != i && orc_dist2(r + 3 * i, r + 3 * j) < sup2) {
            d->nneigh += 1;
            if (type[j] != ORC_FLUID)
                d->has_boundary = 1;
            if (ti == ORC_FLUID || type[j] == ORC_FLUID)
                orc_pair(cs, m, ti, r + 3 * i, u + 3 * i, rho[i], Pi, ci, type[j], r + 3 * j, u + 3 * j,
                         rho[j], d);
        }
    });
    if (cs->delta_mode == 1 && !d->has_boundary)
        d->drho += d->delta_sum;
    if (ti == ORC_FLUID)
        d->acc[2] -= cs->g;
}

/* One pair pass over all particles.  Outputs in id order: drho[n], acc[3n],
 * mumax[n], nneigh[n] (-1 and zeros for out-of-domain particles). */
int orc_derivatives(const orc_case *cs, int64_t n, const double *r, const double *u, const double *rho,
                    const int32_t *type, double *drho, double *acc, double *mumax, int32_t *nneigh)
{
    orc_list cl;
    if (orc_list_build(cs, n, r, &cl))
        return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        orc_deriv d;
        orc_particle(cs, &cl, i, r, u, rho, type, &d);
        drho[i] = d.drho;
        acc[3 * i] = d.acc[0];
        acc[3 * i + 1] = d.acc[1];
        acc[3 * i + 2] = d.acc[2];
        mumax[i] = d.mumax;
        nneigh[i] = d.nneigh;
    }
    orc_list_free(&cl);
    return 0;
}

/* The same for a chosen subset of particles (sampled checks at full size). */
int orc_derivatives_subset(const orc_case *cs, int64_t n, const double *r, const double *u, const double *rho,
                           const int32_t *type, int64_t nsel, const int64_t *sel, double *drho, double *acc,
                           double *mumax, int32_t *nneigh)
{
    orc_list cl;
    if (orc_list_build(cs, n, r, &cl))
        return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < nsel; ++s) {
        orc_deriv d;
        orc_particle(cs, &cl, sel[s], r, u, rho, type, &d);
        drho[s] = d.drho;
        acc[3 * s] = d.acc[0];
        acc[3 * s + 1] = d.acc[1];
        acc[3 * s + 2] = d.acc[2];
        mumax[s] = d.mumax;
        nneigh[s] = d.nneigh;
    }
    orc_list_free(&cl);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 15.  Readings: i runs over the fluid particles in the domain (boundary */
/* particles do not move); |f_i| is the magnitude of the full acceleration    */
/* including gravity; the inner max is the signed mu_ij with the running max  */
/* started at 0.  With no fluid particle the step falls back to Cr h / c0.    */
/* ------------------------------------------------------------------------ */
double orc_dt(const orc_case *cs, int64_t n, const int32_t *type, const int32_t *nneigh, const double *acc,
              const double *mumax)
{
    double h = cs->h;
    double best_f = INFINITY, best_v = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        if (type[i] != ORC_FLUID || nneigh[i] < 0)
            continue;
        double f = sqrt(acc[3 * i] * acc[3 * i] + acc[3 * i + 1] * acc[3 * i + 1] + acc[3 * i + 2] * acc[3 * i + 2]);
        if (f > 0.0) {
            double t = sqrt(h / f);
            if (t < best_f)
                best_f = t;
        }
        double v = h / (cs->c0 + mumax[i]);
        if (v < best_v)
            best_v = v;
    }
    double m = best_f < best_v ? best_f : best_v;
    if (!(m < INFINITY))
        m = h / cs->c0;
    return cs->cfl * m;
}

/* ------------------------------------------------------------------------ */
/* One time step: neighbour structure, Eqs. 3-8, Eq. 15 (or a fixed dt), then */
/* Eqs. 9-14.  Readings: the first-order step runs when step mod ns == 0,     */
/* step 0 included (there is no t - dt level yet); the Verlet step uses the   */
/* current dt; boundary particles update density only and keep u = 0 (gate   */
/* particles move at their prescribed velocity);                              */
/* out-of-domain particles are frozen.                                         */
/* State in id order: r, u, rho (level t) and uprev, rhoprev (level t - dt). */
/* ------------------------------------------------------------------------ */
static int orc_step_symplectic(const orc_case *cs, int64_t n, double *r, double *u, double *rho, double *uprev,
                               double *rhoprev, const int32_t *type, double dt_fixed, double *dt_used);

int orc_step(const orc_case *cs, int64_t n, double *r, double *u, double *rho, double *uprev, double *rhoprev,
             const int32_t *type, int64_t step, double dt_fixed, double *dt_used)
{
    if (cs->integrator == 1)
        return orc_step_symplectic(cs, n, r, u, rho, uprev, rhoprev, type, dt_fixed, dt_used);
    double *drho = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *acc = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double *mumax = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    int32_t *nn = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    if (!drho || !acc || !mumax || !nn)
        return -1;
    if (orc_derivatives(cs, n, r, u, rho, type, drho, acc, mumax, nn))
        return -1;
    double dt = dt_fixed > 0.0 ? dt_fixed : orc_dt(cs, n, type, nn, acc, mumax);
    int euler = (step % cs->ns) == 0;
    for (int64_t i = 0; i < n; ++i) {
        if (nn[i] < 0)
            continue;
        double rho_new = euler ? rho[i] + dt * drho[i] : rhoprev[i] + 2.0 * dt * drho[i];
        rhoprev[i] = rho[i];
        rho[i] = rho_new;
        if (type[i] == ORC_GATE) { /* prescribed motion at constant velocity */
            for (int a = 0; a < 3; ++a) {
                r[3 * i + a] = r[3 * i + a] + dt * cs->gate_v[a];
                uprev[3 * i + a] = cs->gate_v[a];
                u[3 * i + a] = cs->gate_v[a];
            }
            continue;
        }
        if (type[i] != ORC_FLUID)
            continue;
        for (int a = 0; a < 3; ++a) {
            double ua = u[3 * i + a], aa = acc[3 * i + a];
            double u_new = euler ? ua + dt * aa : uprev[3 * i + a] + 2.0 * dt * aa;
            r[3 * i + a] = r[3 * i + a] + dt * ua + 0.5 * dt * dt * aa;
            uprev[3 * i + a] = ua;
            u[3 * i + a] = u_new;
        }
    }
    free(drho);
    free(acc);
    free(mumax);
    free(nn);
    if (dt_used)
        *dt_used = dt;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Symplectic position-Verlet predictor-corrector (the reading taken for the  */
/* integrator the paper leaves to the literature it cites after Eq. 15), two  */
/* evaluations of Eqs. 3-8 per step:                                           */
/*   dt from Eq. 15 on the derivatives at level n (or the fixed dt);           */
/*   predictor, half a step:  rho' = rho + dt/2 Drho,  u' = u + dt/2 Du,       */
/*                            r'   = r + dt/2 u;                               */
/*   derivatives at the predicted state (neighbour structure rebuilt);        */
/*   corrector, a full kick from level n with the mid-step acceleration and   */
/*   the second half drift:  u'' = u + dt Du',  r'' = r' + dt/2 u'',           */
/*               rho'' = rho (2 - e)/(2 + e),  e = -(Drho'/rho') dt,           */
/*   the density update being the exact solution of Drho/Dt = rho k for a     */
/*   constant rate k = Drho'/rho' taken to its (1,1) Pade form.  u' enters    */
/*   only the mid-step derivatives (viscosity and continuity terms).           */
/* Boundary particles integrate density only and keep u = 0 (gate particles   */
/* move at their prescribed velocity, half a step in each stage).  A particle out */
/* of the grid at level n stays frozen; one that leaves the grid in the        */
/* predictor keeps its predicted state.  uprev, rhoprev receive the level-n    */
/* state.                                                                       */
/* ------------------------------------------------------------------------ */
static int orc_step_symplectic(const orc_case *cs, int64_t n, double *r, double *u, double *rho, double *uprev,
                               double *rhoprev, const int32_t *type, double dt_fixed, double *dt_used)
{
    const int64_t m = n > 0 ? n : 1;
    double *drho = (double *)malloc(sizeof(double) * m);
    double *acc = (double *)malloc(sizeof(double) * 3 * m);
    double *mumax = (double *)malloc(sizeof(double) * m);
    int32_t *nn = (int32_t *)malloc(sizeof(int32_t) * m);
    int rc = -1;
    if (!drho || !acc || !mumax || !nn)
        goto out;
    if (orc_derivatives(cs, n, r, u, rho, type, drho, acc, mumax, nn))
        goto out;
    double dt = dt_fixed > 0.0 ? dt_fixed : orc_dt(cs, n, type, nn, acc, mumax);
    double hdt = 0.5 * dt;
    /* predictor */
    for (int64_t i = 0; i < n; ++i) {
        if (nn[i] < 0)
            continue;
        rhoprev[i] = rho[i];
        rho[i] = rho[i] + hdt * drho[i];
        if (type[i] == ORC_GATE) {
            for (int a = 0; a < 3; ++a) {
                r[3 * i + a] = r[3 * i + a] + hdt * cs->gate_v[a];
                uprev[3 * i + a] = cs->gate_v[a];
                u[3 * i + a] = cs->gate_v[a];
            }
            continue;
        }
        if (type[i] != ORC_FLUID)
            continue;
        for (int a = 0; a < 3; ++a) {
            uprev[3 * i + a] = u[3 * i + a];
            r[3 * i + a] = r[3 * i + a] + hdt * u[3 * i + a];
            u[3 * i + a] = u[3 * i + a] + hdt * acc[3 * i + a];
        }
    }
    /* derivatives at the predicted state; corrector */
    if (orc_derivatives(cs, n, r, u, rho, type, drho, acc, mumax, nn))
        goto out;
    for (int64_t i = 0; i < n; ++i) {
        if (nn[i] < 0)
            continue;
        double e = -(drho[i] / rho[i]) * dt;
        rho[i] = rhoprev[i] * (2.0 - e) / (2.0 + e);
        if (type[i] == ORC_GATE) {
            for (int a = 0; a < 3; ++a)
                r[3 * i + a] = r[3 * i + a] + hdt * cs->gate_v[a];
            continue;
        }
        if (type[i] != ORC_FLUID)
            continue;
        for (int a = 0; a < 3; ++a) {
            u[3 * i + a] = uprev[3 * i + a] + dt * acc[3 * i + a];
            r[3 * i + a] = r[3 * i + a] + hdt * u[3 * i + a];
        }
    }
    if (dt_used)
        *dt_used = dt;
    rc = 0;
out:
    free(drho);
    free(acc);
    free(mumax);
    free(nn);
    return rc;
}

/* nsteps steps from step index step0; dts[nsteps] receives each dt. */
int orc_run(const orc_case *cs, int64_t n, double *r, double *u, double *rho, double *uprev, double *rhoprev,
            const int32_t *type, int64_t step0, int64_t nsteps, double dt_fixed, double *dts)
{
    for (int64_t s = 0; s < nsteps; ++s)
        if (orc_step(cs, n, r, u, rho, uprev, rhoprev, type, step0 + s, dt_fixed, dts ? dts + s : NULL))
            return -1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Probes (Sections 3.1 and 3.2), brute force over all particles.             */
/* ------------------------------------------------------------------------ */

static int orc_in_domain(const orc_case *cs, const double *x)
{
    orc_grid gr;
    int64_t c[3];
    orc_make_grid(cs, &gr);
    return orc_cell_coords(&gr, x, c);
}

/* Eq. 33: P_a = sum_b P_b W_ab / sum_b W_ab over fluid particles b (the
 * printed sum index j is read as b).  With no fluid particle within 2h the
 * probe returns 0. */
int orc_probe_pressure(const orc_case *cs, int64_t n, const double *r, const double *rho, const int32_t *type,
                       int64_t npts, const double *pts, double *out)
{
    for (int64_t a = 0; a < npts; ++a) {
        double num = 0.0, den = 0.0;
        for (int64_t b = 0; b < n; ++b) {
            if (type[b] != ORC_FLUID || !orc_in_domain(cs, r + 3 * b))
                continue;
            double d = sqrt(orc_dist2(pts + 3 * a, r + 3 * b));
            double w = orc_kernel_w(d, cs->h);
            num += orc_tait(cs, rho[b]) * w;
            den += w;
        }
        out[a] = den > 0.0 ? num / den : 0.0;
    }
    return 0;
}

/* Wave height at (x, y).  The paper reports wave heights but does not state
 * how they are measured.  Reading: scan z = k dp/4, k = 0, 1, ... up to the
 * grid top; the height is the largest z at which the kernel-summed fluid
 * density sum_b m W(|p - r_b|) reaches rho0 / 2 (0 if it never does). */
int orc_probe_wave_height(const orc_case *cs, int64_t n, const double *r, const int32_t *type, int64_t npts,
                          const double *pts_xy, double *out)
{
    double m = cs->rho0 * cs->dp * cs->dp * cs->dp;
    double ztop = cs->tank[2] + 4.0 * cs->h;
    double dz = 0.25 * cs->dp;
    for (int64_t a = 0; a < npts; ++a) {
        double best = 0.0;
        for (int64_t k = 0; k * dz <= ztop; ++k) {
            double p[3] = {pts_xy[2 * a], pts_xy[2 * a + 1], k * dz};
            double s = 0.0;
            for (int64_t b = 0; b < n; ++b) {
                if (type[b] != ORC_FLUID || !orc_in_domain(cs, r + 3 * b))
                    continue;
                s += m * orc_kernel_w(sqrt(orc_dist2(p, r + 3 * b)), cs->h);
            }
            if (s >= 0.5 * cs->rho0)
                best = p[2];
        }
        out[a] = best;
    }
    return 0;
}

/* Force on the obstacle (Section 3.2): the sum over its particles of m a_b,
 * with a_b the Eq. 3 acceleration from fluid neighbours only and no gravity,
 * evaluated on the current state. */
int orc_probe_force(const orc_case *cs, int64_t n, const double *r, const double *u, const double *rho,
                    const int32_t *type, double out[3])
{
    orc_list cl;
    if (orc_list_build(cs, n, r, &cl))
        return -1;
    double m = cs->rho0 * cs->dp * cs->dp * cs->dp;
    out[0] = out[1] = out[2] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (type[i] != ORC_OBSTACLE)
            continue;
        orc_deriv d;
        orc_particle(cs, &cl, i, r, u, rho, type, &d);
        if (d.nneigh < 0)
            continue;
        out[0] += m * d.acc[0];
        out[1] += m * d.acc[1];
        out[2] += m * d.acc[2];
    }
    orc_list_free(&cl);
    return 0;
}

/* Diagnostics over in-domain particles: [0] total mass, [1] fluid volume
 * sum m/rho, [2..4] fluid momentum, [5] kinetic energy, [6] potential energy
 * m g z, [7] internal energy m e(rho) of the fluid, [8] out-of-domain count,
 * [9] fluid particles in the domain. */
int orc_diagnostics(const orc_case *cs, int64_t n, const double *r, const double *u, const double *rho,
                    const int32_t *type, double out[10])
{
    double m = cs->rho0 * cs->dp * cs->dp * cs->dp;
    for (int k = 0; k < 10; ++k)
        out[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (!orc_in_domain(cs, r + 3 * i)) {
            out[8] += 1.0;
            continue;
        }
        out[0] += m;
        if (type[i] != ORC_FLUID)
            continue;
        const double *ui = u + 3 * i;
        out[1] += m / rho[i];
        out[2] += m * ui[0];
        out[3] += m * ui[1];
        out[4] += m * ui[2];
        out[5] += 0.5 * m * (ui[0] * ui[0] + ui[1] * ui[1] + ui[2] * ui[2]);
        out[6] += m * cs->g * r[3 * i + 2];
        out[7] += m * orc_internal_energy(cs, rho[i]);
        out[9] += 1.0;
    }
    return 0;
}

/* Thread control for the CPU baseline (1 thread = fully serial). */
int orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}
