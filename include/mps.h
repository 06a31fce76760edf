/*
 * mps.h - C ABI of the GB300 (sm_103a) MPS time step: the semi-implicit method
 * that "A comparison between WCSPH and MPS methods for 3D dam-break flows"
 * (Amaro Jr., Cheng, Buruchenko) compares WCSPH against, Section 2.3.
 *
 * One step (mps_step), all on the device:
 *  1. explicit prediction (Eqs. 21-22): u* = u + dt (nu <lap u> + g) with the
 *     Laplacian of Eq. 19 and the weight of Eq. 16, r* = r + dt u*;
 *  2. at r*: particle number density n* (Eq. 17), free-surface detection by
 *     both criteria of Eqs. 28-30, the pressure Poisson equation (Eq. 23)
 *     assembled as a sparse symmetric positive definite system and solved by
 *     the conjugate gradient method to a relative residual of cg_tol;
 *  3. the first-order pressure gradient of Eq. 24 and the correction of
 *     Eqs. 25-26.
 * Readings where the paper is silent: Eq. 16's second case "|r_ij| > 0" is read
 * as |r_ij| > r_e; the wall is `layers` layers of fixed particles, the one
 * touching the fluid with a solved pressure, the outer ones dummy particles
 * that count in n* but carry no pressure and take no part in the Laplacian of
 * Eq. 23 or the gradient of Eq. 24; a free-surface neighbour enters with its
 * Dirichlet pressure 0; the solve starts from P = 0; negative pressures from
 * the solve are set to zero before the gradient; a moment matrix of Eq. 24
 * that cannot be inverted gives a zero gradient; particles leaving the grid
 * are frozen.
 *
 * Conventions are those of sph.h: SPH_OK or a negative SPH_E* code (the codes
 * of sph.h), SI units, gravity along -z, the column against the x = 0 wall,
 * caller-owned host arrays borrowed for the call, a caller-owned device
 * workspace borrowed for the handle's lifetime (the library never calls
 * cudaMalloc), work enqueued on the stream given at creation.  Particle
 * arrays are in id order: fluid (x fastest over the column lattice), then the
 * wall and dummy particles.  A handle is not thread-safe.
 */
#ifndef MPS_H
#define MPS_H

#include <stddef.h>
#include <stdint.h>

#include "sph.h"

#ifdef __cplusplus
extern "C" {
#endif

#define MPS_FLUID 0
#define MPS_WALL 1  /* wall layer touching the fluid: pressure solved */
#define MPS_DUMMY 2 /* outer wall layers: number density only */

typedef struct mps_s mps_t;

/* Parameters; fill with mps_params_default() (the values of Section 3). */
typedef struct mps_params {
    uint32_t size;      /* sizeof(mps_params) */
    int32_t layers;     /* wall layers, 1 wall + (layers - 1) dummy (3) */
    double re_factor;   /* effective radius r_e = re_factor l0, Eq. 16 (2.1) */
    double nu;          /* kinematic viscosity of Eq. 21 [m^2/s] (1e-6) */
    double rho;         /* density [kg/m^3] (1000) */
    double g;           /* gravity [m/s^2] (9.81) */
    double kappa_c;     /* artificial compressibility of Eq. 23 [m s^2/kg] (1e-8) */
    double kappa_r;     /* relaxation coefficient of Eq. 23 (0.01) */
    double beta1;       /* free-surface threshold n* < beta1 n0, Eq. 28 (0.98) */
    double varrho1;     /* free-surface threshold sigma > varrho1 l0, Eq. 29 (0.2) */
    double cg_tol;      /* relative residual |r| <= cg_tol |b| of the CG solve (1e-6) */
    int32_t cg_max;     /* iteration cap of the CG solve (20000) */
    int32_t row_width;  /* stored off-diagonal entries per row of Eq. 23, at most (64) */
    int32_t reserved[6];
} mps_params;

void mps_params_default(mps_params *p);

/* Device bytes needed for this tank.  Errors: SPH_EINVAL. */
int mps_workspace_size(const double tank[3], const double column[3], double l0, const mps_params *p,
                       size_t *bytes);

/* Create a dam-break tank: water column `column` at rest against x = 0 in
 * tank `tank`, lattice spacing l0, fixed time step dt (Eq. 27).  Workspace and
 * stream as for sph_create.  Errors: SPH_EINVAL, SPH_ENOMEM, SPH_ECUDA. */
int mps_create(mps_t **out, const double tank[3], const double column[3], double l0, double dt,
               const mps_params *p, void *dev_workspace, size_t workspace_bytes, uintptr_t cuda_stream);

void mps_destroy(mps_t *s);

/* Advance nsteps steps.  Each step waits for its CG solve (the convergence
 * test reads one flag back every 16 iterations).  Errors: SPH_EINVAL,
 * SPH_ECUDA, SPH_ESTATE (a row of Eq. 23 with more than row_width entries),
 * SPH_EUNSTABLE (the solve did not reach cg_tol within cg_max iterations, or a
 * non-finite state). */
int mps_step(mps_t *s, int32_t nsteps);

/* The pressure system of the current state without advancing it (test seam):
 * n* (Eq. 17), free-surface flags (Eqs. 28-30) and the CG solution of Eq. 23
 * (0 for particles that are not unknowns; not clamped), in id order; any
 * pointer may be NULL.  Synchronous. */
int mps_pressure(mps_t *s, double *P, double *nd, int32_t *surf, int64_t *iterations, double *residual);

/* Copy the state out (id order, any pointer may be NULL): r (3n), u (3n),
 * the pressure of the last step after the clamp (n), type (n), the step
 * counter.  Synchronous. */
int mps_get_state(mps_t *s, double *r, double *u, double *P, int32_t *type, int64_t *step);

/* Load positions and velocities (id order; wall and dummy velocities are held
 * at zero).  Synchronous. */
int mps_set_state(mps_t *s, const double *r, const double *u);

/* CG iterations and final relative residual of the last solve. */
int mps_last_solve(mps_t *s, int64_t *iterations, double *residual);

/* Phase timing: with profiling on, every step records CUDA events around its
 * phases; mps_phase_times fills ms[4] with the summed milliseconds of
 * [0] neighbour lists and prediction (Eqs. 21-22), [1] number density, free
 * surface and assembly (Eqs. 17, 28-30, 23), [2] the CG solve, [3] gradient and
 * correction (Eqs. 24-26), then clears them.  Profiling synchronises each
 * step. */
int mps_set_profiling(mps_t *s, int32_t on);
int mps_phase_times(mps_t *s, double ms[4]);

/* Size of the last pressure system of Eq. 23: out[0] rows (every particle,
 * the non-unknowns as identity rows), out[1] stored off-diagonal entries.
 * Synchronous. */
int mps_system_size(mps_t *s, int64_t out[2]);

/* Particle counts: fluid, wall, dummy, total. */
int mps_counts(const mps_t *s, int64_t out[4]);

/* Description of the last failure on this handle (never NULL). */
const char *mps_last_error(const mps_t *s);

#ifdef __cplusplus
}
#endif
#endif /* MPS_H */
