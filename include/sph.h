/*
 * sph.h - C ABI of the GB300 (sm_103a) WCSPH particle-interaction pass.
 *
 * The library advances weakly-compressible SPH dam-break simulations as in
 * "A comparison between WCSPH and MPS methods for 3D dam-break flows"
 * (Amaro Jr., Cheng, Buruchenko), Section 2.2: the cell-linked neighbour
 * structure over the kernel support 2h (Eq. 6), the continuity equation with
 * the delta-SPH term (Eq. 7) and the Tait equation of state (Eq. 8), the
 * momentum equation with Monaghan artificial viscosity (Eqs. 3-5), the
 * Verlet scheme with a first-order step every Ns steps (Eqs. 9-14) or a
 * symplectic predictor-corrector, and the adaptive time step (Eq. 15);
 * optionally a gate of boundary particles moving at a prescribed velocity
 * (Section 3.2).  Probes give the Shepard-averaged pressure of
 * Eq. 33 (Section 3.1), wave heights (Section 3.1) and the force on the
 * obstacle (Section 3.2).
 *
 * Conventions for every entry point:
 *  - Return value: SPH_OK (0) or a negative SPH_E* code.  sph_last_error()
 *    gives a one-line description of the last failure on a handle.
 *  - Units are SI.  Gravity acts along -z.  Coordinates have their origin at
 *    the inner corner of the tank floor; the water column sits against the
 *    x = 0 end wall.
 *  - Host arrays are caller-owned and only borrowed for the duration of the
 *    call.  The device workspace passed to sph_create/sph_batch_create is
 *    borrowed for the lifetime of the handle (the library never calls
 *    cudaMalloc for it; the caller frees it after sph_destroy).
 *  - Particle arrays at the boundary are in particle-id order: for every
 *    instance, fluid particles first (x fastest, then y, then z over the
 *    column lattice), then wall/floor particles, then obstacle particles,
 *    then gate particles; instances follow one another.  Vectors are
 *    interleaved xyz (n x 3).
 *  - Work is enqueued on the CUDA stream given at creation; sph_step returns
 *    without waiting.  Calls that fill host arrays synchronise that stream.
 *    A handle is not thread-safe.
 */
#ifndef SPH_H
#define SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SPH_OK 0
#define SPH_EINVAL (-1)    /* an argument is out of range or inconsistent */
#define SPH_ENOMEM (-2)    /* workspace smaller than sph_workspace_size() */
#define SPH_ECUDA (-3)     /* a CUDA runtime call failed */
#define SPH_EUNSTABLE (-4) /* non-finite state, or dt fell below dt_min */
#define SPH_ETIMEOUT (-5)  /* a bounded device-side wait ran out */
#define SPH_ESTATE (-6)    /* device state inconsistent (cell counters out of step with the particle keys) */

/* ---- enumerations -------------------------------------------------------- */
#define SPH_FP64 0  /* every step of the pass in IEEE double */
#define SPH_MIXED 1 /* FP32 pair arithmetic on cell-relative offsets, FP64
                       position update, dt reduction and diagnostics */

#define SPH_INIT_HYDROSTATIC 0 /* fluid density from Eq. 8 inverted for rho0 g (Hc - z) */
#define SPH_INIT_UNIFORM 1     /* rho0 everywhere */

/* Time integration.  SPH_VERLET: the scheme of Eqs. 9-14 (one pair pass per
 * step).  SPH_SYMPLECTIC: a symplectic position-Verlet predictor-corrector,
 * a reading (the paper cites alternative schemes after Eq. 15 without printing
 * one): predictor rho' = rho + dt/2 Drho, u' = u + dt/2 Du, r' = r + dt/2 u;
 * a second pair pass at the predicted state; corrector u'' = u + dt Du',
 * r'' = r' + dt/2 u'', rho'' = rho (2 - e)/(2 + e) with e = -dt Drho'/rho'.
 * dt (Eq. 15) comes from the first pass.  Two pair passes per step. */
#define SPH_VERLET 0
#define SPH_SYMPLECTIC 1

#define SPH_CSOUND_EOS 0      /* c_i = c0 (rho_i/rho0)^((gamma-1)/2), i.e. sqrt(dP/drho) of Eq. 8 */
#define SPH_CSOUND_CONSTANT 1 /* c_i = c0 */

/* Where the delta term of Eq. 7 acts (the paper gives delta = 0.1 but does not
 * say how the term treats boundary particles).  SPH_DELTA_ALL_FLUID: on every
 * fluid particle, summed over its fluid neighbours.  SPH_DELTA_FULL_SUPPORT:
 * the same, except that a fluid particle with any boundary particle within 2h
 * takes no delta term at all; near a wall the fluid-only sum does not vanish
 * for a hydrostatic density field and drains the deep density, which this
 * mode avoids.  The mixed form always uses compensated sums in this mode. */
#define SPH_DELTA_ALL_FLUID 0
#define SPH_DELTA_FULL_SUPPORT 1

#define SPH_PROBE_PRESSURE 0    /* Eq. 33 at points (x,y,z): n outputs [Pa] */
#define SPH_PROBE_WAVE_HEIGHT 1 /* free-surface height above (x,y): n outputs [m] */
#define SPH_PROBE_FORCE 2       /* force on the obstacle: 3 outputs [N] */

#define SPH_FLUID 0
#define SPH_WALL 1
#define SPH_OBSTACLE 2
#define SPH_GATE 3

typedef struct sph_s sph_t;

/* Method switches and tuning knobs.  Fill with sph_params_default() and
 * override fields; `size` must be sizeof(sph_params). */
typedef struct sph_params {
    uint32_t size;
    int32_t precision;       /* SPH_FP64 or SPH_MIXED */
    double gamma;            /* Tait index, Eq. 8 (7) */
    double g;                /* gravity (9.81) */
    double delta;            /* delta-SPH coefficient of Eq. 7 (0.1; 0 disables) */
    double cfl;              /* Courant number Cr of Eq. 15 (0.2) */
    double dt_min;           /* adaptive dt below this sets SPH_EUNSTABLE (1e-12) */
    int32_t ns;              /* first-order step every ns steps, Eqs. 12-14 (40) */
    int32_t boundary_layers; /* boundary particle layers (2) */
    int32_t init;            /* SPH_INIT_HYDROSTATIC or SPH_INIT_UNIFORM */
    int32_t csound;          /* SPH_CSOUND_EOS or SPH_CSOUND_CONSTANT */
    int32_t cell_div;        /* grid cells per support radius 2h: 1, 2 or 3; 0 = automatic
                                (1 for SPH_MIXED, 2 for SPH_FP64) */
    int32_t use_graph;       /* replay multi-step launches from CUDA graphs (1) */
    int32_t graph_steps;     /* steps per captured graph (16) */
    int32_t pair_warps;      /* warps per CTA of the pair kernel, 0 = default */
    int32_t pair_ctas_per_sm;/* resident pair CTAs per SM, 0 = default */
    int32_t compensated;     /* mixed form: compensated FP32 pair sums (1) */
    int32_t pair_group;      /* mixed form: particles per warp sharing candidate loads (1, 2 or 4), 0 = default 4 */
    int32_t integrator;      /* SPH_VERLET (default) or SPH_SYMPLECTIC */
    int32_t delta_mode;      /* SPH_DELTA_ALL_FLUID (default) or SPH_DELTA_FULL_SUPPORT */
    int32_t persistent;      /* 1: sph_step runs all its steps in one persistent cooperative launch
                                (SPH_MIXED with SPH_VERLET only; the pair pass takes its default
                                shape, compensated sums); 0 (default): per-phase launches */
    int32_t spin_limit;      /* polls before a grid-barrier wait of the persistent launch gives up
                                (SPH_ETIMEOUT); 0 = default, about 2 s */
    int32_t list_capacity;   /* neighbour lists: entries per particle, 0 = automatic (the lattice
                                count within 2h + s, plus a third) */
    double list_skin;        /* neighbour lists with skin s = list_skin * h (SPH_MIXED with
                                SPH_VERLET, per-phase launches, cell_div 1): cells of 2h + s, each
                                particle's partners within 2h + s listed at a rebuild and reused
                                until a particle has moved s/2 (or left the grid); every step
                                still applies the exact |r_ij| < 2h test.  0 (default): the
                                neighbour structure is rebuilt and swept every step */
    int32_t pair_symmetric;  /* 1 (SPH_FP64 with SPH_DELTA_ALL_FLUID): each interacting pair is
                                evaluated once and its partner's share added through FP64
                                atomics, so the order of those additions, and the last bits of
                                the sums, can change from run to run; 44 more workspace bytes
                                per particle.  0 (default): each ordered pair, deterministic */
    int32_t reserved[1];
} sph_params;

/* One dam-break instance (batched creation). */
typedef struct sph_instance {
    double tank[3];     /* tank length, width, height */
    double column[3];   /* water column length, width, height */
    int32_t has_obstacle;
    int32_t has_gate;
    double obstacle[6]; /* lower corner x0,y0,z0 and size lx,ly,lz */
    double dp;          /* particle spacing l0 */
    double h;           /* smoothing length */
    double c0;          /* artificial speed of sound */
    double rho0;        /* reference density */
    double alpha;       /* artificial viscosity coefficient (Eq. 4) */
    /* Moving gate (Section 3.2: the Case 2 column is held by a gate opened at
     * a constant vertical speed): a filled lattice box of boundary particles
     * (type SPH_GATE, lower corner x0,y0,z0 and size lx,ly,lz like the
     * obstacle) moving at the constant velocity gate_velocity from t = 0.
     * Gate particles obey the dynamic boundary condition like the walls
     * (density by Eq. 7 over fluid neighbours, no forces applied), carry their
     * prescribed velocity into the pair terms and leave the domain for good
     * once they pass the grid.  Used when has_gate != 0; sph_create has no
     * gate argument, so an instance with a gate is created with
     * sph_batch_create (a batch of one behaves as a single tank). */
    double gate[6];
    double gate_velocity[3];
} sph_instance;

/* Defaults of the paper (Section 2.2 and Section 3): gamma 7, g 9.81,
 * delta 0.1, Cr 0.2, Ns 40; FP64 precision, 2 boundary layers, hydrostatic
 * start, c_i from the EOS, automatic cell size. */
void sph_params_default(sph_params *p);

/* Device bytes the caller must provide for these instances (n_inst >= 1).
 * Errors: SPH_EINVAL for invalid geometry or parameters. */
int sph_workspace_size(int32_t n_inst, const sph_instance *inst, const sph_params *p, size_t *bytes);

/* Create a single-instance simulation (the interface of the method:
 * tank, column, optional obstacle (NULL for none), dp, h, c0, rho0, alpha).
 * dev_workspace: device pointer to at least sph_workspace_size() bytes,
 * 256-byte aligned, owned by the caller.  cuda_stream: a cudaStream_t cast to
 * uintptr_t (0 = legacy default stream).  The initial lattice is generated
 * on the host and uploaded; the call returns after the upload has finished.
 * Errors: SPH_EINVAL, SPH_ENOMEM, SPH_ECUDA. */
int sph_create(sph_t **out, const double tank[3], const double column[3], const double *obstacle, double dp,
               double h, double c0, double rho0, double alpha, const sph_params *p, void *dev_workspace,
               size_t workspace_bytes, uintptr_t cuda_stream);

/* Create n_inst independent instances advanced together (an alpha sweep);
 * every kernel of a step covers all instances in one launch, each with its
 * own cell grid and its own adaptive dt. */
int sph_batch_create(sph_t **out, int32_t n_inst, const sph_instance *inst, const sph_params *p,
                     void *dev_workspace, size_t workspace_bytes, uintptr_t cuda_stream);

/* Release host resources of the handle (the workspace stays the caller's). */
void sph_destroy(sph_t *s);

/* Enqueue nsteps time steps.  dt > 0: fixed step; dt == 0: adaptive step of
 * Eq. 15 per instance.  Asynchronous: device-side failures (non-finite state,
 * dt < dt_min, a persistent launch's barrier wait running out) are reported by
 * the next synchronising call.  With params.persistent = 1 the nsteps steps of
 * every instance run in one cooperative launch whose phases are separated by
 * grid barriers (the per-phase launches compute the same steps bit for bit);
 * after SPH_ETIMEOUT the handle's state is undefined (destroy it). */
int sph_step(sph_t *s, double dt, int32_t nsteps);

/* Wait for the stream; return the device status (SPH_OK, SPH_EUNSTABLE...). */
int sph_sync(sph_t *s);

/* Probe instance `inst` on its current state.  kind SPH_PROBE_PRESSURE: pts
 * holds n points (x,y,z) and out receives n pressures (0 where no fluid
 * particle lies within 2h).  SPH_PROBE_WAVE_HEIGHT: pts holds n (x,y) pairs
 * and out receives n heights (largest z = k dp/4 whose kernel-summed fluid
 * density reaches rho0/2; 0 if none).  SPH_PROBE_FORCE: pts ignored, out
 * receives (Fx,Fy,Fz) = sum over obstacle particles of m a, a from fluid
 * neighbours by Eq. 3 without gravity.  Synchronous.  n <= 65536. */
int sph_probe(sph_t *s, int32_t inst, int32_t kind, const double *pts, int32_t n, double *out);

/* Particle counts of instance inst (inst = -1: all): fluid, walls and floor
 * (with the gate, if any), obstacle, total.  Ids run fluid, walls and floor,
 * obstacle, gate. */
int sph_counts(const sph_t *s, int32_t inst, int64_t out[4]);

/* Number of instances, total particles and total grid cells. */
int sph_sizes(const sph_t *s, int32_t *n_inst, int64_t *n_particles, int64_t *n_cells);

/* Copy the state out, id order, any pointer may be NULL: r (3n), u (3n),
 * rho (n), type (n), previous Verlet level uprev (3n) and rhoprev (n), the
 * step counter and the per-instance times (n_inst).  Synchronous. */
int sph_get_state(sph_t *s, double *r, double *u, double *rho, int32_t *type, double *uprev, double *rhoprev,
                  int64_t *step, double *time);

/* Load a state (id order; uprev/rhoprev NULL = same as u/rho), set the step
 * counter and, when time is not NULL, the simulated time of every instance
 * (time[n_inst]), then rebuild the neighbour structure.  Particle types are
 * fixed by the scene and unchanged.  Boundary velocities are prescribed, not
 * loaded: zero for walls and obstacle, the gate velocity for gate particles.
 * Checkpoint restore and test seam: a state read by sph_get_state and loaded
 * into a handle of the same cases continues as the saved handle does, bit
 * for bit in the FP64 form; in the mixed form the FP32 density offsets
 * rho - rho0 pass through the FP64 rho, which holds them exactly down to
 * about 1e-6 kg/m^3 (for rho0 = 1000).  Synchronous. */
int sph_set_state(sph_t *s, const double *r, const double *u, const double *rho, const double *uprev,
                  const double *rhoprev, int64_t step, const double *time);

/* One pair pass (Eqs. 3-8) on the current state without advancing it; outputs
 * in id order, any pointer may be NULL: drho (n), acc (3n, gravity included
 * for fluid), mumax (n, the inner max of Eq. 15, >= 0), nneigh (n, number of
 * in-domain j != i with |r_ij| < 2h; -1 for out-of-domain particles; with
 * neighbour lists (list_skin > 0) a boundary particle counts its fluid
 * neighbours only, since boundary pairs are not listed).  Synchronous. */
int sph_derivatives(sph_t *s, double *drho, double *acc, double *mumax, int32_t *nneigh);

/* The neighbour structure of the current state: cell (n, global cell id per
 * particle, id order; n_cells for out-of-domain particles), sorted (n_in,
 * ids in ascending (cell, id) order for the in-domain particles in the FP64
 * form, ascending (cell, x, id) in the mixed form, whose pair kernel relies on
 * cells sorted along x), cell_start
 * (n_cells + 1, index in `sorted` of the first particle of each cell; cell c
 * holds sorted[cell_start[c] .. cell_start[c+1])).  n_in receives the count of
 * in-domain particles.  Synchronous. */
int sph_cells(sph_t *s, int64_t *cell, int64_t *sorted, int64_t *cell_start, int64_t *n_in);

/* dt of the most recent step per instance (n_inst values).  Synchronous. */
int sph_last_dt(sph_t *s, double *dt);

/* FP64 diagnostics of instance inst on the current state: [0] mass,
 * [1] fluid volume sum m/rho, [2..4] fluid momentum, [5] kinetic energy,
 * [6] potential energy m g z, [7] internal energy (de/drho = P/rho^2,
 * e(rho0) = 0), [8] out-of-domain particles, [9] fluid particles in the
 * domain.  Synchronous. */
int sph_diagnostics(sph_t *s, int32_t inst, double out[10]);

/* Kernel timing: on = 1 records CUDA events around every kernel phase of
 * sph_step on the handle's stream; sph_phase_times fills ms[k] (total
 * milliseconds) and launches[k] for k < nphase of the phases named by
 * sph_phase_name(k), then clears the counters.  Synchronous. */
int sph_set_profiling(sph_t *s, int32_t on);
int sph_phase_times(sph_t *s, double *ms, int64_t *launches, int32_t nphase);
const char *sph_phase_name(int32_t k);
int32_t sph_num_phases(void);

/* Autotuner, on the current state (not advanced), each candidate timed with
 * CUDA events over `steps` passes: (1) the cell size 2h/cell_div (cell_div 1
 * or 2 for SPH_MIXED, 1-3 for SPH_FP64: cells per support radius, i.e. the
 * cells each work tile of the pair kernel covers), timed on the pair passes
 * plus one rebuild of the neighbour structure, the grid switched and the
 * structure rebuilt for each; (2) the pair kernel's launch shape (warps per
 * CTA, CTAs per SM, particles per warp); (3) the sort granularity: resident
 * CTAs per SM of the per-cell sort and gather.  The fastest of each is kept.
 * best[3] receives the chosen pair shape (may be NULL); sph_tuned_config gives
 * all five choices.  The cell count (sph_sizes) can change.  Synchronous. */
int sph_autotune(sph_t *s, int32_t steps, int32_t best[3]);

/* The tuned configuration: out[0..2] pair warps per CTA, CTAs per SM and
 * particles per warp (0 = the kernel's default), out[3] cell_div, out[4] sort
 * CTAs per SM. */
int sph_tuned_config(const sph_t *s, int32_t out[5]);

/* Runs one pair pass on the current state (the state is not advanced; the
 * derivative buffers are overwritten, as by sph_derivatives) with work
 * counting enabled, and returns its counts, summed over in-domain particles:
 * out[0] in-support ordered pairs (sum of nneigh), out[1] pairs whose terms
 * were evaluated (fluid-fluid, fluid-boundary and boundary-fluid), out[2]
 * candidates tested against |r_ij| < 2h (mixed form: per particle group
 * sharing a candidate load), out[3] evaluated fluid-fluid pairs (delta term)
 * and out[4] evaluated approaching pairs (viscosity term); out[3] and out[4]
 * are -1 for the FP64 form.  Synchronous. */
int sph_pair_stats(sph_t *s, int64_t out[5]);

/* Kernels launched by sph_step per time step (for launch accounting); with
 * params.persistent, 1: the kernels of one sph_step call, whatever its number
 * of steps. */
int32_t sph_launches_per_step(const sph_t *s);

/* Neighbour-list counters (list_skin > 0; zeros otherwise) since creation or
 * the last call, which clears them: out[0] list rebuilds, out[1] pair passes
 * that reused the lists, out[2] particles whose partners exceeded
 * list_capacity at a rebuild (evaluated by a direct scan of the 27 cells
 * instead), out[3] the longest list seen.  Synchronous. */
int sph_list_stats(sph_t *s, int64_t out[4]);

/* Allocation-free adaptive time step.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc - plug-ins whose
 * host application's caching allocator owns the device memory, real-time
 * loops that must not risk an allocation's implicit synchronisation, code
 * whose device-memory budget is fixed before it starts.  It computes the
 * adaptive step Cr min(min_i sqrt(h/|a_i|), min_i h/(c0 + mumax_i)) over the
 * particles with type[i] == SPH_FLUID (type NULL: all n particles) and writes
 * it to dt_out.  All pointers are caller-owned DEVICE pointers: acc (3n
 * doubles, interleaved xyz, gravity included), mumax (n doubles), type (n
 * int32 or NULL), dt_out (1 double).  Work is enqueued on cuda_stream (a
 * cudaStream_t cast to uintptr_t) and the call returns without waiting.
 * dt_out receives NaN when any acc or mumax value of a counted particle is
 * NaN; the call still returns SPH_OK, so check dt_out before using it.
 * It allocates nothing: its scratch is a fixed 32 KB device array in the
 * library, held on every device that loads the library until exit, so n must
 * not exceed 16,777,216 (SPH_EINVAL otherwise, as for n < 1, null pointers or
 * h, c0, cfl <= 0).  The scratch address (cudaGetSymbolAddress) belongs to
 * the CUDA context current at the call: it is looked up on every call whose
 * stream is not being captured, and remembered for that context; a call on a
 * stream under capture only reuses the address remembered for its context
 * (SPH_ECUDA if there is none).  So the first call in a context - which does
 * this set-up - must come before any stream capture.  Every call in a context
 * shares the scratch, and each call overwrites what it reads before reading
 * it, but calls whose work overlaps on the GPU (different streams, no
 * ordering) race on it: order them.  Errors: SPH_EINVAL, SPH_ECUDA. */
int sph_cfl_dt_noalloc(const double *acc, const double *mumax, const int32_t *type, int64_t n, double h,
                       double c0, double cfl, double *dt_out, uintptr_t cuda_stream);

/* Measured ALU peak for the roofline of the pair kernels (the paper has no
 * counterpart).  precision SPH_MIXED: FP32 fused multiply-adds (the better of
 * scalar and packed FP32x2 instructions); SPH_FP64: FP64 fused multiply-adds;
 * each counted as 2 flop.  Runs independent FMA chains on every SM for about
 * `millis` milliseconds per launch (1..60000), three timed launches, on
 * cuda_stream (a cudaStream_t cast to uintptr_t), and writes the fastest rate
 * in flop/s to *flops_per_s.  Synchronous; allocates nothing.
 * Errors: SPH_EINVAL, SPH_ECUDA. */
int sph_alu_peak(int32_t precision, int32_t millis, uintptr_t cuda_stream, double *flops_per_s);

/* Description of the last failure on this handle (never NULL). */
const char *sph_last_error(const sph_t *s);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
