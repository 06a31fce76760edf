// Internal declarations of the WCSPH library: per-instance constants, the
// device buffers carved from the caller's workspace, and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "sph.h"

namespace sph {

// Four doubles aligned to 32 bytes, so that one element is one 256-bit access;
// every array of them starts on a 256-byte boundary of the workspace.
using dvec4 = double4_32a;
__host__ __device__ __forceinline__ dvec4 make_dvec4(double x, double y, double z, double w)
{
    return make_double4_32a(x, y, z, w);
}

enum : uint8_t { T_FLUID = 0, T_WALL = 1, T_OBST = 2, T_GATE = 3 };

// Device status bits (ORed by kernels, read by sph_sync).
enum : int32_t { ST_UNSTABLE = 1, ST_TIMEOUT = 2, ST_OVERFLOW = 4, ST_BOUNDS = 8 };

// Debug builds (-DSPH_DEBUG) check shared-memory indices of the pair kernels
// before each access: a failing check records ST_BOUNDS and skips the access.
#ifdef SPH_DEBUG
#define SPH_BOUNDS_OK(cond, status) ((cond) ? true : (atomicOr((status), ST_BOUNDS), false))
#else
#define SPH_BOUNDS_OK(cond, status) true
#endif

// Constants of one instance, resident in device memory.  Grid: cells of size
// cs over [lo, lo + n cs) per axis; global cell id = cell_base +
// (cz n[1] + cy) n[0] + cx.  Particles [pbase, pbase + np): fluid first
// (nf), then walls (nw), then obstacle (no).
struct Inst {
    double lo[3];
    double cs, inv_cs;
    double h, c0, rho0, alpha, delta, gamma, g, cfl, mass, B, eta2, sup2, dt_min, ztop, dp;
    double kF;  // 105 / (16 pi h^5): grad_i W_ij = -kF (1 - q/2)^3 (r_i - r_j)
    double kW;  // 21 / (16 pi h^3)
    int32_t n[3];
    int32_t cell_base, ncells;
    int32_t pbase, np, nf, nw, no, ng;
    int32_t csound;
    int32_t delta_mode;  // SPH_DELTA_ALL_FLUID or SPH_DELTA_FULL_SUPPORT
    double gate_v[3];  // prescribed velocity of the gate particles
    // FP32 copies for the mixed form
    float csf, hf, inv_hf, c0f, rho0f, inv_rho0f, alphaf, massf, Bf, eta2f, sup2f, kFf, dfac;  // dfac = 2 delta h c0
    float gammaf, gf;
    float gate_vf[3];
    // FP64 form: squared radius of a conservative FP32 pre-test on the FP32
    // copies of the positions (2h widened by their worst rounding error), so
    // that the exact FP64 test is skipped only for pairs certainly beyond 2h
    float sup2_filter;
    float sup2_inner;  // below this FP32 squared distance a pair is certainly within 2h
    // neighbour lists: skin s, (s/2)^2 (the displacement that forces a rebuild)
    // and the FP32 list radius (2h + s)^2
    double skin, half_skin2;
    float list_r2f;
};

// Pointers into the workspace.  "id" arrays are in particle-id order, "s"
// arrays in sorted (cell, id) order.
struct Bufs {
    // canonical state (id order)
    dvec4 *pos;            // x, y, z, unused
    void *vel;               // FP64: dvec4 (u, rho); mixed: float4 (u, rho - rho0)
    void *velp;              // previous Verlet level, same layout as vel
    uint8_t *type;           // SPH_FLUID / SPH_WALL / SPH_OBSTACLE
    uint16_t *inst_of;       // instance of each particle
    uint32_t *key;           // cell of each particle (C = out of domain)
    // neighbour structure
    uint32_t *count;         // C + 1 per-cell counters (zero between steps)
    int32_t *cell_start;     // C + 2 lower bounds into the sorted order
    int32_t *active;         // non-empty cells in ascending order
    uint64_t *scan_blocks;   // block partials of the cell scan
    int32_t *perm;           // sorted index -> particle id
    int32_t *ptmp;           // scatter target before the per-cell id sort
    int32_t *scell;          // sorted index -> cell
    // sorted particle data for the pair kernel
    void *sA;                // FP64: dvec4 (x, y, z, rho); mixed: float4 (offset to cell origin, rho - rho0)
    void *sB;                // FP64: dvec4 (u, P); mixed: float4 (u, P)
    double2 *sC;             // FP64 form: (1 / rho, c) per sorted particle; unused by the mixed form
    float4 *sD;              // FP64 form: FP32 copies of the sorted positions, for the pre-test
    uint8_t *sflag;          // type per sorted index
    // pair outputs (sorted)
    void *deriv;             // FP64: dvec4 (a, Drho); mixed: float4
    void *mumax;             // double or float
    int32_t *nneigh;
    int32_t *npair;          // pairs evaluated per particle (interacting neighbours)
    int32_t *ncand;          // candidates staged for each particle's home cell
    // neighbour lists (list_skin > 0; null otherwise), sorted order of the last rebuild
    int32_t *nlist;          // [N][list_cap]: (j << 5) | offset code of j's cell from i's
    int32_t *ncnt;           // partners listed per particle (> list_cap: overflow)
    dvec4 *xbuild;           // id order: position at the last rebuild
    int32_t *lflag;          // [0] rebuild request (set by the update, cleared by the list pass);
                             // counters: [1] rebuilds, [2] overflowing particles, [3] longest
                             // list, [4] list passes
    int32_t list_cap;
    // FP64 pass evaluating each pair once (pair_symmetric; null otherwise):
    // sorted order, the partners' shares (t^3 units) of D u/Dt, D rho/Dt, mu/h
    // (bits) and the neighbour counts
    dvec4 *fjacc;
    long long *fjmu;
    int32_t *fjnn;
    unsigned long long *pstat; // [4] last pair pass: fluid-fluid pairs, approaching pairs, windowed candidates
    // per-instance reductions and time stepping
    unsigned long long *red; // [ninst][2]: max |a|^2 bits, max mu bits
    double *dt;              // [ninst]
    double *time;            // [ninst]
    double *dt_fixed;        // [1]
    long long *step;         // [1] step counter
    int32_t *euler;          // [1] 1 when the current step is first-order
    int32_t *misc;           // [0] n_in, [1] n_active, [2] status, [3] pair work queue
    unsigned *bar;           // grid-barrier counter of the persistent time loop
    Inst *inst;              // [ninst]
    // probes and diagnostics scratch
    double *probe_in;        // up to kMaxProbe * 3
    double *probe_out;       // up to kMaxProbe * 4
    int32_t *probe_k;        // up to kMaxProbe
    double *diag;            // [diag_blocks][10]
};

constexpr int kMaxProbe = 65536;
constexpr int kDiagBlocks = 256;
constexpr int kScanTile = 4096;

// Kernel launchers (implemented in the .cu files).  All launch on `st`.
void launch_bin(const Bufs &b, int mode, int64_t N, int32_t C, cudaStream_t st);
void launch_cells(const Bufs &b, int64_t N, int32_t C, cudaStream_t st);
void launch_reorder(const Bufs &b, int mode, int64_t N, int32_t C, int32_t ninst, int32_t max_active,
                    int32_t ctas_per_sm, cudaStream_t st);
// neighbours: the pass must write every particle's nneigh (with
// pair_symmetric the partners' counts are left out of time steps).
void launch_pair_fp64(const Bufs &b, int64_t N, int32_t ninst, int32_t cell_div, int32_t warps, int32_t ctas,
                      int32_t delta_mode, bool neighbours, cudaStream_t st);
void launch_pair_mixed(const Bufs &b, int64_t N, int32_t ninst, int32_t cell_div, int32_t warps,
                       int32_t ctas, int32_t group, int32_t compensated, int32_t max_active, bool count,
                       int32_t delta_mode, cudaStream_t st);
// Neighbour lists (pair_list.cu): the build (when lflag[0] requests it) and
// the list pass; the gather of a step that keeps the lists.
void launch_list_pass(const Bufs &b, int64_t N, int32_t ninst, int32_t delta_mode, cudaStream_t st);
void launch_list_regather(const Bufs &b, int64_t N, int32_t ninst, cudaStream_t st);
void launch_dt(const Bufs &b, int mode, int64_t N, int32_t ninst, int32_t ns, cudaStream_t st);
void launch_integrate(const Bufs &b, int mode, int64_t N, int32_t C, int32_t ninst, cudaStream_t st);
void launch_predict(const Bufs &b, int mode, int64_t N, int32_t C, cudaStream_t st);
void launch_correct(const Bufs &b, int mode, int64_t N, int32_t C, cudaStream_t st);
void launch_probe_pressure(const Bufs &b, int mode, int32_t inst, int32_t ninst, int32_t cell_div,
                           int32_t npts, cudaStream_t st);
void launch_probe_wave(const Bufs &b, int mode, int32_t inst, int32_t ninst, int32_t cell_div, int32_t npts,
                       int32_t nlev, cudaStream_t st);
void launch_probe_force(const Bufs &b, int mode, int32_t inst, int32_t ninst, int32_t cell_div, int64_t N,
                        cudaStream_t st);
// One cooperative launch of nsteps Verlet steps of the mixed form over all
// instances (persist.cu); spin_limit bounds every grid-barrier wait.
cudaError_t launch_persistent_steps(const Bufs &b, int32_t ninst, int32_t nsteps, int32_t ns, int32_t cell_div,
                                    int32_t delta_mode, int64_t N, int32_t C, long long spin_limit, cudaStream_t st);
void launch_diagnostics(const Bufs &b, int mode, int32_t inst, int32_t C, cudaStream_t st);

// Host-side instance description after validation.
struct HostInst {
    sph_instance d;
    int64_t nf, nw, no, ng;
    Inst dev;
};

int validate_instance(const sph_instance &in, const sph_params &p, std::string &err);
int effective_cell_div(const sph_params &p);
void fill_inst(HostInst &hi, const sph_params &p);
void build_scene(const HostInst &hi, const sph_params &p, double *r, double *rho, uint8_t *type);

}  // namespace sph
