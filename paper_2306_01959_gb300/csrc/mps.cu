// MPS time step (Section 2.3, Eqs. 16-30) on the GPU, FP64 throughout: the
// explicit prediction, the particle number density and free-surface detection,
// the pressure Poisson equation assembled row by row into a fixed-width sparse
// layout and solved by the conjugate gradient method, the first-order pressure
// gradient and the correction.  The readings are listed in include/mps.h.
//
// Layout: canonical state in particle-id order (position, velocity, type);
// every neighbour query runs on a cell list of cell size r_e rebuilt at r^t and
// at r* (counting sort by cell, per-cell sort by id, so the candidate order is
// (cell, id) as in the method's definition of the neighbourhood).  The system
// of Eq. 23 lives in sorted-index space: row i holds the diagonal and up to
// `row_width` off-diagonal entries stored column-major (entry k of every row
// contiguous), so that the one-thread-per-row product reads coalesced; rows of
// particles that are not unknowns are identity rows with a zero right-hand
// side, which keeps every vector the length of the sorted order.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cells.cuh"
#include "mps.h"

namespace {

using namespace sph;

constexpr int kCgBlocks = 1024;  // fixed block count of the reductions (deterministic sums)
constexpr int kCgThreads = 256;
constexpr int kCgChunk = 16;     // CG iterations launched between convergence checks

struct MpsConst {
    double lo[3];
    double cs;  // cell size r_e
    int32_t n[3];
    int32_t ncells;
    double re, l0, nu, rho, g, kc, kr, beta1, varrho1, dt, n0, lambda0, lapc, tol;
    float re2f;  // squared FP32 pre-test radius: r_e widened by the rounding of FP32 coordinates
    int32_t width;
};

struct MpsBufs {
    dvec4 *pos, *vel, *ustar;  // id order
    uint8_t *type;             // id order
    uint8_t *moved;            // id order: predicted in this step (reset by k_mps_finish)
    double *P;                 // id order: pressure of the last step (clamped)
    uint32_t *key, *count;
    int32_t *cell_start, *active, *perm, *ptmp, *misc;  // misc: [0] n_in, [1] n_active, [2] status
    uint64_t *scan_blocks;
    dvec4 *spos;               // sorted: x, y, z, type
    float4 *sposf;             // sorted: FP32 copies of x, y, z (the candidate pre-test)
    double *snd, *ssig;        // sorted: n*, centroid deviation
    uint8_t *surf;             // sorted: free-surface flag
    int32_t *ecnt, *ecol;      // sorted rows: entry count; entry k of row i at [k * N + i]
    double *eval, *diag, *rhs;
    double *x, *r, *p, *q, *part, *scal;  // scal: [0] rho, [1] |b|^2, [2] alpha, [3] beta
    int32_t *cgi;              // [0] iterations, [1] done
    MpsConst *c;
};

// The weight of Eq. 16 (r_e / |r_ij| - 1 within r_e, 0 beyond and for
// coincident particles) from the squared distance, through one reciprocal
// square root (the FP64 pipe of this GPU is narrow: a square root and a
// division per pair cost several times more); inv receives 1/|r_ij|.
__device__ __forceinline__ double mps_w2(double d2, const MpsConst &C, double &inv)
{
    if (!(d2 > 0.0) || d2 > C.re * C.re) {
        inv = 0.0;
        return 0.0;
    }
    inv = rsqrt(d2);
    return C.re * inv - 1.0;
}

__device__ __forceinline__ bool mps_cell(const MpsConst &C, double x, double y, double z, int &cx, int &cy, int &cz)
{
    const double fx = floor((x - C.lo[0]) / C.cs), fy = floor((y - C.lo[1]) / C.cs), fz = floor((z - C.lo[2]) / C.cs);
    if (!(fx >= 0.0) || fx >= C.n[0] || !(fy >= 0.0) || fy >= C.n[1] || !(fz >= 0.0) || fz >= C.n[2])
        return false;
    cx = (int)fx;
    cy = (int)fy;
    cz = (int)fz;
    return true;
}

// ---------------------------------------------------------------- cell list
__global__ void k_mps_bin(MpsBufs b, int64_t N)
{
    const MpsConst &C = *b.c;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < N; id += (int64_t)gridDim.x * blockDim.x) {
        const dvec4 p = b.pos[id];
        int cx, cy, cz;
        uint32_t c = (uint32_t)C.ncells;
        if (mps_cell(C, p.x, p.y, p.z, cx, cy, cz))
            c = (uint32_t)((cz * C.n[1] + cy) * C.n[0] + cx);
        b.key[id] = c;
        atomicAdd(&b.count[c], 1u);
    }
}

__global__ void k_mps_scan_reduce(MpsBufs b, int64_t C) { scan_reduce_tile(b.count, b.scan_blocks, C, blockIdx.x); }
__global__ void k_mps_scan_blocks(MpsBufs b, int nb) { scan_blocks_block(b.scan_blocks, nb); }
__global__ void k_mps_scan_final(MpsBufs b, int64_t C)
{
    scan_final_tile(b.count, b.scan_blocks, b.cell_start, b.active, b.misc, C, blockIdx.x);
}
__global__ void k_mps_scatter(MpsBufs b, int64_t N)
{
    scatter_range(b.key, b.count, b.cell_start, b.ptmp, b.misc, N, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                  (int64_t)gridDim.x * blockDim.x);
}

// One warp per non-empty cell: rank its particles by id, gather the sorted
// positions (type in w).
__global__ void __launch_bounds__(256) k_mps_sort(MpsBufs b)
{
    __shared__ int32_t sid[8][256];
    const int lane = threadIdx.x & 31;
    int32_t *K = sid[threadIdx.x >> 5];
    const int32_t n_active = b.misc[1];
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_active; w += warps) {
        const int32_t c = b.active[w];
        const int32_t s0 = b.cell_start[c], n = b.cell_start[c + 1] - s0;
        const bool smem = n <= 256;
        if (smem)
            for (int e = lane; e < n; e += 32)
                K[e] = b.ptmp[s0 + e];
        __syncwarp();
        for (int e = lane; e < n; e += 32) {
            const int32_t id = smem ? K[e] : b.ptmp[s0 + e];
            int32_t rank = 0;
            for (int k = 0; k < n; ++k)
                rank += (smem ? K[k] : b.ptmp[s0 + k]) < id;
            const int32_t s = s0 + rank;
            b.perm[s] = id;
            const dvec4 p = b.pos[id];
            b.spos[s] = make_dvec4(p.x, p.y, p.z, (double)b.type[id]);
            b.sposf[s] = make_float4((float)p.x, (float)p.y, (float)p.z, 0.f);
        }
        __syncwarp();
    }
}

// The 9 rows (cells x-1 .. x+1 of each (y, z) neighbour) of sorted particle s:
// calls f(j, valid) for the candidates in (cell, id) order, on all lanes of
// the warp (lane k takes candidates k, k + 32, ...); `valid` is false past the
// end of a row, for j = s, and for a candidate that an FP32 distance test on
// the FP32 copies of the positions puts beyond r_e by more than their rounding
// (so every pair within r_e stays valid and takes the exact FP64 test).
template <class F>
__device__ __forceinline__ void for_candidates(const MpsBufs &b, const MpsConst &C, int32_t s, F &&f)
{
    const int lane = threadIdx.x & 31;
    const dvec4 pi = b.spos[s];
    const float4 pif = b.sposf[s];
    int cx, cy, cz;
    mps_cell(C, pi.x, pi.y, pi.z, cx, cy, cz);
    const int x0 = max(cx - 1, 0), x1 = min(cx + 1, C.n[0] - 1);
    for (int z = max(cz - 1, 0); z <= min(cz + 1, C.n[2] - 1); ++z)
        for (int y = max(cy - 1, 0); y <= min(cy + 1, C.n[1] - 1); ++y) {
            const int32_t row = (z * C.n[1] + y) * C.n[0];
            const int32_t j0 = b.cell_start[row + x0], j1 = b.cell_start[row + x1 + 1];
            for (int32_t base = j0; base < j1; base += 32) {
                const int32_t j = base + lane;
                bool valid = j < j1 && j != s;
                if (valid) {
                    const float4 a = b.sposf[j];
                    const float dx = a.x - pif.x, dy = a.y - pif.y, dz = a.z - pif.z;
                    valid = dx * dx + dy * dy + dz * dz <= C.re2f;
                }
                f(j, valid);
            }
        }
}

// The candidates of for_candidates that pass its pre-test, compacted by ballot
// (in the same order) into the warp's 64-entry shared buffer and handed to
// f(j, on) 32 at a time, so that the FP64 arithmetic of a pair runs on full
// lanes (about 40 of the ~250 candidates of a particle pass).  f is called on
// all lanes of the warp; `on` is false only on the lanes of the last, partial
// batch that hold no candidate.
constexpr int kMpsWarps = 8;  // warps per CTA of the neighbour kernels (blockDim 256)

template <class F>
__device__ __forceinline__ void for_near(const MpsBufs &b, const MpsConst &C, int32_t s, int32_t *buf, F &&f)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int cnt = 0;
    for_candidates(b, C, s, [&](int32_t j, bool valid) {
        const unsigned m = __ballot_sync(0xffffffffu, valid);
        if (valid)
            buf[cnt + __popc(m & lt)] = j;
        cnt += __popc(m);
        if (cnt >= 32) {
            __syncwarp();
            f(buf[lane], true);
            __syncwarp();
            if (lane < cnt - 32)
                buf[lane] = buf[32 + lane];
            cnt -= 32;
            __syncwarp();
        }
    });
    __syncwarp();
    if (cnt > 0)
        f(lane < cnt ? buf[lane] : s, lane < cnt);
    __syncwarp();
}

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- Eqs. 21-22
__global__ void __launch_bounds__(kMpsWarps * 32) k_mps_predict(MpsBufs b)
{
    __shared__ int32_t nbuf[kMpsWarps][64];
    int32_t *buf = nbuf[threadIdx.x >> 5];
    const MpsConst &C = *b.c;
    const int32_t n_in = b.misc[0];
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n_in; s += warps) {
        const dvec4 pi = b.spos[s];
        if ((int)pi.w != MPS_FLUID)
            continue;
        const int32_t id = b.perm[s];
        const dvec4 ui = b.vel[id];
        double lx = 0.0, ly = 0.0, lz = 0.0;
        for_near(b, C, s, buf, [&](int32_t j, bool valid) {
            if (!valid)
                return;
            const dvec4 pj = b.spos[j];
            const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            double inv;
            const double w = mps_w2(dx * dx + dy * dy + dz * dz, C, inv);
            if (w == 0.0)
                return;
            const dvec4 uj = b.vel[b.perm[j]];
            lx += (uj.x - ui.x) * w;
            ly += (uj.y - ui.y) * w;
            lz += (uj.z - ui.z) * w;
        });
        {
            double t[4] = {lx, ly, lz, 0.0};
            warp_totals<4>(t);
            lx = t[0];
            ly = t[1];
            lz = t[2];
        }
        if ((threadIdx.x & 31) == 0) {
            b.moved[id] = 1;
            const double k = C.nu * C.lapc;
            const dvec4 us = make_dvec4(ui.x + C.dt * (k * lx), ui.y + C.dt * (k * ly), ui.z + C.dt * (k * lz - C.g), 0.0);
            b.ustar[id] = us;
            const dvec4 p = b.pos[id];
            b.pos[id] = make_dvec4(p.x + C.dt * us.x, p.y + C.dt * us.y, p.z + C.dt * us.z, 0.0);
        }
    }
}

// ---------------------------------------------------------------- Eq. 17, Eqs. 28-30
__global__ void __launch_bounds__(kMpsWarps * 32) k_mps_density(MpsBufs b)
{
    __shared__ int32_t nbuf[kMpsWarps][64];
    int32_t *buf = nbuf[threadIdx.x >> 5];
    const MpsConst &C = *b.c;
    const int32_t n_in = b.misc[0];
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n_in; s += warps) {
        const dvec4 pi = b.spos[s];
        double sw = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for_near(b, C, s, buf, [&](int32_t j, bool valid) {
            if (!valid)
                return;
            const dvec4 pj = b.spos[j];
            const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            double inv;
            const double w = mps_w2(dx * dx + dy * dy + dz * dz, C, inv);
            sw += w;
            sx += dx * w;
            sy += dy * w;
            sz += dz * w;
        });
        {
            double t[4] = {sw, sx, sy, sz};
            warp_totals<4>(t);
            sw = t[0];
            sx = t[1];
            sy = t[2];
            sz = t[3];
        }
        if ((threadIdx.x & 31) == 0) {
            const double sig = sw > 0.0 ? sqrt(sx * sx + sy * sy + sz * sz) / sw : 0.0;
            b.snd[s] = sw;
            b.ssig[s] = sig;
            b.surf[s] = ((int)pi.w != MPS_DUMMY && sw < C.beta1 * C.n0 && sig > C.varrho1 * C.l0) ? 1 : 0;
        }
    }
}

// ---------------------------------------------------------------- Eq. 23
// Row of sorted particle s (times -1, so that the system is SPD):
//   (lapc sum_{j non-dummy} w_ij + rho kappa_c / dt^2) P_s - lapc sum_{j unknown} w_ij P_j
//     = kappa_r rho / dt^2 (n*_s - n0) / n0.
__global__ void __launch_bounds__(kMpsWarps * 32) k_mps_assemble(MpsBufs b, int32_t Ns)
{
    __shared__ int32_t nbuf[kMpsWarps][64];
    int32_t *buf = nbuf[threadIdx.x >> 5];
    const MpsConst &C = *b.c;
    const int32_t n_in = b.misc[0];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n_in; s += warps) {
        const dvec4 pi = b.spos[s];
        const bool unknown = (int)pi.w != MPS_DUMMY && !b.surf[s];
        if (!unknown) {
            if (lane == 0) {
                b.diag[s] = 1.0;
                b.ecnt[s] = 0;
                b.rhs[s] = 0.0;
            }
            continue;
        }
        double sw = 0.0;
        int cnt = 0;
        bool over = false;
        for_near(b, C, s, buf, [&](int32_t j, bool valid) {
            double w = 0.0;
            bool take = false;
            if (valid) {
                const dvec4 pj = b.spos[j];
                if ((int)pj.w != MPS_DUMMY) {
                    const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                    const double d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 > 0.0 && d2 <= C.re * C.re) {
                        double inv;
                        w = mps_w2(d2, C, inv);
                        sw += w;
                        take = !b.surf[j];
                    }
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, take);
            if (take) {
                const int k = cnt + __popc(m & lt);
                if (k < C.width) {
                    b.ecol[(int64_t)k * Ns + s] = j;
                    b.eval[(int64_t)k * Ns + s] = -C.lapc * w;
                } else {
                    over = true;
                }
            }
            cnt += __popc(m);
        });
        sw = wsum(sw);
        over = __any_sync(0xffffffffu, over);
        if (lane == 0) {
            b.diag[s] = C.lapc * sw + C.rho * C.kc / (C.dt * C.dt);
            b.ecnt[s] = min(cnt, C.width);
            b.rhs[s] = C.kr * C.rho / (C.dt * C.dt) * (b.snd[s] - C.n0) / C.n0;
            if (over)
                atomicOr(&b.misc[2], ST_OVERFLOW);
        }
    }
}

// ---------------------------------------------------------------- CG
// Block sums over a fixed grid of kCgBlocks blocks; the partials are summed by
// one block in a fixed order, so every dot product is deterministic.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = wsum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0)
        sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        t = wsum(t);
    }
    return t;  // valid in thread 0
}

__global__ void k_cg_init(MpsBufs b, int32_t Ns)
{
    __shared__ double sh[32];
    const int32_t n_in = b.misc[0];
    double bb = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < Ns; i += gridDim.x * blockDim.x) {
        const double v = i < n_in ? b.rhs[i] : 0.0;
        b.x[i] = 0.0;
        b.r[i] = v;
        b.p[i] = v;
        bb += v * v;
    }
    bb = block_sum(bb, sh);
    if (threadIdx.x == 0)
        b.part[blockIdx.x] = bb;
}

// One block: total of the partials into scal[slot]; init also sets rho and
// the counters.
__global__ void k_cg_total(MpsBufs b, int slot, int init)
{
    __shared__ double sh[32];
    if (!init && b.cgi[1])
        return;
    double v = 0.0;
    for (int k = threadIdx.x; k < kCgBlocks; k += blockDim.x)
        v += b.part[k];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) {
        if (init) {
            b.scal[1] = v;  // |b|^2
            b.scal[0] = v;  // rho = r.r with r = b
            b.cgi[0] = 0;
            b.cgi[1] = v == 0.0;  // a zero right-hand side is solved by P = 0
        } else if (slot == 2) {
            b.scal[2] = b.scal[0] / v;  // alpha = rho / p.q
        } else {
            const double rho_new = v;
            b.scal[3] = rho_new / b.scal[0];  // beta
            b.scal[0] = rho_new;
            b.cgi[0] += 1;
            if (sqrt(rho_new) <= b.c->tol * sqrt(b.scal[1]) || !(rho_new == rho_new))
                b.cgi[1] = 1;
        }
    }
}

__global__ void k_cg_spmv(MpsBufs b, int32_t Ns)
{
    __shared__ double sh[32];
    if (b.cgi[1])
        return;
    const int32_t n_in = b.misc[0];
    double pq = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < Ns; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        if (i < n_in) {
            s = b.diag[i] * b.p[i];
            const int cnt = b.ecnt[i];
            for (int k = 0; k < cnt; ++k)
                s += b.eval[(int64_t)k * Ns + i] * b.p[b.ecol[(int64_t)k * Ns + i]];
        }
        b.q[i] = s;
        pq += b.p[i] * s;
    }
    pq = block_sum(pq, sh);
    if (threadIdx.x == 0)
        b.part[blockIdx.x] = pq;
}

__global__ void k_cg_update(MpsBufs b, int32_t Ns)
{
    __shared__ double sh[32];
    if (b.cgi[1])
        return;
    const double alpha = b.scal[2];
    double rr = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < Ns; i += gridDim.x * blockDim.x) {
        b.x[i] += alpha * b.p[i];
        const double ri = b.r[i] - alpha * b.q[i];
        b.r[i] = ri;
        rr += ri * ri;
    }
    rr = block_sum(rr, sh);
    if (threadIdx.x == 0)
        b.part[blockIdx.x] = rr;
}

__global__ void k_cg_direction(MpsBufs b, int32_t Ns)
{
    // the iteration that reached the tolerance has set the flag; its direction
    // update is not needed
    if (b.cgi[1])
        return;
    const double beta = b.scal[3];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < Ns; i += gridDim.x * blockDim.x)
        b.p[i] = b.r[i] + beta * b.p[i];
}

// ---------------------------------------------------------------- clamp, Eq. 24, Eqs. 25-26
__global__ void k_mps_clamp(MpsBufs b, int32_t Ns)
{
    const int32_t n_in = b.misc[0];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_in; i += gridDim.x * blockDim.x) {
        const dvec4 pi = b.spos[i];
        const bool unknown = (int)pi.w != MPS_DUMMY && !b.surf[i];
        const double P = unknown ? fmax(b.x[i], 0.0) : 0.0;
        b.q[i] = P;  // the clamped pressure in sorted order, read by the gradient
        b.P[b.perm[i]] = P;
    }
    (void)Ns;
}

__global__ void __launch_bounds__(kMpsWarps * 32) k_mps_correct(MpsBufs b)
{
    __shared__ int32_t nbuf[kMpsWarps][64];
    int32_t *buf = nbuf[threadIdx.x >> 5];
    const MpsConst &C = *b.c;
    const int32_t n_in = b.misc[0];
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const double *P = b.q;
    for (int32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n_in; s += warps) {
        const dvec4 pi = b.spos[s];
        if ((int)pi.w != MPS_FLUID)
            continue;
        // P_hat: minimum of P over i and its neighbours with a pressure
        double pmin = P[s];
        double m00 = 0, m01 = 0, m02 = 0, m11 = 0, m12 = 0, m22 = 0, vx = 0, vy = 0, vz = 0, ax = 0, ay = 0, az = 0;
        for_near(b, C, s, buf, [&](int32_t j, bool valid) {
            if (!valid)
                return;
            const dvec4 pj = b.spos[j];
            if ((int)pj.w == MPS_DUMMY)
                return;
            const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            const double d2 = dx * dx + dy * dy + dz * dz;
            if (!(d2 > 0.0 && d2 <= C.re * C.re))
                return;
            double inv;
            const double w = mps_w2(d2, C, inv);
            const double ex = dx * inv, ey = dy * inv, ez = dz * inv;
            m00 += ex * ex * w;
            m01 += ex * ey * w;
            m02 += ex * ez * w;
            m11 += ey * ey * w;
            m12 += ey * ez * w;
            m22 += ez * ez * w;
            // sum (P_j - P_hat) r_ij w / d^2 = sum P_j r_ij w / d^2 - P_hat sum r_ij w / d^2
            const double f = w * (inv * inv);
            vx += P[j] * dx * f;
            vy += P[j] * dy * f;
            vz += P[j] * dz * f;
            ax += dx * f;
            ay += dy * f;
            az += dz * f;
            pmin = fmin(pmin, P[j]);
        });
        {
            double t[16] = {m00, m01, m02, m11, m12, m22, vx, vy, vz, ax, ay, az, 0.0, 0.0, 0.0, 0.0};
            warp_totals<16>(t);
            m00 = t[0]; m01 = t[1]; m02 = t[2]; m11 = t[3]; m12 = t[4]; m22 = t[5];
            vx = t[6]; vy = t[7]; vz = t[8]; ax = t[9]; ay = t[10]; az = t[11];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            pmin = fmin(pmin, __shfl_xor_sync(0xffffffffu, pmin, o));
        if ((threadIdx.x & 31) == 0) {
            const double v0 = vx - pmin * ax, v1 = vy - pmin * ay, v2 = vz - pmin * az;
            // M^{-1} v by the adjugate of the symmetric moment matrix
            const double c00 = m11 * m22 - m12 * m12, c01 = m02 * m12 - m01 * m22, c02 = m01 * m12 - m02 * m11;
            const double c11 = m00 * m22 - m02 * m02, c12 = m02 * m01 - m00 * m12, c22 = m00 * m11 - m01 * m01;
            const double det = m00 * c00 + m01 * c01 + m02 * c02;
            const double scale = (m00 + m11 + m22) / 3.0;
            double gx = 0.0, gy = 0.0, gz = 0.0;
            if (fabs(det) > 1e-12 * scale * scale * scale) {
                gx = (c00 * v0 + c01 * v1 + c02 * v2) / det;
                gy = (c01 * v0 + c11 * v1 + c12 * v2) / det;
                gz = (c02 * v0 + c12 * v1 + c22 * v2) / det;
            }
            const int32_t id = b.perm[s];
            const dvec4 us = b.ustar[id];
            const double k = C.dt / C.rho;
            const dvec4 un = make_dvec4(us.x - k * gx, us.y - k * gy, us.z - k * gz, 0.0);
            b.vel[id] = un;
            const dvec4 p = b.pos[id];
            b.pos[id] = make_dvec4(p.x + C.dt * (un.x - us.x), p.y + C.dt * (un.y - us.y), p.z + C.dt * (un.z - us.z),
                                   0.0);
            if (!(un.x == un.x && un.y == un.y && un.z == un.z))
                atomicOr(&b.misc[2], ST_UNSTABLE);
        }
    }
}

// A fluid particle that the prediction carried out of the grid takes no part in
// the pressure step: it keeps u* and r* and is frozen from then on.
__global__ void k_mps_finish(MpsBufs b, int64_t N)
{
    const uint32_t out = (uint32_t)b.c->ncells;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < N; id += (int64_t)gridDim.x * blockDim.x) {
        if (!b.moved[id])
            continue;
        if (b.key[id] == out)
            b.vel[id] = b.ustar[id];
        b.moved[id] = 0;
    }
}

struct Layout {
    size_t off = 0;
    char *base = nullptr;
    template <class T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * (count ? count : 1);
        return p;
    }
};

int64_t nint(double x) { return (int64_t)std::floor(x + 0.5); }

struct Geometry {
    int64_t nf = 0, nw = 0, ndum = 0, N = 0;
    MpsConst c{};
};

int geometry(const double tank[3], const double column[3], double l0, double dt, const mps_params *p, Geometry &g,
             std::string &err)
{
    if (!p || p->size != sizeof(mps_params)) {
        err = "mps_params.size must equal sizeof(mps_params)";
        return SPH_EINVAL;
    }
    if (!tank || !column || !(l0 > 0) || !(dt >= 0) || p->layers < 1 || p->layers > 8 || !(p->re_factor >= 1.0) ||
        !(p->re_factor <= 4.0) || !(p->rho > 0) || !(p->kappa_c >= 0) || !(p->kappa_r >= 0) || !(p->cg_tol > 0) ||
        p->cg_max < 1 || p->row_width < 1 || p->row_width > 512) {
        err = "invalid parameters";
        return SPH_EINVAL;
    }
    int64_t ncx = nint(column[0] / l0), ncy = nint(column[1] / l0), ncz = nint(column[2] / l0);
    int64_t ntx = nint(tank[0] / l0), nty = nint(tank[1] / l0), ntz = nint(tank[2] / l0);
    if (ncx < 0 || ncy < 0 || ncz < 0 || ncx > ntx || ncy > nty || ncz > ntz || ntx < 1 || nty < 1 || ntz < 1) {
        err = "the column must fit in the tank";
        return SPH_EINVAL;
    }
    const int64_t L = p->layers;
    g.nf = ncx * ncy * ncz;
    for (int64_t k = -L; k < ntz; ++k)
        for (int64_t j = -L; j < nty + L; ++j)
            for (int64_t i = -L; i < ntx + L; ++i) {
                int64_t dx = i < 0 ? -1 - i : (i >= ntx ? i - ntx : -1);
                int64_t dy = j < 0 ? -1 - j : (j >= nty ? j - nty : -1);
                int64_t dz = k < 0 ? -1 - k : -1;
                int64_t layer = std::max(dx, std::max(dy, dz));
                if (layer < 0)
                    continue;
                (layer == 0 ? g.nw : g.ndum) += 1;
            }
    g.N = g.nf + g.nw + g.ndum;
    MpsConst &c = g.c;
    std::memset(&c, 0, sizeof(c));
    c.re = p->re_factor * l0;
    c.cs = c.re;
    const double Ld = L * l0;
    const double hi[3] = {tank[0] + Ld, tank[1] + Ld, tank[2] + 4.0 * c.re};
    int64_t ncells = 1;
    for (int a = 0; a < 3; ++a) {
        c.lo[a] = -Ld;
        c.n[a] = (int32_t)std::ceil((hi[a] - c.lo[a]) / c.cs);
        ncells *= c.n[a];
    }
    if (g.N >= ((int64_t)1 << 31) / 2 || ncells >= ((int64_t)1 << 31) - 4) {
        err = "too many particles or cells";
        return SPH_EINVAL;
    }
    c.ncells = (int32_t)ncells;
    c.l0 = l0;
    c.nu = p->nu;
    c.rho = p->rho;
    c.g = p->g;
    c.kc = p->kappa_c;
    c.kr = p->kappa_r;
    c.beta1 = p->beta1;
    c.varrho1 = p->varrho1;
    c.dt = dt;
    c.tol = p->cg_tol;
    c.width = p->row_width;
    // n0 and lambda0 (Eq. 20) of the full initial lattice
    const int k = (int)std::ceil(c.re / l0);
    double sw = 0.0, sr2w = 0.0;
    for (int a = -k; a <= k; ++a)
        for (int bb = -k; bb <= k; ++bb)
            for (int d = -k; d <= k; ++d) {
                if (!a && !bb && !d)
                    continue;
                const double r2 = (double)(a * a + bb * bb + d * d) * l0 * l0;
                const double r = std::sqrt(r2);
                const double w = (r > c.re) ? 0.0 : c.re / r - 1.0;
                sw += w;
                sr2w += r2 * w;
            }
    c.n0 = sw;
    c.lambda0 = sr2w / sw;
    c.lapc = 2.0 * 3.0 / (c.lambda0 * c.n0);
    {
        // an FP32 copy of a coordinate inside the grid differs from it by at most
        // coord_max 2^-24, a difference of two copies by twice that per axis: the
        // radius is widened by the resulting bound on the distance (doubled) and
        // by the rounding of the FP32 test itself
        double coord_max = 0.0;
        for (int a = 0; a < 3; ++a)
            coord_max = std::fmax(coord_max, std::fmax(std::fabs(c.lo[a]), std::fabs(c.lo[a] + c.n[a] * c.cs)));
        const double R = c.re + 2.0 * std::sqrt(3.0) * std::ldexp(coord_max, -22);
        c.re2f = std::nextafter((float)(R * R * (1.0 + std::ldexp(1.0, -18))), 3.0e38f);
    }
    return SPH_OK;
}

size_t layout(MpsBufs &b, char *base, int64_t N, int32_t C, int width)
{
    Layout L;
    L.base = base;
    b.pos = L.take<dvec4>(N);
    b.vel = L.take<dvec4>(N);
    b.ustar = L.take<dvec4>(N);
    b.type = L.take<uint8_t>(N);
    b.moved = L.take<uint8_t>(N);
    b.P = L.take<double>(N);
    b.key = L.take<uint32_t>(N);
    b.count = L.take<uint32_t>((size_t)C + 1);
    b.cell_start = L.take<int32_t>((size_t)C + 2);
    b.active = L.take<int32_t>((size_t)C);
    b.scan_blocks = L.take<uint64_t>(((size_t)C + 1 + kScanTile - 1) / kScanTile);
    b.perm = L.take<int32_t>(N);
    b.ptmp = L.take<int32_t>(N);
    b.misc = L.take<int32_t>(16);
    b.spos = L.take<dvec4>(N);
    b.sposf = L.take<float4>(N);
    b.snd = L.take<double>(N);
    b.ssig = L.take<double>(N);
    b.surf = L.take<uint8_t>(N);
    b.ecnt = L.take<int32_t>(N);
    b.ecol = L.take<int32_t>((size_t)N * width);
    b.eval = L.take<double>((size_t)N * width);
    b.diag = L.take<double>(N);
    b.rhs = L.take<double>(N);
    b.x = L.take<double>(N);
    b.r = L.take<double>(N);
    b.p = L.take<double>(N);
    b.q = L.take<double>(N);
    b.part = L.take<double>(kCgBlocks);
    b.scal = L.take<double>(8);
    b.cgi = L.take<int32_t>(4);
    b.c = L.take<MpsConst>(1);
    return (L.off + 255) & ~(size_t)255;
}

}  // namespace

struct mps_s {
    mps_params p{};
    Geometry g;
    MpsBufs b{};
    cudaStream_t st = nullptr;
    std::string err;
    int64_t step = 0;
    int64_t last_it = 0;
    double last_res = 0.0;
    bool prof = false;
    cudaEvent_t ev[5] = {};
    double phase_ms[4] = {};
};

static int mfail(mps_t *s, int code, const std::string &m)
{
    if (s)
        s->err = m;
    return code;
}

#define MCK(call)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return mfail(s, SPH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static int warp_grid(int64_t items)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((items + 7) / 8, (int64_t)sm_count() * 16));
}

static int flat_grid(int64_t items)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, (int64_t)sm_count() * 8));
}

// Cell list of the current positions.
static void build_cells(mps_t *s)
{
    const int64_t N = s->g.N;
    const int32_t C = s->g.c.ncells;
    cudaMemsetAsync(s->b.count, 0, sizeof(uint32_t) * ((size_t)C + 1), s->st);
    k_mps_bin<<<flat_grid(N), 256, 0, s->st>>>(s->b, N);
    const int nb = (int)((C + 1 + kScanTile - 1) / kScanTile);
    k_mps_scan_reduce<<<nb, kScanThreads, 0, s->st>>>(s->b, C);
    k_mps_scan_blocks<<<1, 1024, 0, s->st>>>(s->b, nb);
    k_mps_scan_final<<<nb, kScanThreads, 0, s->st>>>(s->b, C);
    k_mps_scatter<<<flat_grid(N), 256, 0, s->st>>>(s->b, N);
    k_mps_sort<<<warp_grid(std::min<int64_t>(N, C)), 256, 0, s->st>>>(s->b);
}

static void mark(mps_t *s, int k)
{
    if (s->prof)
        cudaEventRecord(s->ev[k], s->st);
}

// Eqs. 17, 28-30 and 23 at the current positions (cell list built), then the
// CG solve; leaves the solution in b.x (sorted order).
static int solve_pressure(mps_t *s)
{
    const int64_t N = s->g.N;
    const int32_t Ns = (int32_t)N;
    k_mps_density<<<warp_grid(N), 256, 0, s->st>>>(s->b);
    k_mps_assemble<<<warp_grid(N), 256, 0, s->st>>>(s->b, Ns);
    mark(s, 2);
    k_cg_init<<<kCgBlocks, kCgThreads, 0, s->st>>>(s->b, Ns);
    k_cg_total<<<1, kCgThreads, 0, s->st>>>(s->b, 1, 1);
    int32_t cgi[2] = {0, 0};
    for (int it = 0; it < s->p.cg_max; it += kCgChunk) {
        for (int k = 0; k < kCgChunk; ++k) {
            k_cg_spmv<<<kCgBlocks, kCgThreads, 0, s->st>>>(s->b, Ns);
            k_cg_total<<<1, kCgThreads, 0, s->st>>>(s->b, 2, 0);
            k_cg_update<<<kCgBlocks, kCgThreads, 0, s->st>>>(s->b, Ns);
            k_cg_total<<<1, kCgThreads, 0, s->st>>>(s->b, 3, 0);
            k_cg_direction<<<kCgBlocks, kCgThreads, 0, s->st>>>(s->b, Ns);
        }
        MCK(cudaGetLastError());
        MCK(cudaMemcpyAsync(cgi, s->b.cgi, sizeof(cgi), cudaMemcpyDeviceToHost, s->st));
        MCK(cudaStreamSynchronize(s->st));
        if (cgi[1])
            break;
    }
    double scal[2];
    int32_t misc[4];
    MCK(cudaMemcpyAsync(scal, s->b.scal, sizeof(scal), cudaMemcpyDeviceToHost, s->st));
    MCK(cudaMemcpyAsync(misc, s->b.misc, sizeof(misc), cudaMemcpyDeviceToHost, s->st));
    MCK(cudaStreamSynchronize(s->st));
    s->last_it = cgi[0];
    s->last_res = scal[1] > 0.0 ? std::sqrt(scal[0] / scal[1]) : 0.0;
    if (misc[2] & ST_OVERFLOW)
        return mfail(s, SPH_ESTATE, "a row of the pressure system has more entries than row_width");
    if (!cgi[1] || !(s->last_res <= s->p.cg_tol))
        return mfail(s, SPH_EUNSTABLE, "the CG solve did not reach its tolerance within cg_max iterations");
    return SPH_OK;
}

extern "C" {

void mps_params_default(mps_params *p)
{
    std::memset(p, 0, sizeof(*p));
    p->size = sizeof(mps_params);
    p->layers = 3;
    p->re_factor = 2.1;
    p->nu = 1e-6;
    p->rho = 1000.0;
    p->g = 9.81;
    p->kappa_c = 1e-8;
    p->kappa_r = 0.01;
    p->beta1 = 0.98;
    p->varrho1 = 0.2;
    p->cg_tol = 1e-6;
    p->cg_max = 20000;
    p->row_width = 64;
}

int mps_workspace_size(const double tank[3], const double column[3], double l0, const mps_params *p, size_t *bytes)
{
    if (!bytes)
        return SPH_EINVAL;
    Geometry g;
    std::string err;
    int rc = geometry(tank, column, l0, 0.0, p, g, err);
    if (rc)
        return rc;
    MpsBufs b{};
    *bytes = layout(b, nullptr, g.N, g.c.ncells, p->row_width);
    return SPH_OK;
}

int mps_create(mps_t **out, const double tank[3], const double column[3], double l0, double dt, const mps_params *p,
               void *ws, size_t bytes, uintptr_t stream)
{
    if (!out)
        return SPH_EINVAL;
    *out = nullptr;
    if (!(dt > 0))
        return SPH_EINVAL;
    mps_t *s = new mps_t();
    int rc = geometry(tank, column, l0, dt, p, s->g, s->err);
    if (rc) {
        delete s;
        return rc;
    }
    s->p = *p;
    MpsBufs tmp{};
    const size_t need = layout(tmp, nullptr, s->g.N, s->g.c.ncells, p->row_width);
    if (!ws || bytes < need || ((uintptr_t)ws & 255)) {
        delete s;
        return ws && bytes < need ? SPH_ENOMEM : SPH_EINVAL;
    }
    layout(s->b, (char *)ws, s->g.N, s->g.c.ncells, p->row_width);
    s->st = (cudaStream_t)stream;
    // scene: fluid lattice, then wall and dummy layers (id order of mps.h)
    const int64_t N = s->g.N, L = p->layers;
    std::vector<dvec4> pos(N), vel(N, make_dvec4(0, 0, 0, 0));
    std::vector<uint8_t> type(N);
    const int64_t ncx = nint(column[0] / l0), ncy = nint(column[1] / l0), ncz = nint(column[2] / l0);
    const int64_t ntx = nint(tank[0] / l0), nty = nint(tank[1] / l0), ntz = nint(tank[2] / l0);
    int64_t id = 0;
    for (int64_t k = 0; k < ncz; ++k)
        for (int64_t j = 0; j < ncy; ++j)
            for (int64_t i = 0; i < ncx; ++i) {
                pos[id] = make_dvec4((i + 0.5) * l0, (j + 0.5) * l0, (k + 0.5) * l0, 0.0);
                type[id++] = MPS_FLUID;
            }
    for (int64_t k = -L; k < ntz; ++k)
        for (int64_t j = -L; j < nty + L; ++j)
            for (int64_t i = -L; i < ntx + L; ++i) {
                int64_t dx = i < 0 ? -1 - i : (i >= ntx ? i - ntx : -1);
                int64_t dy = j < 0 ? -1 - j : (j >= nty ? j - nty : -1);
                int64_t dz = k < 0 ? -1 - k : -1;
                int64_t layer = std::max(dx, std::max(dy, dz));
                if (layer < 0)
                    continue;
                pos[id] = make_dvec4((i + 0.5) * l0, (j + 0.5) * l0, (k + 0.5) * l0, 0.0);
                type[id++] = layer == 0 ? MPS_WALL : MPS_DUMMY;
            }
    auto up = [&](void *dst, const void *src, size_t n) {
        if (rc == SPH_OK && cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s->st) != cudaSuccess)
            rc = SPH_ECUDA;
    };
    up(s->b.pos, pos.data(), sizeof(dvec4) * N);
    up(s->b.vel, vel.data(), sizeof(dvec4) * N);
    up(s->b.ustar, vel.data(), sizeof(dvec4) * N);
    up(s->b.type, type.data(), N);
    up(s->b.c, &s->g.c, sizeof(MpsConst));
    if (rc == SPH_OK) {
        cudaMemsetAsync(s->b.P, 0, sizeof(double) * N, s->st);
        cudaMemsetAsync(s->b.moved, 0, N, s->st);
        cudaMemsetAsync(s->b.misc, 0, sizeof(int32_t) * 16, s->st);
        if (cudaStreamSynchronize(s->st) != cudaSuccess)
            rc = SPH_ECUDA;
    }
    if (rc) {
        delete s;
        return rc;
    }
    *out = s;
    return SPH_OK;
}

void mps_destroy(mps_t *s)
{
    if (!s)
        return;
    if (s->st)
        cudaStreamSynchronize(s->st);
    for (cudaEvent_t e : s->ev)
        if (e)
            cudaEventDestroy(e);
    delete s;
}

int mps_set_profiling(mps_t *s, int32_t on)
{
    if (!s)
        return SPH_EINVAL;
    if (on && !s->ev[0])
        for (cudaEvent_t &e : s->ev)
            MCK(cudaEventCreate(&e));
    s->prof = on != 0;
    return SPH_OK;
}

int mps_phase_times(mps_t *s, double ms[4])
{
    if (!s || !ms)
        return SPH_EINVAL;
    for (int q = 0; q < 4; ++q) {
        ms[q] = s->phase_ms[q];
        s->phase_ms[q] = 0.0;
    }
    return SPH_OK;
}

int mps_step(mps_t *s, int32_t nsteps)
{
    if (!s || nsteps < 0)
        return SPH_EINVAL;
    const int64_t N = s->g.N;
    for (int32_t k = 0; k < nsteps; ++k) {
        mark(s, 0);
        build_cells(s);
        k_mps_predict<<<warp_grid(N), 256, 0, s->st>>>(s->b);
        build_cells(s);
        mark(s, 1);
        int rc = solve_pressure(s);
        if (rc)
            return rc;
        mark(s, 3);
        k_mps_clamp<<<flat_grid(N), 256, 0, s->st>>>(s->b, (int32_t)N);
        k_mps_correct<<<warp_grid(N), 256, 0, s->st>>>(s->b);
        k_mps_finish<<<flat_grid(N), 256, 0, s->st>>>(s->b, N);
        mark(s, 4);
        MCK(cudaGetLastError());
        if (s->prof) {
            MCK(cudaEventSynchronize(s->ev[4]));
            for (int q = 0; q < 4; ++q) {
                float ms = 0.f;
                MCK(cudaEventElapsedTime(&ms, s->ev[q], s->ev[q + 1]));
                s->phase_ms[q] += ms;
            }
        }
        s->step += 1;
    }
    int32_t misc[4];
    MCK(cudaMemcpyAsync(misc, s->b.misc, sizeof(misc), cudaMemcpyDeviceToHost, s->st));
    MCK(cudaStreamSynchronize(s->st));
    if (misc[2] & ST_UNSTABLE)
        return mfail(s, SPH_EUNSTABLE, "non-finite velocity");
    return SPH_OK;
}

int mps_pressure(mps_t *s, double *P, double *nd, int32_t *surf, int64_t *iterations, double *residual)
{
    if (!s)
        return SPH_EINVAL;
    const int64_t N = s->g.N;
    build_cells(s);
    int rc = solve_pressure(s);
    if (rc)
        return rc;
    int32_t misc[4];
    std::vector<double> x(N), snd(N);
    std::vector<int32_t> perm(N);
    std::vector<uint8_t> sf(N);
    MCK(cudaMemcpyAsync(misc, s->b.misc, sizeof(misc), cudaMemcpyDeviceToHost, s->st));
    MCK(cudaStreamSynchronize(s->st));
    const int32_t n_in = misc[0];
    if (n_in > 0) {
        MCK(cudaMemcpyAsync(x.data(), s->b.x, sizeof(double) * n_in, cudaMemcpyDeviceToHost, s->st));
        MCK(cudaMemcpyAsync(snd.data(), s->b.snd, sizeof(double) * n_in, cudaMemcpyDeviceToHost, s->st));
        MCK(cudaMemcpyAsync(perm.data(), s->b.perm, sizeof(int32_t) * n_in, cudaMemcpyDeviceToHost, s->st));
        MCK(cudaMemcpyAsync(sf.data(), s->b.surf, n_in, cudaMemcpyDeviceToHost, s->st));
    }
    MCK(cudaStreamSynchronize(s->st));
    for (int64_t i = 0; i < N; ++i) {
        if (P)
            P[i] = 0.0;
        if (nd)
            nd[i] = 0.0;
        if (surf)
            surf[i] = 0;
    }
    for (int32_t k = 0; k < n_in; ++k) {
        const int32_t id = perm[k];
        if (P)
            P[id] = x[k];
        if (nd)
            nd[id] = snd[k];
        if (surf)
            surf[id] = sf[k];
    }
    if (iterations)
        *iterations = s->last_it;
    if (residual)
        *residual = s->last_res;
    return SPH_OK;
}

int mps_get_state(mps_t *s, double *r, double *u, double *P, int32_t *type, int64_t *step)
{
    if (!s)
        return SPH_EINVAL;
    const int64_t N = s->g.N;
    std::vector<dvec4> pos(N), vel(N);
    std::vector<double> pr(N);
    std::vector<uint8_t> ty(N);
    MCK(cudaMemcpyAsync(pos.data(), s->b.pos, sizeof(dvec4) * N, cudaMemcpyDeviceToHost, s->st));
    MCK(cudaMemcpyAsync(vel.data(), s->b.vel, sizeof(dvec4) * N, cudaMemcpyDeviceToHost, s->st));
    MCK(cudaMemcpyAsync(pr.data(), s->b.P, sizeof(double) * N, cudaMemcpyDeviceToHost, s->st));
    MCK(cudaMemcpyAsync(ty.data(), s->b.type, N, cudaMemcpyDeviceToHost, s->st));
    MCK(cudaStreamSynchronize(s->st));
    for (int64_t i = 0; i < N; ++i) {
        if (r) {
            r[3 * i] = pos[i].x;
            r[3 * i + 1] = pos[i].y;
            r[3 * i + 2] = pos[i].z;
        }
        if (u) {
            u[3 * i] = vel[i].x;
            u[3 * i + 1] = vel[i].y;
            u[3 * i + 2] = vel[i].z;
        }
        if (P)
            P[i] = pr[i];
        if (type)
            type[i] = ty[i];
    }
    if (step)
        *step = s->step;
    return SPH_OK;
}

int mps_set_state(mps_t *s, const double *r, const double *u)
{
    if (!s || !r || !u)
        return SPH_EINVAL;
    const int64_t N = s->g.N;
    std::vector<dvec4> pos(N), vel(N);
    const int64_t nf = s->g.nf;
    for (int64_t i = 0; i < N; ++i) {
        pos[i] = make_dvec4(r[3 * i], r[3 * i + 1], r[3 * i + 2], 0.0);
        vel[i] = i < nf ? make_dvec4(u[3 * i], u[3 * i + 1], u[3 * i + 2], 0.0) : make_dvec4(0, 0, 0, 0);
    }
    MCK(cudaMemcpyAsync(s->b.pos, pos.data(), sizeof(dvec4) * N, cudaMemcpyHostToDevice, s->st));
    MCK(cudaMemcpyAsync(s->b.vel, vel.data(), sizeof(dvec4) * N, cudaMemcpyHostToDevice, s->st));
    MCK(cudaStreamSynchronize(s->st));
    return SPH_OK;
}

int mps_last_solve(mps_t *s, int64_t *iterations, double *residual)
{
    if (!s)
        return SPH_EINVAL;
    if (iterations)
        *iterations = s->last_it;
    if (residual)
        *residual = s->last_res;
    return SPH_OK;
}

int mps_system_size(mps_t *s, int64_t out[2])
{
    if (!s || !out)
        return SPH_EINVAL;
    const int64_t N = s->g.N;
    std::vector<int32_t> cnt((size_t)N);
    MCK(cudaMemcpyAsync(cnt.data(), s->b.ecnt, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToHost, s->st));
    MCK(cudaStreamSynchronize(s->st));
    int64_t nnz = 0;
    for (int64_t i = 0; i < N; ++i)
        nnz += cnt[(size_t)i];
    out[0] = N;
    out[1] = nnz;
    return SPH_OK;
}

int mps_counts(const mps_t *s, int64_t out[4])
{
    if (!s || !out)
        return SPH_EINVAL;
    out[0] = s->g.nf;
    out[1] = s->g.nw;
    out[2] = s->g.ndum;
    out[3] = s->g.N;
    return SPH_OK;
}

const char *mps_last_error(const mps_t *s)
{
    if (!s)
        return "null handle";
    return s->err.c_str();
}

}  // extern "C"
