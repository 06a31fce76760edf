// Device bodies of the time-stepping phases: the adaptive step (Eq. 15) and the
// Verlet scheme with a first-order step every Ns steps (Eqs. 9-14) fused with
// the rebinning of the moved particles.  The kernels of integrate.cu run them
// one launch per phase; the persistent kernel of persist.cu runs them between
// grid barriers.
#pragma once

#include "device.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// Eq. 15 is a min over fluid particles of sqrt(h/|f_i|) and h/(c0 + mu_i);
// both are decreasing in |f_i| and mu_i, so the reduction keeps the maxima of
// |f_i|^2 and mu_i per instance (exact, order independent) and the final
// formula runs once per instance in double.
// ---------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void dt_reduce_part(const Bufs &b, int ninst, int part, int nparts)
{
    const int32_t n_in = b.misc[0];
    const int32_t per = (n_in + nparts - 1) / nparts;
    const int32_t s_begin = part * per, s_end = min(n_in, s_begin + per);
    int cur = -1;
    double amax = 0.0, mmax = 0.0;
    for (int32_t s = s_begin + threadIdx.x; s < s_end; s += blockDim.x) {
        if (b.sflag[s] != T_FLUID)
            continue;
        double ax, ay, az, mu;
        if (MODE == SPH_FP64) {
            dvec4 d = reinterpret_cast<const dvec4 *>(b.deriv)[s];
            ax = d.x;
            ay = d.y;
            az = d.z;
            mu = reinterpret_cast<const double *>(b.mumax)[s];
        } else {
            float4 d = reinterpret_cast<const float4 *>(b.deriv)[s];
            ax = d.x;
            ay = d.y;
            az = d.z;
            mu = reinterpret_cast<const float *>(b.mumax)[s];
        }
        int k = inst_of_cell(b.inst, ninst, b.scell[s]);
        if (k != cur) {
            if (cur >= 0) {
                atomic_max_pos(&b.red[2 * cur], amax);
                atomic_max_pos(&b.red[2 * cur + 1], mmax);
            }
            cur = k;
            amax = 0.0;
            mmax = 0.0;
        }
        double a2 = ax * ax + ay * ay + az * az;
        // a NaN replaces the running max so that it reaches the status check
        amax = (a2 > amax || a2 != a2) ? a2 : amax;
        mmax = (mu > mmax || mu != mu) ? mu : mmax;
    }
    // block-level combine when every thread saw at most one instance, all the same
    const int lane = threadIdx.x & 31;
    int first = __shfl_sync(0xffffffffu, cur, 0);
    bool same = __all_sync(0xffffffffu, cur == first || cur < 0);
    if (same && first >= 0) {
        for (int o = 16; o > 0; o >>= 1) {
            double ya = __shfl_xor_sync(0xffffffffu, amax, o), ym = __shfl_xor_sync(0xffffffffu, mmax, o);
            amax = (ya > amax || ya != ya) ? ya : amax;
            mmax = (ym > mmax || ym != ym) ? ym : mmax;
        }
        if (lane == 0) {
            atomic_max_pos(&b.red[2 * first], amax);
            atomic_max_pos(&b.red[2 * first + 1], mmax);
        }
    } else if (cur >= 0) {
        atomic_max_pos(&b.red[2 * cur], amax);
        atomic_max_pos(&b.red[2 * cur + 1], mmax);
    }
}

// One block: dt of every instance, its clock, and the step counter.
__device__ __forceinline__ void dt_finalize_block(const Bufs &b, int ninst, int ns)
{
    for (int k = threadIdx.x; k < ninst; k += blockDim.x) {
        const Inst &I = b.inst[k];
        double a2 = __longlong_as_double((long long)b.red[2 * k]);
        double mu = __longlong_as_double((long long)b.red[2 * k + 1]);
        double fixed = b.dt_fixed[0];
        double dt;
        bool bad = (a2 != a2) || (mu != mu);
        if (fixed > 0.0) {
            dt = fixed;
        } else {
            double t1 = a2 > 0.0 ? sqrt(I.h / sqrt(a2)) : INFINITY;
            double t2 = I.h / (I.c0 + mu);
            dt = I.cfl * fmin(t1, t2);
            bad = bad || !(dt >= I.dt_min);
        }
        if (bad) {
            atomicOr(&b.misc[2], ST_UNSTABLE);
            dt = 0.0;  // freeze the instance; the host reports SPH_EUNSTABLE
        }
        b.dt[k] = dt;
        b.time[k] += dt;
        b.red[2 * k] = 0ull;
        b.red[2 * k + 1] = 0ull;
    }
    if (threadIdx.x == 0) {
        long long n = b.step[0];
        b.euler[0] = (n % ns) == 0;
        b.step[0] = n + 1;
    }
}

// ---------------------------------------------------------------------------
// Eqs. 9-14 for every in-domain particle (sorted order), writing the new state
// back in id order and binning the new position for the next step.  Fluid
// particles move; boundary particles update only their density (dynamic
// boundary conditions) and keep u = 0, except gate particles, which move at
// their prescribed velocity.  Out-of-domain particles stay frozen in the last
// bucket.
// ---------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void integrate_range(const Bufs &b, int64_t N, uint32_t C, int32_t thread0, int32_t stride)
{
    const int32_t n_in = b.misc[0];
    // neighbour lists: no binning here (a rebuild bins by itself); a particle
    // that moved more than s/2 since the last rebuild, or left the grid,
    // requests the next one
    const bool lists = b.lflag != nullptr;
    if (thread0 == 0 && N > n_in && !lists)
        atomicAdd(&b.count[C], (uint32_t)(N - n_in));
    const bool euler = b.euler[0] != 0;
    for (int32_t s = thread0; s < n_in; s += stride) {
        const int32_t id = b.perm[s];
        const int k = b.inst_of[id];
        const Inst &I = b.inst[k];
        const double dt = b.dt[k];
        const bool fluid = b.type[id] == T_FLUID;
        dvec4 p = b.pos[id];
        if (MODE == SPH_FP64) {
            const dvec4 d = reinterpret_cast<const dvec4 *>(b.deriv)[s];
            dvec4 *vel = reinterpret_cast<dvec4 *>(b.vel);
            dvec4 *velp = reinterpret_cast<dvec4 *>(b.velp);
            dvec4 v = vel[id], vp = velp[id];
            double rho_new = euler ? v.w + dt * d.w : vp.w + 2.0 * dt * d.w;
            if (fluid) {
                double ux = euler ? v.x + dt * d.x : vp.x + 2.0 * dt * d.x;
                double uy = euler ? v.y + dt * d.y : vp.y + 2.0 * dt * d.y;
                double uz = euler ? v.z + dt * d.z : vp.z + 2.0 * dt * d.z;
                double hdt2 = 0.5 * dt * dt;
                p.x = p.x + dt * v.x + hdt2 * d.x;
                p.y = p.y + dt * v.y + hdt2 * d.y;
                p.z = p.z + dt * v.z + hdt2 * d.z;
                b.pos[id] = p;
                velp[id] = v;
                vel[id] = make_dvec4(ux, uy, uz, rho_new);
            } else if (b.type[id] == T_GATE) {
                const double *gv = I.gate_v;
                p.x = p.x + dt * gv[0];
                p.y = p.y + dt * gv[1];
                p.z = p.z + dt * gv[2];
                b.pos[id] = p;
                velp[id] = make_dvec4(gv[0], gv[1], gv[2], v.w);
                vel[id] = make_dvec4(gv[0], gv[1], gv[2], rho_new);
            } else {
                velp[id] = make_dvec4(0.0, 0.0, 0.0, v.w);
                vel[id] = make_dvec4(0.0, 0.0, 0.0, rho_new);
            }
        } else {
            const float4 d = reinterpret_cast<const float4 *>(b.deriv)[s];
            float4 *vel = reinterpret_cast<float4 *>(b.vel);
            float4 *velp = reinterpret_cast<float4 *>(b.velp);
            float4 v = vel[id], vp = velp[id];
            const float dtf = (float)dt;
            float r_new = euler ? v.w + dtf * d.w : vp.w + 2.f * dtf * d.w;
            if (fluid) {
                float ux = euler ? v.x + dtf * d.x : vp.x + 2.f * dtf * d.x;
                float uy = euler ? v.y + dtf * d.y : vp.y + 2.f * dtf * d.y;
                float uz = euler ? v.z + dtf * d.z : vp.z + 2.f * dtf * d.z;
                double hdt2 = 0.5 * dt * dt;
                p.x = p.x + dt * (double)v.x + hdt2 * (double)d.x;
                p.y = p.y + dt * (double)v.y + hdt2 * (double)d.y;
                p.z = p.z + dt * (double)v.z + hdt2 * (double)d.z;
                b.pos[id] = p;
                velp[id] = v;
                vel[id] = make_float4(ux, uy, uz, r_new);
            } else if (b.type[id] == T_GATE) {
                const double *gv = I.gate_v;
                p.x = p.x + dt * gv[0];
                p.y = p.y + dt * gv[1];
                p.z = p.z + dt * gv[2];
                b.pos[id] = p;
                velp[id] = make_float4(I.gate_vf[0], I.gate_vf[1], I.gate_vf[2], v.w);
                vel[id] = make_float4(I.gate_vf[0], I.gate_vf[1], I.gate_vf[2], r_new);
            } else {
                velp[id] = make_float4(0.f, 0.f, 0.f, v.w);
                vel[id] = make_float4(0.f, 0.f, 0.f, r_new);
            }
        }
        int cx, cy, cz;
        uint32_t c = C;
        bool in = MODE == SPH_FP64 ? cell_coords_exact(I, p.x, p.y, p.z, cx, cy, cz)
                                   : cell_coords_fast(I, p.x, p.y, p.z, cx, cy, cz);
        if (lists) {
            const dvec4 q = b.xbuild[id];
            const double ex = p.x - q.x, ey = p.y - q.y, ez = p.z - q.z;
            if (!in || ex * ex + ey * ey + ez * ez > I.half_skin2)
                b.lflag[0] = 1;
            continue;
        }
        if (in)
            c = (uint32_t)(I.cell_base + (cz * I.n[1] + cy) * I.n[0] + cx);
        b.key[id] = c;
        atomicAdd(&b.count[c], 1u);
    }
}

}  // namespace sph
