// Adaptive time step (Eq. 15), the Verlet scheme with a first-order step every
// Ns steps (Eqs. 9-14) fused with the rebinning of the moved particles, and the
// FP64 diagnostics.
#include "step.cuh"

namespace sph {

// One launch per phase; the bodies live in step.cuh.
template <int MODE>
__global__ void k_dt_reduce(Bufs b, int ninst)
{
    dt_reduce_part<MODE>(b, ninst, blockIdx.x, gridDim.x);
}

__global__ void k_dt_finalize(Bufs b, int ninst, int ns) { dt_finalize_block(b, ninst, ns); }

void launch_dt(const Bufs &b, int mode, int64_t N, int32_t ninst, int32_t ns, cudaStream_t st)
{
    int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((N + 2047) / 2048, sm_count() * 4));
    if (mode == SPH_FP64)
        k_dt_reduce<SPH_FP64><<<blocks, 256, 0, st>>>(b, ninst);
    else
        k_dt_reduce<SPH_MIXED><<<blocks, 256, 0, st>>>(b, ninst);
    k_dt_finalize<<<1, 256, 0, st>>>(b, ninst, ns);
}

template <int MODE>
__global__ void k_integrate(Bufs b, int64_t N, uint32_t C)
{
    integrate_range<MODE>(b, N, C, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

void launch_integrate(const Bufs &b, int mode, int64_t N, int32_t C, int32_t ninst, cudaStream_t st)
{
    (void)ninst;
    int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, sm_count() * 8));
    if (mode == SPH_FP64)
        k_integrate<SPH_FP64><<<blocks, 256, 0, st>>>(b, N, (uint32_t)C);
    else
        k_integrate<SPH_MIXED><<<blocks, 256, 0, st>>>(b, N, (uint32_t)C);
}

// ---------------------------------------------------------------------------
// Symplectic position-Verlet predictor-corrector (the integrator the paper
// leaves to the literature cited after Eq. 15; two pair passes per step).
// Predictor, half a step from level n with the level-n derivatives:
//   rho' = rho + dt/2 Drho,  u' = u + dt/2 Du,  r' = r + dt/2 u,
// level n kept in velp.  Corrector, with the derivatives at the predicted
// state: u'' = u + dt Du' (a full kick from level n), r'' = r' + dt/2 u'',
// rho'' = rho (2 - e)/(2 + e), e = -dt Drho'/rho'.  Boundary particles update
// density only and keep u = 0 (gate particles: their prescribed velocity, half
// a step of it in each kernel).  Both kernels rebin the moved particles like
// k_integrate; a particle out of the grid after the predictor keeps its
// predicted state.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rebin_particle(const Bufs &b, const Inst &I, int32_t id, const dvec4 p,
                                               uint32_t C, bool exact)
{
    int cx, cy, cz;
    uint32_t c = C;
    const bool in = exact ? cell_coords_exact(I, p.x, p.y, p.z, cx, cy, cz)
                          : cell_coords_fast(I, p.x, p.y, p.z, cx, cy, cz);
    if (in)
        c = (uint32_t)(I.cell_base + (cz * I.n[1] + cy) * I.n[0] + cx);
    b.key[id] = c;
    atomicAdd(&b.count[c], 1u);
}

template <int MODE>
__global__ void k_predict(Bufs b, int64_t N, uint32_t C)
{
    const int32_t n_in = b.misc[0];
    if (blockIdx.x == 0 && threadIdx.x == 0 && N > n_in)
        atomicAdd(&b.count[C], (uint32_t)(N - n_in));
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_in; s += gridDim.x * blockDim.x) {
        const int32_t id = b.perm[s];
        const Inst &I = b.inst[b.inst_of[id]];
        const double dt = b.dt[b.inst_of[id]], hdt = 0.5 * dt;
        const bool fluid = b.type[id] == T_FLUID;
        dvec4 p = b.pos[id];
        if (MODE == SPH_FP64) {
            const dvec4 d = reinterpret_cast<const dvec4 *>(b.deriv)[s];
            dvec4 *vel = reinterpret_cast<dvec4 *>(b.vel);
            const dvec4 v = vel[id];
            reinterpret_cast<dvec4 *>(b.velp)[id] = v;
            const double rho_h = v.w + hdt * d.w;
            if (fluid) {
                p.x = p.x + hdt * v.x;
                p.y = p.y + hdt * v.y;
                p.z = p.z + hdt * v.z;
                b.pos[id] = p;
                vel[id] = make_dvec4(v.x + hdt * d.x, v.y + hdt * d.y, v.z + hdt * d.z, rho_h);
            } else if (b.type[id] == T_GATE) {
                const double *gv = I.gate_v;
                p.x = p.x + hdt * gv[0];
                p.y = p.y + hdt * gv[1];
                p.z = p.z + hdt * gv[2];
                b.pos[id] = p;
                vel[id] = make_dvec4(gv[0], gv[1], gv[2], rho_h);
            } else {
                vel[id] = make_dvec4(0.0, 0.0, 0.0, rho_h);
            }
        } else {
            const float4 d = reinterpret_cast<const float4 *>(b.deriv)[s];
            float4 *vel = reinterpret_cast<float4 *>(b.vel);
            const float4 v = vel[id];
            reinterpret_cast<float4 *>(b.velp)[id] = v;
            const float hf = (float)hdt;
            const float drho_h = v.w + hf * d.w;  // density offset rho - rho0
            if (fluid) {
                p.x = p.x + hdt * (double)v.x;
                p.y = p.y + hdt * (double)v.y;
                p.z = p.z + hdt * (double)v.z;
                b.pos[id] = p;
                vel[id] = make_float4(v.x + hf * d.x, v.y + hf * d.y, v.z + hf * d.z, drho_h);
            } else if (b.type[id] == T_GATE) {
                const double *gv = I.gate_v;
                p.x = p.x + hdt * gv[0];
                p.y = p.y + hdt * gv[1];
                p.z = p.z + hdt * gv[2];
                b.pos[id] = p;
                vel[id] = make_float4(I.gate_vf[0], I.gate_vf[1], I.gate_vf[2], drho_h);
            } else {
                vel[id] = make_float4(0.f, 0.f, 0.f, drho_h);
            }
        }
        rebin_particle(b, I, id, p, C, MODE == SPH_FP64);
    }
}

template <int MODE>
__global__ void k_correct(Bufs b, int64_t N, uint32_t C)
{
    const int32_t n_in = b.misc[0];
    if (blockIdx.x == 0 && threadIdx.x == 0 && N > n_in)
        atomicAdd(&b.count[C], (uint32_t)(N - n_in));
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_in; s += gridDim.x * blockDim.x) {
        const int32_t id = b.perm[s];
        const Inst &I = b.inst[b.inst_of[id]];
        const double dt = b.dt[b.inst_of[id]], hdt = 0.5 * dt;
        const bool fluid = b.type[id] == T_FLUID;
        dvec4 p = b.pos[id];
        if (MODE == SPH_FP64) {
            const dvec4 d = reinterpret_cast<const dvec4 *>(b.deriv)[s];
            dvec4 *vel = reinterpret_cast<dvec4 *>(b.vel);
            const dvec4 v = vel[id], vn = reinterpret_cast<const dvec4 *>(b.velp)[id];
            const double e = -(d.w / v.w) * dt;
            const double rho_new = vn.w * (2.0 - e) / (2.0 + e);
            if (fluid) {
                const double ux = vn.x + dt * d.x, uy = vn.y + dt * d.y, uz = vn.z + dt * d.z;
                p.x = p.x + hdt * ux;
                p.y = p.y + hdt * uy;
                p.z = p.z + hdt * uz;
                b.pos[id] = p;
                vel[id] = make_dvec4(ux, uy, uz, rho_new);
            } else if (b.type[id] == T_GATE) {
                const double *gv = I.gate_v;
                p.x = p.x + hdt * gv[0];
                p.y = p.y + hdt * gv[1];
                p.z = p.z + hdt * gv[2];
                b.pos[id] = p;
                vel[id] = make_dvec4(gv[0], gv[1], gv[2], rho_new);
            } else {
                vel[id] = make_dvec4(0.0, 0.0, 0.0, rho_new);
            }
        } else {
            const float4 d = reinterpret_cast<const float4 *>(b.deriv)[s];
            float4 *vel = reinterpret_cast<float4 *>(b.vel);
            const float4 v = vel[id], vn = reinterpret_cast<const float4 *>(b.velp)[id];
            const float dtf = (float)dt;
            const float e = -dtf * d.w / (I.rho0f + v.w);
            // rho0 + d'' = (rho0 + dn)(2 - e)/(2 + e), written for the offset d''
            // so that no rho0-sized terms cancel
            const float drho_new = (2.f * vn.w - e * (2.f * I.rho0f + vn.w)) / (2.f + e);
            if (fluid) {
                const float ux = vn.x + dtf * d.x, uy = vn.y + dtf * d.y, uz = vn.z + dtf * d.z;
                p.x = p.x + hdt * (double)ux;
                p.y = p.y + hdt * (double)uy;
                p.z = p.z + hdt * (double)uz;
                b.pos[id] = p;
                vel[id] = make_float4(ux, uy, uz, drho_new);
            } else if (b.type[id] == T_GATE) {
                const double *gv = I.gate_v;
                p.x = p.x + hdt * gv[0];
                p.y = p.y + hdt * gv[1];
                p.z = p.z + hdt * gv[2];
                b.pos[id] = p;
                vel[id] = make_float4(I.gate_vf[0], I.gate_vf[1], I.gate_vf[2], drho_new);
            } else {
                vel[id] = make_float4(0.f, 0.f, 0.f, drho_new);
            }
        }
        rebin_particle(b, I, id, p, C, MODE == SPH_FP64);
    }
}

void launch_predict(const Bufs &b, int mode, int64_t N, int32_t C, cudaStream_t st)
{
    int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, sm_count() * 8));
    if (mode == SPH_FP64)
        k_predict<SPH_FP64><<<blocks, 256, 0, st>>>(b, N, (uint32_t)C);
    else
        k_predict<SPH_MIXED><<<blocks, 256, 0, st>>>(b, N, (uint32_t)C);
}

void launch_correct(const Bufs &b, int mode, int64_t N, int32_t C, cudaStream_t st)
{
    int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, sm_count() * 8));
    if (mode == SPH_FP64)
        k_correct<SPH_FP64><<<blocks, 256, 0, st>>>(b, N, (uint32_t)C);
    else
        k_correct<SPH_MIXED><<<blocks, 256, 0, st>>>(b, N, (uint32_t)C);
}

// ---------------------------------------------------------------------------
// Diagnostics of one instance in double (canonical state, id order):
// mass, fluid volume, fluid momentum, kinetic, potential and internal energy
// (de/drho = P/rho^2 integrated from Eq. 8 with e(rho0) = 0), out-of-domain
// count, fluid count.  Two stages with a fixed summation order.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void k_diag(Bufs b, int inst, uint32_t C)
{
    __shared__ double part[8][10];
    const Inst &I = b.inst[inst];
    double acc[10];
#pragma unroll
    for (int q = 0; q < 10; ++q)
        acc[q] = 0.0;
    const double m = I.mass, gm1 = I.gamma - 1.0;
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < I.np; t += gridDim.x * blockDim.x) {
        const int32_t id = I.pbase + t;
        if (b.key[id] == C) {
            acc[8] += 1.0;
            continue;
        }
        acc[0] += m;
        if (b.type[id] != T_FLUID)
            continue;
        double ux, uy, uz, rho;
        if (MODE == SPH_FP64) {
            dvec4 v = reinterpret_cast<const dvec4 *>(b.vel)[id];
            ux = v.x;
            uy = v.y;
            uz = v.z;
            rho = v.w;
        } else {
            float4 v = reinterpret_cast<const float4 *>(b.vel)[id];
            ux = v.x;
            uy = v.y;
            uz = v.z;
            rho = I.rho0 + (double)v.w;
        }
        double x = rho / I.rho0;
        acc[1] += m / rho;
        acc[2] += m * ux;
        acc[3] += m * uy;
        acc[4] += m * uz;
        acc[5] += 0.5 * m * (ux * ux + uy * uy + uz * uz);
        acc[6] += m * I.g * b.pos[id].z;
        acc[7] += m * (I.B / I.rho0 * (pow(x, gm1) / gm1 + 1.0 / x - I.gamma / gm1));
        acc[9] += 1.0;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        double v = warp_sum(acc[q]);
        if (lane == 0)
            part[w][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k)
            s += part[k][threadIdx.x];
        b.diag[blockIdx.x * 10 + threadIdx.x] = s;
    }
}

__global__ void k_diag_final(const double *part, int nb, double *out)
{
    if (threadIdx.x < 10) {
        double s = 0.0;
        for (int k = 0; k < nb; ++k)
            s += part[k * 10 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

void launch_diagnostics(const Bufs &b, int mode, int32_t inst, int32_t C, cudaStream_t st)
{
    if (mode == SPH_FP64)
        k_diag<SPH_FP64><<<kDiagBlocks, 256, 0, st>>>(b, inst, (uint32_t)C);
    else
        k_diag<SPH_MIXED><<<kDiagBlocks, 256, 0, st>>>(b, inst, (uint32_t)C);
    k_diag_final<<<1, 32, 0, st>>>(b.diag, kDiagBlocks, b.probe_out);
}

}  // namespace sph
