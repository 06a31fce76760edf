// Probes on the current state, accumulated in double:
//  - Eq. 33: Shepard-averaged pressure P_a = sum_b P_b W_ab / sum_b W_ab over
//    fluid particles b within 2h of the point (0 when there is none);
//  - wave height: the largest level z = k dp/4 at which the kernel-summed
//    fluid density sum_b m W(|p - r_b|) reaches rho0/2 (the paper reports
//    wave heights without stating how they are measured; this is the reading).
// One warp per point (pressure) or per (point, level) (wave height); lanes
// sweep the rows of cells around the point.
#include "device.cuh"

namespace sph {

template <int MODE>
__device__ __forceinline__ void canon(const Bufs &b, const Inst &I, int32_t id, double &x, double &y, double &z,
                                      double &rho)
{
    dvec4 p = b.pos[id];
    x = p.x;
    y = p.y;
    z = p.z;
    if (MODE == SPH_FP64)
        rho = reinterpret_cast<const dvec4 *>(b.vel)[id].w;
    else
        rho = I.rho0 + (double)reinterpret_cast<const float4 *>(b.vel)[id].w;
}

__device__ __forceinline__ double kernel_w(const Inst &I, double r)
{
    double q = r / I.h;
    if (q >= 2.0)
        return 0.0;
    double t = 1.0 - 0.5 * q;
    return I.kW * t * t * t * t * (2.0 * q + 1.0);
}

// Sum over fluid particles near point (px,py,pz): s0 = sum W, s1 = sum P W
// (want_p) or s0 = sum m W.
template <int MODE>
__device__ void point_sums(const Bufs &b, const Inst &I, int kdiv, double px, double py, double pz, bool want_p,
                           double &s0, double &s1)
{
    const int lane = threadIdx.x & 31;
    // cell of the point, clamped so that far-away points convert safely
    auto cell = [&](double v, double lo, int n) {
        double f = floor((v - lo) / I.cs);
        f = fmin(fmax(f, -(double)kdiv - 1.0), (double)n + kdiv);
        return (int)f;
    };
    const int fx = cell(px, I.lo[0], I.n[0]), fy = cell(py, I.lo[1], I.n[1]), fz = cell(pz, I.lo[2], I.n[2]);
    s0 = 0.0;
    s1 = 0.0;
    for (int z = max(fz - kdiv, 0); z <= min(fz + kdiv, I.n[2] - 1); ++z)
        for (int y = max(fy - kdiv, 0); y <= min(fy + kdiv, I.n[1] - 1); ++y) {
            int x0 = max(fx - kdiv, 0), x1 = min(fx + kdiv, I.n[0] - 1);
            if (x0 > x1)
                continue;
            int32_t row = I.cell_base + (z * I.n[1] + y) * I.n[0];
            int32_t s_0 = b.cell_start[row + x0], s_1 = b.cell_start[row + x1 + 1];
            for (int32_t j = s_0 + lane; j < s_1; j += 32) {
                if (b.sflag[j] != T_FLUID)
                    continue;
                double x, y2, z2, rho;
                canon<MODE>(b, I, b.perm[j], x, y2, z2, rho);
                double dx = x - px, dy = y2 - py, dz = z2 - pz;
                double w = kernel_w(I, sqrt(dx * dx + dy * dy + dz * dz));
                if (want_p) {
                    s0 += w;
                    s1 += tait_d(I, rho) * w;
                } else {
                    s0 += I.mass * w;
                }
            }
        }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
}

template <int MODE>
__global__ void k_probe_pressure(Bufs b, int inst, int kdiv, int npts)
{
    const Inst &I = b.inst[inst];
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < npts; a += nwarps) {
        double s0, s1;
        point_sums<MODE>(b, I, kdiv, b.probe_in[3 * a], b.probe_in[3 * a + 1], b.probe_in[3 * a + 2], true, s0, s1);
        if ((threadIdx.x & 31) == 0)
            b.probe_out[a] = s0 > 0.0 ? s1 / s0 : 0.0;
    }
}

template <int MODE>
__global__ void k_probe_wave(Bufs b, int inst, int kdiv, int npts, int nlev)
{
    const Inst &I = b.inst[inst];
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const double dz = 0.25 * I.dp;
    const int64_t total = (int64_t)npts * nlev;
    for (int64_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nwarps) {
        int a = (int)(w / nlev), k = (int)(w % nlev);
        double s0, s1;
        point_sums<MODE>(b, I, kdiv, b.probe_in[2 * a], b.probe_in[2 * a + 1], k * dz, false, s0, s1);
        if ((threadIdx.x & 31) == 0 && s0 >= 0.5 * I.rho0)
            atomicMax(&b.probe_k[a], k);
    }
}

void launch_probe_pressure(const Bufs &b, int mode, int32_t inst, int32_t ninst, int32_t cell_div, int32_t npts,
                           cudaStream_t st)
{
    (void)ninst;
    int blocks = std::max(1, std::min((npts + 7) / 8, 1024));
    if (mode == SPH_FP64)
        k_probe_pressure<SPH_FP64><<<blocks, 256, 0, st>>>(b, inst, cell_div, npts);
    else
        k_probe_pressure<SPH_MIXED><<<blocks, 256, 0, st>>>(b, inst, cell_div, npts);
}

void launch_probe_wave(const Bufs &b, int mode, int32_t inst, int32_t ninst, int32_t cell_div, int32_t npts,
                       int32_t nlev, cudaStream_t st)
{
    (void)ninst;
    int64_t work = (int64_t)npts * nlev;
    int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((work + 7) / 8, 4096));
    if (mode == SPH_FP64)
        k_probe_wave<SPH_FP64><<<blocks, 256, 0, st>>>(b, inst, cell_div, npts, nlev);
    else
        k_probe_wave<SPH_MIXED><<<blocks, 256, 0, st>>>(b, inst, cell_div, npts, nlev);
}

}  // namespace sph
