// Device helpers shared by the kernels: cell coordinates, the Tait equation of
// state (Eq. 8), the sound speed and small warp utilities.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace sph {

// Cell coordinates with the exact IEEE division (x - lo) / cs, as the
// definition of the grid states it; false when outside the grid.
__device__ __forceinline__ bool cell_coords_exact(const Inst &I, double x, double y, double z, int &cx, int &cy,
                                                  int &cz)
{
    double fx = floor((x - I.lo[0]) / I.cs);
    double fy = floor((y - I.lo[1]) / I.cs);
    double fz = floor((z - I.lo[2]) / I.cs);
    if (!(fx >= 0.0) || fx >= (double)I.n[0] || !(fy >= 0.0) || fy >= (double)I.n[1] || !(fz >= 0.0) ||
        fz >= (double)I.n[2])
        return false;
    cx = (int)fx;
    cy = (int)fy;
    cz = (int)fz;
    return true;
}

// The same with a multiplication by 1/cs (mixed form: cell assignment only
// has to be consistent with the FP32 offsets, which it always is).
__device__ __forceinline__ bool cell_coords_fast(const Inst &I, double x, double y, double z, int &cx, int &cy,
                                                 int &cz)
{
    double fx = floor((x - I.lo[0]) * I.inv_cs);
    double fy = floor((y - I.lo[1]) * I.inv_cs);
    double fz = floor((z - I.lo[2]) * I.inv_cs);
    if (!(fx >= 0.0) || fx >= (double)I.n[0] || !(fy >= 0.0) || fy >= (double)I.n[1] || !(fz >= 0.0) ||
        fz >= (double)I.n[2])
        return false;
    cx = (int)fx;
    cy = (int)fy;
    cz = (int)fz;
    return true;
}

// Streaming multiprocessors of the current device (queried once per device;
// grids of the memory-bound kernels are capped at a multiple of it).
inline int sm_count()
{
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64)
        dev = 0;
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
        cached[dev] = n;
    }
    return cached[dev];
}

__device__ __forceinline__ double pow7(double x)
{
    double x2 = x * x;
    return x2 * x2 * x2 * x;
}

// Eq. 8 in double.
__device__ __forceinline__ double tait_d(const Inst &I, double rho)
{
    double x = rho / I.rho0;
    double p = I.gamma == 7.0 ? pow7(x) : pow(x, I.gamma);
    return I.B * (p - 1.0);
}

// Eq. 8 in float from the density offset d = rho - rho0:
// (1 + x)^7 - 1 expanded by the binomial theorem, which keeps full relative
// precision for small x = d / rho0.
__device__ __forceinline__ float tait_f(const Inst &I, float d)
{
    float x = d * I.inv_rho0f;
    if (I.gamma == 7.0)
        return I.Bf * x * (7.f + x * (21.f + x * (35.f + x * (35.f + x * (21.f + x * (7.f + x))))));
    return I.Bf * expm1f(I.gammaf * log1pf(x));
}

// c_i: sqrt(dP/drho) of Eq. 8, c0 (rho/rho0)^((gamma-1)/2), or c0.
__device__ __forceinline__ double sound_d(const Inst &I, double rho)
{
    if (I.csound == SPH_CSOUND_CONSTANT)
        return I.c0;
    double x = rho / I.rho0;
    if (I.gamma == 7.0)
        return I.c0 * x * x * x;
    return I.c0 * pow(x, 0.5 * (I.gamma - 1.0));
}

// Max of a non-negative double through its bit pattern (order preserving for
// x >= 0; a NaN result propagates as the largest pattern).
__device__ __forceinline__ void atomic_max_pos(unsigned long long *addr, double x)
{
    atomicMax(addr, (unsigned long long)__double_as_longlong(x));
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Warp totals of K values (K a power of two, at most 32) by a value-splitting
// butterfly: at each of the first log2 K levels a lane keeps half of its
// values and adds its partner's copies of them, the remaining levels add the
// one value left, so K values cost K FP64 additions per lane (5 K for K
// separate butterflies).  On return v[k] of lane 0 holds the total of value k
// (other lanes: undefined).  The order of the additions is fixed.
template <int K>
__device__ __forceinline__ void warp_totals(double (&v)[K])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = K, o = 16; k > 1; k >>= 1, o >>= 1) {
        const bool upper = (lane & o) != 0;
        const int half = k >> 1;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const double keep = upper ? v[i + half] : v[i];
            const double send = upper ? v[i] : v[i + half];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = 16 / K; o > 0; o >>= 1)
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    // lane (32 / K) k holds the total of value k
    const double mine = v[0];
#pragma unroll
    for (int k = 0; k < K; ++k)
        v[k] = __shfl_sync(0xffffffffu, mine, k * (32 / K));
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Instance owning a global cell id (instances hold consecutive cell ranges).
__device__ __forceinline__ int inst_of_cell(const Inst *inst, int ninst, int32_t c)
{
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (inst[mid].cell_base <= c)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void decompose(const Inst &I, int32_t c, int &cx, int &cy, int &cz)
{
    int lc = c - I.cell_base;
    cx = lc % I.n[0];
    int t = lc / I.n[0];
    cy = t % I.n[1];
    cz = t / I.n[1];
}

}  // namespace sph
