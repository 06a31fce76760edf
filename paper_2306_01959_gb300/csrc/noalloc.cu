// Allocation-free variant of the adaptive time-step reduction (Eq. 15).
//
// Some callers cannot call cudaMalloc: plug-ins living inside an application
// whose caching allocator already owns the device memory, real-time loops that
// must not risk the implicit device synchronisation of an allocation, and code
// whose device-memory budget is fixed before it starts.  For them,
// sph_cfl_dt_noalloc computes the step from caller-provided device arrays and
// keeps its only scratch (per-block partial maxima) in a fixed, file-scope
// device array.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "sph.h"

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocItems = 32;  // elements per thread and block tile
constexpr int64_t kNoAllocTile = (int64_t)kNoAllocThreads * kNoAllocItems;
constexpr int kNoAllocMaxBlocks = 2048;  // tiles: at most 2048 x 8192 = 16,777,216 particles
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: [block][0] max |f|^2, [block][1]
// max mu.  Each call overwrites the slots of its own blocks before reading
// them, so nothing has to start at zero.  32 KB per device, held until exit.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * 2];

// The device address of g_noalloc_partials belongs to one CUDA context (a
// module is loaded once per context).  It is looked up with the caller's
// context current and remembered per context, for calls that cannot look it up.
typedef int (*CtxGetCurrentFn)(void **);
struct ScratchAddr {
    void *ctx;
    double *addr;
};
std::mutex g_setup_mutex;
CtxGetCurrentFn g_ctx_get_current = nullptr;
bool g_ctx_fn_tried = false;
ScratchAddr g_addr[kMaxDevices] = {};
int g_naddr = 0;

// Current context handle (driver API, reached through the runtime), or nullptr.
void *current_context()
{
    if (!g_ctx_fn_tried) {
        g_ctx_fn_tried = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    }
    void *ctx = nullptr;
    if (!g_ctx_get_current || g_ctx_get_current(&ctx) != 0)
        return nullptr;
    return ctx;
}

// Scratch address in the current context.  Looked up afresh (and remembered)
// whenever the stream is not being captured, so that a context created anew
// (after cudaDeviceReset, or a caller's own context) gets its own address; a
// call on a capturing stream reuses the address remembered for its context.
double *scratch_address(cudaStream_t st)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone;
    void *ctx = current_context();
    int k = 0;
    while (k < g_naddr && g_addr[k].ctx != ctx)
        ++k;
    if (capturing)
        return (ctx && k < g_naddr) ? g_addr[k].addr : nullptr;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p)
        return nullptr;
    ctx = current_context();  // the lookup may have made the primary context current
    k = 0;
    while (k < g_naddr && g_addr[k].ctx != ctx)
        ++k;
    if (ctx && k == g_naddr && g_naddr < kMaxDevices)
        g_addr[g_naddr++] = ScratchAddr{ctx, nullptr};
    if (ctx && k < g_naddr)
        g_addr[k].addr = static_cast<double *>(p);
    return static_cast<double *>(p);
}

__global__ void k_noalloc_partials(const double *__restrict__ acc, const double *__restrict__ mumax,
                                   const int32_t *__restrict__ type, int64_t n, double *__restrict__ partials)
{
    __shared__ double sa[kNoAllocThreads / 32], sm[kNoAllocThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kNoAllocTile;
    double amax = 0.0, mmax = 0.0;
    for (int k = 0; k < kNoAllocItems; ++k) {
        const int64_t i = base + (int64_t)k * kNoAllocThreads + threadIdx.x;
        if (i >= n || (type && type[i] != SPH_FLUID))
            continue;
        const double ax = acc[3 * i], ay = acc[3 * i + 1], az = acc[3 * i + 2];
        const double a2 = ax * ax + ay * ay + az * az;
        const double mu = mumax[i];
        amax = (a2 > amax || a2 != a2) ? a2 : amax;  // a NaN is carried to the result
        mmax = (mu > mmax || mu != mu) ? mu : mmax;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ya = __shfl_xor_sync(0xffffffffu, amax, o), ym = __shfl_xor_sync(0xffffffffu, mmax, o);
        amax = (ya > amax || ya != ya) ? ya : amax;
        mmax = (ym > mmax || ym != ym) ? ym : mmax;
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sa[w] = amax;
        sm[w] = mmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kNoAllocThreads / 32; ++k) {
            amax = (sa[k] > amax || sa[k] != sa[k]) ? sa[k] : amax;
            mmax = (sm[k] > mmax || sm[k] != sm[k]) ? sm[k] : mmax;
        }
        partials[2 * blockIdx.x] = amax;
        partials[2 * blockIdx.x + 1] = mmax;
    }
}

__global__ void k_noalloc_finish(const double *__restrict__ partials, int nblocks, double h, double c0, double cfl,
                                 double *__restrict__ dt_out)
{
    if (threadIdx.x != 0)
        return;
    double amax = 0.0, mmax = 0.0;
    for (int k = 0; k < nblocks; ++k) {
        const double a = partials[2 * k], m = partials[2 * k + 1];
        amax = (a > amax || a != a) ? a : amax;
        mmax = (m > mmax || m != m) ? m : mmax;
    }
    // Eq. 15: Cr min(min_i sqrt(h/|f_i|), min_i h/(c0 + max_j mu_ij)); both
    // terms decrease with |f_i| and mu_i, so the maxima give the minima.
    const double t1 = amax > 0.0 ? sqrt(h / sqrt(amax)) : INFINITY;
    const double t2 = h / (c0 + mmax);
    dt_out[0] = cfl * fmin(t1, t2);
    if (amax != amax || mmax != mmax)
        dt_out[0] = amax + mmax;  // NaN in, NaN out
}

}  // namespace

extern "C" int sph_cfl_dt_noalloc(const double *acc, const double *mumax, const int32_t *type, int64_t n,
                                  double h, double c0, double cfl, double *dt_out, uintptr_t cuda_stream)
{
    if (!acc || !mumax || !dt_out || n < 1 || !(h > 0.0) || !(c0 > 0.0) || !(cfl > 0.0))
        return SPH_EINVAL;
    if (n > kNoAllocTile * kNoAllocMaxBlocks)
        return SPH_EINVAL;  // beyond the fixed scratch: 16,777,216 particles at most
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // The host-side name of a __device__ array is not a device address: the
    // address is looked up in the current context (see scratch_address).
    double *partials = scratch_address(st);
    if (!partials)
        return SPH_ECUDA;
    const int nblocks = (int)((n + kNoAllocTile - 1) / kNoAllocTile);
    k_noalloc_partials<<<nblocks, kNoAllocThreads, 0, st>>>(acc, mumax, type, n, partials);
    k_noalloc_finish<<<1, 32, 0, st>>>(partials, nblocks, h, c0, cfl, dt_out);
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ECUDA;
}
