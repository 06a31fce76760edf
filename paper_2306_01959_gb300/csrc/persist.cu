// Persistent form of the time loop: one cooperative launch advances every
// instance of a handle (a batch of dam breaks, e.g. an alpha sweep) by nsteps
// Verlet steps of the mixed form.  Each step runs the phases of the per-phase
// launches in the same order - pair pass (Eqs. 3-8), adaptive dt (Eq. 15),
// Verlet update with rebinning (Eqs. 9-14), cell scan, scatter, per-cell sort
// and gather - with a grid-wide barrier between phases instead of a kernel
// boundary.  The phase bodies are the ones the per-phase kernels run
// (pair_mixed.cuh, step.cuh, cells.cuh), so a persistent step computes what a
// launched step computes, bit for bit.
//
// The barrier is a counter in the workspace that every CTA increments once per
// barrier; a CTA waits until it reaches (barriers passed) x (CTAs).  Every wait
// is bounded: after spin_limit polls the CTA records ST_TIMEOUT in the device
// status (reported as SPH_ETIMEOUT) and returns, and every other CTA then runs
// out at its next barrier, so the launch always ends.  A cooperative launch
// guarantees that all CTAs are resident at once.
#include "cells.cuh"
#include "pair_mixed.cuh"
#include "step.cuh"

namespace sph {

namespace {

constexpr int kPersistWarps = 8;  // the pair pass's default shape: 8 warps,
constexpr int kPersistGroup = 4;  // 4 particles per warp

// Grid barrier with a bounded wait; returns false (for every thread of the
// CTA) when the wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned &target, long long spin_limit, int32_t *status,
                                             int *s_ok)
{
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(bar, 1u);
        long long polls = 0;
        while (*((volatile unsigned *)bar) < target) {
            if (++polls > spin_limit) {
                atomicOr(status, ST_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <bool DFS>
__global__ void __launch_bounds__(kPersistWarps * 32, 2)
    k_persistent_steps(Bufs b, int ninst, int nsteps, int ns, int kdiv, int max_stage, int64_t N, uint32_t C,
                       int ntiles, long long spin_limit)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ PairSmem S;
    __shared__ int s_ok;
    unsigned target = 0;
    const int tid = threadIdx.x;
    const int gthread = blockIdx.x * blockDim.x + tid, gstride = gridDim.x * blockDim.x;
    const int gwarp = gthread >> 5, nwarps = gstride >> 5;
    int32_t *status = &b.misc[2];
#define SPH_BARRIER()                                                       \
    if (!grid_barrier(b.bar, target, spin_limit, status, &s_ok))            \
        return;
    for (int step = 0; step < nsteps; ++step) {
        pair_mixed_body<kPersistWarps, kPersistGroup, true, false, DFS>(b, ninst, kdiv, max_stage, dyn, S);
        SPH_BARRIER();
        dt_reduce_part<SPH_MIXED>(b, ninst, blockIdx.x, gridDim.x);
        SPH_BARRIER();
        if (blockIdx.x == 0) {
            dt_finalize_block(b, ninst, ns);
            if (tid == 0)
                b.misc[3] = 0;  // the pair pass's work queue, for the next step
        }
        SPH_BARRIER();
        integrate_range<SPH_MIXED>(b, N, C, gthread, gstride);
        SPH_BARRIER();
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
            scan_reduce_tile(b.count, b.scan_blocks, C, t);
        SPH_BARRIER();
        if (blockIdx.x == 0)
            scan_blocks_block(b.scan_blocks, ntiles);
        SPH_BARRIER();
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
            scan_final_tile(b.count, b.scan_blocks, b.cell_start, b.active, b.misc, C, t);
        SPH_BARRIER();
        scatter_range(b.key, b.count, b.cell_start, b.ptmp, b.misc, N, gthread, gstride);
        SPH_BARRIER();
        // the sort keys use the pair pass's staging memory, idle in this phase
        sort_reorder_warps<SPH_MIXED>(b, ninst, reinterpret_cast<uint64_t *>(dyn) + (tid >> 5) * kSortCap, gwarp,
                                      nwarps);
        SPH_BARRIER();
    }
#undef SPH_BARRIER
}

template <bool DFS>
cudaError_t launch_typed(const Bufs &b, int ninst, int nsteps, int ns, int cell_div, int64_t N, int32_t C,
                         long long spin_limit, cudaStream_t st)
{
    const int max_stage = mixed_max_stage(cell_div);
    const size_t dyn = mixed_dyn_smem(max_stage, kPersistWarps, kPersistGroup);
    static size_t dyn_set = 0;
    cudaError_t e;
    if (dyn > dyn_set) {
        e = cudaFuncSetAttribute(k_persistent_steps<DFS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess)
            return e;
        dyn_set = dyn;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent_steps<DFS>, kPersistWarps * 32, dyn);
    if (e != cudaSuccess)
        return e;
    if (per_sm < 1)
        return cudaErrorLaunchOutOfResources;
    const int grid = per_sm * sm_count();
    int ntiles = (int)((C + 1 + kScanTile - 1) / kScanTile);
    uint32_t Cu = (uint32_t)C;
    void *args[] = {(void *)&b, &ninst, &nsteps, &ns, &cell_div, (void *)&max_stage, &N, &Cu, &ntiles, &spin_limit};
    e = cudaMemsetAsync(b.bar, 0, sizeof(unsigned), st);
    if (e != cudaSuccess)
        return e;
    e = cudaMemsetAsync(b.misc + 3, 0, sizeof(int32_t), st);
    if (e != cudaSuccess)
        return e;
    return cudaLaunchCooperativeKernel((const void *)k_persistent_steps<DFS>, grid, kPersistWarps * 32, args, dyn, st);
}

}  // namespace

cudaError_t launch_persistent_steps(const Bufs &b, int32_t ninst, int32_t nsteps, int32_t ns, int32_t cell_div,
                                    int32_t delta_mode, int64_t N, int32_t C, long long spin_limit, cudaStream_t st)
{
    if (delta_mode == SPH_DELTA_FULL_SUPPORT)
        return launch_typed<true>(b, ninst, nsteps, ns, cell_div, N, C, spin_limit, st);
    return launch_typed<false>(b, ninst, nsteps, ns, cell_div, N, C, spin_limit, st);
}

}  // namespace sph
