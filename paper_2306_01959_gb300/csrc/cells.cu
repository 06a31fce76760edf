// Cell-linked neighbour structure: binning, per-cell counts, a scan of the
// counts into cell starts and the list of non-empty cells, a counting-sort
// scatter, and a per-cell sort by particle id fused with the gather of the
// sorted particle data (including the Tait pressure, Eq. 8).
//
// The resulting order is ascending (cell, id) for every in-domain particle;
// out-of-domain particles fill the bucket after the last cell in arbitrary
// order and take no further part.
#include "cells.cuh"

namespace sph {

// With neighbour lists, `gate` is the rebuild request: these kernels run only
// when it is set (steps that reuse the lists keep the last sorted order); a
// null gate always runs.
__device__ __forceinline__ bool gated_off(const int32_t *gate) { return gate && *gate == 0; }

// ---------------------------------------------------------------------------
// Binning of the canonical state (used at creation, after a state load and,
// with neighbour lists, at a rebuild).
// ---------------------------------------------------------------------------
__global__ void k_bin(const dvec4 *__restrict__ pos, const uint16_t *__restrict__ inst_of,
                      const Inst *__restrict__ inst, uint32_t *__restrict__ key, uint32_t *__restrict__ count,
                      int64_t N, uint32_t C, const int32_t *gate)
{
    if (gated_off(gate))
        return;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < N; id += (int64_t)gridDim.x * blockDim.x) {
        const Inst &I = inst[inst_of[id]];
        dvec4 p = pos[id];
        int cx, cy, cz;
        uint32_t c = C;
        if (cell_coords_exact(I, p.x, p.y, p.z, cx, cy, cz))
            c = (uint32_t)(I.cell_base + (cz * I.n[1] + cy) * I.n[0] + cx);
        key[id] = c;
        atomicAdd(&count[c], 1u);
    }
}

void launch_bin(const Bufs &b, int mode, int64_t N, int32_t C, cudaStream_t st)
{
    (void)mode;
    int blocks = (int)std::min<int64_t>((N + 255) / 256, 4096);
    if (blocks < 1)
        blocks = 1;
    k_bin<<<blocks, 256, 0, st>>>(b.pos, b.inst_of, b.inst, b.key, b.count, N, (uint32_t)C, b.lflag);
}

// One launch per phase; the bodies live in cells.cuh.
__global__ void k_scan_reduce(const uint32_t *__restrict__ count, uint64_t *__restrict__ blocks, int64_t C,
                              const int32_t *gate)
{
    if (gated_off(gate))
        return;
    scan_reduce_tile(count, blocks, C, blockIdx.x);
}

__global__ void k_scan_blocks(uint64_t *__restrict__ blocks, int nb, const int32_t *gate)
{
    if (gated_off(gate))
        return;
    scan_blocks_block(blocks, nb);
}

__global__ void k_scan_final(const uint32_t *__restrict__ count, const uint64_t *__restrict__ blocks,
                             int32_t *__restrict__ cell_start, int32_t *__restrict__ active,
                             int32_t *__restrict__ misc, int64_t C, const int32_t *gate)
{
    if (gated_off(gate))
        return;
    scan_final_tile(count, blocks, cell_start, active, misc, C, blockIdx.x);
}

__global__ void k_scatter(const uint32_t *__restrict__ key, uint32_t *__restrict__ count,
                          const int32_t *__restrict__ cell_start, int32_t *__restrict__ tmp, int32_t *misc,
                          int64_t N, const int32_t *gate)
{
    if (gated_off(gate))
        return;
    scatter_range(key, count, cell_start, tmp, misc, N, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                  (int64_t)gridDim.x * blockDim.x);
}

void launch_cells(const Bufs &b, int64_t N, int32_t C, cudaStream_t st)
{
    int nb = (int)((C + 1 + kScanTile - 1) / kScanTile);
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(b.count, b.scan_blocks, C, b.lflag);
    k_scan_blocks<<<1, 1024, 0, st>>>(b.scan_blocks, nb, b.lflag);
    k_scan_final<<<nb, kScanThreads, 0, st>>>(b.count, b.scan_blocks, b.cell_start, b.active, b.misc, C, b.lflag);
    int blocks = (int)std::min<int64_t>((N + 255) / 256, 8192);
    if (blocks < 1)
        blocks = 1;
    k_scatter<<<blocks, 256, 0, st>>>(b.key, b.count, b.cell_start, b.ptmp, b.misc, N, b.lflag);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_sort_reorder(Bufs b, int32_t C, int32_t ninst)
{
    (void)C;
    if (gated_off(b.lflag))
        return;
    __shared__ uint64_t skeys[8][kSortCap];
    sort_reorder_warps<MODE>(b, ninst, skeys[threadIdx.x >> 5], (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                             (gridDim.x * blockDim.x) >> 5);
}

void launch_reorder(const Bufs &b, int mode, int64_t N, int32_t C, int32_t ninst, int32_t max_active,
                    int32_t ctas_per_sm, cudaStream_t st)
{
    (void)N;
    int blocks = std::max(1, std::min((max_active + 7) / 8, sm_count() * std::max(1, ctas_per_sm)));
    if (mode == SPH_FP64)
        k_sort_reorder<SPH_FP64><<<blocks, 256, 0, st>>>(b, C, ninst);
    else
        k_sort_reorder<SPH_MIXED><<<blocks, 256, 0, st>>>(b, C, ninst);
}

}  // namespace sph
