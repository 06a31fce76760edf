// Device bodies of the neighbour-structure phases: the scan of the per-cell
// counts into cell starts and the list of non-empty cells, the counting-sort
// scatter, and the per-cell sort fused with the gather of the sorted particle
// data (including the Tait pressure, Eq. 8).  The kernels of cells.cu run them
// one launch per phase; the persistent kernel of persist.cu runs them between
// grid barriers.  Each body takes the index of the unit it works on (tile,
// block or warp) and the number of such units, not blockIdx/gridDim.  Their
// pointers carry no __restrict__: in the persistent kernel the arrays they read
// were written by other CTAs earlier in the same launch, so the loads must not
// take the read-only (non-coherent) path.
#pragma once

#include "device.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// Scan of the per-cell counts.  Value per cell: (nonempty << 32) | count, so
// that one exclusive scan yields both the cell start and the index of the
// cell in the list of non-empty cells.  The out-of-domain bucket C is never
// marked non-empty.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = kScanTile / kScanThreads;

__device__ __forceinline__ uint64_t scan_value(const uint32_t *count, int64_t c, int64_t C)
{
    if (c > C)
        return 0;
    uint32_t n = count[c];
    return ((uint64_t)(n > 0 && c < C) << 32) | n;
}

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *warp_tot, uint64_t &total)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        uint64_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o)
                t += y;
        }
        if (lane < nw)
            warp_tot[lane] = t;
    }
    __syncthreads();
    uint64_t before = w > 0 ? warp_tot[w - 1] : 0;
    total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

// Tile `tile` of the cell counts (kScanTile cells, kScanThreads threads):
// its total goes to blocks[tile].
__device__ __forceinline__ void scan_reduce_tile(const uint32_t *count, uint64_t *blocks,
                                                 int64_t C, int64_t tile)
{
    __shared__ uint64_t warp_tot[32];
    int64_t base = tile * kScanTile + threadIdx.x * kScanItems;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        s += scan_value(count, base + k, C);
    uint64_t total;
    block_exclusive_scan(s, warp_tot, total);
    if (threadIdx.x == 0)
        blocks[tile] = total;
}

// Exclusive scan of the nb tile totals, by one block.
__device__ __forceinline__ void scan_blocks_block(uint64_t *blocks, int nb)
{
    __shared__ uint64_t warp_tot[32];
    uint64_t carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        int i = base + threadIdx.x;
        uint64_t v = i < nb ? blocks[i] : 0;
        uint64_t total;
        uint64_t ex = block_exclusive_scan(v, warp_tot, total);
        if (i < nb)
            blocks[i] = carry + ex;
        carry += total;
    }
}

// Tile `tile`: cell starts, non-empty cell list, and (last cell) the counts.
__device__ __forceinline__ void scan_final_tile(const uint32_t *count,
                                                const uint64_t *blocks, int32_t *cell_start,
                                                int32_t *active, int32_t *misc, int64_t C,
                                                int64_t tile)
{
    __shared__ uint64_t warp_tot[32];
    int64_t base = tile * kScanTile + threadIdx.x * kScanItems;
    uint64_t v[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = scan_value(count, base + k, C);
        s += v[k];
    }
    uint64_t total;
    uint64_t run = blocks[tile] + block_exclusive_scan(s, warp_tot, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t c = base + k;
        if (c <= C) {
            cell_start[c] = (int32_t)(uint32_t)run;
            if (v[k] >> 32)
                active[(uint32_t)(run >> 32)] = (int32_t)c;
            if (c == C) {
                misc[0] = (int32_t)(uint32_t)run;        // in-domain particles
                misc[1] = (int32_t)(run >> 32);          // non-empty cells
                cell_start[C + 1] = (int32_t)(uint32_t)(run + (v[k] & 0xffffffffu));
            }
        }
        run += v[k];
    }
}

// Counting-sort scatter over particles [thread0, N) with stride `stride`;
// decrementing the counters returns them to zero.
__device__ __forceinline__ void scatter_range(const uint32_t *key, uint32_t *count,
                                              const int32_t *cell_start, int32_t *tmp,
                                              int32_t *misc, int64_t N, int64_t thread0, int64_t stride)
{
    for (int64_t id = thread0; id < N; id += stride) {
        uint32_t c = key[id];
        uint32_t v = atomicSub(&count[c], 1u);
        int64_t slot = (int64_t)cell_start[c] + (int64_t)v - 1;
        if (v == 0u || slot < 0 || slot >= N) {  // counters out of step with the keys
            atomicOr(&misc[2], ST_OVERFLOW);
            continue;
        }
        tmp[slot] = (int32_t)id;
    }
}

// ---------------------------------------------------------------------------
// Per-cell sort + gather (one warp per non-empty cell).  The FP64 form orders
// each cell by particle id, which gives the (cell, id) order of the method's
// definition.  The mixed form orders each cell by (x offset, id): rows of
// cells along x are then sorted by x, which the mixed pair kernel uses to cut
// its candidate ranges.
// ---------------------------------------------------------------------------
constexpr int kSortCap = 256;

__device__ __forceinline__ uint32_t orderable(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <int MODE>
__device__ __forceinline__ uint64_t sort_key(const Bufs &b, int32_t id, double x_origin)
{
    if (MODE == SPH_FP64)
        return (uint64_t)(uint32_t)id;
    const float ox = (float)(b.pos[id].x - x_origin);
    return ((uint64_t)orderable(ox) << 32) | (uint32_t)id;
}

// Warps [warp0, n_active) with stride `warps`; K is this warp's kSortCap-entry
// key scratch in shared memory.
template <int MODE>
__device__ __forceinline__ void sort_reorder_warps(const Bufs &b, int32_t ninst, uint64_t *K, int warp0, int warps)
{
    const int lane = threadIdx.x & 31;
    const int32_t n_active = b.misc[1];
    const int32_t *tmp = b.ptmp;
    for (int w = warp0; w < n_active; w += warps) {
        const int32_t c = b.active[w];
        const int32_t s0 = b.cell_start[c], s1 = b.cell_start[c + 1];
        const int32_t n = s1 - s0;
        const Inst &I = b.inst[inst_of_cell(b.inst, ninst, c)];
        int cx, cy, cz;
        decompose(I, c, cx, cy, cz);
        const double ox0 = I.lo[0] + cx * I.cs, oy0 = I.lo[1] + cy * I.cs, oz0 = I.lo[2] + cz * I.cs;
        const bool in_smem = n <= kSortCap;
        if (in_smem) {
            for (int e = lane; e < n; e += 32)
                K[e] = sort_key<MODE>(b, tmp[s0 + e], ox0);
            __syncwarp();
        }
        for (int e = lane; e < ((n + 31) & ~31); e += 32) {
            uint64_t key = ~0ull;
            if (e < n)
                key = in_smem ? K[e] : sort_key<MODE>(b, tmp[s0 + e], ox0);
            int32_t rank = 0;
            if (in_smem) {
                for (int k = 0; k < n; ++k)
                    rank += K[k] < key;
            } else {
                for (int k = 0; k < n; ++k)
                    rank += sort_key<MODE>(b, tmp[s0 + k], ox0) < key;
            }
            if (e < n) {
                const int32_t id = (int32_t)(uint32_t)(key & 0xffffffffu);
                const int32_t s = s0 + rank;
                b.perm[s] = id;
                b.scell[s] = c;
                b.sflag[s] = b.type[id];
                const dvec4 p = b.pos[id];
                if (b.xbuild)
                    b.xbuild[id] = p;  // neighbour lists: reference of the displacement test
                if (MODE == SPH_FP64) {
                    const dvec4 v = reinterpret_cast<const dvec4 *>(b.vel)[id];
                    reinterpret_cast<dvec4 *>(b.sA)[s] = make_dvec4(p.x, p.y, p.z, v.w);
                    reinterpret_cast<dvec4 *>(b.sB)[s] = make_dvec4(v.x, v.y, v.z, tait_d(I, v.w));
                    b.sC[s] = make_double2(1.0 / v.w, sound_d(I, v.w));
                    b.sD[s] = make_float4((float)p.x, (float)p.y, (float)p.z, 0.f);
                } else {
                    const float4 v = reinterpret_cast<const float4 *>(b.vel)[id];
                    reinterpret_cast<float4 *>(b.sA)[s] =
                        make_float4((float)(p.x - ox0), (float)(p.y - oy0), (float)(p.z - oz0), v.w);
                    reinterpret_cast<float4 *>(b.sB)[s] = make_float4(v.x, v.y, v.z, tait_f(I, v.w));
                }
            }
        }
        __syncwarp();
    }
}

}  // namespace sph
