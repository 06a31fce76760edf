// Cell-linked neighbour structure: binning, per-cell counts, a scan of the
// counts into cell starts and the list of non-empty cells, a counting-sort
// scatter, and a per-cell sort by particle id fused with the gather of the
// sorted particle data (including the Tait pressure, Eq. 8).
//
// The resulting order is ascending (cell, id) for every in-domain particle;
// out-of-domain particles fill the bucket after the last cell in arbitrary
// order and take no further part.
#include "device.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// Binning of the canonical state (used at creation and after a state load).
// ---------------------------------------------------------------------------
__global__ void k_bin(const dvec4 *__restrict__ pos, const uint16_t *__restrict__ inst_of,
                      const Inst *__restrict__ inst, uint32_t *__restrict__ key, uint32_t *__restrict__ count,
                      int64_t N, uint32_t C)
{
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
    k_bin<<<blocks, 256, 0, st>>>(b.pos, b.inst_of, b.inst, b.key, b.count, N, (uint32_t)C);
}

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

__global__ void k_scan_reduce(const uint32_t *__restrict__ count, uint64_t *__restrict__ blocks, int64_t C)
{
    __shared__ uint64_t warp_tot[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        s += scan_value(count, base + k, C);
    uint64_t total;
    block_exclusive_scan(s, warp_tot, total);
    if (threadIdx.x == 0)
        blocks[blockIdx.x] = total;
}

__global__ void k_scan_blocks(uint64_t *__restrict__ blocks, int nb)
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

__global__ void k_scan_final(const uint32_t *__restrict__ count, const uint64_t *__restrict__ blocks,
                             int32_t *__restrict__ cell_start, int32_t *__restrict__ active,
                             int32_t *__restrict__ misc, int64_t C)
{
    __shared__ uint64_t warp_tot[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint64_t v[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = scan_value(count, base + k, C);
        s += v[k];
    }
    uint64_t total;
    uint64_t run = blocks[blockIdx.x] + block_exclusive_scan(s, warp_tot, total);
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

// Counting-sort scatter; decrementing the counters returns them to zero.
__global__ void k_scatter(const uint32_t *__restrict__ key, uint32_t *__restrict__ count,
                          const int32_t *__restrict__ cell_start, int32_t *__restrict__ tmp, int32_t *misc,
                          int64_t N)
{
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < N; id += (int64_t)gridDim.x * blockDim.x) {
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

void launch_cells(const Bufs &b, int64_t N, int32_t C, cudaStream_t st)
{
    int nb = (int)((C + 1 + kScanTile - 1) / kScanTile);
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(b.count, b.scan_blocks, C);
    k_scan_blocks<<<1, 1024, 0, st>>>(b.scan_blocks, nb);
    k_scan_final<<<nb, kScanThreads, 0, st>>>(b.count, b.scan_blocks, b.cell_start, b.active, b.misc, C);
    int blocks = (int)std::min<int64_t>((N + 255) / 256, 8192);
    if (blocks < 1)
        blocks = 1;
    k_scatter<<<blocks, 256, 0, st>>>(b.key, b.count, b.cell_start, b.ptmp, b.misc, N);
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

template <int MODE>
__global__ void __launch_bounds__(256) k_sort_reorder(Bufs b, int32_t C, int32_t ninst)
{
    __shared__ uint64_t skeys[8][kSortCap];
    const int lane = threadIdx.x & 31;
    uint64_t *K = skeys[threadIdx.x >> 5];
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int32_t n_active = b.misc[1];
    const int32_t *tmp = b.ptmp;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_active; w += warps) {
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

void launch_reorder(const Bufs &b, int mode, int64_t N, int32_t C, int32_t ninst, int32_t max_active,
                    cudaStream_t st)
{
    (void)N;
    int blocks = std::max(1, std::min((max_active + 7) / 8, 152 * 16));
    if (mode == SPH_FP64)
        k_sort_reorder<SPH_FP64><<<blocks, 256, 0, st>>>(b, C, ninst);
    else
        k_sort_reorder<SPH_MIXED><<<blocks, 256, 0, st>>>(b, C, ninst);
}

}  // namespace sph
