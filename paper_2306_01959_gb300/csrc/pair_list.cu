// Neighbour lists with a skin for the mixed form of the pair pass (Eqs. 3-8).
//
// With params.list_skin = s/h > 0 the cells hold the list radius 2h + s.  At a
// rebuild the neighbour structure is rebuilt as every step does without lists
// (binning, counting sort, per-cell sort by x and gather), the positions are
// kept as the reference of the displacement test, and k_list_build writes, for
// every in-domain particle i, the sorted indices j of its partners within
// 2h + s (pairs of two boundary particles are never evaluated and are left
// out) together with the offset of j's cell from i's.  Until a particle has
// moved s/2 from its reference (or left the grid), every pair within 2h is in
// these lists: two particles within 2h now were within 2h + s at the rebuild.
// The steps in between keep the sorted order of the rebuild: k_list_regather
// gathers the new state into it, each position relative to the origin of the
// cell the particle had at the rebuild, and k_pair_list evaluates the listed
// pairs with the exact FP32 test |r_ij|^2 < (2h)^2 and the pair arithmetic of
// the staged kernel (pair_term_f): on the rebuild's own state each pair term
// is bit-identical to the staged kernel's, only the order of the sums differs.
// The update kernel raises the rebuild request (lflag[0]); the rebuild kernels
// run only when it is set and the gather only when it is not, so that every
// step launches the same kernels (graph capture is unchanged).
#include "pair_mixed.cuh"

namespace sph {

// Entry code of the offset (dx, dy, dz) in -1..1 of j's cell from i's.
__device__ __forceinline__ int32_t list_code(int dx, int dy, int dz) { return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1); }

constexpr int kListNW = 8, kListG = 4;  // warps per CTA and particles per warp of the build
constexpr int kListBuildStage = 2048;   // staged candidates per chunk of the build

struct ListSmem {
    int32_t item;
    int32_t longest;
    int32_t pre[10];
    int32_t bnd[9][4];  // cell_start of the row's cells x0 .. x1 + 1; -1 outside the grid
};

// ---------------------------------------------------------------------------
// Build: the staged candidate sweep of pair_mixed.cuh at the list radius,
// appending to global per-particle lists instead of evaluating.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kListNW * 32, 2) k_list_build(Bufs b, int ninst, int max_stage)
{
    constexpr int NW = kListNW, G = kListG;
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ ListSmem S;
    if (b.lflag[0] == 0)
        return;  // the lists are current
    float4 *stA = reinterpret_cast<float4 *>(dyn);          // positions in the home-cell frame
    int32_t *stE = reinterpret_cast<int32_t *>(stA + max_stage);  // list entries
    uint8_t *stF = reinterpret_cast<uint8_t *>(stE + max_stage);   // type flags
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const float4 *gA = reinterpret_cast<const float4 *>(b.sA);
    const int32_t n_active = b.misc[1];
    const int32_t cap = b.list_cap;
    int32_t longest = 0;
    if (tid == 0)
        S.longest = 0;

    for (;;) {
        if (tid == 0)
            S.item = atomicAdd(&b.misc[3], 1);
        __syncthreads();
        const int32_t item = S.item;
        if (item >= n_active)
            break;
        const int32_t c = b.active[item];
        const Inst &I = b.inst[inst_of_cell(b.inst, ninst, c)];
        const float cs = I.csf, r2 = I.list_r2f;
        int cx, cy, cz;
        decompose(I, c, cx, cy, cz);
        const int x0 = max(cx - 1, 0), x1 = min(cx + 1, I.n[0] - 1), nb = x1 - x0 + 2;
        const int32_t h0 = b.cell_start[c], h1 = b.cell_start[c + 1];
        if (tid < 9 * 4) {
            const int r = tid >> 2, m = tid & 3;
            const int z = cz + r / 3 - 1, y = cy + r % 3 - 1;
            int32_t v = -1;
            if (m < nb && z >= 0 && z < I.n[2] && y >= 0 && y < I.n[1])
                v = b.cell_start[I.cell_base + (z * I.n[1] + y) * I.n[0] + x0 + m];
            S.bnd[r][m] = v;
        }
        __syncthreads();
        if (tid == 0) {
            int carry = 0;
            for (int r = 0; r < 9; ++r) {
                S.pre[r] = carry;
                if (S.bnd[r][0] >= 0)
                    carry += S.bnd[r][nb - 1] - S.bnd[r][0];
            }
            S.pre[9] = carry;
        }
        __syncthreads();
        const int32_t total = S.pre[9];
        const int32_t home_flat0 = S.pre[4] + (h0 - S.bnd[4][0]);  // row 4 is (dy, dz) = (0, 0)

        for (int32_t f0 = 0; f0 < total; f0 += max_stage) {
            const int32_t f1 = min(total, f0 + max_stage);
            __syncthreads();
            for (int32_t t = tid; t < f1 - f0; t += blockDim.x) {
                const int32_t T = f0 + t;
                int r = 0;
                while (r < 8 && T >= S.pre[r + 1])
                    ++r;
                const int32_t j = S.bnd[r][0] + (T - S.pre[r]);
                int xc = x0;
                for (int m = 1; m < nb - 1; ++m)
                    xc += j >= S.bnd[r][m];
                const int dy = r % 3 - 1, dz = r / 3 - 1;
                float4 a = gA[j];
                a.x += (float)(xc - cx) * cs;
                a.y += (float)dy * cs;
                a.z += (float)dz * cs;
                stA[t] = a;
                stE[t] = (j << 5) | list_code(xc - cx, dy, dz);
                stF[t] = b.sflag[j];
            }
            __syncthreads();
            for (int32_t ib = h0 + G * wib; ib < h1; ib += G * NW) {
                const int32_t ie = min(ib + G, h1);
                const int nreal = ie - ib;  // slots g >= nreal repeat the last particle
                float px[G], py[G], pz[G];
                int32_t cnt[G];
                unsigned fl = 0;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int32_t ii = min(ib + g, ie - 1);
                    const float4 Ai = gA[ii];
                    px[g] = Ai.x;
                    py[g] = Ai.y;
                    pz[g] = Ai.z;
                    fl |= (b.sflag[ii] == T_FLUID ? 1u : 0u) << g;
                    cnt[g] = f0 == 0 ? 0 : b.ncnt[ii];
                }
                SweepPos<G> sp;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    float2 &vx = sp.nx[g / 2], &vy = sp.ny[g / 2], &vz = sp.nz[g / 2];
                    if (g % 2 == 0) {
                        vx.x = -px[g];
                        vy.x = -py[g];
                        vz.x = -pz[g];
                    } else {
                        vx.y = -px[g];
                        vy.y = -py[g];
                        vz.y = -pz[g];
                    }
                }
                // x-window of each row at the list radius (one lane per row)
                int wlo = 0, whi = 0;
                if (lane < 9) {
                    const int r = lane;
                    const int32_t ra = max(S.pre[r], f0) - f0, rb = min(S.pre[r + 1], f1) - f0;
                    if (ra < rb) {
                        const float ry = (float)(r % 3 - 1), rz = (float)(r / 3 - 1);
                        float xl = 3.0e38f, xh = -3.0e38f;
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            float dy = ry > 0.f ? cs - py[g] : (ry < 0.f ? py[g] : 0.f);
                            float dz = rz > 0.f ? cs - pz[g] : (rz < 0.f ? pz[g] : 0.f);
                            dy = fmaxf(dy, 0.f);
                            dz = fmaxf(dz, 0.f);
                            const float rem = r2 - dy * dy - dz * dz;
                            if (rem > 0.f) {
                                const float w = sqrtf(rem) * 1.0001f + 1e-6f * cs;
                                xl = fminf(xl, px[g] - w);
                                xh = fmaxf(xh, px[g] + w);
                            }
                        }
                        if (xl <= xh) {
                            int a0 = ra, a1 = rb;
                            while (a0 < a1) {
                                const int m = (a0 + a1) >> 1;
                                if (stA[m].x < xl)
                                    a0 = m + 1;
                                else
                                    a1 = m;
                            }
                            wlo = a0;
                            a1 = rb;
                            while (a0 < a1) {
                                const int m = (a0 + a1) >> 1;
                                if (stA[m].x <= xh)
                                    a0 = m + 1;
                                else
                                    a1 = m;
                            }
                            whi = a0;
                        }
                    }
                }
                for (int r = 0; r < 9; ++r) {
                    const int lo = __shfl_sync(0xffffffffu, wlo, r);
                    const int hi = __shfl_sync(0xffffffffu, whi, r);
                    for (int32_t base = lo; base < hi; base += 32) {
                        const int32_t t = base + lane;
                        const bool valid = t < hi;
                        float4 a = stA[valid ? t : lo];
                        a.x = valid ? a.x : 1.0e30f;
                        bool hits[G];
                        hit_tests<G>(sp, a, r2, hits);
                        const bool fj = stF[valid ? t : lo] == T_FLUID;
                        const int32_t e = stE[valid ? t : lo];
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            // i itself and pairs of two boundary particles are not listed
                            const bool take = hits[g] && g < nreal && (((fl >> g) & 1u) || fj) &&
                                              f0 + t != home_flat0 + (ib + g - h0);
                            const unsigned m = __ballot_sync(0xffffffffu, take);
                            const int32_t pos = cnt[g] + __popc(m & lt);
                            if (take && pos < cap)
                                b.nlist[(size_t)(ib + g) * cap + pos] = e;
                            cnt[g] += __popc(m);
                        }
                    }
                }
                if (lane == 0) {
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        if (g < nreal) {
                            b.ncnt[ib + g] = cnt[g];
                            if (f1 == total) {
                                longest = max(longest, cnt[g]);
                                if (cnt[g] > cap)
                                    atomicAdd(&b.lflag[2], 1);
                            }
                        }
                }
            }
        }
        __syncthreads();
    }
    if (lane == 0)
        atomicMax(&S.longest, longest);
    __syncthreads();
    if (tid == 0) {
        atomicMax(&b.lflag[3], S.longest);
        if (blockIdx.x == 0)
            atomicAdd(&b.lflag[1], 1);
    }
}

// ---------------------------------------------------------------------------
// List pass: one warp per particle.
// ---------------------------------------------------------------------------
// The 4 sums (d rho/dt, a) of the 32 lanes, TwoSum-compensated: the first two
// levels split the values between lane halves, the last three add one value;
// lane 8 v then holds value v (its sum and error term).
__device__ __forceinline__ void warp_total4(float (&v)[4], float (&e)[4], int lane)
{
    int idx = 0;
#pragma unroll
    for (int k = 4, o = 16; k > 1; k >>= 1, o >>= 1) {
        const bool upper = (lane & o) != 0;
        const int half = k >> 1;
        idx += upper ? half : 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float keep = upper ? v[i + half] : v[i];
            const float send = upper ? v[i] : v[i + half];
            const float ke = upper ? e[i + half] : e[i];
            const float se = upper ? e[i] : e[i + half];
            const float recv = __shfl_xor_sync(0xffffffffu, send, o);
            float ee = ke + __shfl_xor_sync(0xffffffffu, se, o);
            float sum = keep;
            two_sum(sum, ee, recv);
            v[i] = sum;
            e[i] = ee;
        }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        const float recv = __shfl_xor_sync(0xffffffffu, v[0], o);
        float ee = e[0] + __shfl_xor_sync(0xffffffffu, e[0], o);
        two_sum(v[0], ee, recv);
        e[0] = ee;
    }
    (void)idx;
}

// Candidate j (sorted index) of particle i in the FP32 frame of i's cell
// ((ox, oy, oz): offset of j's cell from i's): its shifted position and
// whether |r_ij| < 2h.
__device__ __forceinline__ bool list_test(const float4 *gA, const PairConst &kc, const PartI &P, int32_t j, int ox,
                                          int oy, int oz, float4 &a)
{
    a = gA[j];
    a.x += (float)ox * kc.cs;
    a.y += (float)oy * kc.cs;
    a.z += (float)oz * kc.cs;
    const float dx = P.x - a.x, dy = P.y - a.y, dz = P.z - a.z;
    return dx * dx + dy * dy + dz * dz < kc.sup2;
}

constexpr int kListPassNW = 8;  // warps per CTA of the list pass

// One warp per particle.  Phase 1 tests 32 candidates (listed partners, or
// the 27 cells when the list overflowed) at a time and compacts the hits by
// ballot into the warp's shared buffer; every 32 hits, phase 2 evaluates them
// on 32 full lanes (the pair terms read j's velocity, pressure and type only
// there).
template <bool DFS>
__global__ void __launch_bounds__(kListPassNW * 32, 4) k_pair_list(Bufs b, int ninst)
{
    __shared__ float4 hitA[kListPassNW][64];
    __shared__ int32_t hitJ[kListPassNW][64];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t n_in = b.misc[0];
    const int32_t cap = b.list_cap;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        b.lflag[0] = 0;  // the build (launched before) has read the request
        b.lflag[4] += 1; // list passes
    }
    const float4 *gA = reinterpret_cast<const float4 *>(b.sA);
    const float4 *gB = reinterpret_cast<const float4 *>(b.sB);
    float4 *gD = reinterpret_cast<float4 *>(b.deriv);
    float *gM = reinterpret_cast<float *>(b.mumax);
    float4 *HA = hitA[wib];
    int32_t *HJ = hitJ[wib];
    const int32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (int32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n_in; s += warps) {
        const int32_t c = b.scell[s];
        const Inst &I = b.inst[inst_of_cell(b.inst, ninst, c)];
        const PairConst kc = pair_const(I);
        const bool fluid = b.sflag[s] == T_FLUID;
        const PartI P = load_part(kc, gA[s], gB[s], fluid);
        const int32_t n = b.ncnt[s];
        LaneAcc acc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int nh = 0, cnt = 0;
        unsigned bnd = 0;  // a boundary particle within 2h (DFS)
        // evaluate buffer entries [0, 32) or [0, cnt) and keep the rest
        auto drain = [&](int upto) {
            __syncwarp();
            if (lane < upto) {
                const int32_t j = HJ[lane];
                const bool jf = b.sflag[j] == T_FLUID;
                if (DFS && !jf)
                    bnd = 1u;
                pair_term_f<DFS>(kc, P, HA[lane], gB[j], P.fluid && jf, acc);
            }
            __syncwarp();
            if (lane < cnt - upto) {
                HA[lane] = HA[upto + lane];
                HJ[lane] = HJ[upto + lane];
            }
            cnt -= upto;
            __syncwarp();
        };
        auto push = [&](bool hit, const float4 &a, int32_t j) {
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int pos = cnt + __popc(m & lt);
                HA[pos] = a;
                HJ[pos] = j;
            }
            cnt += __popc(m);
            nh += __popc(m);
            if (cnt >= 32)
                drain(32);
        };
        if (n <= cap) {
            const int32_t *L = b.nlist + (size_t)s * cap;
            for (int32_t k = 0; k < n; k += 32) {
                bool hit = false;
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
                int32_t j = 0;
                if (k + lane < n) {
                    const int32_t e = L[k + lane];
                    const int code = e & 31;
                    j = e >> 5;
                    hit = list_test(gA, kc, P, j, code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1, a);
                }
                push(hit, a, j);
            }
        } else {
            // more partners than the list holds: scan the 27 cells directly
            int cx, cy, cz;
            decompose(I, c, cx, cy, cz);
            const int x0 = max(cx - 1, 0), x1 = min(cx + 1, I.n[0] - 1);
            for (int r = 0; r < 9; ++r) {
                const int z = cz + r / 3 - 1, y = cy + r % 3 - 1;
                if (z < 0 || z >= I.n[2] || y < 0 || y >= I.n[1])
                    continue;
                const int32_t row = I.cell_base + (z * I.n[1] + y) * I.n[0];
                for (int x = x0; x <= x1; ++x) {
                    const int32_t j0 = b.cell_start[row + x], j1 = b.cell_start[row + x + 1];
                    for (int32_t jb = j0; jb < j1; jb += 32) {
                        const int32_t j = jb + lane;
                        bool hit = false;
                        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (j < j1 && j != s && (fluid || b.sflag[j] == T_FLUID))
                            hit = list_test(gA, kc, P, j, x - cx, r % 3 - 1, r / 3 - 1, a);
                        push(hit, a, j);
                    }
                }
            }
        }
        if (cnt > 0)
            drain(cnt);
        if (DFS)
            bnd = __any_sync(0xffffffffu, bnd != 0u) ? 1u : 0u;
        float v[4] = {acc.drho, acc.ax, acc.ay, acc.az}, e[4] = {0.f, 0.f, 0.f, 0.f};
        warp_total4(v, e, lane);
        float mu = acc.mumax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        float dv = 0.f, de = 0.f;
        if (DFS) {
            dv = acc.dd;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float recv = __shfl_xor_sync(0xffffffffu, dv, o);
                float ee = de + __shfl_xor_sync(0xffffffffu, de, o);
                two_sum(dv, ee, recv);
                de = ee;
            }
        }
        // lane 8 v holds total v: bring a to lane 0
        const float ax = __shfl_sync(0xffffffffu, v[0] + e[0], 8);
        const float ay = __shfl_sync(0xffffffffu, v[0] + e[0], 16);
        const float az = __shfl_sync(0xffffffffu, v[0] + e[0], 24);
        if (lane == 0) {
            float drho = v[0] + e[0];
            if (DFS && bnd == 0) {  // the delta term only with a fluid-only support
                float sum = v[0], err = e[0];
                two_sum(sum, err, dv);
                drho = sum + (err + de);
            }
            gD[s] = make_float4(ax, ay, fluid ? az - I.gf : az, drho);
            gM[s] = I.hf * mu;
            b.nneigh[s] = nh;
            b.npair[s] = nh;
            b.ncand[s] = n;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Gather of a step that keeps the lists: the sorted order and the cells of the
// last rebuild; positions relative to the rebuild cell's origin.
// ---------------------------------------------------------------------------
__global__ void k_list_regather(Bufs b, int ninst)
{
    if (b.lflag[0] != 0)
        return;  // a rebuild gathers by itself
    const int32_t n_in = b.misc[0];
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_in; s += gridDim.x * blockDim.x) {
        const int32_t id = b.perm[s], c = b.scell[s];
        const Inst &I = b.inst[inst_of_cell(b.inst, ninst, c)];
        int cx, cy, cz;
        decompose(I, c, cx, cy, cz);
        const dvec4 p = b.pos[id];
        const float4 v = reinterpret_cast<const float4 *>(b.vel)[id];
        reinterpret_cast<float4 *>(b.sA)[s] = make_float4((float)(p.x - (I.lo[0] + cx * I.cs)),
                                                          (float)(p.y - (I.lo[1] + cy * I.cs)),
                                                          (float)(p.z - (I.lo[2] + cz * I.cs)), v.w);
        reinterpret_cast<float4 *>(b.sB)[s] = make_float4(v.x, v.y, v.z, tait_f(I, v.w));
    }
}

size_t list_build_smem() { return (size_t)kListBuildStage * (sizeof(float4) + sizeof(int32_t) + 1); }

void launch_list_pass(const Bufs &b, int64_t N, int32_t ninst, int32_t delta_mode, cudaStream_t st)
{
    const int sms = sm_count();
    static bool attr = false;
    const size_t dyn = list_build_smem();
    if (!attr) {
        cudaFuncSetAttribute(k_list_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        attr = true;
    }
    cudaMemsetAsync(b.misc + 3, 0, sizeof(int32_t), st);
    k_list_build<<<sms * 2, kListNW * 32, dyn, st>>>(b, ninst, kListBuildStage);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((N + kListPassNW - 1) / kListPassNW, (int64_t)sms * 16));
    if (delta_mode == SPH_DELTA_FULL_SUPPORT)
        k_pair_list<true><<<blocks, kListPassNW * 32, 0, st>>>(b, ninst);
    else
        k_pair_list<false><<<blocks, kListPassNW * 32, 0, st>>>(b, ninst);
}

void launch_list_regather(const Bufs &b, int64_t N, int32_t ninst, cudaStream_t st)
{
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, (int64_t)sm_count() * 8));
    k_list_regather<<<blocks, 256, 0, st>>>(b, ninst);
}

}  // namespace sph
