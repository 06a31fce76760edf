// Mixed-precision form of the pair pass (Eqs. 3-8): FP32 pair arithmetic on
// cell-relative offsets, with compensated FP32 accumulation.
//
// Work decomposition (persistent CTAs, one work item = one non-empty home
// cell):
//  1. The CTA stages the particles of every cell within cell_div cells of the
//     home cell into shared memory.  Rows of cells along x are contiguous in
//     the sorted order, so each (dy, dz) row is one copy.  Every staged
//     position is shifted from its own cell origin to the home cell origin;
//     the FP32 offsets stay small (|x| < (cell_div + 1) cs), so the relative
//     distances keep full FP32 precision however large the tank is.
//  2. Each warp takes one particle i of the home cell at a time.  Lanes test
//     32 staged candidates per step (|r_ij|^2 < (2h)^2); hits are compacted by
//     ballot into a per-warp queue and the pair arithmetic runs on 32 full
//     lanes whenever 32 hits are queued.  Each lane accumulates its pair terms;
//     the 32 lane sums are combined by a shuffle tree.
//  3. If a neighbourhood holds more particles than the staging buffer, it is
//     processed in chunks and the per-particle partial sums are carried in
//     shared memory between chunks.
//
// Compensated sums: each lane keeps (sum, error) pairs updated by Knuth's
// TwoSum for the density rate and the three acceleration components; the
// lane errors are added to the lane sums before the shuffle tree.
#include "device.cuh"

namespace sph {

constexpr int kMaxRowsM = 49;  // (2 * 3 + 1)^2 rows at cell_div = 3
constexpr int kMaxI = 128;     // particles of a home cell handled per pass
constexpr int kQM = 64;        // per-warp hit queue

struct RowM {
    int32_t s0;      // first sorted index of the row's x-range
    int16_t dy, dz;  // row offset from the home cell
    int32_t bnd[8];  // cell_start of cells x0 .. x1 + 1 (x-cell boundaries)
};

struct PairSmem {
    int32_t item;
    int32_t nrows;
    int32_t pre[kMaxRowsM + 1];
    RowM row[kMaxRowsM];
    float acc[kMaxI][9];  // drho, ax, ay, az, mumax, and the error terms of the 4 sums
    int32_t nn[kMaxI];
    uint16_t q[16][kQM];
};

__device__ __forceinline__ void two_sum(float &s, float &e, float x)
{
    // Knuth's TwoSum: s + x = t + err exactly, err accumulated in e.
    float t = s + x;
    float bp = t - s;
    float err = (s - (t - bp)) + (x - bp);
    s = t;
    e += err;
}

template <bool COMP>
struct LaneAcc {
    float drho = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
    float edrho = 0.f, eax = 0.f, eay = 0.f, eaz = 0.f;
    float mumax = 0.f;
    __device__ __forceinline__ void add(float d, float x, float y, float z)
    {
        if (COMP) {
            two_sum(drho, edrho, d);
            two_sum(ax, eax, x);
            two_sum(ay, eay, y);
            two_sum(az, eaz, z);
        } else {
            drho += d;
            ax += x;
            ay += y;
            az += z;
        }
    }
};

// Pair term of neighbour j on particle i in FP32.  dx = x_i - x_j (home-cell
// relative), du = u_i - u_j.  grad_i W_ij = F (r_i - r_j) with
// F = -kF (1 - q/2)^3; Eq. 7 continuity (standard sign) and delta term between
// fluid particles; Eqs. 4-5 viscosity when u_ij . r_ij < 0; Eq. 3 momentum.
template <bool COMP>
__device__ __forceinline__ void pair_term_f(const Inst &I, float dx, float dy, float dz, float dux, float duy,
                                            float duz, float drho_i, float drho_j, float inv_rho_i,
                                            float rho_i, float Pi, float Pj, float ci, bool fluid_pair,
                                            LaneAcc<COMP> &a)
{
    float r2 = dx * dx + dy * dy + dz * dz;
    float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
    float t = fmaf(-0.5f * I.inv_hf, r, 1.f);
    float F = -I.kFf * t * t * t;
    float udr = dux * dx + duy * dy + duz * dz;  // u_ij . r_ij
    float rho_j = I.rho0f + drho_j;
    float inv_rho_j = __fdividef(1.f, rho_j);
    float mF = I.massf * F;
    // continuity: m_j (u_i - u_j) . grad_i W_ij = m F udr
    float dd = mF * udr;
    if (fluid_pair)
        dd += I.dfac * (drho_j - drho_i) * (-mF) * inv_rho_j;
    // viscosity (Eqs. 4-5)
    float mu = I.hf * udr * __fdividef(1.f, r2 + I.eta2f);
    float visc = 0.f;
    if (udr < 0.f) {
        float xj = 1.f + drho_j * I.inv_rho0f;
        float cj = I.csound == SPH_CSOUND_CONSTANT ? I.c0f : I.c0f * xj * xj * xj;
        visc = -I.alphaf * (ci + cj) * mu * __fdividef(1.f, rho_i + rho_j);
    }
    // Eq. 3: a_i -= m_j ((P_i + P_j)/(rho_i rho_j) + Pi_ij) grad_i W_ij
    float coef = mF * ((Pi + Pj) * inv_rho_i * inv_rho_j + visc);
    a.add(dd, -coef * dx, -coef * dy, -coef * dz);
    a.mumax = fmaxf(a.mumax, mu);
}

template <int NW, bool COMP>
__global__ void __launch_bounds__(NW * 32) k_pair_mixed(Bufs b, int ninst, int kdiv, int max_stage)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ PairSmem S;
    float4 *stA = reinterpret_cast<float4 *>(dyn);
    float4 *stB = stA + max_stage;
    uint8_t *stF = reinterpret_cast<uint8_t *>(stB + max_stage);

    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const float4 *gA = reinterpret_cast<const float4 *>(b.sA);
    const float4 *gB = reinterpret_cast<const float4 *>(b.sB);
    float4 *gD = reinterpret_cast<float4 *>(b.deriv);
    float *gM = reinterpret_cast<float *>(b.mumax);
    const int32_t n_active = b.misc[1];
    uint16_t *q = S.q[wib];

    for (;;) {
        if (tid == 0)
            S.item = atomicAdd(&b.misc[3], 1);
        __syncthreads();
        const int32_t item = S.item;
        if (item >= n_active)
            break;
        const int32_t c = b.active[item];
        const Inst &I = b.inst[inst_of_cell(b.inst, ninst, c)];
        int cx, cy, cz;
        decompose(I, c, cx, cy, cz);
        const int x0 = max(cx - kdiv, 0), x1 = min(cx + kdiv, I.n[0] - 1);
        const int32_t h0 = b.cell_start[c], h1 = b.cell_start[c + 1];
        // rows of the neighbourhood and their prefix in the flattened list
        if (tid == 0) {
            int nr = 0, tot = 0;
            for (int dz = -kdiv; dz <= kdiv; ++dz) {
                int z = cz + dz;
                if (z < 0 || z >= I.n[2])
                    continue;
                for (int dy = -kdiv; dy <= kdiv; ++dy) {
                    int y = cy + dy;
                    if (y < 0 || y >= I.n[1])
                        continue;
                    int32_t rowc = I.cell_base + (z * I.n[1] + y) * I.n[0];
                    RowM &R = S.row[nr];
                    for (int x = x0; x <= x1 + 1; ++x)
                        R.bnd[x - x0] = b.cell_start[rowc + x];
                    R.s0 = R.bnd[0];
                    R.dy = (int16_t)dy;
                    R.dz = (int16_t)dz;
                    S.pre[nr] = tot;
                    tot += R.bnd[x1 + 1 - x0] - R.s0;
                    ++nr;
                }
            }
            S.pre[nr] = tot;
            S.nrows = nr;
        }
        __syncthreads();
        const int nrows = S.nrows;
        const int32_t total = S.pre[nrows];
        // flattened index of particle i of the home cell: home row (dy = dz = 0)
        int home_row = 0;
        for (int r = 0; r < nrows; ++r)
            if (S.row[r].dy == 0 && S.row[r].dz == 0)
                home_row = r;
        const int32_t home_flat0 = S.pre[home_row] - S.row[home_row].s0;

        for (int32_t g0 = h0; g0 < h1; g0 += kMaxI) {
            const int32_t g1 = min(h1, g0 + kMaxI);
            for (int m = tid; m < (g1 - g0) * 9; m += blockDim.x)
                (&S.acc[0][0])[m] = 0.f;
            for (int m = tid; m < g1 - g0; m += blockDim.x)
                S.nn[m] = 0;
            for (int32_t f0 = 0; f0 < total; f0 += max_stage) {
                const int32_t f1 = min(total, f0 + max_stage);
                __syncthreads();
                // stage [f0, f1)
                for (int32_t t = f0 + tid; t < f1; t += blockDim.x) {
                    int lo = 0, hi = nrows - 1;
                    while (lo < hi) {
                        int mid = (lo + hi + 1) >> 1;
                        if (S.pre[mid] <= t)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    const RowM &R = S.row[lo];
                    const int32_t j = R.s0 + (t - S.pre[lo]);
                    int xc = x0;
                    for (int m = 1; m <= x1 - x0; ++m)
                        xc += j >= R.bnd[m];
                    float4 a = gA[j];
                    a.x += (float)(xc - cx) * I.csf;
                    a.y += (float)R.dy * I.csf;
                    a.z += (float)R.dz * I.csf;
                    stA[t - f0] = a;
                    stB[t - f0] = gB[j];
                    stF[t - f0] = b.sflag[j];
                }
                __syncthreads();
                const int32_t nst = f1 - f0;
                for (int32_t ii = g0 + wib; ii < g1; ii += NW) {
                    const float4 Ai = gA[ii], Bi = gB[ii];
                    const bool fluid_i = b.sflag[ii] == T_FLUID;
                    const int32_t self = home_flat0 + ii - f0;  // staged slot of i (may be outside the chunk)
                    const float rho_i = I.rho0f + Ai.w;
                    const float inv_rho_i = __fdividef(1.f, rho_i);
                    const float xi3 = 1.f + Ai.w * I.inv_rho0f;
                    const float ci = I.csound == SPH_CSOUND_CONSTANT ? I.c0f : I.c0f * xi3 * xi3 * xi3;
                    LaneAcc<COMP> acc;
                    int nn = 0, qn = 0;
                    auto flush = [&](int cnt) {
                        if (lane < cnt) {
                            const int t = q[lane];
                            const float4 a = stA[t], bb = stB[t];
                            const bool fj = stF[t] == T_FLUID;
                            pair_term_f<COMP>(I, Ai.x - a.x, Ai.y - a.y, Ai.z - a.z, Bi.x - bb.x, Bi.y - bb.y,
                                              Bi.z - bb.z, Ai.w, a.w, inv_rho_i, rho_i, Bi.w, bb.w, ci,
                                              fluid_i && fj, acc);
                        }
                    };
                    for (int32_t base = 0; base < nst; base += 32) {
                        const int32_t t = base + lane;
                        bool take = false;
                        if (t < nst && t != self) {
                            const float4 a = stA[t];
                            const float dx = Ai.x - a.x, dy = Ai.y - a.y, dz = Ai.z - a.z;
                            if (dx * dx + dy * dy + dz * dz < I.sup2f) {
                                ++nn;
                                take = fluid_i || stF[t] == T_FLUID;
                            }
                        }
                        const unsigned msk = __ballot_sync(0xffffffffu, take);
                        if (take)
                            q[qn + __popc(msk & lt)] = (uint16_t)t;
                        qn += __popc(msk);
                        __syncwarp();
                        if (qn >= 32) {
                            flush(32);
                            __syncwarp();
                            if (lane < qn - 32)
                                q[lane] = q[lane + 32];
                            qn -= 32;
                            __syncwarp();
                        }
                    }
                    flush(qn);
                    __syncwarp();
                    float d = acc.drho + acc.edrho, x = acc.ax + acc.eax, y = acc.ay + acc.eay,
                          z = acc.az + acc.eaz;
                    // shuffle tree; the error of each level is kept when compensating
                    float ed = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        float od = __shfl_xor_sync(0xffffffffu, d, o), ox = __shfl_xor_sync(0xffffffffu, x, o);
                        float oy = __shfl_xor_sync(0xffffffffu, y, o), oz = __shfl_xor_sync(0xffffffffu, z, o);
                        if (COMP) {
                            float oed = __shfl_xor_sync(0xffffffffu, ed, o), oex = __shfl_xor_sync(0xffffffffu, ex, o);
                            float oey = __shfl_xor_sync(0xffffffffu, ey, o), oez = __shfl_xor_sync(0xffffffffu, ez, o);
                            ed += oed;
                            ex += oex;
                            ey += oey;
                            ez += oez;
                            two_sum(d, ed, od);
                            two_sum(x, ex, ox);
                            two_sum(y, ey, oy);
                            two_sum(z, ez, oz);
                        } else {
                            d += od;
                            x += ox;
                            y += oy;
                            z += oz;
                        }
                    }
                    float mu = acc.mumax;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
                        mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
                    const int nsum = warp_sum(nn);
                    if (lane == 0) {
                        float *A = S.acc[ii - g0];
                        if (COMP) {
                            two_sum(A[0], A[5], d + ed);
                            two_sum(A[1], A[6], x + ex);
                            two_sum(A[2], A[7], y + ey);
                            two_sum(A[3], A[8], z + ez);
                        } else {
                            A[0] += d;
                            A[1] += x;
                            A[2] += y;
                            A[3] += z;
                        }
                        A[4] = fmaxf(A[4], mu);
                        S.nn[ii - g0] += nsum;
                    }
                }
            }
            __syncthreads();
            for (int32_t ii = g0 + tid; ii < g1; ii += blockDim.x) {
                const float *A = S.acc[ii - g0];
                float az = A[3] + A[8];
                if (b.sflag[ii] == T_FLUID)
                    az -= I.gf;
                gD[ii] = make_float4(A[1] + A[6], A[2] + A[7], az, A[0] + A[5]);
                gM[ii] = A[4];
                b.nneigh[ii] = S.nn[ii - g0];
            }
        }
        __syncthreads();
    }
}

template <int NW, bool COMP>
static void launch_nw(const Bufs &b, int ninst, int kdiv, int ctas, int max_stage, cudaStream_t st)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    size_t dyn = (size_t)max_stage * (2 * sizeof(float4) + 1);
    dyn = (dyn + 15) & ~(size_t)15;
    static size_t dyn_set = 0;  // attribute set once per instantiation, outside any capture
    if (dyn > dyn_set) {
        cudaFuncSetAttribute(k_pair_mixed<NW, COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        dyn_set = dyn;
    }
    k_pair_mixed<NW, COMP><<<sms * ctas, NW * 32, dyn, st>>>(b, ninst, kdiv, max_stage);
}

void launch_pair_mixed(const Bufs &b, int64_t N, int32_t ninst, int32_t cell_div, int32_t warps, int32_t ctas,
                       int32_t compensated, int32_t max_active, cudaStream_t st)
{
    (void)N;
    (void)max_active;
    if (warps <= 0)
        warps = 8;
    if (ctas <= 0)
        ctas = 2;
    // staging capacity: the whole neighbourhood of a typical home cell
    const int max_stage = cell_div == 1 ? 2560 : (cell_div == 2 ? 1536 : 1280);
    cudaMemsetAsync(b.misc + 3, 0, sizeof(int32_t), st);
    if (compensated) {
        if (warps <= 4)
            launch_nw<4, true>(b, ninst, cell_div, ctas, max_stage, st);
        else if (warps <= 8)
            launch_nw<8, true>(b, ninst, cell_div, ctas, max_stage, st);
        else
            launch_nw<16, true>(b, ninst, cell_div, ctas, max_stage, st);
    } else {
        if (warps <= 4)
            launch_nw<4, false>(b, ninst, cell_div, ctas, max_stage, st);
        else if (warps <= 8)
            launch_nw<8, false>(b, ninst, cell_div, ctas, max_stage, st);
        else
            launch_nw<16, false>(b, ninst, cell_div, ctas, max_stage, st);
    }
}

}  // namespace sph
