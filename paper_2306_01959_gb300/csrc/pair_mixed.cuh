#pragma once
// Mixed-precision form of the pair pass (Eqs. 3-8), device body: FP32 pair
// arithmetic on cell-relative offsets, with compensated FP32 accumulation.
//
// Work decomposition (persistent CTAs, one work item = one non-empty home
// cell):
//  1. The CTA stages the particles of every cell within cell_div cells of the
//     home cell into shared memory.  Rows of cells along x are contiguous in
//     the sorted order, so each (dy, dz) row is one copy (one warp per row).
//     Every staged position is shifted from its own cell origin to the home
//     cell origin; the FP32 offsets stay small (|x| < (cell_div + 1) cs), so
//     relative distances keep full FP32 precision however large the tank is.
//  2. A warp takes G particles i of the home cell at a time (G = 1, 2 or 4).
//     Lanes test 32 staged candidates per step against the G particles
//     (|r_ij|^2 < (2h)^2), one shared-memory load serving all G tests; the
//     interacting candidates are compacted by ballot into one list per
//     particle.  The pair arithmetic then runs over each list on 32 full
//     lanes (only the last batch of a list is partial).
//  3. Each lane accumulates its pair terms; the 32 lane sums of a particle are
//     combined by a shuffle tree.  If a neighbourhood holds more particles
//     than the staging buffer, it is processed in chunks and the partial sums
//     are carried in shared memory between chunks.
//
// Compensated sums: the lane sums (at most a few tens of terms each) are
// combined across lanes and across chunks with Knuth's TwoSum, carrying the
// rounding error of every addition, so the result is the compensated sum of
// the lane partials.
#include "device.cuh"

namespace sph {

constexpr int kMaxRowsM = 49;  // (2 * 3 + 1)^2 rows at cell_div = 3
constexpr int kMaxI = 128;     // particles of a home cell handled per pass
// capacity of a per-particle candidate list (entries); a list without room for
// the next row window is drained first, so the capacity only bounds shared memory
constexpr int kList = 512;

// Staging capacity of a CTA (a multiple of 32): the whole neighbourhood of a
// typical home cell at each cell size.
__host__ __device__ __forceinline__ int mixed_max_stage(int cell_div)
{
    return cell_div == 1 ? 2048 : (cell_div == 2 ? 1536 : 1280);
}

// Dynamic shared memory of a CTA of NW warps with G particles per warp.
__host__ __device__ __forceinline__ size_t mixed_dyn_smem(int max_stage, int NW, int G)
{
    size_t dyn = (size_t)max_stage * (2 * sizeof(float4) + 1);
    dyn = (dyn + 15) & ~(size_t)15;
    return dyn + (size_t)NW * G * kList * sizeof(uint16_t);
}

struct RowM {
    int32_t bnd[8];  // cell_start of cells x0 .. x1 + 1 (x-cell boundaries); -1 outside the grid
};

struct PairSmem {
    int32_t item;
    unsigned long long st_ff, st_visc, st_cand;  // work counts of this CTA
    int32_t pre[kMaxRowsM + 1];
    RowM row[kMaxRowsM];
    float acc[kMaxI][9];  // drho, ax, ay, az, mumax, and the error terms of the 4 sums
    float dd[kMaxI][2];   // SPH_DELTA_FULL_SUPPORT: the delta term of Eq. 7 and its error term
    int32_t nb[kMaxI];    // SPH_DELTA_FULL_SUPPORT: the particle has a boundary neighbour
    int32_t nn[kMaxI];
    int32_t np[kMaxI];
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

// FP32 constants of one instance, held in registers for a work item.
struct PairConst {
    float half_inv_h, mkF, rho0, inv_rho0, dfac, eta2, c0, nah, nahc0, sup2, cs;  // nah = -alpha h
    bool csound_const;
};

__device__ __forceinline__ PairConst pair_const(const Inst &I)
{
    PairConst k;
    k.half_inv_h = 0.5f * I.inv_hf;
    k.mkF = -I.massf * I.kFf;  // m_j F = mkF (1 - q/2)^3
    k.rho0 = I.rho0f;
    k.inv_rho0 = I.inv_rho0f;
    k.dfac = I.dfac;
    k.eta2 = I.eta2f;
    k.c0 = I.c0f;
    k.nah = -I.alphaf * I.hf;
    k.nahc0 = k.nah * I.c0f;
    k.sup2 = I.sup2f;
    k.cs = I.csf;
    k.csound_const = I.csound == SPH_CSOUND_CONSTANT;
    return k;
}

// ---------------------------------------------------------------------------
// Scalar path (one particle per warp)
// ---------------------------------------------------------------------------
struct PartI {
    float x, y, z, ux, uy, uz, rho, inv_rho;
    float Pr;   // P_i / rho_i
    float ndd;  // -2 delta h c0 (rho_i - rho0)
    float nac;  // -alpha h c_i
    bool fluid;
};

__device__ __forceinline__ PartI load_part(const PairConst &k, const float4 A, const float4 B, bool fluid)
{
    PartI p;
    p.x = A.x;
    p.y = A.y;
    p.z = A.z;
    p.ux = B.x;
    p.uy = B.y;
    p.uz = B.z;
    p.rho = k.rho0 + A.w;
    p.inv_rho = __fdividef(1.f, p.rho);
    p.Pr = B.w * p.inv_rho;
    p.ndd = -k.dfac * A.w;
    const float xi = fmaf(A.w, k.inv_rho0, 1.f);
    p.nac = k.csound_const ? k.nahc0 : k.nahc0 * xi * xi * xi;
    p.fluid = fluid;
    return p;
}

struct LaneAcc {
    float drho, ax, ay, az, mumax;
    float dd;  // delta term of Eq. 7 summed apart (SPH_DELTA_FULL_SUPPORT only)
};

// Pair term of neighbour j on particle i in FP32.  dx = x_i - x_j (home-cell
// relative), du = u_i - u_j.  grad_i W_ij = F (r_i - r_j) with
// F = -kF (1 - q/2)^3; Eq. 7 continuity (standard sign) and delta term between
// fluid particles; Eqs. 4-5 viscosity when u_ij . r_ij < 0; Eq. 3 momentum.
// For j = i (dx = du = 0) every term is exactly zero.  The running maximum is
// of mu / h (the caller scales it by h).  Returns bit 0 for a fluid-fluid pair
// (delta term evaluated) and bit 1 for an approaching pair (viscosity
// evaluated).  With DFS the delta term goes to acc.dd instead of acc.drho.
template <bool DFS>
__device__ __forceinline__ int pair_term_f(const PairConst &k, const PartI &p, const float4 a, const float4 bb,
                                           bool fluid_pair, LaneAcc &acc)
{
    const float dx = p.x - a.x, dy = p.y - a.y, dz = p.z - a.z;
    const float dux = p.ux - bb.x, duy = p.uy - bb.y, duz = p.uz - bb.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float r = r2 * rsqrtf(r2 + 1e-30f);  // 0 for j = i
    const float t = fmaf(-k.half_inv_h, r, 1.f);
    const float mF = k.mkF * (t * t * t);  // m_j F
    const float udr = dux * dx + duy * dy + duz * dz;  // u_ij . r_ij
    const float rho_j = k.rho0 + a.w;
    const float inv_rho_j = __fdividef(1.f, rho_j);
    // continuity: m_j (u_i - u_j) . grad_i W_ij = m F udr, plus between fluid
    // particles the delta term -m F 2 delta h c0 (rho_j - rho_i) / rho_j
    const float ud = DFS ? udr : (fluid_pair ? fmaf(-fmaf(k.dfac, a.w, p.ndd), inv_rho_j, udr) : udr);
    // viscosity (Eqs. 4-5): mu = h muh
    const float muh = udr * __fdividef(1.f, r2 + k.eta2);
    // evaluated on every lane: a batch of 32 pairs almost always holds an
    // approaching pair, so a branch would only add overhead; muh < 0 exactly
    // when u_ij . r_ij < 0, so min(muh, 0) switches the term on
    const float xj = fmaf(a.w, k.inv_rho0, 1.f);
    const float nac = k.csound_const ? p.nac + k.nahc0 : fmaf(k.nahc0 * (xj * xj), xj, p.nac);  // -alpha h (c_i + c_j)
    const float visc = nac * fminf(muh, 0.f) * __fdividef(1.f, p.rho + rho_j);
    // Eq. 3: a_i -= m_j ((P_i + P_j)/(rho_i rho_j) + Pi_ij) grad_i W_ij
    const float coef = mF * fmaf(fmaf(bb.w, p.inv_rho, p.Pr), inv_rho_j, visc);
    acc.drho = fmaf(mF, ud, acc.drho);
    if (DFS)
        acc.dd = fmaf(mF, fluid_pair ? -fmaf(k.dfac, a.w, p.ndd) * inv_rho_j : 0.f, acc.dd);
    acc.ax = fmaf(-coef, dx, acc.ax);
    acc.ay = fmaf(-coef, dy, acc.ay);
    acc.az = fmaf(-coef, dz, acc.az);
    acc.mumax = fmaxf(acc.mumax, muh);
    return (fluid_pair ? 1 : 0) | (udr < 0.f ? 2 : 0);  // pair classes for the work counts
}

// Positions of the G particles of a warp, negated and packed in pairs, for the
// candidate sweep: r_j - r_i is then one packed add, and one packed FP32x2
// instruction (sm_100 and later) advances the |r_ij|^2 < (2h)^2 test of two
// particles.  For G = 1 the scalar halves are used.
template <int G>
struct SweepPos {
    float2 nx[(G + 1) / 2], ny[(G + 1) / 2], nz[(G + 1) / 2];
};

template <int G>
__device__ __forceinline__ void hit_tests(const SweepPos<G> &sp, const float4 a, float sup2, bool (&hit)[G])
{
    if constexpr (G == 1) {
        const float dx = a.x + sp.nx[0].x, dy = a.y + sp.ny[0].x, dz = a.z + sp.nz[0].x;
        hit[0] = dx * dx + dy * dy + dz * dz < sup2;
    } else {
        const float2 ax = make_float2(a.x, a.x), ay = make_float2(a.y, a.y), az = make_float2(a.z, a.z);
#pragma unroll
        for (int q = 0; q < G / 2; ++q) {
            const float2 dx = __fadd2_rn(ax, sp.nx[q]), dy = __fadd2_rn(ay, sp.ny[q]), dz = __fadd2_rn(az, sp.nz[q]);
            const float2 d2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            hit[2 * q] = d2.x < sup2;
            hit[2 * q + 1] = d2.y < sup2;
        }
    }
}

// ---------------------------------------------------------------------------
// Combination of the 32 lane sums of one particle and of the chunks.
// ---------------------------------------------------------------------------
// The 4G sums (d rho/dt and the three acceleration components of each of the G
// particles of a warp) are combined across the 32 lanes by a value-splitting
// butterfly: at each of the first log2(4G) levels a lane keeps half of its
// values and adds its partner's copies of them, so a level moves half as many
// values as the one before; the remaining levels are a plain butterfly on the
// one value left.  Lane 32/(4G) * v then holds the total of value v and adds it
// to the particle's running sums in shared memory (TwoSum-compensated when
// COMP).  mumax is a plain max butterfly; the counts are warp-uniform.
template <int G, bool COMP, bool DFS>
__device__ __forceinline__ void combine_group(PairSmem &S, const LaneAcc (&acc)[G], const int32_t (&slot)[G],
                                              const bool (&valid)[G], const int (&nsum)[G], const int (&npair)[G],
                                              unsigned nbits)
{
    constexpr int K = 4 * G;
    const int lane = threadIdx.x & 31;
    float v[K], e[K];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        v[4 * g + 0] = acc[g].drho;
        v[4 * g + 1] = acc[g].ax;
        v[4 * g + 2] = acc[g].ay;
        v[4 * g + 3] = acc[g].az;
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
        e[k] = 0.f;
    int idx = 0;  // which of the K values this lane ends up holding
#pragma unroll
    for (int k = K, o = 16; k > 1; k >>= 1, o >>= 1) {
        const bool upper = (lane & o) != 0;
        const int half = k >> 1;
        idx += upper ? half : 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float keep = upper ? v[i + half] : v[i];
            const float send = upper ? v[i] : v[i + half];
            const float recv = __shfl_xor_sync(0xffffffffu, send, o);
            if (COMP) {
                const float ke = upper ? e[i + half] : e[i];
                const float se = upper ? e[i] : e[i + half];
                float ee = ke + __shfl_xor_sync(0xffffffffu, se, o);
                float sum = keep;
                two_sum(sum, ee, recv);
                v[i] = sum;
                e[i] = ee;
            } else {
                v[i] = keep + recv;
            }
        }
    }
#pragma unroll
    for (int o = 16 / K; o > 0; o >>= 1) {
        const float recv = __shfl_xor_sync(0xffffffffu, v[0], o);
        if (COMP) {
            float ee = e[0] + __shfl_xor_sync(0xffffffffu, e[0], o);
            two_sum(v[0], ee, recv);
            e[0] = ee;
        } else {
            v[0] += recv;
        }
    }
    float mu[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        mu[g] = acc[g].mumax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            mu[g] = fmaxf(mu[g], __shfl_xor_sync(0xffffffffu, mu[g], o));
    }
    if ((lane & (32 / K - 1)) == 0) {
        const int gsel = idx >> 2, c = idx & 3;
        int32_t sl = slot[0];
        bool ok = valid[0];
#pragma unroll
        for (int g = 1; g < G; ++g)
            if (gsel == g) {
                sl = slot[g];
                ok = valid[g];
            }
        if (ok) {
            float *A = S.acc[sl];
            if (COMP)
                two_sum(A[c], A[5 + c], v[0] + e[0]);
            else
                A[c] += v[0];
        }
    }
    if (DFS) {
        // the delta sums: a TwoSum butterfly per particle; the boundary-neighbour
        // flags: an OR over the lanes
        const unsigned nball = __reduce_or_sync(0xffffffffu, nbits);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            float dv = acc[g].dd, de = 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float recv = __shfl_xor_sync(0xffffffffu, dv, o);
                float ee = de + __shfl_xor_sync(0xffffffffu, de, o);
                two_sum(dv, ee, recv);
                de = ee;
            }
            if (lane == 0 && valid[g]) {
                float *D = S.dd[slot[g]];
                two_sum(D[0], D[1], dv + de);
                S.nb[slot[g]] |= (nball >> g) & 1u;
            }
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (valid[g]) {
                float *A = S.acc[slot[g]];
                A[4] = fmaxf(A[4], mu[g]);
                S.nn[slot[g]] += nsum[g];
                S.np[slot[g]] += npair[g];
            }
    }
}

// The pair pass of one CTA: pulls home cells from the work queue b.misc[3]
// until it is exhausted.  dyn: the dynamic shared memory (staging buffers and
// candidate lists), S: the CTA's bookkeeping.
template <int NW, int G, bool COMP, bool CNT, bool DFS>
__device__ __forceinline__ void pair_mixed_body(const Bufs &b, int ninst, int kdiv, int max_stage, unsigned char *dyn,
                                                PairSmem &S)
{
    float4 *stA = reinterpret_cast<float4 *>(dyn);
    float4 *stB = stA + max_stage;
    uint8_t *stF = reinterpret_cast<uint8_t *>(stB + max_stage);
    constexpr int LC = kList;
    // interacting-candidate lists, one per (warp, particle slot), after the staged data
    uint16_t *lists = reinterpret_cast<uint16_t *>(dyn + ((size_t)max_stage * (2 * sizeof(float4) + 1) + 15) / 16 * 16);

    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const float4 *gA = reinterpret_cast<const float4 *>(b.sA);
    const float4 *gB = reinterpret_cast<const float4 *>(b.sB);
    float4 *gD = reinterpret_cast<float4 *>(b.deriv);
    float *gM = reinterpret_cast<float *>(b.mumax);
    const int32_t n_active = b.misc[1];
    uint32_t lc_ff = 0, lc_visc = 0;  // evaluated fluid-fluid and approaching pairs of this lane
    unsigned long long wc_cand = 0;   // windowed candidates tested by this warp
    if (tid == 0) {
        S.st_ff = 0ull;
        S.st_visc = 0ull;
        S.st_cand = 0ull;
    }

    for (;;) {
        if (tid == 0)
            S.item = atomicAdd(&b.misc[3], 1);
        __syncthreads();
        const int32_t item = S.item;
        if (item >= n_active)
            break;
        const int32_t c = b.active[item];
        const Inst &I = b.inst[inst_of_cell(b.inst, ninst, c)];
        const PairConst kc = pair_const(I);
        int cx, cy, cz;
        decompose(I, c, cx, cy, cz);
        const int x0 = max(cx - kdiv, 0), x1 = min(cx + kdiv, I.n[0] - 1);
        const int32_t h0 = b.cell_start[c], h1 = b.cell_start[c + 1];
        // Rows of the neighbourhood: slot r = (dz + k) side + (dy + k).  One
        // thread per (row, x-boundary) loads the cell starts; warp 0 turns the
        // row lengths into offsets of the flattened candidate list.
        const int side = 2 * kdiv + 1, nrow = side * side, nb = x1 - x0 + 2;
        for (int t = tid; t < nrow * nb; t += blockDim.x) {
            const int r = t / nb, m = t - r * nb;
            const int z = cz + r / side - kdiv, y = cy + r % side - kdiv;
            int32_t v = -1;
            if (z >= 0 && z < I.n[2] && y >= 0 && y < I.n[1])
                v = b.cell_start[I.cell_base + (z * I.n[1] + y) * I.n[0] + x0 + m];
            S.row[r].bnd[m] = v;
        }
        __syncthreads();
        if (wib == 0) {
            int carry = 0;
            for (int r0 = 0; r0 < nrow; r0 += 32) {
                const int r = r0 + lane;
                int len = 0;
                if (r < nrow && S.row[r].bnd[0] >= 0)
                    len = S.row[r].bnd[nb - 1] - S.row[r].bnd[0];
                int x = len;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o)
                        x += y;
                }
                if (r < nrow)
                    S.pre[r] = carry + x - len;
                carry += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0)
                S.pre[nrow] = carry;
        }
        __syncthreads();
        const int32_t total = S.pre[nrow];
        // flattened index of the home cell's first particle (home row dy = dz = 0)
        const int home_row = kdiv * side + kdiv;
        const int32_t home_flat0 = S.pre[home_row] + (h0 - S.row[home_row].bnd[0]);

        for (int32_t g0 = h0; g0 < h1; g0 += kMaxI) {
            const int32_t g1 = min(h1, g0 + kMaxI);
            __syncthreads();
            for (int m = tid; m < (g1 - g0) * 9; m += blockDim.x)
                (&S.acc[0][0])[m] = 0.f;
            for (int m = tid; m < g1 - g0; m += blockDim.x) {
                S.nn[m] = 0;
                S.np[m] = 0;
                S.dd[m][0] = 0.f;
                S.dd[m][1] = 0.f;
                S.nb[m] = 0;
            }
            for (int32_t f0 = 0; f0 < total; f0 += max_stage) {
                const int32_t f1 = min(total, f0 + max_stage);
                                __syncthreads();
                // stage [f0, f1): one warp per row, lanes along the row
                for (int r = wib; r < nrow; r += NW) {
                    const int32_t p0 = S.pre[r], len = S.pre[r + 1] - p0;
                    const int32_t l0 = max(f0 - p0, 0), l1 = min(f1 - p0, len);
                    if (l0 >= l1)
                        continue;
                    const RowM &R = S.row[r];
                    const float sy = (float)(r % side - kdiv) * kc.cs, sz = (float)(r / side - kdiv) * kc.cs;
                    for (int32_t l = l0 + lane; l < l1; l += 32) {
                        const int32_t j = R.bnd[0] + l;
                        int xc = x0;
                        for (int m = 1; m < nb - 1; ++m)
                            xc += j >= R.bnd[m];
                        float4 a = gA[j];
                        a.x += (float)(xc - cx) * kc.cs;
                        a.y += sy;
                        a.z += sz;
                        const int32_t t = p0 + l - f0;
                        if (!SPH_BOUNDS_OK(t >= 0 && t < max_stage, &b.misc[2]))
                            continue;
                        stA[t] = a;
                        stB[t] = gB[j];
                        stF[t] = b.sflag[j];
                    }
                }
                __syncthreads();
                // Each warp takes G particles of the home cell.  Phase 1 sweeps the
                // staged candidates once for all G particles and appends the
                // interacting ones to one list per particle; phase 2 evaluates the
                // pair terms 32 at a time.  A list short of room is drained early.
                // Warps take G consecutive home particles at a time; in a short
                // last group the empty slots repeat the last particle and are
                // swept but neither evaluated nor stored.
                for (int32_t ib = g0 + G * wib; ib < g1; ib += G * NW) {
                    const int32_t ie = min(ib + G, g1);
                    // Only the positions and type flags of the G particles stay in
                    // registers through the sweep; the rest of a particle's state is
                    // reloaded when its list is evaluated.
                    float px[G], py[G], pz[G];
                    LaneAcc acc[G];
                    int cnt[G], nn[G], np[G];
                    unsigned fl = 0;  // bit g: particle g is fluid
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const int32_t ii = min(ib + g, ie - 1);
                        const float4 Ai = gA[ii];
                        px[g] = Ai.x;
                        py[g] = Ai.y;
                        pz[g] = Ai.z;
                        fl |= (b.sflag[ii] == T_FLUID ? 1u : 0u) << g;
                        acc[g] = LaneAcc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                        cnt[g] = 0;
                        nn[g] = 0;
                        np[g] = 0;
                    }
                    const bool all_fluid = fl == (1u << G) - 1u;
                    unsigned nbits = 0;  // DFS: bit g set when a listed neighbour of particle g is a boundary particle
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
                    uint16_t *const wl0 = lists + wib * G * LC;
                    auto drain = [&](int g, int upto) {
                        // evaluate list entries [0, upto) of particle g, upto a multiple of 32 or cnt
                        const int32_t ii = min(ib + g, ie - 1);
                        const PartI P = load_part(kc, gA[ii], gB[ii], (fl >> g) & 1u);
                        const uint16_t *lg = wl0 + g * LC;
                        int k = 0;
                        if (!CNT) {
                            // two full batches at a time: two independent chains per lane
                            for (; k + 64 <= upto; k += 64) {
                                const int t0 = lg[k + lane], t1 = lg[k + 32 + lane];
                                LaneAcc a1{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                                const bool f0 = stF[t0] == T_FLUID, f1 = stF[t1] == T_FLUID;
                                pair_term_f<DFS>(kc, P, stA[t0], stB[t0], P.fluid && f0, acc[g]);
                                pair_term_f<DFS>(kc, P, stA[t1], stB[t1], P.fluid && f1, a1);
                                if (DFS) {
                                    nbits |= (f0 && f1 ? 0u : 1u) << g;
                                    acc[g].dd += a1.dd;
                                }
                                acc[g].drho += a1.drho;
                                acc[g].ax += a1.ax;
                                acc[g].ay += a1.ay;
                                acc[g].az += a1.az;
                                acc[g].mumax = fmaxf(acc[g].mumax, a1.mumax);
                            }
                        }
                        for (; k < upto; k += 32) {
                            if (lane < upto - k) {
                                const int t = lg[k + lane];
                                const bool fj = stF[t] == T_FLUID;
                                const int f = pair_term_f<DFS>(kc, P, stA[t], stB[t], P.fluid && fj, acc[g]);
                                if (DFS)
                                    nbits |= (fj ? 0u : 1u) << g;
                                if (CNT && ib + g < ie) {  // a repeated particle is not counted
                                    lc_ff += f & 1;
                                    lc_visc += f >> 1;
                                }
                            }
                        }
                    };
                    // Exact x-windows per row: a candidate j of row r can lie within 2h
                    // of i only if |x_j - x_i| <= w_r = sqrt((2h)^2 - d_r^2), d_r the
                    // distance from i to the row's y-z cross-section.  Cells are sorted
                    // by x, so each row is sorted by x and each window is a contiguous
                    // range, found by binary search (one lane per row); the windows of
                    // the G particles are merged.
                    int wlo[2] = {0, 0}, whi[2] = {0, 0};
#pragma unroll
                    for (int pass = 0; pass < 2; ++pass) {
                        const int r = pass * 32 + lane;
                        if (pass * 32 < nrow && r < nrow) {
                            const int32_t ra = max(S.pre[r], f0) - f0, rb = min(S.pre[r + 1], f1) - f0;
                            if (ra < rb) {
                                const float ry = (float)(r % side - kdiv), rz = (float)(r / side - kdiv);
                                float xl = 3.0e38f, xh = -3.0e38f;
#pragma unroll
                                for (int g = 0; g < G; ++g) {
                                    float dy = ry > 0.f ? ry * kc.cs - py[g] : (ry < 0.f ? py[g] - (ry + 1.f) * kc.cs : 0.f);
                                    float dz = rz > 0.f ? rz * kc.cs - pz[g] : (rz < 0.f ? pz[g] - (rz + 1.f) * kc.cs : 0.f);
                                    dy = fmaxf(dy, 0.f);
                                    dz = fmaxf(dz, 0.f);
                                    const float rem = kc.sup2 - dy * dy - dz * dz;
                                    if (rem > 0.f) {
                                        const float w = sqrtf(rem) * 1.0001f + 1e-6f * kc.cs;
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
                                    wlo[pass] = a0;
                                    a1 = rb;
                                    while (a0 < a1) {
                                        const int m = (a0 + a1) >> 1;
                                        if (stA[m].x <= xh)
                                            a0 = m + 1;
                                        else
                                            a1 = m;
                                    }
                                    whi[pass] = a0;
                                }
                            }
                        }
                    }
                    if (CNT) {
                        const int wsum = warp_sum((whi[0] - wlo[0]) + (whi[1] - wlo[1]));
                        if (lane == 0)
                            wc_cand += (unsigned long long)wsum;
                    }
                    // Drain the full 32-entry batches of every list and keep the rest.
                    auto flush = [&]() {
                        __syncwarp();
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            const int done = cnt[g] & ~31;
                            if (ib + g < ie)
                                drain(g, done);
                            __syncwarp();
                            if (lane < cnt[g] - done)
                                if (SPH_BOUNDS_OK(done + lane < LC, &b.misc[2]))
                                    wl0[g * LC + lane] = wl0[g * LC + done + lane];
                            np[g] += done;
                            cnt[g] -= done;
                            __syncwarp();
                        }
                    };
                    // One 32-candidate step: G tests per candidate, ballot compaction.
                    auto sweep = [&](int32_t base, int32_t lo, int32_t hi) {
                        const int32_t t = base + lane;
                        const bool valid = t < hi;
                        float4 a = stA[valid ? t : lo];
                        a.x = valid ? a.x : 1.0e30f;  // a lane past the window misses every test
                        bool hits[G];
                        hit_tests<G>(sp, a, kc.sup2, hits);
                        if (all_fluid) {
#pragma unroll
                            for (int g = 0; g < G; ++g) {
                                const bool take = hits[g];
                                const unsigned m = __ballot_sync(0xffffffffu, take);
                                if (take && SPH_BOUNDS_OK(cnt[g] + __popc(m & lt) < LC && t < max_stage, &b.misc[2]))
                                    wl0[g * LC + cnt[g] + __popc(m & lt)] = (uint16_t)t;
                                cnt[g] += __popc(m);
                            }
                        } else {
                            const bool fj = stF[valid ? t : lo] == T_FLUID;
#pragma unroll
                            for (int g = 0; g < G; ++g) {
                                const bool hit = hits[g];
                                const bool take = hit && (((fl >> g) & 1u) || fj);
                                nn[g] += __popc(__ballot_sync(0xffffffffu, hit));
                                const unsigned m = __ballot_sync(0xffffffffu, take);
                                if (take && SPH_BOUNDS_OK(cnt[g] + __popc(m & lt) < LC && t < max_stage, &b.misc[2]))
                                    wl0[g * LC + cnt[g] + __popc(m & lt)] = (uint16_t)t;
                                cnt[g] += __popc(m);
                            }
                        }
                    };
                    for (int r = 0; r < nrow; ++r) {
                        const int lo = __shfl_sync(0xffffffffu, r < 32 ? wlo[0] : wlo[1], r & 31);
                        const int hi = __shfl_sync(0xffffffffu, r < 32 ? whi[0] : whi[1], r & 31);
                        // Room for the whole row window in every list is made before the
                        // row; only a window longer than LC - 32 is checked step by step.
                        bool need = false;
#pragma unroll
                        for (int g = 0; g < G; ++g)
                            need = need || cnt[g] + (hi - lo) > LC;
                        if (need)
                            flush();
                        if (hi - lo <= LC - 32) {
                            for (int32_t base = lo; base < hi; base += 32)
                                sweep(base, lo, hi);
                        } else {
                            for (int32_t base = lo; base < hi; base += 32) {
                                sweep(base, lo, hi);
                                bool full = false;
#pragma unroll
                                for (int g = 0; g < G; ++g)
                                    full = full || cnt[g] > LC - 32;
                                if (full)
                                    flush();
                            }
                        }
                    }
                    __syncwarp();
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        if (ib + g < ie)
                            drain(g, cnt[g]);
                        np[g] += cnt[g];
                    }
                    {
                        int32_t slot[G];
                        bool valid[G];
                        int nsum[G], npair[G];
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            const int32_t ii = ib + g;
                            // the staged copy of i itself is a hit (and a zero term) in its chunk
                            const int32_t self = home_flat0 + (ii - h0);
                            const int selfc = (ii < ie && self >= f0 && self < f1) ? 1 : 0;
                            slot[g] = ii - g0;
                            valid[g] = ii < ie;
                            // every hit of a fluid particle is evaluated, so nn = np there
                            nsum[g] = (((fl >> g) & 1u) ? np[g] : nn[g]) - selfc;
                            npair[g] = np[g] - selfc;
                        }
                        combine_group<G, COMP, DFS>(S, acc, slot, valid, nsum, npair, nbits);
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            for (int32_t ii = g0 + tid; ii < g1; ii += blockDim.x) {
                const float *A = S.acc[ii - g0];
                float az = A[3] + A[8];
                if (b.sflag[ii] == T_FLUID)
                    az -= I.gf;
                float drho = A[0] + A[5];
                if (DFS && !S.nb[ii - g0]) {  // the delta term only with a fluid-only support
                    float e = A[5];
                    float sum = A[0];
                    two_sum(sum, e, S.dd[ii - g0][0]);
                    drho = sum + (e + S.dd[ii - g0][1]);
                }
                gD[ii] = make_float4(A[1] + A[6], A[2] + A[7], az, drho);
                gM[ii] = I.hf * A[4];
                b.nneigh[ii] = S.nn[ii - g0];
                b.npair[ii] = S.np[ii - g0];
                b.ncand[ii] = total;
            }
        }
        __syncthreads();
    }
    if (!CNT)
        return;
    // work counts: lanes -> warp -> CTA -> device
    const uint32_t wff = (uint32_t)warp_sum((int)lc_ff), wvi = (uint32_t)warp_sum((int)lc_visc);
    if (lane == 0) {
        atomicAdd(&S.st_ff, (unsigned long long)wff);
        atomicAdd(&S.st_visc, (unsigned long long)wvi);
        atomicAdd(&S.st_cand, wc_cand);
    }
    __syncthreads();
    if (tid == 0) {
        atomicAdd(&b.pstat[0], S.st_ff);
        atomicAdd(&b.pstat[1], S.st_visc);
        atomicAdd(&b.pstat[2], S.st_cand);
    }
}

}  // namespace sph
