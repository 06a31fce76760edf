// FP64 form of the pair pass (Eqs. 3-8) and the obstacle-force probe.
//
// One warp per particle i (sorted order).  The lanes sweep i's candidate
// rows: for every (dy, dz) cell offset the cells cx-k .. cx+k of that row are
// consecutive in the sorted order, so each row is one contiguous range.  A
// candidate j is a neighbour when |r_j - r_i|^2 < (2h)^2, evaluated as
// ((dx dx + dy dy) + dz dz) with every operation rounded separately, so the
// neighbour set is the same set the definition gives; an FP32 pre-test on
// FP32 copies of the positions, with radii moved out and in by their worst
// rounding error, settles every candidate certainly out of reach or certainly
// inside, so that only a thin shell around 2h takes the exact test.  Neighbours that
// interact are compacted through a per-warp queue by ballot, so that the
// expensive pair arithmetic runs on full 32-lane batches (all but the last
// batch of each particle); the lane partial sums are combined by warp shuffles.
#include "device.cuh"

namespace sph {

constexpr int kQ = 64;  // per-warp queue of neighbour indices

struct AccD {
    double drho, ax, ay, az;
    double dd;  // the delta term of Eq. 7, kept apart when it may be dropped (SPH_DELTA_FULL_SUPPORT)
    // running max of mu / h as the bit pattern of a double read as a signed
    // integer: non-negative doubles order like their bit patterns and negative
    // ones fall below the starting 0 (+0.0), so the integer max is the max of
    // mu started at 0, taken on the integer units instead of the FP64 pipe
    long long mumax_bits;
};

// Constants of an instance used by every pair, computed once per particle.
struct PairConstD {
    double half_inv_h, kFm, dfac, nah, eta2;  // kFm = kF m, dfac = 2 delta h c0, nah = -alpha h
};

__device__ __forceinline__ PairConstD pair_const_d(const Inst &I)
{
    return PairConstD{0.5 / I.h, I.kF * I.mass, 2.0 * I.delta * I.h * I.c0, -I.alpha * I.h, I.eta2};
}

// Contribution of neighbour j to particle i (Eqs. 3-7), in double.
// Continuity uses the standard sign (u_i - u_j) . grad_i W_ij; the delta
// term acts between fluid particles; the viscosity of Eq. 4 applies when
// u_ij . r_ij < 0.  1/rho and c of both particles come precomputed, so a pair
// costs one reciprocal square root and two correctly rounded reciprocals (mu,
// and the viscosity's mean density when it applies).  m_j F = -kF m t^3 with
// t = 1 - q/2: the sums of D rho/Dt and of the acceleration are accumulated
// with t^3 in place of m_j F and the caller scales them by -kF m, and the
// running maximum is of mu / h, which the caller scales by h.  With DFS the
// delta term is summed apart (the caller drops it for a fluid particle that
// has a boundary neighbour).
template <bool DFS>
__device__ __forceinline__ void pair_term_d(const PairConstD &k, double xi, double yi, double zi, double uxi,
                                            double uyi, double uzi, double rhoi, double inv_rhoi, double Pi,
                                            double ci, bool fluid_i, double xj, double yj, double zj, double uxj,
                                            double uyj, double uzj, double rhoj, double inv_rhoj, double Pj,
                                            double cj, bool fluid_j, AccD &a)
{
    double rx = xj - xi, ry = yj - yi, rz = zj - zi;  // r_ij = r_j - r_i
    double ux = uxj - uxi, uy = uyj - uyi, uz = uzj - uzi;  // u_ij = u_j - u_i
    double r2 = rx * rx + ry * ry + rz * rz;
    // |r_ij| = r2 / sqrt(r2); the integer max (on the bit pattern) lifts r2 = 0
    // (coincident particles) to the smallest subnormal, so that r = 0 there
    double r = r2 * rsqrt(__longlong_as_double(max(__double_as_longlong(r2), 1LL)));
    double t = 1.0 - r * k.half_inv_h;
    double t3 = t * t * t;  // m_j F / (-kF m), grad_i W_ij = F (r_i - r_j) = -F r_ij
    double udotr = ux * rx + uy * ry + uz * rz;  // u_ij . r_ij
    // Eq. 7: sum_j m_j (u_i - u_j) . grad_i W_ij = m_j F (u_ij . r_ij), plus the delta term
    // 2 delta h c0 (rho_j - rho_i) (r_ij . grad_i W_ij) / |r_ij|^2 m_j / rho_j, where
    // (r_ij . grad_i W_ij) / |r_ij|^2 = -F and (rho_j - rho_i) / rho_j = 1 - rho_i / rho_j
    double g = (fluid_i && fluid_j) ? fma(-k.dfac * rhoi, inv_rhoj, k.dfac) : 0.0;
    if (DFS) {
        a.drho = fma(t3, udotr, a.drho);
        a.dd = fma(t3, g, a.dd);
    } else {
        a.drho = fma(t3, udotr - g, a.drho);
    }
    // Eqs. 4-5: Pi_ij = -alpha c_bar mu / rho_bar, c_bar / rho_bar = (c_i + c_j) / (rho_i + rho_j),
    // mu = h (u_ij . r_ij) / (|r_ij|^2 + eta^2) = h muh
    double muh = udotr * __drcp_rn(r2 + k.eta2);
    double visc = 0.0;
    if (__double2hiint(udotr) < 0)  // u_ij . r_ij < 0 (a -0.0 gives a zero term)
        visc = fma(k.nah, cj, k.nah * ci) * muh * __drcp_rn(rhoi + rhoj);
    // Eq. 3: a_i -= m_j (...) grad_i W_ij = m_j (...) F r_ij, with
    // (P_i + P_j) / (rho_i rho_j) = (P_i / rho_i + P_j / rho_i) / rho_j
    double coef = fma(fma(Pj, inv_rhoi, Pi * inv_rhoi), inv_rhoj, visc) * t3;
    a.ax += coef * rx;
    a.ay += coef * ry;
    a.az += coef * rz;
    a.mumax_bits = max(a.mumax_bits, __double_as_longlong(muh));
}

// Partner's share of a pair evaluated once (params.pair_symmetric): the terms
// of Eqs. 3, 7 and 15 for j from the same pair, added to j's accumulators in
// global memory by FP64 atomics (performed in L2).  Eq. 3 is antisymmetric
// ((P_i + P_j)/(rho_i rho_j) and Pi_ij are symmetric, r_ji = -r_ij), Eq. 7
// has the same continuity term and j's own delta term
// 2 delta h c0 (1 - rho_j / rho_i), mu is the same; units as pair_term_d
// (t^3 in place of m F, mu / h).  i's own share is accumulated in a.
__device__ __forceinline__ void pair_share_j(const PairConstD &k, double xi, double yi, double zi, double uxi,
                                             double uyi, double uzi, double rhoi, double inv_rhoi, double Pi,
                                             double ci, bool fluid_i, double xj, double yj, double zj, double uxj,
                                             double uyj, double uzj, double rhoj, double inv_rhoj, double Pj,
                                             double cj, bool fluid_j, dvec4 *jacc, long long *jmu, int32_t j,
                                             AccD &a)
{
    double rx = xj - xi, ry = yj - yi, rz = zj - zi;
    double ux = uxj - uxi, uy = uyj - uyi, uz = uzj - uzi;
    double r2 = rx * rx + ry * ry + rz * rz;
    double r = r2 * rsqrt(__longlong_as_double(max(__double_as_longlong(r2), 1LL)));
    double t = 1.0 - r * k.half_inv_h;
    double t3 = t * t * t;
    double udotr = ux * rx + uy * ry + uz * rz;
    const bool ff = fluid_i && fluid_j;
    double g = ff ? fma(-k.dfac * rhoi, inv_rhoj, k.dfac) : 0.0;
    double gj = ff ? fma(-k.dfac * rhoj, inv_rhoi, k.dfac) : 0.0;
    a.drho = fma(t3, udotr - g, a.drho);
    double muh = udotr * __drcp_rn(r2 + k.eta2);
    double visc = 0.0;
    if (__double2hiint(udotr) < 0)
        visc = fma(k.nah, cj, k.nah * ci) * muh * __drcp_rn(rhoi + rhoj);
    double coef = fma(fma(Pj, inv_rhoi, Pi * inv_rhoi), inv_rhoj, visc) * t3;
    a.ax += coef * rx;
    a.ay += coef * ry;
    a.az += coef * rz;
    a.mumax_bits = max(a.mumax_bits, __double_as_longlong(muh));
    double *J = reinterpret_cast<double *>(jacc + j);
    atomicAdd(J + 0, -coef * rx);
    atomicAdd(J + 1, -coef * ry);
    atomicAdd(J + 2, -coef * rz);
    atomicAdd(J + 3, t3 * (udotr - gj));
    if (muh > 0.0)
        atomicMax(jmu + j, __double_as_longlong(muh));  // positive doubles order like their bits
}

__device__ __forceinline__ double dist2_rn(double xi, double yi, double zi, double xj, double yj, double zj)
{
    double dx = __dsub_rn(xj, xi), dy = __dsub_rn(yj, yi), dz = __dsub_rn(zj, zi);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// SYM: each interacting pair once (the forward half of i's neighbourhood:
// rows with dz > 0, rows with dz = 0 and dy > 0, and the home row after i),
// the partner's share by pair_share_j; k_pair_fp64_finish adds the shares.
// CNT (with SYM): also count the partners' neighbours (nneigh is read by
// sph_derivatives and the work counts, not by a time step).
template <bool DFS, bool SYM, bool CNT = true>
__global__ void __launch_bounds__(256) k_pair_fp64(Bufs b, int ninst, int kdiv)
{
    extern __shared__ int32_t smem_q[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int32_t *q = smem_q + wib * kQ;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t n_in = b.misc[0];
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const dvec4 *sA = reinterpret_cast<const dvec4 *>(b.sA);
    const dvec4 *sB = reinterpret_cast<const dvec4 *>(b.sB);

    for (int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_in; i += nwarps) {
        const int32_t ci_cell = b.scell[i];
        const Inst &I = b.inst[inst_of_cell(b.inst, ninst, ci_cell)];
        int cx, cy, cz;
        decompose(I, ci_cell, cx, cy, cz);
        const dvec4 Ai = sA[i], Bi = sB[i];
        const double2 Ci = b.sC[i];
        const float4 Di = b.sD[i];
        const bool fluid_i = b.sflag[i] == T_FLUID;
        const PairConstD kc = pair_const_d(I);
        AccD acc = {0.0, 0.0, 0.0, 0.0, 0.0, 0};
        bool touches_boundary = false;  // DFS: some neighbour j is a boundary particle
        int nn = 0;
        int qn = 0;
        int npair = 0, ncand = 0;

        auto flush = [&](int cnt) {
            if (lane < cnt) {
                int32_t j = q[lane];
                dvec4 Aj = sA[j], Bj = sB[j];
                double2 Cj = b.sC[j];
                if (SYM)
                    pair_share_j(kc, Ai.x, Ai.y, Ai.z, Bi.x, Bi.y, Bi.z, Ai.w, Ci.x, Bi.w, Ci.y, fluid_i, Aj.x, Aj.y,
                                 Aj.z, Bj.x, Bj.y, Bj.z, Aj.w, Cj.x, Bj.w, Cj.y, b.sflag[j] == T_FLUID, b.fjacc, b.fjmu,
                                 j, acc);
                else
                    pair_term_d<DFS>(kc, Ai.x, Ai.y, Ai.z, Bi.x, Bi.y, Bi.z, Ai.w, Ci.x, Bi.w, Ci.y, fluid_i, Aj.x,
                                     Aj.y, Aj.z, Bj.x, Bj.y, Bj.z, Aj.w, Cj.x, Bj.w, Cj.y, b.sflag[j] == T_FLUID, acc);
            }
        };

        for (int dz = SYM ? 0 : -kdiv; dz <= kdiv; ++dz) {
            int z = cz + dz;
            if (z < 0 || z >= I.n[2])
                continue;
            for (int dy = (SYM && dz == 0) ? 0 : -kdiv; dy <= kdiv; ++dy) {
                int y = cy + dy;
                if (y < 0 || y >= I.n[1])
                    continue;
                int x0 = max(cx - kdiv, 0), x1 = min(cx + kdiv, I.n[0] - 1);
                int32_t row = I.cell_base + (z * I.n[1] + y) * I.n[0];
                int32_t s0 = b.cell_start[row + x0], s1 = b.cell_start[row + x1 + 1];
                if (SYM && dz == 0 && dy == 0)
                    s0 = i + 1;  // the home row from the home cell on (cells hold ascending ids), after i
                for (int32_t base = s0; base < s1; base += 32) {
                    int32_t j = base + lane;
                    bool take = false;
                    if (j < s1 && j != i) {
                        // FP32 pre-test with radii that cover every rounding of the
                        // FP32 copies: certainly inside, certainly outside, or (in a
                        // thin shell around 2h) decided by the exact FP64 test
                        const float4 Dj = b.sD[j];
                        const float fx = Dj.x - Di.x, fy = Dj.y - Di.y, fz = Dj.z - Di.z;
                        const float d2f = fx * fx + fy * fy + fz * fz;
                        bool hit = d2f < I.sup2_inner;
                        if (!hit && d2f < I.sup2_filter) {
                            dvec4 Aj = sA[j];
                            hit = dist2_rn(Ai.x, Ai.y, Ai.z, Aj.x, Aj.y, Aj.z) < I.sup2;
                        }
                        if (hit) {
                            ++nn;
                            if (SYM && CNT)
                                atomicAdd(b.fjnn + j, 1);
                            const bool fluid_j = b.sflag[j] == T_FLUID;
                            take = fluid_i || fluid_j;
                            if (DFS)
                                touches_boundary = touches_boundary || !fluid_j;
                        }
                    }
                    unsigned m = __ballot_sync(0xffffffffu, take);
                    if (take)
                        q[qn + __popc(m & lt)] = j;
                    qn += __popc(m);
                    npair += __popc(m);
                    ncand += min(32, s1 - base);
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
            }
        }
        flush(qn);
        __syncwarp();
        const double sF = -kc.kFm;  // t^3 -> m_j F
        constexpr int K = DFS ? 8 : 4;
        double tot[K] = {acc.drho, acc.ax, acc.ay, acc.az};
        if (DFS)
            tot[4] = acc.dd;
        warp_totals<K>(tot);  // lane 0 holds the totals
        double drho_sum = tot[0];
        if (DFS && !__any_sync(0xffffffffu, touches_boundary))
            drho_sum -= tot[K > 4 ? 4 : 0];
        double drho = sF * drho_sum;
        double ax = sF * tot[1], ay = sF * tot[2], az = sF * tot[3];
        double mumax = I.h * warp_max(__longlong_as_double(acc.mumax_bits));
        int nsum = warp_sum(nn);
        if (lane == 0) {
            if (fluid_i)
                az -= I.g;
            reinterpret_cast<dvec4 *>(b.deriv)[i] = make_dvec4(ax, ay, az, drho);
            reinterpret_cast<double *>(b.mumax)[i] = mumax;
            b.nneigh[i] = nsum;
            b.npair[i] = npair;
            b.ncand[i] = ncand;
        }
    }
}

// Adds the partners' shares of the symmetric pass, scaled as the owner's.
template <bool CNT>
__global__ void k_pair_fp64_finish(Bufs b, int ninst)
{
    const int32_t n_in = b.misc[0];
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_in; s += gridDim.x * blockDim.x) {
        const Inst &I = b.inst[inst_of_cell(b.inst, ninst, b.scell[s])];
        const double sF = -I.kF * I.mass;
        const dvec4 j = b.fjacc[s];
        dvec4 *D = reinterpret_cast<dvec4 *>(b.deriv) + s;
        const dvec4 d = *D;
        *D = make_dvec4(d.x + sF * j.x, d.y + sF * j.y, d.z + sF * j.z, d.w + sF * j.w);
        double *M = reinterpret_cast<double *>(b.mumax) + s;
        *M = fmax(*M, I.h * __longlong_as_double(b.fjmu[s]));
        if (CNT)
            b.nneigh[s] += b.fjnn[s];
    }
}

void launch_pair_fp64(const Bufs &b, int64_t N, int32_t ninst, int32_t cell_div, int32_t warps, int32_t ctas,
                      int32_t delta_mode, bool neighbours, cudaStream_t st)
{
    if (warps <= 0 || warps > 8)
        warps = 8;  // the kernel is compiled for at most 256 threads per CTA
    if (ctas <= 0)
        ctas = 8;
    const int sms = sm_count();
    if (b.fjacc) {
        // the partners' accumulators start at zero (mu / h >= 0 as bits)
        cudaMemsetAsync(b.fjacc, 0, sizeof(dvec4) * (size_t)N, st);
        cudaMemsetAsync(b.fjmu, 0, sizeof(long long) * (size_t)N, st);
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, (int64_t)sms * 8));
        if (neighbours) {
            cudaMemsetAsync(b.fjnn, 0, sizeof(int32_t) * (size_t)N, st);
            k_pair_fp64<false, true, true><<<sms * ctas, warps * 32, warps * kQ * sizeof(int32_t), st>>>(b, ninst,
                                                                                                      cell_div);
            k_pair_fp64_finish<true><<<blocks, 256, 0, st>>>(b, ninst);
        } else {
            k_pair_fp64<false, true, false><<<sms * ctas, warps * 32, warps * kQ * sizeof(int32_t), st>>>(b, ninst,
                                                                                                       cell_div);
            k_pair_fp64_finish<false><<<blocks, 256, 0, st>>>(b, ninst);
        }
        return;
    }
    if (delta_mode == SPH_DELTA_FULL_SUPPORT)
        k_pair_fp64<true, false><<<sms * ctas, warps * 32, warps * kQ * sizeof(int32_t), st>>>(b, ninst, cell_div);
    else
        k_pair_fp64<false, false><<<sms * ctas, warps * 32, warps * kQ * sizeof(int32_t), st>>>(b, ninst, cell_div);
}

// ---------------------------------------------------------------------------
// Force on the obstacle (Section 3.2): sum over its particles of m a_b, a_b
// from fluid neighbours by Eq. 3 without gravity, in double on the current
// state (read through the canonical arrays, so both precision forms agree).
// ---------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void load_state(const Bufs &b, const Inst &I, int32_t id, double &x, double &y,
                                           double &z, double &ux, double &uy, double &uz, double &rho)
{
    dvec4 p = b.pos[id];
    x = p.x;
    y = p.y;
    z = p.z;
    if (MODE == SPH_FP64) {
        dvec4 v = reinterpret_cast<const dvec4 *>(b.vel)[id];
        ux = v.x;
        uy = v.y;
        uz = v.z;
        rho = v.w;
    } else {
        float4 v = reinterpret_cast<const float4 *>(b.vel)[id];
        ux = v.x;
        uy = v.y;
        uz = v.z;
        rho = I.rho0 + (double)v.w;
    }
}

template <int MODE>
__global__ void k_probe_force(Bufs b, int inst, int kdiv)
{
    __shared__ double part[8][3];
    const Inst &I = b.inst[inst];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int32_t s_begin = b.cell_start[I.cell_base], s_end = b.cell_start[I.cell_base + I.ncells];
    double fx = 0, fy = 0, fz = 0;
    for (int32_t s = s_begin + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); s < s_end; s += nwarps) {
        if (b.sflag[s] != T_OBST)
            continue;
        int32_t idb = b.perm[s];
        double xb, yb, zb, uxb, uyb, uzb, rhob;
        load_state<MODE>(b, I, idb, xb, yb, zb, uxb, uyb, uzb, rhob);
        double Pb = tait_d(I, rhob), cb = sound_d(I, rhob);
        const PairConstD kc = pair_const_d(I);
        int cx, cy, cz;
        decompose(I, b.scell[s], cx, cy, cz);
        AccD acc = {0, 0, 0, 0, 0};
        for (int dz = -kdiv; dz <= kdiv; ++dz) {
            int z = cz + dz;
            if (z < 0 || z >= I.n[2])
                continue;
            for (int dy = -kdiv; dy <= kdiv; ++dy) {
                int y = cy + dy;
                if (y < 0 || y >= I.n[1])
                    continue;
                int x0 = max(cx - kdiv, 0), x1 = min(cx + kdiv, I.n[0] - 1);
                int32_t row = I.cell_base + (z * I.n[1] + y) * I.n[0];
                int32_t s0 = b.cell_start[row + x0], s1 = b.cell_start[row + x1 + 1];
                for (int32_t j = s0 + lane; j < s1; j += 32) {
                    if (b.sflag[j] != T_FLUID)
                        continue;
                    int32_t idj = b.perm[j];
                    double xj, yj, zj, uxj, uyj, uzj, rhoj;
                    load_state<MODE>(b, I, idj, xj, yj, zj, uxj, uyj, uzj, rhoj);
                    if (dist2_rn(xb, yb, zb, xj, yj, zj) < I.sup2)
                        pair_term_d<false>(kc, xb, yb, zb, uxb, uyb, uzb, rhob, 1.0 / rhob, Pb, cb, false, xj, yj, zj, uxj,
                                    uyj, uzj, rhoj, 1.0 / rhoj, tait_d(I, rhoj), sound_d(I, rhoj), true, acc);
                }
            }
        }
        const double sF = -kc.kFm * I.mass;  // t^3 -> m_j F, times the obstacle particle's mass
        fx += sF * acc.ax;
        fy += sF * acc.ay;
        fz += sF * acc.az;
    }
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    fz = warp_sum(fz);
    if (lane == 0) {
        part[wib][0] = fx;
        part[wib][1] = fy;
        part[wib][2] = fz;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            s += part[w][threadIdx.x];
        b.diag[blockIdx.x * 3 + threadIdx.x] = s;
    }
}

__global__ void k_sum_blocks3(const double *part, int nb, double *out)
{
    if (threadIdx.x < 3) {
        double s = 0;
        for (int k = 0; k < nb; ++k)
            s += part[k * 3 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

void launch_probe_force(const Bufs &b, int mode, int32_t inst, int32_t ninst, int32_t cell_div, int64_t N,
                        cudaStream_t st)
{
    (void)ninst;
    (void)N;
    const int nb = kDiagBlocks;
    if (mode == SPH_FP64)
        k_probe_force<SPH_FP64><<<nb, 256, 0, st>>>(b, inst, cell_div);
    else
        k_probe_force<SPH_MIXED><<<nb, 256, 0, st>>>(b, inst, cell_div);
    k_sum_blocks3<<<1, 32, 0, st>>>(b.diag, nb, b.probe_out);
}

}  // namespace sph
