// Launchers of the mixed-precision pair pass (Eqs. 3-8); the kernel body, its
// work decomposition and its compensated sums are described in pair_mixed.cuh.
#include "pair_mixed.cuh"

namespace sph {

// One CTA per resident slot; the body lives in pair_mixed.cuh.
template <int NW, int G, bool COMP, bool CNT, bool DFS>
__global__ void __launch_bounds__(NW * 32, NW >= 16 ? 1 : 2) k_pair_mixed(Bufs b, int ninst, int kdiv, int max_stage)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ PairSmem S;
    pair_mixed_body<NW, G, COMP, CNT, DFS>(b, ninst, kdiv, max_stage, dyn, S);
}

template <int NW, int G, bool COMP, bool CNT, bool DFS>
static void launch_nw(const Bufs &b, int ninst, int kdiv, int ctas, int max_stage, cudaStream_t st)
{
    const int sms = sm_count();
    const size_t dyn = mixed_dyn_smem(max_stage, NW, G);
    static size_t dyn_set = 0;  // attribute set once per instantiation, outside any capture
    if (dyn > dyn_set) {
        cudaFuncSetAttribute(k_pair_mixed<NW, G, COMP, CNT, DFS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn);
        dyn_set = dyn;
    }
    k_pair_mixed<NW, G, COMP, CNT, DFS><<<sms * ctas, NW * 32, dyn, st>>>(b, ninst, kdiv, max_stage);
}

template <bool COMP, bool CNT, bool DFS>
static void launch_comp(const Bufs &b, int ninst, int kdiv, int warps, int group, int ctas, int max_stage,
                        cudaStream_t st)
{
    if (group >= 4) {
        if (warps <= 4)
            launch_nw<4, 4, COMP, CNT, DFS>(b, ninst, kdiv, ctas, max_stage, st);
        else
            launch_nw<8, 4, COMP, CNT, DFS>(b, ninst, kdiv, ctas, max_stage, st);
    } else if (group >= 2) {
        if (warps <= 4)
            launch_nw<4, 2, COMP, CNT, DFS>(b, ninst, kdiv, ctas, max_stage, st);
        else
            launch_nw<8, 2, COMP, CNT, DFS>(b, ninst, kdiv, ctas, max_stage, st);
    } else {
        if (warps <= 4)
            launch_nw<4, 1, COMP, CNT, DFS>(b, ninst, kdiv, ctas, max_stage, st);
        else if (warps <= 8)
            launch_nw<8, 1, COMP, CNT, DFS>(b, ninst, kdiv, ctas, max_stage, st);
        else
            launch_nw<16, 1, COMP, CNT, DFS>(b, ninst, kdiv, ctas, max_stage, st);
    }
}

void launch_pair_mixed(const Bufs &b, int64_t N, int32_t ninst, int32_t cell_div, int32_t warps, int32_t ctas,
                       int32_t group, int32_t compensated, int32_t max_active, bool count, int32_t delta_mode,
                       cudaStream_t st)
{
    (void)N;
    (void)max_active;
    // defaults: the fastest launch shape measured on GB300 for cells of size 2h
    if (warps <= 0)
        warps = 8;
    if (ctas <= 0)
        ctas = 2;
    if (group <= 0)
        group = 4;
    const int max_stage = mixed_max_stage(cell_div);
    cudaMemsetAsync(b.misc + 3, 0, sizeof(int32_t), st);
    if (count)
        cudaMemsetAsync(b.pstat, 0, 4 * sizeof(unsigned long long), st);
    if (delta_mode == SPH_DELTA_FULL_SUPPORT) {  // always compensated
        if (count)
            launch_comp<true, true, true>(b, ninst, cell_div, warps, group, ctas, max_stage, st);
        else
            launch_comp<true, false, true>(b, ninst, cell_div, warps, group, ctas, max_stage, st);
    } else if (count) {
        if (compensated)
            launch_comp<true, true, false>(b, ninst, cell_div, warps, group, ctas, max_stage, st);
        else
            launch_comp<false, true, false>(b, ninst, cell_div, warps, group, ctas, max_stage, st);
    } else if (compensated) {
        launch_comp<true, false, false>(b, ninst, cell_div, warps, group, ctas, max_stage, st);
    } else {
        launch_comp<false, false, false>(b, ninst, cell_div, warps, group, ctas, max_stage, st);
    }
}

}  // namespace sph
