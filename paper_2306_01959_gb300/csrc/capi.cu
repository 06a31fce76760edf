// C ABI and engine: workspace layout, step sequencing, CUDA-graph replay,
// per-phase event timing, probes and state transfer.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "device.cuh"

using namespace sph;

namespace {

enum Phase { PH_PAIR = 0, PH_DT, PH_INTEGRATE, PH_CELLS, PH_REORDER, PH_PERSIST, PH_COUNT };
const char *kPhaseNames[PH_COUNT] = {"pair", "dt", "integrate", "cells", "reorder", "persistent"};

// Host staging buffer of n bytes, 32-byte aligned like the device arrays of
// dvec4 or float4 it mirrors.
struct HostBytes {
    std::vector<dvec4> v;
    explicit HostBytes(size_t n) : v((n + sizeof(dvec4) - 1) / sizeof(dvec4)) {}
    char *data() { return reinterpret_cast<char *>(v.data()); }
};

struct Layout {
    size_t off = 0;
    char *base = nullptr;
    template <class T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * (count ? count : 1);
        return p;
    }
};

}  // namespace

struct sph_s {
    sph_params p{};
    int mode = SPH_FP64;
    std::vector<HostInst> inst;
    int64_t N = 0;
    int32_t C = 0;
    int32_t ninst = 0;
    int32_t max_active = 0;
    int32_t C_alloc = 0;      // cells the workspace holds: the largest grid, at cell_div 3
    int32_t reorder_ctas = 16; // resident CTAs per SM of the per-cell sort and gather (tuned)
    int32_t list_cap = 0;      // neighbour-list entries per particle (0: no lists)
    Bufs b{};
    cudaStream_t st = nullptr;
    cudaStream_t cap = nullptr;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    std::string err;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    double dt_host = 0.0;
    bool dt_uploaded = false;
    int pair_warps = 0, pair_ctas = 0, pair_group = 0;
    bool prof = false;
    std::vector<cudaEvent_t> ev;  // 2 per phase per profiled step
    std::vector<int> ev_phase;    // phase of each event pair
    size_t ev_used = 0;
    double phase_ms[PH_COUNT] = {};
    int64_t phase_n[PH_COUNT] = {};
    int64_t nf_tot = 0, nw_tot = 0, no_tot = 0, ng_tot = 0;
};

static int fail(sph_t *s, int code, const std::string &m)
{
    if (s)
        s->err = m;
    return code;
}

static int cuda_fail(sph_t *s, cudaError_t e, const char *where)
{
    return fail(s, SPH_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess)                    \
            return cuda_fail(s, e_, #call);       \
    } while (0)

static size_t layout(Bufs &b, char *base, int64_t N, int32_t C, int32_t ninst, int mode, int32_t list_cap,
                     bool fp64_sym)
{
    Layout L;
    L.base = base;
    const size_t vsz = mode == SPH_FP64 ? sizeof(dvec4) : sizeof(float4);
    b.pos = L.take<dvec4>(N);
    b.vel = L.take<char>(N * vsz);
    b.velp = L.take<char>(N * vsz);
    b.type = L.take<uint8_t>(N);
    b.inst_of = L.take<uint16_t>(N);
    b.key = L.take<uint32_t>(N);
    b.count = L.take<uint32_t>((size_t)C + 1);
    b.cell_start = L.take<int32_t>((size_t)C + 2);
    b.active = L.take<int32_t>((size_t)C);
    b.scan_blocks = L.take<uint64_t>(((size_t)C + 1 + kScanTile - 1) / kScanTile);
    b.perm = L.take<int32_t>(N);
    b.ptmp = L.take<int32_t>(N);
    b.scell = L.take<int32_t>(N);
    b.sA = L.take<char>(N * vsz);
    b.sB = L.take<char>(N * vsz);
    b.sC = mode == SPH_FP64 ? L.take<double2>(N) : nullptr;
    b.sD = mode == SPH_FP64 ? L.take<float4>(N) : nullptr;
    b.sflag = L.take<uint8_t>(N);
    b.deriv = L.take<char>(N * vsz);
    b.mumax = L.take<char>(N * (mode == SPH_FP64 ? sizeof(double) : sizeof(float)));
    b.nneigh = L.take<int32_t>(N);
    b.npair = L.take<int32_t>(N);
    b.ncand = L.take<int32_t>(N);
    b.pstat = L.take<unsigned long long>(4);
    b.red = L.take<unsigned long long>(2 * (size_t)ninst);
    b.dt = L.take<double>(ninst);
    b.time = L.take<double>(ninst);
    b.dt_fixed = L.take<double>(1);
    b.step = L.take<long long>(1);
    b.euler = L.take<int32_t>(1);
    b.misc = L.take<int32_t>(16);
    b.bar = L.take<unsigned>(4);
    b.inst = L.take<Inst>(ninst);
    b.probe_in = L.take<double>((size_t)kMaxProbe * 3);
    b.probe_out = L.take<double>((size_t)kMaxProbe * 4);
    b.probe_k = L.take<int32_t>(kMaxProbe);
    b.diag = L.take<double>((size_t)kDiagBlocks * 10);
    b.list_cap = list_cap;
    b.nlist = list_cap ? L.take<int32_t>((size_t)N * list_cap) : nullptr;
    b.ncnt = list_cap ? L.take<int32_t>(N) : nullptr;
    b.xbuild = list_cap ? L.take<dvec4>(N) : nullptr;
    b.lflag = list_cap ? L.take<int32_t>(8) : nullptr;
    b.fjacc = fp64_sym ? L.take<dvec4>(N) : nullptr;
    b.fjmu = fp64_sym ? L.take<long long>(N) : nullptr;
    b.fjnn = fp64_sym ? L.take<int32_t>(N) : nullptr;
    return (L.off + 255) & ~(size_t)255;
}

static int prepare_sizes(sph_t *s, int32_t n_inst, const sph_instance *in, const sph_params *p)
{
    if (!p || p->size != sizeof(sph_params))
        return fail(s, SPH_EINVAL, "sph_params.size must equal sizeof(sph_params)");
    if (p->persistent && (p->precision != SPH_MIXED || p->integrator != SPH_VERLET))
        return fail(s, SPH_EINVAL, "persistent launches run the mixed form with the Verlet scheme only");
    if (p->spin_limit < 0)
        return fail(s, SPH_EINVAL, "spin_limit must be >= 0");
    if (n_inst < 1 || n_inst > 65535 || !in)
        return fail(s, SPH_EINVAL, "n_inst must be in [1, 65535] with a non-NULL instance array");
    s->p = *p;
    s->mode = p->precision;
    s->p.cell_div = effective_cell_div(*p);
    s->inst.resize(n_inst);
    int64_t N = 0, C = 0;
    for (int k = 0; k < n_inst; ++k) {
        std::string e;
        int rc = validate_instance(in[k], *p, e);
        if (rc)
            return fail(s, rc, "instance " + std::to_string(k) + ": " + e);
        HostInst &hi = s->inst[k];
        hi.d = in[k];
        fill_inst(hi, *p);
        hi.dev.pbase = (int32_t)N;
        hi.dev.cell_base = (int32_t)C;
        N += hi.nf + hi.nw + hi.no + hi.ng;
        C += hi.dev.ncells;
        s->nf_tot += hi.nf;
        s->nw_tot += hi.nw;
        s->no_tot += hi.no;
        s->ng_tot += hi.ng;
        if (N >= (int64_t)1 << 31 || C >= ((int64_t)1 << 31) - 4)
            return fail(s, SPH_EINVAL, "too many particles or cells (limit 2^31)");
    }
    if (N == 0)
        return fail(s, SPH_EINVAL, "no particles");
    // room for the finest grid the autotuner may choose (cells of 2h/3)
    int64_t C3 = 0;
    {
        sph_params p3 = *p;
        p3.cell_div = std::max(3, effective_cell_div(*p));
        for (int k = 0; k < n_inst; ++k) {
            HostInst tmp = s->inst[k];
            fill_inst(tmp, p3);
            C3 += tmp.dev.ncells;
        }
    }
    if (C3 >= ((int64_t)1 << 31) - 4)
        return fail(s, SPH_EINVAL, "too many cells (limit 2^31)");
    s->C_alloc = (int32_t)std::max<int64_t>(C3, C);
    s->list_cap = 0;
    if (p->list_skin > 0) {
        // entries (j << 5 | cell offset) hold sorted indices below 2^26
        if (N >= (int64_t)1 << 26)
            return fail(s, SPH_EINVAL, "neighbour lists hold at most 2^26 particles");
        if (p->list_capacity > 0) {
            s->list_cap = p->list_capacity;
        } else {
            // the lattice count within 2h + s, plus a third, in multiples of 32
            double most = 0.0;
            for (int k = 0; k < n_inst; ++k) {
                const Inst &d = s->inst[k].dev;
                const double R = (2.0 * d.h + d.skin) / d.dp;
                most = std::max(most, 4.0 / 3.0 * 3.14159265358979323846 * R * R * R);
            }
            s->list_cap = (int32_t)std::min(65536.0, std::ceil(most * 4.0 / 3.0 / 32.0) * 32.0);
        }
    }
    s->N = N;
    s->C = (int32_t)C;
    s->ninst = n_inst;
    s->max_active = (int32_t)std::min<int64_t>(C, N);
    return SPH_OK;
}

extern "C" {

void sph_params_default(sph_params *p)
{
    std::memset(p, 0, sizeof(*p));
    p->size = sizeof(sph_params);
    p->precision = SPH_FP64;
    p->gamma = 7.0;
    p->g = 9.81;
    p->delta = 0.1;
    p->cfl = 0.2;
    p->dt_min = 1e-12;
    p->ns = 40;
    p->boundary_layers = 2;
    p->init = SPH_INIT_HYDROSTATIC;
    p->csound = SPH_CSOUND_EOS;
    p->cell_div = 0;
    p->use_graph = 1;
    p->graph_steps = 16;
    p->pair_warps = 0;
    p->pair_ctas_per_sm = 0;
    p->pair_group = 0;
    p->compensated = 1;
    p->integrator = SPH_VERLET;
}

int sph_workspace_size(int32_t n_inst, const sph_instance *inst, const sph_params *p, size_t *bytes)
{
    if (!bytes)
        return SPH_EINVAL;
    sph_s tmp;
    int rc = prepare_sizes(&tmp, n_inst, inst, p);
    if (rc)
        return rc;
    Bufs b{};
    *bytes = layout(b, nullptr, tmp.N, tmp.C_alloc, tmp.ninst, tmp.mode, tmp.list_cap, tmp.p.pair_symmetric != 0);
    return SPH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Engine steps
// ---------------------------------------------------------------------------
// With profiling on, CUDA events bracket each phase on the stream (their
// times are summed by sph_phase_times) and NVTX ranges name the phases on the
// host timeline of a profiler.
static void rec(sph_t *s, int phase, bool start)
{
    if (!s->prof)
        return;
    if (start)
        nvtxRangePushA(kPhaseNames[phase]);
    else
        nvtxRangePop();
    if (s->ev_used + 1 > s->ev.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        s->ev.push_back(e);
    }
    cudaEventRecord(s->ev[s->ev_used++], s->st);
    if (start)
        s->ev_phase.push_back(phase);
}

static void enqueue_prepare(sph_t *s, cudaStream_t st)
{
    if (s->b.lflag)
        cudaMemsetAsync(s->b.lflag, 1, 1, st);  // rebuild request: the structure and then the lists
    launch_bin(s->b, s->mode, s->N, s->C, st);
    launch_cells(s->b, s->N, s->C, st);
    launch_reorder(s->b, s->mode, s->N, s->C, s->ninst, s->max_active, s->reorder_ctas, st);
}

// count: also sum the per-class work counts of the mixed form (a separate
// instantiation, so that time steps pay nothing for them).  neighbours: the
// pass must write every particle's nneigh (sph_derivatives).
static void enqueue_pair(sph_t *s, cudaStream_t st, bool count = false, bool neighbours = false)
{
    if (s->mode == SPH_FP64) {
        launch_pair_fp64(s->b, s->N, s->ninst, s->p.cell_div, s->pair_warps, s->pair_ctas, s->p.delta_mode,
                         count || neighbours, st);
    } else if (s->b.lflag && !count) {
        launch_list_pass(s->b, s->N, s->ninst, s->p.delta_mode, st);
    } else
        launch_pair_mixed(s->b, s->N, s->ninst, s->p.cell_div, s->pair_warps, s->pair_ctas, s->pair_group,
                          s->p.compensated, s->max_active, count, s->p.delta_mode, st);
}

// Neighbour structure of the rebinned state and the sorted gather.  With
// neighbour lists the binning is its own kernel; binning, structure and
// sorted gather run only on a rebuild request, the gather into the kept order
// only without one.
static void enqueue_rebuild(sph_t *s, cudaStream_t st)
{
    rec(s, PH_CELLS, true);
    if (s->b.lflag)
        launch_bin(s->b, s->mode, s->N, s->C, st);
    launch_cells(s->b, s->N, s->C, st);
    rec(s, PH_CELLS, false);
    rec(s, PH_REORDER, true);
    launch_reorder(s->b, s->mode, s->N, s->C, s->ninst, s->max_active, s->reorder_ctas, st);
    if (s->b.lflag)
        launch_list_regather(s->b, s->N, s->ninst, st);
    rec(s, PH_REORDER, false);
}

// One time step.  Verlet (Eqs. 9-14): pair pass, dt, update + rebin,
// neighbour structure of the new state, sorted gather.  Symplectic: pair pass,
// dt, predictor + rebin, neighbour structure, pair pass at the predicted
// state, corrector + rebin, neighbour structure.  With profiling on, events
// bracket each phase.
static void enqueue_step(sph_t *s, cudaStream_t st)
{
    if (s->p.integrator == SPH_SYMPLECTIC) {
        rec(s, PH_PAIR, true);
        enqueue_pair(s, st);
        rec(s, PH_PAIR, false);
        rec(s, PH_DT, true);
        launch_dt(s->b, s->mode, s->N, s->ninst, s->p.ns, st);
        rec(s, PH_DT, false);
        rec(s, PH_INTEGRATE, true);
        launch_predict(s->b, s->mode, s->N, s->C, st);
        rec(s, PH_INTEGRATE, false);
        enqueue_rebuild(s, st);
        rec(s, PH_PAIR, true);
        enqueue_pair(s, st);
        rec(s, PH_PAIR, false);
        rec(s, PH_INTEGRATE, true);
        launch_correct(s->b, s->mode, s->N, s->C, st);
        rec(s, PH_INTEGRATE, false);
        enqueue_rebuild(s, st);
        return;
    }
    rec(s, PH_PAIR, true);
    enqueue_pair(s, st);
    rec(s, PH_PAIR, false);
    rec(s, PH_DT, true);
    launch_dt(s->b, s->mode, s->N, s->ninst, s->p.ns, st);
    rec(s, PH_DT, false);
    rec(s, PH_INTEGRATE, true);
    launch_integrate(s->b, s->mode, s->N, s->C, s->ninst, st);
    rec(s, PH_INTEGRATE, false);
    enqueue_rebuild(s, st);
}

static int collect_profile(sph_t *s)
{
    if (!s->prof || s->ev_used == 0)
        return SPH_OK;
    CK(cudaStreamSynchronize(s->st));
    for (size_t k = 0; k + 1 < s->ev_used; k += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, s->ev[k], s->ev[k + 1]));
        const int ph = s->ev_phase[k / 2];
        s->phase_ms[ph] += ms;
        s->phase_n[ph] += 1;
    }
    s->ev_used = 0;
    s->ev_phase.clear();
    return SPH_OK;
}

static int check_status(sph_t *s)
{
    int32_t misc[4];
    CK(cudaMemcpyAsync(misc, s->b.misc, sizeof(misc), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (misc[2] & ST_UNSTABLE)
        return fail(s, SPH_EUNSTABLE, "non-finite state or dt below dt_min");
    if (misc[2] & ST_TIMEOUT)
        return fail(s, SPH_ETIMEOUT, "a bounded device wait ran out");
    if (misc[2] & ST_OVERFLOW)
        return fail(s, SPH_ESTATE, "cell counters out of step with the particle keys");
    if (misc[2] & ST_BOUNDS)
        return fail(s, SPH_ESTATE, "a shared-memory bounds check of the pair kernel failed (debug build)");
    return SPH_OK;
}

static int create_common(sph_t **out, int32_t n_inst, const sph_instance *in, const sph_params *p, void *ws,
                         size_t bytes, uintptr_t stream)
{
    if (!out)
        return SPH_EINVAL;
    *out = nullptr;
    sph_t *s = new sph_t();
    int rc = prepare_sizes(s, n_inst, in, p);
    if (rc) {
        std::fprintf(stderr, "sph_create: %s\n", s->err.c_str());
        delete s;
        return rc;
    }
    Bufs tmpb{};
    size_t need = layout(tmpb, nullptr, s->N, s->C_alloc, s->ninst, s->mode, s->list_cap, s->p.pair_symmetric != 0);
    if (!ws || bytes < need || ((uintptr_t)ws & 255)) {
        std::fprintf(stderr, "sph_create: workspace needs %zu bytes, 256-byte aligned\n", need);
        delete s;
        return ws && bytes < need ? SPH_ENOMEM : SPH_EINVAL;
    }
    s->ws = (char *)ws;
    s->ws_bytes = bytes;
    layout(s->b, s->ws, s->N, s->C_alloc, s->ninst, s->mode, s->list_cap, s->p.pair_symmetric != 0);
    s->st = (cudaStream_t)stream;
    s->pair_warps = p->pair_warps;
    s->pair_ctas = p->pair_ctas_per_sm;
    s->pair_group = p->pair_group;
    cudaError_t e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return SPH_ECUDA;
    }
    // host scene
    std::vector<double> r(3 * s->N), rho(s->N);
    std::vector<uint8_t> type(s->N);
    std::vector<uint16_t> inst_of(s->N);
    std::vector<Inst> idev(s->ninst);
    for (int k = 0; k < s->ninst; ++k) {
        HostInst &hi = s->inst[k];
        int64_t pb = hi.dev.pbase;
        build_scene(hi, s->p, r.data() + 3 * pb, rho.data() + pb, type.data() + pb);
        for (int64_t q = 0; q < hi.dev.np; ++q)
            inst_of[pb + q] = (uint16_t)k;
        idev[k] = hi.dev;
    }
    rc = SPH_OK;
    {
        const size_t vsz = s->mode == SPH_FP64 ? sizeof(dvec4) : sizeof(float4);
        std::vector<dvec4> pos(s->N);
        HostBytes vel(s->N * vsz);
        for (int64_t i = 0; i < s->N; ++i) {
            pos[i] = make_dvec4(r[3 * i], r[3 * i + 1], r[3 * i + 2], 0.0);
            const Inst &I = idev[inst_of[i]];
            // gate particles start with their prescribed velocity, all others at rest
            const bool gate = type[i] == T_GATE;
            if (s->mode == SPH_FP64)
                reinterpret_cast<dvec4 *>(vel.data())[i] =
                    gate ? make_dvec4(I.gate_v[0], I.gate_v[1], I.gate_v[2], rho[i])
                         : make_dvec4(0, 0, 0, rho[i]);
            else
                reinterpret_cast<float4 *>(vel.data())[i] =
                    gate ? make_float4(I.gate_vf[0], I.gate_vf[1], I.gate_vf[2], (float)(rho[i] - I.rho0))
                         : make_float4(0, 0, 0, (float)(rho[i] - I.rho0));
        }
        auto up = [&](void *dst, const void *src, size_t n) {
            cudaError_t e2 = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s->st);
            if (e2 != cudaSuccess && rc == SPH_OK)
                rc = cuda_fail(s, e2, "upload");
        };
        up(s->b.pos, pos.data(), sizeof(dvec4) * s->N);
        up(s->b.vel, vel.data(), vsz * s->N);
        up(s->b.velp, vel.data(), vsz * s->N);
        up(s->b.type, type.data(), s->N);
        up(s->b.inst_of, inst_of.data(), 2 * s->N);
        up(s->b.inst, idev.data(), sizeof(Inst) * s->ninst);
        cudaMemsetAsync(s->b.count, 0, sizeof(uint32_t) * ((size_t)s->C_alloc + 1), s->st);
        cudaMemsetAsync(s->b.red, 0, sizeof(unsigned long long) * 2 * s->ninst, s->st);
        cudaMemsetAsync(s->b.dt, 0, sizeof(double) * s->ninst, s->st);
        cudaMemsetAsync(s->b.time, 0, sizeof(double) * s->ninst, s->st);
        cudaMemsetAsync(s->b.dt_fixed, 0, sizeof(double), s->st);
        cudaMemsetAsync(s->b.step, 0, sizeof(long long), s->st);
        cudaMemsetAsync(s->b.misc, 0, sizeof(int32_t) * 16, s->st);
        if (s->b.lflag)
            cudaMemsetAsync(s->b.lflag, 0, sizeof(int32_t) * 8, s->st);
        enqueue_prepare(s, s->st);
        e = cudaStreamSynchronize(s->st);
        if (e != cudaSuccess && rc == SPH_OK)
            rc = cuda_fail(s, e, "create");
        e = cudaGetLastError();
        if (e != cudaSuccess && rc == SPH_OK)
            rc = cuda_fail(s, e, "create launch");
    }
    if (rc) {
        std::fprintf(stderr, "sph_create: %s\n", s->err.c_str());
        cudaStreamDestroy(s->cap);
        delete s;
        return rc;
    }
    *out = s;
    return SPH_OK;
}

extern "C" {

int sph_create(sph_t **out, const double tank[3], const double column[3], const double *obstacle, double dp,
               double h, double c0, double rho0, double alpha, const sph_params *p, void *dev_workspace,
               size_t workspace_bytes, uintptr_t cuda_stream)
{
    if (!tank || !column)
        return SPH_EINVAL;
    sph_instance in;
    std::memset(&in, 0, sizeof(in));
    for (int a = 0; a < 3; ++a) {
        in.tank[a] = tank[a];
        in.column[a] = column[a];
    }
    in.has_obstacle = obstacle ? 1 : 0;
    if (obstacle)
        for (int a = 0; a < 6; ++a)
            in.obstacle[a] = obstacle[a];
    in.dp = dp;
    in.h = h;
    in.c0 = c0;
    in.rho0 = rho0;
    in.alpha = alpha;
    return create_common(out, 1, &in, p, dev_workspace, workspace_bytes, cuda_stream);
}

int sph_batch_create(sph_t **out, int32_t n_inst, const sph_instance *inst, const sph_params *p,
                     void *dev_workspace, size_t workspace_bytes, uintptr_t cuda_stream)
{
    return create_common(out, n_inst, inst, p, dev_workspace, workspace_bytes, cuda_stream);
}

void sph_destroy(sph_t *s)
{
    if (!s)
        return;
    if (s->st)
        cudaStreamSynchronize(s->st);
    if (s->graph)
        cudaGraphExecDestroy(s->graph);
    for (cudaEvent_t e : s->ev)
        cudaEventDestroy(e);
    if (s->cap)
        cudaStreamDestroy(s->cap);
    delete s;
}

int sph_step(sph_t *s, double dt, int32_t nsteps)
{
    if (!s)
        return SPH_EINVAL;
    if (nsteps < 0 || !(dt >= 0.0) || !std::isfinite(dt))
        return fail(s, SPH_EINVAL, "nsteps must be >= 0 and dt finite and >= 0");
    if (nsteps == 0)
        return SPH_OK;
    if (!s->dt_uploaded || dt != s->dt_host) {
        s->dt_host = dt;
        CK(cudaMemcpyAsync(s->b.dt_fixed, &s->dt_host, sizeof(double), cudaMemcpyHostToDevice, s->st));
        s->dt_uploaded = true;
    }
    if (s->p.persistent) {
        // all steps in cooperative launches of at most 100,000 steps each (the
        // barrier counter stays far below 2^32)
        const long long limit = s->p.spin_limit > 0 ? s->p.spin_limit : 20000000LL;
        rec(s, PH_PERSIST, true);
        for (int done = 0; done < nsteps; done += 100000) {
            const int n = std::min(nsteps - done, 100000);
            cudaError_t e = launch_persistent_steps(s->b, s->ninst, n, s->p.ns, s->p.cell_div, s->p.delta_mode, s->N,
                                                    s->C, limit, s->st);
            if (e != cudaSuccess)
                return cuda_fail(s, e, "persistent launch");
        }
        rec(s, PH_PERSIST, false);
        CK(cudaGetLastError());
        if (s->prof)
            return collect_profile(s);
        return SPH_OK;
    }
    int done = 0;
    const int G = std::max(1, s->p.graph_steps);
    if (s->p.use_graph && !s->prof && nsteps >= G) {
        if (!s->graph || s->graph_steps != G) {
            if (s->graph) {
                cudaGraphExecDestroy(s->graph);
                s->graph = nullptr;
            }
            // order the capture stream after the caller's stream
            CK(cudaStreamSynchronize(s->st));
            CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
            for (int k = 0; k < G; ++k)
                enqueue_step(s, s->cap);
            cudaGraph_t g = nullptr;
            CK(cudaStreamEndCapture(s->cap, &g));
            cudaError_t e = cudaGraphInstantiate(&s->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess)
                return cuda_fail(s, e, "cudaGraphInstantiate");
            s->graph_steps = G;
        }
        for (; done + G <= nsteps; done += G)
            CK(cudaGraphLaunch(s->graph, s->st));
    }
    for (; done < nsteps; ++done)
        enqueue_step(s, s->st);
    CK(cudaGetLastError());
    if (s->prof)
        return collect_profile(s);
    return SPH_OK;
}

int sph_sync(sph_t *s)
{
    if (!s)
        return SPH_EINVAL;
    return check_status(s);
}

int sph_counts(const sph_t *s, int32_t inst, int64_t out[4])
{
    if (!s || !out || inst < -1 || inst >= s->ninst)
        return SPH_EINVAL;
    if (inst < 0) {
        out[0] = s->nf_tot;
        out[1] = s->nw_tot + s->ng_tot;
        out[2] = s->no_tot;
        out[3] = s->N;
    } else {
        const HostInst &hi = s->inst[inst];
        out[0] = hi.nf;
        out[1] = hi.nw + hi.ng;
        out[2] = hi.no;
        out[3] = hi.nf + hi.nw + hi.no + hi.ng;
    }
    return SPH_OK;
}

int sph_sizes(const sph_t *s, int32_t *n_inst, int64_t *n_particles, int64_t *n_cells)
{
    if (!s)
        return SPH_EINVAL;
    if (n_inst)
        *n_inst = s->ninst;
    if (n_particles)
        *n_particles = s->N;
    if (n_cells)
        *n_cells = s->C;
    return SPH_OK;
}

int sph_probe(sph_t *s, int32_t inst, int32_t kind, const double *pts, int32_t n, double *out)
{
    if (!s || !out || inst < 0 || inst >= s->ninst)
        return SPH_EINVAL;
    if (kind == SPH_PROBE_FORCE) {
        launch_probe_force(s->b, s->mode, inst, s->ninst, s->p.cell_div, s->N, s->st);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(out, s->b.probe_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
        CK(cudaStreamSynchronize(s->st));
        return check_status(s);
    }
    if (n < 0 || n > kMaxProbe || (n > 0 && !pts))
        return fail(s, SPH_EINVAL, "probe count must be in [0, 65536]");
    if (n == 0)
        return SPH_OK;
    const HostInst &hi = s->inst[inst];
    if (kind == SPH_PROBE_PRESSURE) {
        CK(cudaMemcpyAsync(s->b.probe_in, pts, 3 * sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
        launch_probe_pressure(s->b, s->mode, inst, s->ninst, s->p.cell_div, n, s->st);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(out, s->b.probe_out, sizeof(double) * n, cudaMemcpyDeviceToHost, s->st));
        CK(cudaStreamSynchronize(s->st));
        return check_status(s);
    }
    if (kind == SPH_PROBE_WAVE_HEIGHT) {
        double dz = 0.25 * hi.d.dp;
        int32_t nlev = 0;
        while (nlev * dz <= hi.dev.ztop)
            ++nlev;
        CK(cudaMemcpyAsync(s->b.probe_in, pts, 2 * sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
        CK(cudaMemsetAsync(s->b.probe_k, 0xff, sizeof(int32_t) * n, s->st));
        launch_probe_wave(s->b, s->mode, inst, s->ninst, s->p.cell_div, n, nlev, s->st);
        CK(cudaGetLastError());
        std::vector<int32_t> k(n);
        CK(cudaMemcpyAsync(k.data(), s->b.probe_k, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s->st));
        CK(cudaStreamSynchronize(s->st));
        for (int a = 0; a < n; ++a)
            out[a] = k[a] >= 0 ? k[a] * dz : 0.0;
        return check_status(s);
    }
    return fail(s, SPH_EINVAL, "unknown probe kind");
}

int sph_get_state(sph_t *s, double *r, double *u, double *rho, int32_t *type, double *uprev, double *rhoprev,
                  int64_t *step, double *time)
{
    if (!s)
        return SPH_EINVAL;
    if (!r && !u && !rho && !type && !uprev && !rhoprev) {  // clocks only
        long long st_dev = 0;
        std::vector<double> tm(s->ninst);
        CK(cudaMemcpyAsync(&st_dev, s->b.step, sizeof(long long), cudaMemcpyDeviceToHost, s->st));
        CK(cudaMemcpyAsync(tm.data(), s->b.time, sizeof(double) * s->ninst, cudaMemcpyDeviceToHost, s->st));
        CK(cudaStreamSynchronize(s->st));
        if (step)
            *step = st_dev;
        if (time)
            for (int k = 0; k < s->ninst; ++k)
                time[k] = tm[k];
        return check_status(s);
    }
    const int64_t N = s->N;
    const size_t vsz = s->mode == SPH_FP64 ? sizeof(dvec4) : sizeof(float4);
    std::vector<dvec4> pos(N);
    HostBytes vel(N * vsz), velp(N * vsz);
    std::vector<uint8_t> ty(N);
    CK(cudaMemcpyAsync(pos.data(), s->b.pos, sizeof(dvec4) * N, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(vel.data(), s->b.vel, vsz * N, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(velp.data(), s->b.velp, vsz * N, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(ty.data(), s->b.type, N, cudaMemcpyDeviceToHost, s->st));
    long long st_dev = 0;
    CK(cudaMemcpyAsync(&st_dev, s->b.step, sizeof(long long), cudaMemcpyDeviceToHost, s->st));
    std::vector<double> tm(s->ninst);
    CK(cudaMemcpyAsync(tm.data(), s->b.time, sizeof(double) * s->ninst, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (int k = 0; k < s->ninst; ++k) {
        const Inst &I = s->inst[k].dev;
        for (int64_t i = I.pbase; i < I.pbase + I.np; ++i) {
            if (r) {
                r[3 * i] = pos[i].x;
                r[3 * i + 1] = pos[i].y;
                r[3 * i + 2] = pos[i].z;
            }
            double v[4], vp[4];
            if (s->mode == SPH_FP64) {
                dvec4 a = reinterpret_cast<dvec4 *>(vel.data())[i], c = reinterpret_cast<dvec4 *>(velp.data())[i];
                v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
                vp[0] = c.x, vp[1] = c.y, vp[2] = c.z, vp[3] = c.w;
            } else {
                float4 a = reinterpret_cast<float4 *>(vel.data())[i], c = reinterpret_cast<float4 *>(velp.data())[i];
                v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = I.rho0 + (double)a.w;
                vp[0] = c.x, vp[1] = c.y, vp[2] = c.z, vp[3] = I.rho0 + (double)c.w;
            }
            for (int a = 0; a < 3; ++a) {
                if (u)
                    u[3 * i + a] = v[a];
                if (uprev)
                    uprev[3 * i + a] = vp[a];
            }
            if (rho)
                rho[i] = v[3];
            if (rhoprev)
                rhoprev[i] = vp[3];
            if (type)
                type[i] = ty[i];
        }
    }
    if (step)
        *step = st_dev;
    if (time)
        for (int k = 0; k < s->ninst; ++k)
            time[k] = tm[k];
    return check_status(s);
}

int sph_set_state(sph_t *s, const double *r, const double *u, const double *rho, const double *uprev,
                  const double *rhoprev, int64_t step, const double *time)
{
    if (!s || !r || !u || !rho || step < 0)
        return SPH_EINVAL;
    const int64_t N = s->N;
    const size_t vsz = s->mode == SPH_FP64 ? sizeof(dvec4) : sizeof(float4);
    std::vector<dvec4> pos(N);
    HostBytes vel(N * vsz), velp(N * vsz);
    std::vector<uint8_t> ty(N);
    CK(cudaMemcpyAsync(ty.data(), s->b.type, N, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (int k = 0; k < s->ninst; ++k) {
        const Inst &I = s->inst[k].dev;
        for (int64_t i = I.pbase; i < I.pbase + I.np; ++i) {
            bool fl = ty[i] == T_FLUID;
            pos[i] = make_dvec4(r[3 * i], r[3 * i + 1], r[3 * i + 2], 0.0);
            const double *up = uprev ? uprev : u;
            const double *rp = rhoprev ? rhoprev : rho;
            // boundary velocities are prescribed: zero for walls and obstacle,
            // the gate velocity for gate particles
            const bool gt = ty[i] == T_GATE;
            double ux = fl ? u[3 * i] : (gt ? I.gate_v[0] : 0), uy = fl ? u[3 * i + 1] : (gt ? I.gate_v[1] : 0);
            double uz = fl ? u[3 * i + 2] : (gt ? I.gate_v[2] : 0);
            double px = fl ? up[3 * i] : (gt ? I.gate_v[0] : 0), py = fl ? up[3 * i + 1] : (gt ? I.gate_v[1] : 0);
            double pz = fl ? up[3 * i + 2] : (gt ? I.gate_v[2] : 0);
            if (s->mode == SPH_FP64) {
                reinterpret_cast<dvec4 *>(vel.data())[i] = make_dvec4(ux, uy, uz, rho[i]);
                reinterpret_cast<dvec4 *>(velp.data())[i] = make_dvec4(px, py, pz, rp[i]);
            } else {
                reinterpret_cast<float4 *>(vel.data())[i] =
                    make_float4((float)ux, (float)uy, (float)uz, (float)(rho[i] - I.rho0));
                reinterpret_cast<float4 *>(velp.data())[i] =
                    make_float4((float)px, (float)py, (float)pz, (float)(rp[i] - I.rho0));
            }
        }
    }
    long long st_dev = step;
    CK(cudaMemcpyAsync(s->b.pos, pos.data(), sizeof(dvec4) * N, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->b.vel, vel.data(), vsz * N, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->b.velp, velp.data(), vsz * N, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->b.step, &st_dev, sizeof(long long), cudaMemcpyHostToDevice, s->st));
    if (time)
        CK(cudaMemcpyAsync(s->b.time, time, sizeof(double) * s->ninst, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemsetAsync(s->b.misc + 2, 0, sizeof(int32_t), s->st));
    // the per-cell counters are zero between steps; rebuild the structure
    enqueue_prepare(s, s->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->st));
    return SPH_OK;
}

int sph_derivatives(sph_t *s, double *drho, double *acc, double *mumax, int32_t *nneigh)
{
    if (!s)
        return SPH_EINVAL;
    const int64_t N = s->N;
    enqueue_pair(s, s->st, false, true);
    CK(cudaGetLastError());
    int32_t misc[4];
    CK(cudaMemcpyAsync(misc, s->b.misc, sizeof(misc), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    const int32_t n_in = misc[0];
    const size_t vsz = s->mode == SPH_FP64 ? sizeof(dvec4) : sizeof(float4);
    HostBytes d(vsz * N), m((s->mode == SPH_FP64 ? 8 : 4) * N);
    std::vector<int32_t> nn(N), perm(N);
    if (n_in > 0) {
        CK(cudaMemcpyAsync(d.data(), s->b.deriv, vsz * n_in, cudaMemcpyDeviceToHost, s->st));
        CK(cudaMemcpyAsync(m.data(), s->b.mumax, (s->mode == SPH_FP64 ? 8 : 4) * (size_t)n_in,
                           cudaMemcpyDeviceToHost, s->st));
        CK(cudaMemcpyAsync(nn.data(), s->b.nneigh, 4 * (size_t)n_in, cudaMemcpyDeviceToHost, s->st));
        CK(cudaMemcpyAsync(perm.data(), s->b.perm, 4 * (size_t)n_in, cudaMemcpyDeviceToHost, s->st));
    }
    CK(cudaStreamSynchronize(s->st));
    for (int64_t i = 0; i < N; ++i) {
        if (drho)
            drho[i] = 0.0;
        if (acc)
            acc[3 * i] = acc[3 * i + 1] = acc[3 * i + 2] = 0.0;
        if (mumax)
            mumax[i] = 0.0;
        if (nneigh)
            nneigh[i] = -1;
    }
    for (int32_t sidx = 0; sidx < n_in; ++sidx) {
        int32_t id = perm[sidx];
        double v[4], mu;
        if (s->mode == SPH_FP64) {
            dvec4 a = reinterpret_cast<dvec4 *>(d.data())[sidx];
            v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
            mu = reinterpret_cast<double *>(m.data())[sidx];
        } else {
            float4 a = reinterpret_cast<float4 *>(d.data())[sidx];
            v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
            mu = reinterpret_cast<float *>(m.data())[sidx];
        }
        if (drho)
            drho[id] = v[3];
        if (acc)
            for (int a = 0; a < 3; ++a)
                acc[3 * id + a] = v[a];
        if (mumax)
            mumax[id] = mu;
        if (nneigh)
            nneigh[id] = nn[sidx];
    }
    return SPH_OK;
}

int sph_cells(sph_t *s, int64_t *cell, int64_t *sorted, int64_t *cell_start, int64_t *n_in_out)
{
    if (!s)
        return SPH_EINVAL;
    const int64_t N = s->N;
    if (s->b.lflag)
        enqueue_prepare(s, s->st);  // the lists keep the order of their last rebuild: rebin now
    std::vector<uint32_t> key(N);
    std::vector<int32_t> perm(N), cs((size_t)s->C + 1);
    int32_t misc[4];
    CK(cudaMemcpyAsync(misc, s->b.misc, sizeof(misc), cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(key.data(), s->b.key, 4 * N, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(perm.data(), s->b.perm, 4 * N, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(cs.data(), s->b.cell_start, 4 * ((size_t)s->C + 1), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (cell)
        for (int64_t i = 0; i < N; ++i)
            cell[i] = key[i];
    if (sorted)
        for (int32_t k = 0; k < misc[0]; ++k)
            sorted[k] = perm[k];
    if (cell_start)
        for (int64_t c = 0; c <= s->C; ++c)
            cell_start[c] = cs[c];
    if (n_in_out)
        *n_in_out = misc[0];
    return SPH_OK;
}

int sph_last_dt(sph_t *s, double *dt)
{
    if (!s || !dt)
        return SPH_EINVAL;
    CK(cudaMemcpyAsync(dt, s->b.dt, sizeof(double) * s->ninst, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return SPH_OK;
}

int sph_diagnostics(sph_t *s, int32_t inst, double out[10])
{
    if (!s || !out || inst < 0 || inst >= s->ninst)
        return SPH_EINVAL;
    launch_diagnostics(s->b, s->mode, inst, s->C, s->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, s->b.probe_out, 10 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return check_status(s);
}

int sph_set_profiling(sph_t *s, int32_t on)
{
    if (!s)
        return SPH_EINVAL;
    s->prof = on != 0;
    s->ev_used = 0;
    return SPH_OK;
}

int sph_phase_times(sph_t *s, double *ms, int64_t *launches, int32_t nphase)
{
    if (!s || nphase < 0)
        return SPH_EINVAL;
    int rc = collect_profile(s);
    if (rc)
        return rc;
    for (int k = 0; k < nphase && k < PH_COUNT; ++k) {
        if (ms)
            ms[k] = s->phase_ms[k];
        if (launches)
            launches[k] = s->phase_n[k];
        s->phase_ms[k] = 0.0;
        s->phase_n[k] = 0;
    }
    return SPH_OK;
}

const char *sph_phase_name(int32_t k) { return k >= 0 && k < PH_COUNT ? kPhaseNames[k] : ""; }

int32_t sph_num_phases(void) { return PH_COUNT; }

// Switch the grid to cells of size 2h/d: new per-instance constants, the
// neighbour structure of the current state rebuilt on the new grid.
static int apply_cell_div(sph_t *s, int d)
{
    if (d == s->p.cell_div)
        return SPH_OK;
    sph_params p = s->p;
    p.cell_div = d;
    int64_t C = 0;
    std::vector<Inst> idev(s->ninst);
    for (int k = 0; k < s->ninst; ++k) {
        HostInst &hi = s->inst[k];
        const int32_t pbase = hi.dev.pbase;
        fill_inst(hi, p);
        hi.dev.pbase = pbase;
        hi.dev.cell_base = (int32_t)C;
        C += hi.dev.ncells;
        idev[k] = hi.dev;
    }
    if (C > s->C_alloc)
        return fail(s, SPH_EINVAL, "grid larger than the workspace holds");
    CK(cudaStreamSynchronize(s->st));
    s->p.cell_div = d;
    s->C = (int32_t)C;
    s->max_active = (int32_t)std::min<int64_t>(C, s->N);
    CK(cudaMemcpyAsync(s->b.inst, idev.data(), sizeof(Inst) * s->ninst, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemsetAsync(s->b.count, 0, sizeof(uint32_t) * ((size_t)s->C_alloc + 1), s->st));
    enqueue_prepare(s, s->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->st));
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    return SPH_OK;
}

int sph_autotune(sph_t *s, int32_t steps, int32_t best[3])
{
    if (!s || steps < 1)
        return SPH_EINVAL;
    // cell size: each candidate grid timed on the pair passes and one rebuild
    // of the neighbour structure (the pair kernel in its current shape)
    {
        const int divs_mixed[] = {1, 2}, divs_fp64[] = {1, 2, 3};
        const int *divs = s->mode == SPH_MIXED ? divs_mixed : divs_fp64;
        const int nd = s->b.lflag ? 0 : (s->mode == SPH_MIXED ? 2 : 3);  // lists: cells of 2h + s only
        const int d0 = s->p.cell_div;
        int best_d = d0;
        float best_d_ms = 1e30f;
        cudaEvent_t a0, a1;
        CK(cudaEventCreate(&a0));
        CK(cudaEventCreate(&a1));
        for (int k = 0; k < nd; ++k) {
            int rc = apply_cell_div(s, divs[k]);
            if (rc)
                return rc;
            enqueue_pair(s, s->st);  // warm-up
            CK(cudaEventRecord(a0, s->st));
            for (int r = 0; r < steps; ++r)
                enqueue_pair(s, s->st);
            enqueue_prepare(s, s->st);  // binning, scan, scatter, sort: leaves the structure as it was
            CK(cudaEventRecord(a1, s->st));
            CK(cudaEventSynchronize(a1));
            CK(cudaGetLastError());
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, a0, a1));
            if (ms < best_d_ms) {
                best_d_ms = ms;
                best_d = divs[k];
            }
        }
        cudaEventDestroy(a0);
        cudaEventDestroy(a1);
        int rc = apply_cell_div(s, best_d);
        if (rc)
            return rc;
    }
    // (warps per CTA, CTAs per SM, particles per warp)
    const int cand_mixed[][3] = {{8, 2, 4}, {8, 2, 2}, {8, 2, 1}, {4, 3, 2}, {16, 1, 1}};
    const int cand_fp64[][3] = {{8, 4, 1}, {8, 8, 1}, {4, 8, 1}, {4, 16, 1}};
    const bool mixed = s->mode == SPH_MIXED;
    const int nc = mixed ? (int)(sizeof(cand_mixed) / sizeof(cand_mixed[0])) : (int)(sizeof(cand_fp64) / sizeof(cand_fp64[0]));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int bw = s->pair_warps, bc = s->pair_ctas, bg = s->pair_group;
    for (int k = 0; k < (s->b.lflag ? 0 : nc); ++k) {  // the list pass has one shape
        const int *cd = mixed ? cand_mixed[k] : cand_fp64[k];
        s->pair_warps = cd[0];
        s->pair_ctas = cd[1];
        s->pair_group = cd[2];
        enqueue_pair(s, s->st);  // warm-up
        CK(cudaEventRecord(e0, s->st));
        for (int r = 0; r < steps; ++r)
            enqueue_pair(s, s->st);
        CK(cudaEventRecord(e1, s->st));
        CK(cudaEventSynchronize(e1));
        CK(cudaGetLastError());
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) {
            best_ms = ms;
            bw = s->pair_warps;
            bc = s->pair_ctas;
            bg = s->pair_group;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->pair_warps = bw;
    s->pair_ctas = bc;
    s->pair_group = bg;
    // sort granularity: resident CTAs per SM of the per-cell sort and gather
    {
        const int cand[] = {8, 16, 32};
        float best_r = 1e30f;
        int br = s->reorder_ctas;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        for (int k = 0; k < 3; ++k) {
            s->reorder_ctas = cand[k];
            if (s->b.lflag)
                CK(cudaMemsetAsync(s->b.lflag, 1, 1, s->st));  // the sort runs on rebuild requests only
            CK(cudaEventRecord(e0, s->st));
            for (int r = 0; r < steps; ++r)
                launch_reorder(s->b, s->mode, s->N, s->C, s->ninst, s->max_active, s->reorder_ctas, s->st);
            CK(cudaEventRecord(e1, s->st));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_r) {
                best_r = ms;
                br = cand[k];
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        s->reorder_ctas = br;
    }
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    if (best) {
        best[0] = bw;
        best[1] = bc;
        best[2] = bg;
    }
    return SPH_OK;
}

int sph_tuned_config(const sph_t *s, int32_t out[5])
{
    if (!s || !out)
        return SPH_EINVAL;
    out[0] = s->pair_warps;
    out[1] = s->pair_ctas;
    out[2] = s->pair_group;
    out[3] = s->p.cell_div;
    out[4] = s->reorder_ctas;
    return SPH_OK;
}

int sph_pair_stats(sph_t *s, int64_t out[5])
{
    if (!s || !out)
        return SPH_EINVAL;
    int32_t misc[4];
    unsigned long long ps[4] = {0, 0, 0, 0};
    if (s->b.lflag)
        enqueue_prepare(s, s->st);  // the staged kernel wants the sorted structure of the current state
    enqueue_pair(s, s->st, true);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(misc, s->b.misc, sizeof(misc), cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(ps, s->b.pstat, sizeof(ps), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    const int32_t n_in = misc[0];
    std::vector<int32_t> nn(n_in > 0 ? n_in : 1), np(n_in > 0 ? n_in : 1), nc(n_in > 0 ? n_in : 1);
    if (n_in > 0) {
        CK(cudaMemcpyAsync(nn.data(), s->b.nneigh, 4 * (size_t)n_in, cudaMemcpyDeviceToHost, s->st));
        CK(cudaMemcpyAsync(np.data(), s->b.npair, 4 * (size_t)n_in, cudaMemcpyDeviceToHost, s->st));
        CK(cudaMemcpyAsync(nc.data(), s->b.ncand, 4 * (size_t)n_in, cudaMemcpyDeviceToHost, s->st));
        CK(cudaStreamSynchronize(s->st));
    }
    int64_t tot[3] = {0, 0, 0};
    for (int32_t k = 0; k < n_in; ++k) {
        tot[0] += nn[k];
        tot[1] += np[k];
        tot[2] += nc[k];
    }
    out[0] = tot[0];
    out[1] = tot[1];
    if (s->mode == SPH_MIXED) {
        out[2] = (int64_t)ps[2];  // windowed candidates (per particle pair, counted once per warp)
        out[3] = (int64_t)ps[0];
        out[4] = (int64_t)ps[1];
    } else {
        out[2] = tot[2];
        out[3] = -1;
        out[4] = -1;
    }
    return SPH_OK;
}

int sph_list_stats(sph_t *s, int64_t out[4])
{
    if (!s || !out)
        return SPH_EINVAL;
    int32_t f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (s->b.lflag) {
        CK(cudaMemcpyAsync(f, s->b.lflag, sizeof(f), cudaMemcpyDeviceToHost, s->st));
        CK(cudaStreamSynchronize(s->st));
        CK(cudaMemsetAsync(s->b.lflag + 1, 0, sizeof(int32_t) * 4, s->st));
        CK(cudaStreamSynchronize(s->st));
    }
    out[0] = f[1];
    out[1] = std::max(0, f[4] - f[1]);
    out[2] = f[2];
    out[3] = f[3];
    return SPH_OK;
}

int32_t sph_launches_per_step(const sph_t *s)
{
    if (!s)
        return 0;
    // kernels per step: pair, dt reduce + finalize, integrate, cell scan x3 +
    // scatter, sort/reorder (the mixed form adds one memset node per pair
    // pass); the symplectic step adds a second pair pass, an integrator kernel
    // and a second neighbour structure and gather
    const int32_t verlet = 1 + 2 + 1 + 4 + 1;
    if (s->p.persistent)
        return 1;  // one launch per sph_step call, whatever its number of steps
    if (s->b.lflag)
        return 2 + 2 + 1 + 1 + 4 + 1 + 1;  // list build (gated) + list pass, dt, update, bin, structure, sort, gather
    const int32_t fin = s->b.fjacc ? 1 : 0;  // FP64 each pair once: the kernel adding the partners' shares
    return s->p.integrator == SPH_SYMPLECTIC ? verlet + 1 + 1 + 4 + 1 + 2 * fin : verlet + fin;
}

const char *sph_last_error(const sph_t *s)
{
    if (!s)
        return "null handle";
    return s->err.c_str();
}

}  // extern "C"
