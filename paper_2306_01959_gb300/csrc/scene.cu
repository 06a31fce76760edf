// Host-side scene generation and instance constants.
//
// The paper gives tank, column and obstacle sizes (Sections 3.1, 3.2) but not
// the particle layout.  The layout taken: fluid on the lattice
// ((i+1/2) dp, (j+1/2) dp, (k+1/2) dp) measured from the inner tank corner,
// the column against the x = 0 end wall; `boundary_layers` layers of fixed
// boundary particles outside the floor and the four walls, up to the tank
// height, no lid; the obstacle a filled lattice box whose lower corner is
// rounded to the lattice; an optional moving gate built the same way.
// Particle ids: fluid (x fastest, then y, then z), walls+floor (same loop
// order over the enclosing box), obstacle, gate.  Every
// particle has mass rho0 dp^3.  The cell grid spans
// [-L dp, Lt + L dp] x [-L dp, Wt + L dp] x [-L dp, Ht + 4h] with cells of
// size 2h / cell_div.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace sph {

static int64_t nint(double x) { return (int64_t)std::floor(x + 0.5); }

int effective_cell_div(const sph_params &p)
{
    // automatic: cells of size 2h for the mixed form (its pair kernel stages
    // whole 27-cell neighbourhoods), cells of size h for the FP64 form
    if (p.cell_div > 0)
        return p.cell_div;
    return p.precision == SPH_MIXED ? 1 : 2;
}

int validate_instance(const sph_instance &in, const sph_params &p, std::string &err)
{
    auto bad = [&](const char *m) {
        err = m;
        return SPH_EINVAL;
    };
    if (!(in.dp > 0) || !(in.h > 0) || !(in.c0 > 0) || !(in.rho0 > 0) || !(in.alpha >= 0))
        return bad("dp, h, c0, rho0 must be > 0 and alpha >= 0");
    if (!(in.h >= 0.5 * in.dp) || in.h > 8.0 * in.dp)
        return bad("h must lie in [dp/2, 8 dp]");
    for (int a = 0; a < 3; ++a) {
        if (!(in.tank[a] > 0) || !(in.column[a] >= 0))
            return bad("tank sizes must be > 0 and column sizes >= 0");
        if (nint(in.column[a] / in.dp) > nint(in.tank[a] / in.dp))
            return bad("water column does not fit in the tank");
    }
    if (in.has_obstacle) {
        int64_t o0[3], o1[3];
        for (int a = 0; a < 3; ++a) {
            if (!(in.obstacle[3 + a] > 0) || !(in.obstacle[a] >= 0))
                return bad("obstacle corner must be >= 0 and sizes > 0");
            o0[a] = nint(in.obstacle[a] / in.dp);
            o1[a] = o0[a] + nint(in.obstacle[3 + a] / in.dp);
            if (o1[a] > nint(in.tank[a] / in.dp) || o1[a] <= o0[a])
                return bad("obstacle does not fit in the tank");
        }
        bool overlap = true;
        for (int a = 0; a < 3; ++a)
            overlap = overlap && o0[a] < nint(in.column[a] / in.dp) && 0 < o1[a];
        if (overlap && nint(in.column[0] / in.dp) > 0 && nint(in.column[1] / in.dp) > 0 &&
            nint(in.column[2] / in.dp) > 0)
            return bad("obstacle overlaps the water column");
    }
    if (in.has_gate) {
        int64_t g0[3], g1[3];
        for (int a = 0; a < 3; ++a) {
            if (!(in.gate[3 + a] > 0) || !(in.gate[a] >= 0) || !std::isfinite(in.gate_velocity[a]))
                return bad("gate corner must be >= 0, sizes > 0 and the velocity finite");
            g0[a] = nint(in.gate[a] / in.dp);
            g1[a] = g0[a] + nint(in.gate[3 + a] / in.dp);
            if (g1[a] > nint(in.tank[a] / in.dp) || g1[a] <= g0[a])
                return bad("gate does not fit in the tank");
        }
        bool overlap = true;
        for (int a = 0; a < 3; ++a)
            overlap = overlap && g0[a] < nint(in.column[a] / in.dp) && 0 < g1[a];
        if (overlap && nint(in.column[0] / in.dp) > 0 && nint(in.column[1] / in.dp) > 0 &&
            nint(in.column[2] / in.dp) > 0)
            return bad("gate overlaps the water column");
    }
    if (p.boundary_layers < 1 || p.boundary_layers > 8)
        return bad("boundary_layers must be in [1, 8]");
    if (p.cell_div < 0 || p.cell_div > 3)
        return bad("cell_div must be 0 (automatic), 1, 2 or 3");
    if (p.ns < 1)
        return bad("ns must be >= 1");
    if (!(p.cfl > 0) || p.cfl > 1)
        return bad("cfl must be in (0, 1]");
    if (!(p.gamma >= 1) || !(p.delta >= 0) || !(p.g >= 0) || !(p.dt_min >= 0))
        return bad("gamma >= 1, delta >= 0, g >= 0 and dt_min >= 0 required");
    if (p.precision != SPH_FP64 && p.precision != SPH_MIXED)
        return bad("precision must be SPH_FP64 or SPH_MIXED");
    if (p.integrator != SPH_VERLET && p.integrator != SPH_SYMPLECTIC)
        return bad("integrator must be SPH_VERLET or SPH_SYMPLECTIC");
    if (p.delta_mode != SPH_DELTA_ALL_FLUID && p.delta_mode != SPH_DELTA_FULL_SUPPORT)
        return bad("delta_mode must be SPH_DELTA_ALL_FLUID or SPH_DELTA_FULL_SUPPORT");
    if (p.pair_symmetric && (p.precision != SPH_FP64 || p.delta_mode != SPH_DELTA_ALL_FLUID))
        return bad("pair_symmetric runs the FP64 form with SPH_DELTA_ALL_FLUID");
    if (!(p.list_skin >= 0) || !(p.list_skin <= 4) || p.list_capacity < 0 || p.list_capacity > 65536)
        return bad("list_skin must be in [0, 4] and list_capacity in [0, 65536]");
    if (p.list_skin > 0 && (p.precision != SPH_MIXED || p.integrator != SPH_VERLET || p.persistent ||
                            effective_cell_div(p) != 1))
        return bad("neighbour lists (list_skin > 0) run the mixed form with the Verlet scheme, per-phase "
                   "launches and cell_div 1");
    return SPH_OK;
}

void fill_inst(HostInst &hi, const sph_params &p)
{
    const sph_instance &in = hi.d;
    double dp = in.dp;
    int64_t L = p.boundary_layers;
    int64_t ncx = nint(in.column[0] / dp), ncy = nint(in.column[1] / dp), ncz = nint(in.column[2] / dp);
    int64_t ntx = nint(in.tank[0] / dp), nty = nint(in.tank[1] / dp), ntz = nint(in.tank[2] / dp);
    hi.nf = ncx * ncy * ncz;
    hi.nw = (ntx + 2 * L) * (nty + 2 * L) * (ntz + L) - ntx * nty * ntz;
    hi.no = in.has_obstacle
                ? nint(in.obstacle[3] / dp) * nint(in.obstacle[4] / dp) * nint(in.obstacle[5] / dp)
                : 0;
    hi.ng = in.has_gate ? nint(in.gate[3] / dp) * nint(in.gate[4] / dp) * nint(in.gate[5] / dp) : 0;

    Inst &d = hi.dev;
    std::memset(&d, 0, sizeof(d));
    double Ld = L * dp;
    double hi3[3] = {in.tank[0] + Ld, in.tank[1] + Ld, in.tank[2] + 4.0 * in.h};
    // with neighbour lists the cells hold the list radius 2h + s
    d.skin = p.list_skin * in.h;
    d.cs = (2.0 * in.h + d.skin) / effective_cell_div(p);
    d.inv_cs = 1.0 / d.cs;
    for (int a = 0; a < 3; ++a) {
        d.lo[a] = -Ld;
        d.n[a] = (int32_t)std::ceil((hi3[a] - d.lo[a]) / d.cs);
    }
    d.ncells = d.n[0] * d.n[1] * d.n[2];
    d.h = in.h;
    d.c0 = in.c0;
    d.rho0 = in.rho0;
    d.alpha = in.alpha;
    d.delta = p.delta;
    d.gamma = p.gamma;
    d.g = p.g;
    d.cfl = p.cfl;
    d.dp = dp;
    d.mass = in.rho0 * dp * dp * dp;
    d.B = in.rho0 * in.c0 * in.c0 / p.gamma;
    d.eta2 = 0.01 * in.h * in.h;
    d.sup2 = (2.0 * in.h) * (2.0 * in.h);
    d.dt_min = p.dt_min;
    d.ztop = in.tank[2] + 4.0 * in.h;
    const double pi = 3.14159265358979323846;
    d.kW = 21.0 / (16.0 * pi * in.h * in.h * in.h);
    d.kF = 5.0 * d.kW / (in.h * in.h);
    d.csound = p.csound;
    d.delta_mode = p.delta_mode;
    d.nf = (int32_t)hi.nf;
    d.nw = (int32_t)hi.nw;
    d.no = (int32_t)hi.no;
    d.ng = (int32_t)hi.ng;
    d.np = (int32_t)(hi.nf + hi.nw + hi.no + hi.ng);
    for (int a = 0; a < 3; ++a) {
        d.gate_v[a] = in.has_gate ? in.gate_velocity[a] : 0.0;
        d.gate_vf[a] = (float)d.gate_v[a];
    }
    d.csf = (float)d.cs;
    d.hf = (float)d.h;
    d.inv_hf = (float)(1.0 / d.h);
    d.c0f = (float)d.c0;
    d.rho0f = (float)d.rho0;
    d.inv_rho0f = (float)(1.0 / d.rho0);
    d.alphaf = (float)d.alpha;
    d.massf = (float)d.mass;
    d.Bf = (float)d.B;
    d.eta2f = (float)d.eta2;
    d.sup2f = (float)d.sup2;
    d.list_r2f = (float)((2.0 * in.h + d.skin) * (2.0 * in.h + d.skin));
    d.half_skin2 = 0.25 * d.skin * d.skin;
    {
        // |x_f - x| <= |x| 2^-24 for a coordinate inside the grid; a difference
        // of two such copies is off by at most 2 coord_max 2^-24 per axis
        double coord_max = 0.0;
        for (int a = 0; a < 3; ++a)
            coord_max = std::fmax(coord_max, std::fmax(std::fabs(d.lo[a]), std::fabs(d.lo[a] + d.n[a] * d.cs)));
        const double eps = std::ldexp(coord_max, -22);  // twice the bound
        const double R = 2.0 * in.h + 2.0 * std::sqrt(3.0) * eps;
        d.sup2_filter = std::nextafter((float)(R * R * (1.0 + std::ldexp(1.0, -18))), 3.0e38f);
        const double Ri = std::fmax(2.0 * in.h - 2.0 * std::sqrt(3.0) * eps, 0.0);
        d.sup2_inner = std::nextafter((float)(Ri * Ri * (1.0 - std::ldexp(1.0, -18))), 0.0f);
    }
    d.kFf = (float)d.kF;
    d.dfac = (float)(2.0 * d.delta * d.h * d.c0);
    d.gammaf = (float)d.gamma;
    d.gf = (float)d.g;
}

void build_scene(const HostInst &hi, const sph_params &p, double *r, double *rho, uint8_t *type)
{
    const sph_instance &in = hi.d;
    double dp = in.dp;
    int64_t L = p.boundary_layers;
    int64_t ncx = nint(in.column[0] / dp), ncy = nint(in.column[1] / dp), ncz = nint(in.column[2] / dp);
    int64_t ntx = nint(in.tank[0] / dp), nty = nint(in.tank[1] / dp), ntz = nint(in.tank[2] / dp);
    int64_t id = 0;
    double gamma = p.gamma, g = p.g, c0 = in.c0, rho0 = in.rho0, hc = in.column[2];
    for (int64_t k = 0; k < ncz; ++k)
        for (int64_t j = 0; j < ncy; ++j)
            for (int64_t i = 0; i < ncx; ++i) {
                double z = (k + 0.5) * dp;
                r[3 * id] = (i + 0.5) * dp;
                r[3 * id + 1] = (j + 0.5) * dp;
                r[3 * id + 2] = z;
                // Eq. 8 inverted for the hydrostatic pressure rho0 g (Hc - z)
                rho[id] = p.init == SPH_INIT_HYDROSTATIC
                              ? rho0 * std::pow(1.0 + gamma * g * (hc - z) / (c0 * c0), 1.0 / gamma)
                              : rho0;
                type[id] = T_FLUID;
                ++id;
            }
    for (int64_t k = -L; k < ntz; ++k)
        for (int64_t j = -L; j < nty + L; ++j)
            for (int64_t i = -L; i < ntx + L; ++i) {
                if (i >= 0 && i < ntx && j >= 0 && j < nty && k >= 0)
                    continue;
                r[3 * id] = (i + 0.5) * dp;
                r[3 * id + 1] = (j + 0.5) * dp;
                r[3 * id + 2] = (k + 0.5) * dp;
                rho[id] = rho0;
                type[id] = T_WALL;
                ++id;
            }
    if (in.has_obstacle) {
        int64_t i0 = nint(in.obstacle[0] / dp), j0 = nint(in.obstacle[1] / dp), k0 = nint(in.obstacle[2] / dp);
        int64_t nx = nint(in.obstacle[3] / dp), ny = nint(in.obstacle[4] / dp), nz = nint(in.obstacle[5] / dp);
        for (int64_t k = k0; k < k0 + nz; ++k)
            for (int64_t j = j0; j < j0 + ny; ++j)
                for (int64_t i = i0; i < i0 + nx; ++i) {
                    r[3 * id] = (i + 0.5) * dp;
                    r[3 * id + 1] = (j + 0.5) * dp;
                    r[3 * id + 2] = (k + 0.5) * dp;
                    rho[id] = rho0;
                    type[id] = T_OBST;
                    ++id;
                }
    }
    if (in.has_gate) {
        int64_t i0 = nint(in.gate[0] / dp), j0 = nint(in.gate[1] / dp), k0 = nint(in.gate[2] / dp);
        int64_t nx = nint(in.gate[3] / dp), ny = nint(in.gate[4] / dp), nz = nint(in.gate[5] / dp);
        for (int64_t k = k0; k < k0 + nz; ++k)
            for (int64_t j = j0; j < j0 + ny; ++j)
                for (int64_t i = i0; i < i0 + nx; ++i) {
                    r[3 * id] = (i + 0.5) * dp;
                    r[3 * id + 1] = (j + 0.5) * dp;
                    r[3 * id + 2] = (k + 0.5) * dp;
                    rho[id] = rho0;
                    type[id] = T_GATE;
                    ++id;
                }
    }
}

}  // namespace sph
