// dfv_api.cu -- the C ABI declared in include/dfvrb.h.
//
// Host-side orchestration only: argument checks, placement of all device
// buffers inside the caller's workspace, and the launch sequence of a step
// (seed, three RK stages, finalize), optionally captured once into a CUDA
// graph and replayed.  No device memory is allocated here.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>
#include <array>

#include "../../include/dfvrb.h"
#include "dfv_gas3.cuh"
#include "dfv_gasw.cuh"
#include "dfv_kernels.cuh"
#include "dfv_ops.h"

using dfv::Ctl;
using dfv::GridP;
using dfv::Ops;

struct dfv_grid {
    int dim = 0, precision = 0, nmat_opt = 1, nmat = 0, solid = 0;
    int bc[6] = {0, 0, 0, 0, 0, 0};
    GridP g;
    const Ops *ops = nullptr;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    Ctl *ctl = nullptr;
    double *partials = nullptr;
    void *U = nullptr, *U1 = nullptr, *U3 = nullptr;
    double *staging = nullptr;
    long long nb_stage = 0, nb_cfl = 0;
    bool fields_set = false, smax_valid = false;
    bool dynamic = false;
    std::string err;
    long long launches = 0;
    cudaGraphExec_t graph = nullptr;
    bool graph_ready = false;
    long long graph_launches = 0;   // kernels in one replay of the step graph
    bool dt_valid = false;               // ctl->dt holds the device-computed next dt
    int fin_pending = 0;                 // mode of a finalize deferred to the next seeding launch (0: none)
    bool graph_defer = false;            // the captured step defers its finalize
    double run_cfl = -1.0, run_tend = -1.0;
    bool prof = false;                   // per-kernel event timing (dfv_profile)
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::array<cudaEvent_t, 6>> ev_steps;
    // the 2-D single-gas FP32 stage kernel (dfv_gasw.cuh): its instance record
    // sits in the workspace, written at creation; it runs the stages whenever
    // the material, the options and the body allow it (gas_on)
    bool gas_ready = false;
    bool gas3_ready = false;   // the 3-D gas kernel is prepared (FP32 3-D single-material fluid grid)
    bool gas3_tma = false;     // ... with the tensor maps of its plane boxes over U, U1, U3
    CUtensorMap gas3_map[3];
    bool body_moving = false;
    bool seed_stages = false;  // seed the stage inputs U1, U3 too (dfv_options.seed_stages)
    dfv::GasInst *d_ginst = nullptr;
    int gas_grid = 1;
    long long gas_items = 0;
};

namespace {

const char *k_no_grid = "dfv: null grid";

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

long long cells_of(int dim, const int n[3])
{
    long long c = 1;
    for (int d = 0; d < dim; d++) c *= n[d];
    return c;
}

// solid: 0 fluids, 1 stretch tensor, 2 stretch tensor and plastic-strain planes
int nvar_of(int dim, int nmat, int solid)
{
    const int nv = solid ? (dim == 1 ? 3 : (dim == 2 ? 5 : 9)) : 0;
    return (nmat - 1) + nmat + dim + 1 + nv + 1 + (solid == 2 ? nmat : 0);
}

int solid_kind(int solid) { return solid == 2 ? 2 : (solid ? 1 : 0); }

struct Layout {
    size_t off_ctl, off_part, off_gas, off_U, off_U1, off_U3, off_stage, total;
    long long pitch, nb_stage, nb_cfl;
};

long long stage_blocks(int dim, const int n[3])
{
    // the smallest tile of dfv_kernels.cuh per dimension: an upper bound on the
    // number of stage blocks of either precision
    const int tx = dim == 1 ? 256 : 32, ty = dim == 1 ? 1 : (dim == 2 ? 8 : 4), tz = dim == 3 ? 2 : 1;
    const long long bx = (n[0] + tx - 1) / tx;
    const long long by = dim >= 2 ? (n[1] + ty - 1) / ty : 1;
    const long long bz = dim >= 3 ? (n[2] + tz - 1) / tz : 1;
    return bx * by * bz;
}

Layout plan(int dim, const int n[3], int nmat, int solid, int precision)
{
    Layout L;
    const long long nc = cells_of(dim, n);
    const int nvar = nvar_of(dim, nmat, solid);
    const int w = precision == DFV_FP32 ? 4 : 8;
    L.pitch = (nc + 63) / 64 * 64;
    L.nb_stage = stage_blocks(dim, n);
    L.nb_cfl = dfv::gs_blocks(nc);
    const long long nparts = L.nb_stage > L.nb_cfl ? L.nb_stage : L.nb_cfl;
    size_t off = 0;
    L.off_ctl = off;
    off += align256(sizeof(Ctl));
    L.off_part = off;
    off += align256(sizeof(double) * 4 * (size_t)nparts);
    L.off_gas = off;   // the gas kernel's instance record
    off += align256(sizeof(dfv::GasInst));
    const size_t state = align256((size_t)w * nvar * (size_t)L.pitch);
    L.off_U = off;
    off += state;
    L.off_U1 = off;
    off += state;
    L.off_U3 = off;
    off += state;
    L.off_stage = off;
    off += align256(sizeof(double) * nvar * (size_t)nc);
    L.total = off;
    return L;
}

dfv_status fail(dfv_grid *g, dfv_status s, const std::string &msg)
{
    if (g) g->err = msg;
    return s;
}

dfv_status cuda_fail(dfv_grid *g, cudaError_t e, const char *where)
{
    return fail(g, DFV_ERR_CUDA, std::string("dfv: ") + where + ": " + cudaGetErrorString(e));
}

#define DFV_CU(g, call, where)                              \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(g, e_, where); \
    } while (0)

__global__ void k_init_ctl(Ctl *c)
{
    memset(c, 0, sizeof(Ctl));
    ctl_box_reset(c);
}

__global__ void k_set_body(Ctl *c, double v0, double v1, double v2, double x0, double x1, double x2, double mass,
                           int dynamic)
{
    c->v[0] = v0;
    c->v[1] = v1;
    c->v[2] = v2;
    c->x[0] = x0;
    c->x[1] = x1;
    c->x[2] = x2;
    c->mass = mass;
    c->dynamic = dynamic;
    dfv::ctl_sync_v(c);
}

// A saved FP64 conserved state (packed planes) into the FP32 storage planes
// (pitch elements apart): the narrowing inverts the widening of
// dfv_get_fields exactly.
__global__ void k_state_from_f64(const double *src, float *dst, long long ncell, long long pitch, int nv)
{
    const long long total = ncell * nv;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long v = t / ncell, c = t - v * ncell;
        dst[v * pitch + c] = (float)src[t];
    }
}

__global__ void k_set_run(Ctl *c, double cfl, double t_end)
{
    c->cfl = cfl;
    c->t_end = t_end;
}

dfv_status sync_stream(dfv_grid *g, int timeout_ms)
{
    if (timeout_ms <= 0) {
        DFV_CU(g, cudaStreamSynchronize(g->stream), "cudaStreamSynchronize");
        return DFV_OK;
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(g->stream);
        if (e == cudaSuccess) return DFV_OK;
        if (e != cudaErrorNotReady) return cuda_fail(g, e, "cudaStreamQuery");
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
        if (ms.count() > timeout_ms) return fail(g, DFV_ERR_TIMEOUT, "dfv: wait for the stream timed out");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

dfv_status read_ctl(dfv_grid *g, Ctl *h)
{
    DFV_CU(g, cudaMemcpyAsync(h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, g->stream), "read ctl");
    DFV_CU(g, cudaStreamSynchronize(g->stream), "read ctl sync");
    if (h->err) return fail(g, DFV_ERR_NONPHYSICAL, "dfv: non-physical state (rho <= 0, c^2 <= 0 or NaN)");
    return DFV_OK;
}

// One-block finalize: nb_max partial blocks hold the CFL maxima.
dfv_status finalize(dfv_grid *g, int mode, long long nb_max)
{
    g->launches++;
    if (nb_max == 0 && !(mode & 2)) {
        DFV_CU(g, dfv::launch_pdl(dfv::k_finalize_lite, dim3(1), dim3(32), 0, g->stream, g->ctl, mode, g->dim,
                                  g->g.dx[0], g->g.dx[1], g->g.dx[2]),
               "k_finalize_lite");
        return DFV_OK;
    }
    DFV_CU(g, dfv::launch_pdl(dfv::k_finalize, dim3(1), dim3(1024), 0, g->stream, g->ctl, (const double *)g->partials,
                              nb_max, g->nb_stage, mode, g->dim, g->g.dx[0], g->g.dx[1], g->g.dx[2]),
           "k_finalize");
    return DFV_OK;
}

// A finalize that a device-driven run deferred to the next step's seeding
// launch, run now: before anything else reads or writes the control block.
dfv_status flush_fin(dfv_grid *g)
{
    if (!g->fin_pending) return DFV_OK;
    const int mode = g->fin_pending;
    g->fin_pending = 0;
    return finalize(g, mode, 0);
}

// CFL reduction over the stored state into ctl->smax.
dfv_status reduce_cfl(dfv_grid *g)
{
    DFV_CU(g, g->ops->cfl(g->g, g->U, g->partials, (int)g->nb_cfl, g->stream), "k_cfl");
    g->launches++;
    dfv_status s = finalize(g, 1, g->nb_cfl);
    if (s == DFV_OK) g->smax_valid = true;
    return s;
}

// The launches of one step: seeding (Sec. 3.2), SSP-RK3 (Sec. 3.1), finalize.
// mode_extra = 8 asks the finalize kernel for the next dt (device-driven runs).
cudaEvent_t take_event(dfv_grid *g)
{
    if (!g->ev_free.empty()) {
        cudaEvent_t e = g->ev_free.back();
        g->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// The finalize of a device-driven step of a static body (stepped probe) is
// deferred: the next step's seeding launch runs it beside the seeding, which
// needs only the rigid box that stage 3 folded.
bool can_defer(const dfv_grid *g) { return !g->dynamic && g->g.probe_mode == 0; }

// Whether the stages run in the gas kernel now (its record exists, and
// the material, the options and the body allow it).
bool gas_on(const dfv_grid *g)
{
    return g->gas_ready && g->nmat == 1 &&
           dfv::gas_eligible(g->precision == DFV_FP32, g->dim, g->nmat, g->solid, g->g.mat[0].kind, g->g.periodic,
                             g->g.hllc_lm, g->dynamic || g->body_moving);
}

// Whether the stages of a 3-D grid run in the 3-D gas kernel now: FP32, one
// ideal or stiffened gas, no solid, no periodic side, no HLLC-LM, a static body.
bool gas3_on(const dfv_grid *g)
{
    const int per[3] = {g->g.periodic[0], g->g.periodic[1], 0};
    return g->gas3_ready && g->dim == 3 && g->nmat == 1 && !g->g.periodic[2] &&
           dfv::gas_eligible(g->precision == DFV_FP32, 2, g->nmat, g->solid, g->g.mat[0].kind, per, g->g.hllc_lm,
                             g->dynamic || g->body_moving);
}

// One SSP-RK3 stage: the gas kernel when it applies, else the general one.
dfv_status launch_stage(dfv_grid *g, int s, const void *in, const void *un, void *out, int want_force, int next)
{
    if (gas3_on(g)) {
        dfv::Gas3Args a;
        a.in = (const float *)in;
        a.un = (const float *)un;
        a.out = (float *)out;
        a.ctl = g->ctl;
        a.n0 = g->g.n[0];
        a.n1 = g->g.n[1];
        a.n2 = g->g.n[2];
        a.pitch = g->g.pitch;
        a.idx = (float)g->g.inv_dx[0];
        a.idy = (float)g->g.inv_dx[1];
        a.idz = (float)g->g.inv_dx[2];
        for (int d = 0; d < 3; d++)
            for (int k = 0; k < 2; k++) a.wall[d][k] = g->g.wall[d][k];
        a.zc = dfv::Gas3T::ZCHUNK;
        a.Gam = g->g.mc_f[0].Gam;
        a.invGam = g->g.mc_f[0].invGam;
        a.pref0 = g->g.mc_f[0].pref0;
        // the stage input's tensor map (the plane boxes by TMA), else per-thread copies
        const CUtensorMap *map = nullptr;
        if (g->gas3_tma)
            map = in == g->U ? &g->gas3_map[0] : (in == g->U1 ? &g->gas3_map[1] : (in == g->U3 ? &g->gas3_map[2] : nullptr));
        DFV_CU(g, dfv::gas3_stage(s, a, map, g->stream), "k_gas3_stage");
        return DFV_OK;
    }
    if (gas_on(g)) {
        dfv::GaswArgs a;
        a.inst = g->d_ginst;
        a.items = nullptr;
        a.nitems = g->gas_items;
        a.queue = nullptr;
        a.in = (const float *)in;
        a.un = (const float *)un;
        a.out = (float *)out;
        a.Gam = g->g.mc_f[0].Gam;
        a.invGam = g->g.mc_f[0].invGam;
        a.pref0 = g->g.mc_f[0].pref0;
        DFV_CU(g, dfv::gasw_stage(s, a, g->gas_grid, g->stream), "k_gasw_stage");
        return DFV_OK;
    }
    DFV_CU(g, g->ops->stage(s, g->g, in, un, out, g->ctl, g->partials, want_force, next, g->stream), "k_stage");
    return DFV_OK;
}

// Seeding of a stage input in place (the option seed_stages), the free
// buffer as the fixed probe's scratch.  A moving body's rigid region moves
// within the step: the published box of the step-start state is marked
// invalid first, so that the whole grid is scanned (the step's finalize
// publishes the box again).
dfv_status seed_stage_input(dfv_grid *g, void *buf, void *scratch)
{
    if (g->dynamic || g->body_moving)
        DFV_CU(g, cudaMemsetAsync(&g->ctl->rbox_valid, 0, sizeof(int), g->stream), "stage seeding box");
    DFV_CU(g, g->ops->seed(g->g, buf, scratch, g->ctl, 0, g->stream), "k_seed (stage input)");
    g->launches += g->g.probe_mode == 1 ? 2 : 1;
    return DFV_OK;
}

// fin_in: mode of the previous step's deferred finalize to run in this step's
// seeding launch (0: none); defer: leave this step's finalize pending.
dfv_status launch_step(dfv_grid *g, int mode_extra, bool capturing = false, int fin_in = 0, bool defer = false)
{
    const int want_force = g->dynamic ? 1 : 0;
    const bool rec = g->prof && !capturing;
    std::array<cudaEvent_t, 6> ev{};
    if (rec) {
        for (auto &e : ev) {
            e = take_event(g);
            if (!e) return fail(g, DFV_ERR_CUDA, "dfv: cudaEventCreate failed");
        }
        DFV_CU(g, cudaEventRecord(ev[0], g->stream), "event");
    }
    DFV_CU(g, g->ops->seed(g->g, g->U, g->U1, g->ctl, fin_in, g->stream), "k_seed");
    if (rec) DFV_CU(g, cudaEventRecord(ev[1], g->stream), "event");
    dfv_status ss = launch_stage(g, 1, g->U, g->U, g->U1, want_force, fin_in != 0 ? 1 : 0);
    if (ss != DFV_OK) return ss;
    if (rec) DFV_CU(g, cudaEventRecord(ev[2], g->stream), "event");
    if (g->seed_stages && (ss = seed_stage_input(g, g->U1, g->U3)) != DFV_OK) return ss;
    if ((ss = launch_stage(g, 2, g->U1, g->U, g->U3, 0, 0)) != DFV_OK) return ss;
    if (rec) DFV_CU(g, cudaEventRecord(ev[3], g->stream), "event");
    if (g->seed_stages && (ss = seed_stage_input(g, g->U3, g->U1)) != DFV_OK) return ss;
    if ((ss = launch_stage(g, 3, g->U3, g->U, g->U, 0, 0)) != DFV_OK) return ss;
    if (rec) DFV_CU(g, cudaEventRecord(ev[4], g->stream), "event");
    // one block: CFL maximum (folded by the stage-3 tiles), force sum, body
    // update, next dt
    if (!defer) {
        dfv_status fs = finalize(g, 1 | (want_force ? 2 : 0) | 4 | mode_extra, 0);
        if (fs != DFV_OK) return fs;
    }
    if (rec) {
        DFV_CU(g, cudaEventRecord(ev[5], g->stream), "event");
        g->ev_steps.push_back(ev);
    }
    g->launches += g->g.probe_mode == 1 ? 5 : 4;
    return DFV_OK;
}

const Ops *pick_ops(int precision, int dim, int nmat, int solid)
{
    return dfv::ops_for(precision == DFV_FP32 ? 1 : 0, dim, nmat, solid);
}

}  // namespace

extern "C" {

dfv_status dfv_workspace_bytes(int dim, const int n[3], int nmat, int solid, int precision, size_t *bytes)
{
    if (!n || !bytes || dim < 1 || dim > 3 || nmat < 1 || nmat > 3) return DFV_ERR_ARG;
    if (precision != DFV_FP64 && precision != DFV_FP32) return DFV_ERR_ARG;
    for (int d = 0; d < dim; d++)
        if (n[d] < 1) return DFV_ERR_ARG;
    int n3[3] = {n[0], dim >= 2 ? n[1] : 1, dim >= 3 ? n[2] : 1};
    *bytes = plan(dim, n3, nmat, solid_kind(solid), precision).total;
    return DFV_OK;
}

dfv_status dfv_create_grid(int dim, const int n[3], const double lo[3], const double hi[3], const int bc[6],
                           int precision, const dfv_options *opt, void *workspace, size_t workspace_bytes,
                           void *stream, dfv_grid **out)
{
    if (!out || !n || !lo || !hi || !opt) return DFV_ERR_ARG;
    *out = nullptr;
    if (dim < 1 || dim > 3 || opt->nmat < 1 || opt->nmat > 3) return DFV_ERR_ARG;
    if (precision != DFV_FP64 && precision != DFV_FP32) return DFV_ERR_ARG;
    if (opt->gas_rows < 0 || opt->gas_rows > 4096) return DFV_ERR_ARG;
    int n3[3] = {1, 1, 1};
    for (int d = 0; d < dim; d++) {
        if (n[d] < 1 || !(hi[d] > lo[d])) return DFV_ERR_ARG;
        n3[d] = n[d];
    }
    int bcs[6] = {0, 0, 0, 0, 0, 0};
    if (bc)
        for (int k = 0; k < 2 * dim; k++) bcs[k] = bc[k];
    for (int d = 0; d < dim; d++) {
        if ((bcs[2 * d] == DFV_BC_PERIODIC) != (bcs[2 * d + 1] == DFV_BC_PERIODIC)) return DFV_ERR_ARG;
        for (int s = 0; s < 2; s++)
            if (bcs[2 * d + s] != DFV_BC_PERIODIC && bcs[2 * d + s] != DFV_BC_TRANSMISSIVE &&
                bcs[2 * d + s] != DFV_BC_REFLECTIVE)
                return DFV_ERR_ARG;
    }
    if (opt->normal_method == 1 && dim != 2) return DFV_ERR_UNSUPPORTED;
    const Ops *ops = pick_ops(precision, dim, opt->nmat, solid_kind(opt->solid));
    if (!ops) return DFV_ERR_UNSUPPORTED;
    const Layout L = plan(dim, n3, opt->nmat, solid_kind(opt->solid), precision);
    if (!workspace || workspace_bytes < L.total || ((uintptr_t)workspace & 255u)) return DFV_ERR_WORKSPACE;

    dfv_grid *g = new dfv_grid();
    g->dim = dim;
    g->precision = precision;
    g->nmat_opt = opt->nmat;
    g->solid = solid_kind(opt->solid);
    g->seed_stages = opt->seed_stages != 0;
    for (int k = 0; k < 6; k++) g->bc[k] = bcs[k];
    g->ops = ops;
    g->stream = (cudaStream_t)stream;
    g->ws = (char *)workspace;
    g->ws_bytes = workspace_bytes;
    g->ctl = (Ctl *)(g->ws + L.off_ctl);
    g->partials = (double *)(g->ws + L.off_part);
    g->U = g->ws + L.off_U;
    g->U1 = g->ws + L.off_U1;
    g->U3 = g->ws + L.off_U3;
    g->staging = (double *)(g->ws + L.off_stage);
    g->nb_cfl = L.nb_cfl;

    GridP &p = g->g;
    memset(&p, 0, sizeof(p));
    p.dim = dim;
    p.ncell = 1;
    p.dxmin = 1e300;
    p.dV = 1.0;
    for (int d = 0; d < 3; d++) {
        p.n[d] = n3[d];
        p.periodic[d] = (d < dim) ? (bcs[2 * d] == DFV_BC_PERIODIC) : 0;
        for (int s = 0; s < 2; s++) p.wall[d][s] = (d < dim) ? (bcs[2 * d + s] == DFV_BC_REFLECTIVE) : 0;
        p.lo[d] = d < dim ? lo[d] : 0.0;
        p.dx[d] = d < dim ? (hi[d] - lo[d]) / n3[d] : 1.0;
        p.inv_dx[d] = 1.0 / p.dx[d];
        p.ncell *= n3[d];
        if (d < dim) {
            p.dxmin = std::fmin(p.dxmin, p.dx[d]);
            p.dV *= p.dx[d];
        }
    }
    p.pitch = L.pitch;
    dfv::apply_options(p, opt->use_thinc, opt->thinc_beta, opt->hllc_lm, opt->seed_variant,
                       opt->normal_method, opt->probe_mode);
    dfv::finish_params(p);
    {
        const dim3 sg = ops->stage_grid(p);
        g->nb_stage = (long long)sg.x * sg.y * sg.z;
    }

    cudaError_t e = ops->prepare();
    if (e != cudaSuccess) {
        delete g;
        return DFV_ERR_CUDA;
    }
    if (!opt->general_stage && precision == DFV_FP32 && dim == 3 && opt->nmat == 1 && g->solid == 0) {
        e = dfv::gas3_prepare();
        if (e != cudaSuccess) {
            delete g;
            return DFV_ERR_CUDA;
        }
        g->gas3_ready = true;
        const void *bases[3] = {g->U, g->U1, g->U3};
        g->gas3_tma = true;
        for (int k = 0; k < 3 && g->gas3_tma; k++)
            g->gas3_tma = dfv::gas3_encode_map(&g->gas3_map[k], bases[k], p.n[0], p.n[1], p.n[2], p.pitch);
    }
    // the gas kernel's instance record: strips of 28 columns x chunks of rows
    g->d_ginst = (dfv::GasInst *)(g->ws + L.off_gas);
    if (!opt->general_stage && precision == DFV_FP32 && dim == 2 && opt->nmat == 1 && g->solid == 0 &&
        !p.periodic[0] && !p.periodic[1]) {
        dfv::GasInst I;
        memset(&I, 0, sizeof(I));
        I.n0 = p.n[0];
        I.n1 = p.n[1];
        I.rows = opt->gas_rows > 0 ? opt->gas_rows : dfv::gasw_rows((long long)p.n[0] * p.n[1]);
        I.strips = dfv::gasw_strips(p.n[0]);
        I.nitems = I.strips * ((p.n[1] + I.rows - 1) / I.rows);
        I.off = 0;
        I.pitch = p.pitch;
        I.idx = (float)p.inv_dx[0];
        I.idy = (float)p.inv_dx[1];
        I.wall_x0 = p.wall[0][0];
        I.wall_x1 = p.wall[0][1];
        I.wall_y0 = p.wall[1][0];
        I.wall_y1 = p.wall[1][1];
        I.ctl = g->ctl;
        e = cudaMemcpyAsync(g->d_ginst, &I, sizeof(I), cudaMemcpyHostToDevice, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) {
            delete g;
            return DFV_ERR_CUDA;
        }
        g->gas_items = I.nitems;
        // one CTA of independent warps per four items (the hardware balances
        // them; a persistent grid of five CTAs per SM measured 15 % slower on
        // the 1024^2 and 2048^2 cylinders)
        g->gas_grid = (int)std::max(1LL, (g->gas_items + dfv::GaswT::WARPS - 1) / dfv::GaswT::WARPS);
        g->gas_ready = true;
    }
    k_init_ctl<<<1, 1, 0, g->stream>>>(g->ctl);
    g->launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        delete g;
        return DFV_ERR_CUDA;
    }
    *out = g;
    return DFV_OK;
}

dfv_status dfv_add_material(dfv_grid *g, int kind, const dfv_material_params *m, int *id_out)
{
    if (!g) return DFV_ERR_ARG;
    if (!m) return fail(g, DFV_ERR_ARG, "dfv_add_material: null parameters");
    if (g->nmat >= g->nmat_opt) return fail(g, DFV_ERR_ARG, "dfv_add_material: all materials already added");
    if (const char *why = dfv::material_problem(kind, m->gamma, m->rho0, m->Gamma0, m->alpha, m->jc_c1, m->jc_c2,
                                                m->jc_n, m->jc_tmelt, m->jc_cv))
        return fail(g, DFV_ERR_ARG, std::string("dfv_add_material: ") + why);
    dfv::MatP &p = g->g.mat[g->nmat];
    dfv::set_material(p, kind, *m);
    dfv::finish_params(g->g);
    if (id_out) *id_out = g->nmat;
    g->nmat++;
    g->graph_ready = false;
    return DFV_OK;
}

}  // extern "C"

namespace {

// nvar planes between the caller's buffer (planes `pitch` elements apart)
// and the packed staging planes: one copy when packed, else one per plane
// A host buffer the device can address (page-locked memory registered with
// CUDA): the device address of `p`, else null.  The conversion kernels then
// read or write the host fields in place over the CPU-GPU link instead of
// going through a copy into the staging buffer.
const void *mapped_host(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

dfv_status copy_planes(dfv_grid *g, double *dst, long long dpitch, const double *src, long long spitch,
                       cudaMemcpyKind kind, const char *what)
{
    const long long n = g->g.ncell;
    const int nv = g->ops->nvar;
    if (dpitch == n && spitch == n) {
        DFV_CU(g, cudaMemcpyAsync(dst, src, sizeof(double) * nv * (size_t)n, kind, g->stream), what);
        return DFV_OK;
    }
    for (int v = 0; v < nv; v++)
        DFV_CU(g, cudaMemcpyAsync(dst + v * dpitch, src + v * spitch, sizeof(double) * (size_t)n, kind, g->stream),
               what);
    return DFV_OK;
}

dfv_status set_fields_impl(dfv_grid *g, const double *prim, long long pitch, int on_device)
{
    if (!g) return DFV_ERR_ARG;
    if (!prim) return fail(g, DFV_ERR_ARG, "dfv_set_fields: null field pointer");
    if (pitch < g->g.ncell) return fail(g, DFV_ERR_ARG, "dfv_set_fields: plane pitch below the cell count");
    if (dfv_status fs = flush_fin(g); fs != DFV_OK) return fs;
    if (g->nmat != g->nmat_opt) return fail(g, DFV_ERR_ARG, "dfv_set_fields: materials missing");
    // device and page-locked host fields are converted in place; other host
    // memory goes through the staging buffer
    const double *src = on_device ? prim : static_cast<const double *>(mapped_host(prim));
    long long spitch = pitch;
    if (!src) {
        if (dfv_status cs = copy_planes(g, g->staging, g->g.ncell, prim, pitch, cudaMemcpyHostToDevice,
                                        "dfv_set_fields copy");
            cs != DFV_OK)
            return cs;
        src = g->staging;
        spitch = g->g.ncell;
    }
    DFV_CU(g, g->ops->prim_to_cons(g->g, src, spitch, g->U, g->stream), "k_prim_to_cons");
    g->launches++;
    // new r: the rigid box is unknown until the next stage 3
    DFV_CU(g, cudaMemsetAsync(&g->ctl->rbox_valid, 0, sizeof(int), g->stream), "dfv_set_fields box");
    if (!on_device) DFV_CU(g, cudaStreamSynchronize(g->stream), "dfv_set_fields sync");
    g->fields_set = true;
    g->smax_valid = false;
    g->dt_valid = false;
    return DFV_OK;
}

dfv_status get_fields_impl(dfv_grid *g, double *outp, long long pitch, int which, int on_device)
{
    if (!g) return DFV_ERR_ARG;
    if (!outp) return fail(g, DFV_ERR_ARG, "dfv_get_fields: null output");
    if (!g->fields_set) return fail(g, DFV_ERR_ARG, "dfv_get_fields: fields not set");
    if (pitch < g->g.ncell) return fail(g, DFV_ERR_ARG, "dfv_get_fields: plane pitch below the cell count");
    if (which != DFV_FIELDS_PRIMITIVE && which != DFV_FIELDS_CONSERVED)
        return fail(g, DFV_ERR_ARG, "dfv_get_fields: bad `which`");
    // into device or page-locked host fields in place; other host memory
    // through the staging buffer
    double *dst = on_device ? outp : static_cast<double *>(const_cast<void *>(mapped_host(outp)));
    const bool staged = dst == nullptr;
    const long long dpitch = staged ? g->g.ncell : pitch;
    if (staged) dst = g->staging;
    if (which == DFV_FIELDS_PRIMITIVE) {
        DFV_CU(g, g->ops->cons_to_prim(g->g, g->U, dst, dpitch, g->stream), "k_cons_to_prim");
    } else {
        DFV_CU(g, g->ops->cons_to_f64(g->g, g->U, dst, dpitch, g->ops->nvar, g->stream), "k_cons_to_f64");
    }
    g->launches++;
    if (staged) {
        if (dfv_status cs = copy_planes(g, outp, pitch, g->staging, g->g.ncell, cudaMemcpyDeviceToHost,
                                        "dfv_get_fields copy");
            cs != DFV_OK)
            return cs;
    }
    if (!on_device) DFV_CU(g, cudaStreamSynchronize(g->stream), "dfv_get_fields sync");
    return DFV_OK;
}

}  // namespace

extern "C" {

dfv_status dfv_set_fields(dfv_grid *g, const double *prim, int on_device)
{
    return set_fields_impl(g, prim, g ? g->g.ncell : 0, on_device);
}

dfv_status dfv_set_fields_pitched(dfv_grid *g, const double *prim, long long plane_pitch, int on_device)
{
    return set_fields_impl(g, prim, plane_pitch, on_device);
}

dfv_status dfv_get_fields(dfv_grid *g, double *outp, int which, int on_device)
{
    return get_fields_impl(g, outp, g ? g->g.ncell : 0, which, on_device);
}

dfv_status dfv_get_fields_pitched(dfv_grid *g, double *outp, long long plane_pitch, int which, int on_device)
{
    return get_fields_impl(g, outp, plane_pitch, which, on_device);
}

dfv_status dfv_set_state(dfv_grid *g, const double *cons, int on_device)
{
    if (!g) return DFV_ERR_ARG;
    if (!cons) return fail(g, DFV_ERR_ARG, "dfv_set_state: null state pointer");
    if (dfv_status fs = flush_fin(g); fs != DFV_OK) return fs;
    if (g->nmat != g->nmat_opt) return fail(g, DFV_ERR_ARG, "dfv_set_state: materials missing");
    const long long n = g->g.ncell, P = g->g.pitch;
    const int nv = g->ops->nvar;
    const cudaMemcpyKind in = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (g->precision == DFV_FP64) {
        for (int v = 0; v < nv; v++)
            DFV_CU(g, cudaMemcpyAsync((double *)g->U + v * P, cons + v * n, sizeof(double) * (size_t)n, in, g->stream),
                   "dfv_set_state copy");
    } else {
        DFV_CU(g, cudaMemcpyAsync(g->staging, cons, sizeof(double) * nv * (size_t)n, in, g->stream),
               "dfv_set_state copy");
        const long long blocks = std::min((n * nv + 255) / 256, 152LL * 16);
        k_state_from_f64<<<(unsigned)std::max(1LL, blocks), 256, 0, g->stream>>>(g->staging, (float *)g->U, n, P, nv);
        DFV_CU(g, cudaGetLastError(), "k_state_from_f64");
        g->launches++;
    }
    // the rigid box of the restored state is unknown until the next stage 3
    DFV_CU(g, cudaMemsetAsync(&g->ctl->rbox_valid, 0, sizeof(int), g->stream), "dfv_set_state box");
    if (!on_device) DFV_CU(g, cudaStreamSynchronize(g->stream), "dfv_set_state sync");
    g->fields_set = true;
    g->smax_valid = false;
    g->dt_valid = false;
    return DFV_OK;
}

dfv_status dfv_set_body(dfv_grid *g, const double v[3], const double x[3], double mass, int dynamic)
{
    if (!g) return DFV_ERR_ARG;
    double vv[3] = {0, 0, 0}, xx[3] = {0, 0, 0};
    if (dfv_status fs = flush_fin(g); fs != DFV_OK) return fs;
    for (int d = 0; d < 3; d++) {
        vv[d] = (v && d < g->dim) ? v[d] : 0.0;
        xx[d] = x ? x[d] : 0.0;
    }
    if (dynamic && !(mass > 0.0)) return fail(g, DFV_ERR_ARG, "dfv_set_body: a dynamic body needs mass > 0");
    k_set_body<<<1, 1, 0, g->stream>>>(g->ctl, vv[0], vv[1], vv[2], xx[0], xx[1], xx[2], mass, dynamic ? 1 : 0);
    g->launches++;
    DFV_CU(g, cudaGetLastError(), "k_set_body");
    g->dynamic = dynamic != 0;
    g->body_moving = vv[0] != 0.0 || vv[1] != 0.0 || vv[2] != 0.0;
    g->smax_valid = false;   // the body speed enters the CFL bound
    g->dt_valid = false;
    g->graph_ready = false;
    return DFV_OK;
}

dfv_status dfv_get_body(dfv_grid *g, double force[3], double v[3], double x[3])
{
    if (!g) return DFV_ERR_ARG;
    if (dfv_status fs = flush_fin(g); fs != DFV_OK) return fs;
    Ctl h;
    dfv_status s = read_ctl(g, &h);
    for (int d = 0; d < 3; d++) {
        if (force) force[d] = h.force[d];
        if (v) v[d] = h.v[d];
        if (x) x[d] = h.x[d];
    }
    return s;
}

dfv_status dfv_compute_dt(dfv_grid *g, double cfl, double *dt_out)
{
    if (!g) return DFV_ERR_ARG;
    if (!dt_out || !(cfl > 0.0)) return fail(g, DFV_ERR_ARG, "dfv_compute_dt: bad arguments");
    if (!g->fields_set) return fail(g, DFV_ERR_ARG, "dfv_compute_dt: fields not set");
    if (dfv_status fs = flush_fin(g); fs != DFV_OK) return fs;
    if (!g->smax_valid) {
        dfv_status s = reduce_cfl(g);
        if (s != DFV_OK) return s;
    }
    Ctl h;
    dfv_status s = read_ctl(g, &h);
    *dt_out = cfl / h.smax;
    return s;
}

dfv_status dfv_step(dfv_grid *g, double dt)
{
    if (!g) return DFV_ERR_ARG;
    if (!g->fields_set) return fail(g, DFV_ERR_ARG, "dfv_step: fields not set");
    if (!(dt >= 0.0)) return fail(g, DFV_ERR_ARG, "dfv_step: dt must be >= 0");
    if (dfv_status fs = flush_fin(g); fs != DFV_OK) return fs;
    dfv::k_set_dt<<<1, 1, 0, g->stream>>>(g->ctl, dt);
    g->launches++;
    DFV_CU(g, cudaGetLastError(), "k_set_dt");
    dfv_status s = launch_step(g, 0);
    if (s == DFV_OK) g->smax_valid = true;
    g->dt_valid = false;
    return s;
}

dfv_status dfv_run(dfv_grid *g, int steps, double cfl, double t_end, double *t_out)
{
    if (!g) return DFV_ERR_ARG;
    if (!g->fields_set) return fail(g, DFV_ERR_ARG, "dfv_run: fields not set");
    if (steps < 0 || !(cfl > 0.0)) return fail(g, DFV_ERR_ARG, "dfv_run: bad arguments");
    const double tend = t_end > 0.0 ? t_end : 0.0;
    const bool defer = can_defer(g);
    if (g->fin_pending && (!defer || cfl != g->run_cfl || tend != g->run_tend || !g->smax_valid || !g->dt_valid)) {
        dfv_status fs = flush_fin(g);
        if (fs != DFV_OK) return fs;
    }
    if (cfl != g->run_cfl || tend != g->run_tend) {
        k_set_run<<<1, 1, 0, g->stream>>>(g->ctl, cfl, tend);
        g->launches++;
        DFV_CU(g, cudaGetLastError(), "k_set_run");
        g->run_cfl = cfl;
        g->run_tend = tend;
        g->dt_valid = false;
    }
    if (!g->smax_valid) {
        dfv_status s = reduce_cfl(g);
        if (s != DFV_OK) return s;
        g->dt_valid = false;
    }
    dfv_status s = DFV_OK;
    if (!g->dt_valid) {
        s = finalize(g, 8, 0);   // dt from the current smax
        if (s != DFV_OK) return s;
        g->dt_valid = true;
    }
    const bool use_graph = g->stream != nullptr && steps > 0 && !g->prof;
    const int fin_run = 1 | 4 | 8;   // the finalize mode of a device-driven step (static body)
    if (use_graph && (!g->graph_ready || g->graph_defer != defer)) {
        if (g->graph) {
            cudaGraphExecDestroy(g->graph);
            g->graph = nullptr;
        }
        cudaGraph_t graph = nullptr;
        DFV_CU(g, cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        const long long before = g->launches;
        // the replayed step runs the previous step's deferred finalize
        dfv_status cs = defer ? launch_step(g, 8, true, fin_run, true) : launch_step(g, 8, true);
        cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
        g->graph_launches = g->launches - before;   // kernels of one replay
        g->launches = before;   // capture launches nothing
        if (cs != DFV_OK) return cs;
        if (e != cudaSuccess) return cuda_fail(g, e, "end capture");
        e = cudaGraphInstantiate(&g->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(g, e, "graph instantiate");
        g->graph_ready = true;
        g->graph_defer = defer;
    }
    for (int k = 0; k < steps; k++) {
        if (defer && !g->fin_pending) {
            // nothing to finalize before this step: launched directly
            s = launch_step(g, 8, false, 0, true);
            if (s != DFV_OK) return s;
        } else if (use_graph) {
            DFV_CU(g, cudaGraphLaunch(g->graph, g->stream), "graph launch");
            g->launches += g->graph_launches;
        } else {
            s = defer ? launch_step(g, 8, false, g->fin_pending, true) : launch_step(g, 8);
            if (s != DFV_OK) return s;
        }
        if (defer) g->fin_pending = fin_run;
    }
    g->smax_valid = true;
    if (t_out) {
        if (dfv_status fs = flush_fin(g); fs != DFV_OK) return fs;
        Ctl h;
        s = read_ctl(g, &h);
        *t_out = h.t;
        return s;
    }
    return DFV_OK;
}

dfv_status dfv_check(dfv_grid *g, int timeout_ms)
{
    if (!g) return DFV_ERR_ARG;
    if (dfv_status fs = flush_fin(g); fs != DFV_OK) return fs;
    dfv_status s = sync_stream(g, timeout_ms);
    if (s != DFV_OK) return s;
    Ctl h;
    return read_ctl(g, &h);
}

dfv_status dfv_profile(dfv_grid *g, int enable, double ms_out[5], long long *steps_out)
{
    if (!g) return DFV_ERR_ARG;
    dfv_status s = DFV_OK;
    double ms[5] = {0, 0, 0, 0, 0};
    long long n = 0;
    if (!g->ev_steps.empty()) {
        cudaError_t e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) s = cuda_fail(g, e, "dfv_profile sync");
        for (auto &ev : g->ev_steps) {
            for (int k = 0; k < 5 && s == DFV_OK; k++) {
                float t = 0.f;
                e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
                if (e != cudaSuccess) s = cuda_fail(g, e, "cudaEventElapsedTime");
                ms[k] += t;
            }
            for (auto x : ev) g->ev_free.push_back(x);
            n++;
        }
        g->ev_steps.clear();
    }
    if (ms_out)
        for (int k = 0; k < 5; k++) ms_out[k] = ms[k];
    if (steps_out) *steps_out = n;
    g->prof = enable != 0;
    return s;
}

dfv_status dfv_launch_count(const dfv_grid *g, long long *count)
{
    if (!g || !count) return DFV_ERR_ARG;
    *count = g->launches;
    return DFV_OK;
}

dfv_status dfv_state_layout(const dfv_grid *g, size_t off[3], long long *pitch, int *nvar, int *elem_bytes)
{
    if (!g) return DFV_ERR_ARG;
    if (off) {
        off[0] = (size_t)((const char *)g->U - g->ws);
        off[1] = (size_t)((const char *)g->U1 - g->ws);
        off[2] = (size_t)((const char *)g->U3 - g->ws);
    }
    if (pitch) *pitch = g->g.pitch;
    if (nvar) *nvar = g->ops->nvar;
    if (elem_bytes) *elem_bytes = g->precision == DFV_FP32 ? 4 : 8;
    return DFV_OK;
}

dfv_status dfv_destroy(dfv_grid *g)
{
    if (!g) return DFV_ERR_ARG;
    if (g->graph) cudaGraphExecDestroy(g->graph);
    for (auto &ev : g->ev_steps)
        for (auto x : ev) g->ev_free.push_back(x);
    for (auto x : g->ev_free) cudaEventDestroy(x);
    delete g;
    return DFV_OK;
}

const char *dfv_last_error(const dfv_grid *g)
{
    if (!g) return k_no_grid;
    return g->err.c_str();
}

}  // extern "C"
