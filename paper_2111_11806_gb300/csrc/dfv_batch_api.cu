// dfv_batch_api.cu -- the batched C ABI (include/dfvrb.h, dfv_batch_*):
// many independent 2-D grids of different sizes, each with its own body and
// time step, advanced by one persistent launch per phase over a work list of
// (instance, tile) items; a step is captured once into a CUDA graph.  The
// persistent grid size and the item schedule are chosen by dfv_batch_autotune
// from timed trial steps.  No device memory is allocated here.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/dfvrb.h"
#include "dfv_batch.cuh"
#include "dfv_gasw.cuh"
#include "dfv_ops.h"

using dfv::BatchArgs;
using dfv::BatchInst;
using dfv::Ctl;
using dfv::GridP;
using dfv::Kern;

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Plan {
    size_t off_inst, off_items0, off_items1, off_ctl, off_ctlbak, off_part, off_queue, off_vbody;
    size_t off_ginst, off_gitems0, off_gitems1;   // the gas stage kernel's records
    size_t off_U, off_U1, off_U3, off_Ubak, off_stage, total;
    long long elems, nitems, max_cells, ntiles_total, gas_nitems;
    int gas_rows;
    std::vector<long long> inst_off, inst_part0;
    std::vector<int> tiles_x, tiles_y;
};

// the tile of the 2-D stage kernels that the batch items address
int tile_x(int precision) { return precision == DFV_FP32 ? dfv::Tile<2, 4>::TX : dfv::Tile<2, 8>::TX; }
int tile_y(int precision) { return precision == DFV_FP32 ? dfv::Tile<2, 4>::TY : dfv::Tile<2, 8>::TY; }

int nvar_2d(int nmat) { return (nmat - 1) + nmat + 2 + 1 + 1; }

bool plan_batch(int count, const dfv_instance_desc *desc, int precision, int nmat, int gas_rows, Plan &P)
{
    const int w = precision == DFV_FP32 ? 4 : 8;
    const int nvar = nvar_2d(nmat);
    P.elems = 0;
    P.nitems = 0;
    P.max_cells = 0;
    P.inst_off.resize(count);
    P.inst_part0.resize(count);
    P.tiles_x.resize(count);
    P.tiles_y.resize(count);
    for (int i = 0; i < count; i++) {
        const long long nc = (long long)desc[i].n[0] * desc[i].n[1];
        if (desc[i].n[0] < 1 || desc[i].n[1] < 1) return false;
        const long long pitch = (nc + 63) / 64 * 64;
        P.inst_off[i] = P.elems;
        P.elems += nvar * pitch;
        P.tiles_x[i] = (desc[i].n[0] + tile_x(precision) - 1) / tile_x(precision);
        P.tiles_y[i] = (desc[i].n[1] + tile_y(precision) - 1) / tile_y(precision);
        P.inst_part0[i] = P.nitems;
        P.nitems += (long long)P.tiles_x[i] * P.tiles_y[i];
        P.max_cells = std::max(P.max_cells, nc);
    }
    // the gas stage kernel's work items: strips of 28 columns x chunks of rows
    long long cells = 0;
    for (int i = 0; i < count; i++) cells += (long long)desc[i].n[0] * desc[i].n[1];
    P.gas_rows = gas_rows > 0 ? gas_rows : dfv::gasw_rows(cells);
    P.gas_nitems = 0;
    for (int i = 0; i < count; i++)
        P.gas_nitems += (long long)dfv::gasw_strips(desc[i].n[0]) * ((desc[i].n[1] + P.gas_rows - 1) / P.gas_rows);
    P.ntiles_total = P.nitems;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += al256(bytes);
        return o;
    };
    P.off_inst = take(sizeof(BatchInst) * count);
    P.off_items0 = take(sizeof(int2) * P.nitems);
    P.off_items1 = take(sizeof(int2) * P.nitems);
    P.off_ctl = take(256 * (size_t)count);
    P.off_ctlbak = take(256 * (size_t)count);
    P.off_part = take(sizeof(double) * 4 * P.nitems);
    P.off_queue = take(sizeof(unsigned int) * 8);
    P.off_vbody = take(sizeof(double) * 3 * count);
    P.off_ginst = take(sizeof(dfv::GasInst) * count);
    P.off_gitems0 = take(sizeof(int2) * P.gas_nitems);
    P.off_gitems1 = take(sizeof(int2) * P.gas_nitems);
    P.off_U = take((size_t)w * P.elems);
    P.off_U1 = take((size_t)w * P.elems);
    P.off_U3 = take((size_t)w * P.elems);
    P.off_Ubak = take((size_t)w * P.elems);
    P.off_stage = take(sizeof(double) * nvar * (size_t)P.max_cells);
    P.total = off;
    return true;
}

Kern kernels_for(int precision, int nmat)
{
    return precision == DFV_FP32 ? dfv::batch_kernels_f32(nmat) : dfv::batch_kernels_f64(nmat);
}

}  // namespace

struct dfv_batch {
    int count = 0, precision = 0, nmat_opt = 1, nmat = 0;
    int seed_opt = 0;   // seeding option set of every instance (dfv::seed_opt)
    dfv_options opt{};
    Plan plan;
    std::vector<dfv_instance_desc> desc;
    std::vector<BatchInst> hinst;
    std::vector<char> fields_set;
    Kern kern{};
    const dfv::Ops *ops = nullptr;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    BatchInst *d_inst = nullptr;
    int2 *d_items[2] = {nullptr, nullptr};
    Ctl *d_ctl = nullptr, *d_ctl_bak = nullptr;
    double *d_part = nullptr, *d_vbody = nullptr, *staging = nullptr;
    unsigned int *d_queue = nullptr;
    void *U = nullptr, *U1 = nullptr, *U3 = nullptr, *Ubak = nullptr;
    int sm_count = 152, ctas_per_sm = 1, max_ctas = 1;
    int schedule = 1;          // 0 instance order, static; 1 largest first, static; 2 largest first, dynamic queue
    bool uploaded = false, dt_valid = false;
    double run_cfl = -1.0, run_tend = -1.0;
    cudaGraphExec_t graph = nullptr;
    bool graph_ready = false;
    long long graph_launches = 0;   // kernels in one replay of the step graph
    bool prof = false;
    // the 2-D single-gas FP32 stage kernel (dfv_gasw.cuh): instance records
    // and (instance, item) lists of its strips x chunks
    bool gas = false;
    int gas_max_ctas = 1;
    dfv::GasInst *d_ginst = nullptr;
    int2 *d_gitems[2] = {nullptr, nullptr};
    std::vector<std::array<cudaEvent_t, 5>> ev_steps;
    std::vector<cudaEvent_t> ev_free;
    std::string err;
    long long launches = 0;
};

namespace {

dfv_status bfail(dfv_batch *b, dfv_status s, const std::string &m)
{
    if (b) b->err = m;
    return s;
}

#define B_CU(b, call, where)                                                                            \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return bfail(b, DFV_ERR_CUDA, std::string("dfv_batch: ") + where + ": " + \
                                                                 cudaGetErrorString(e_));               \
    } while (0)

dfv_status upload(dfv_batch *b)
{
    if (b->uploaded) return DFV_OK;
    for (auto &I : b->hinst) dfv::finish_params(I.g);
    B_CU(b, cudaMemcpyAsync(b->d_inst, b->hinst.data(), sizeof(BatchInst) * b->count, cudaMemcpyHostToDevice,
                            b->stream),
         "upload instances");
    B_CU(b, cudaStreamSynchronize(b->stream), "upload sync");
    b->uploaded = true;
    return DFV_OK;
}

BatchArgs args(dfv_batch *b, const void *in, const void *un, void *out, int final_mode)
{
    BatchArgs a;
    a.in = in;
    a.un = un;
    a.out = out;
    a.inst = b->d_inst;
    a.items = b->d_items[b->schedule == 0 ? 0 : 1];
    a.nitems = b->plan.nitems;
    a.partials = b->d_part;
    a.final_mode = final_mode;
    a.queue = nullptr;
    return a;
}

// ctas_per_sm = 0: one CTA per work item (the hardware schedules them);
// otherwise a persistent grid of ctas_per_sm CTAs per SM loops over the items.
int grid_size(dfv_batch *b)
{
    if (b->ctas_per_sm <= 0) return (int)std::max(1LL, b->plan.nitems);
    const long long persistent = (long long)b->sm_count * b->ctas_per_sm;
    return (int)std::max(1LL, std::min(persistent, b->plan.nitems));
}

// one launch of a phase.  The dynamic schedule's counters (slots 1-3, one
// per stage) start at 0 and the finalize phase puts them back to 0 at the end
// of every step, so no memset sits between the step's kernels.  Seeding
// (phase 0) and the CFL reduction (phase 4) do little work per item, so they
// always run one CTA per item and let the hardware overlap the items' memory
// latency.
dfv_status phase(dfv_batch *b, int ph, const void *in, const void *un, void *out, int final_mode, int slot)
{
    BatchArgs a = args(b, in, un, out, final_mode);
    const bool light = (ph == 0 || ph == 4 || ph == 5 || ph == 6 || ph == 7);
    if (b->schedule == 2 && !light) a.queue = b->d_queue + slot;
    if (ph == 7) a.queue = b->d_queue;
    // seeding: SEED_CTAS per instance (the launcher multiplies); finalize: one
    // per instance; CFL: one CTA per work item
    const bool per_inst = (ph == 0 || ph == 5 || ph == 6 || ph == 7);
    if (b->gas && ph >= 1 && ph <= 3) {
        const dfv::MatC<float> &m = b->hinst[0].g.mc_f[0];
        dfv::GaswArgs ga;
        ga.inst = b->d_ginst;
        ga.items = b->d_gitems[b->schedule == 0 ? 0 : 1];
        ga.nitems = b->plan.gas_nitems;
        ga.queue = a.queue;
        ga.in = (const float *)in;
        ga.un = (const float *)un;
        ga.out = (float *)out;
        ga.Gam = m.Gam;
        ga.invGam = m.invGam;
        ga.pref0 = m.pref0;
        // CTAs of independent warps, one warp per item at a time
        const long long n = (b->plan.gas_nitems + dfv::GaswT::WARPS - 1) / dfv::GaswT::WARPS;
        const long long persistent = (long long)b->sm_count * std::min(std::max(b->ctas_per_sm, 1), b->gas_max_ctas);
        const int grid = (int)std::max(1LL, b->ctas_per_sm <= 0 ? n : std::min(persistent, n));
        B_CU(b, dfv::gasw_stage(ph, ga, grid, b->stream), "gas stage kernel");
        b->launches++;
        return DFV_OK;
    }
    const int grid = per_inst ? b->count : (light ? (int)std::max(1LL, b->plan.nitems) : grid_size(b));
    B_CU(b, b->kern.launch(ph, grid, a, b->seed_opt, b->stream), "batch kernel");
    b->launches++;
    return DFV_OK;
}

cudaEvent_t take_ev(dfv_batch *b)
{
    if (!b->ev_free.empty()) {
        cudaEvent_t e = b->ev_free.back();
        b->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

dfv_status batch_step(dfv_batch *b, bool capturing)
{
    const bool rec = b->prof && !capturing;
    std::array<cudaEvent_t, 5> ev{};
    if (rec) {
        for (auto &e : ev) e = take_ev(b);
        B_CU(b, cudaEventRecord(ev[0], b->stream), "event");
    }
    dfv_status s;
    if (b->opt.probe_mode == 1) {
        // the fixed probe may read rigid cells: seed from the step-start state via U1
        if ((s = phase(b, 5, b->U, b->U, b->U1, 0, 0)) != DFV_OK) return s;
        s = phase(b, 6, b->U, b->U, b->U1, 0, 0);
    } else {
        s = phase(b, 0, b->U, b->U, b->U, 0, 0);
    }
    if (s != DFV_OK) return s;
    if (rec) B_CU(b, cudaEventRecord(ev[1], b->stream), "event");
    if ((s = phase(b, 1, b->U, b->U, b->U1, 0, 1)) != DFV_OK) return s;
    if (rec) B_CU(b, cudaEventRecord(ev[2], b->stream), "event");
    if ((s = phase(b, 2, b->U1, b->U, b->U3, 0, 2)) != DFV_OK) return s;
    if (rec) B_CU(b, cudaEventRecord(ev[3], b->stream), "event");
    if ((s = phase(b, 3, b->U3, b->U, b->U, 0, 3)) != DFV_OK) return s;
    if ((s = phase(b, 7, b->U, b->U, b->U, 1 | 4 | 8, 0)) != DFV_OK) return s;
    if (rec) {
        B_CU(b, cudaEventRecord(ev[4], b->stream), "event");
        b->ev_steps.push_back(ev);
    }
    return DFV_OK;
}

dfv_status ensure_dt(dfv_batch *b, double cfl, double t_end)
{
    const double te = t_end > 0.0 ? t_end : 0.0;
    if (cfl != b->run_cfl || te != b->run_tend) {
        dfv::k_batch_set_run<<<(b->count + 255) / 256, 256, 0, b->stream>>>(b->d_ctl, b->count, cfl, te);
        b->launches++;
        B_CU(b, cudaGetLastError(), "set run");
        b->run_cfl = cfl;
        b->run_tend = te;
        b->dt_valid = false;
    }
    if (!b->dt_valid) {
        dfv_status s = phase(b, 4, b->U, b->U, b->U, 1 | 8, 4);
        if (s != DFV_OK) return s;
        b->dt_valid = true;
    }
    return DFV_OK;
}

}  // namespace

extern "C" {

dfv_status dfv_batch_workspace_bytes(int dim, int count, const dfv_instance_desc *desc, int precision,
                                     const dfv_options *opt, size_t *bytes)
{
    if (!desc || !opt || !bytes || count < 1) return DFV_ERR_ARG;
    if (dim != 2 || opt->solid || opt->nmat < 1 || opt->nmat > 3) return DFV_ERR_UNSUPPORTED;
    if (precision != DFV_FP64 && precision != DFV_FP32) return DFV_ERR_ARG;
    if (opt->gas_rows < 0 || opt->gas_rows > 4096) return DFV_ERR_ARG;
    if (opt->seed_stages) return DFV_ERR_UNSUPPORTED;
    Plan P;
    if (!plan_batch(count, desc, precision, opt->nmat, opt->gas_rows, P)) return DFV_ERR_ARG;
    *bytes = P.total;
    return DFV_OK;
}

dfv_status dfv_batch_create(int dim, int count, const dfv_instance_desc *desc, int precision,
                            const dfv_options *opt, void *workspace, size_t workspace_bytes, void *stream,
                            dfv_batch **out)
{
    if (!out || !desc || !opt || count < 1) return DFV_ERR_ARG;
    *out = nullptr;
    if (dim != 2 || opt->solid || opt->nmat < 1 || opt->nmat > 3) return DFV_ERR_UNSUPPORTED;
    if (precision != DFV_FP64 && precision != DFV_FP32) return DFV_ERR_ARG;
    if (opt->gas_rows < 0 || opt->gas_rows > 4096) return DFV_ERR_ARG;
    if (opt->seed_stages) return DFV_ERR_UNSUPPORTED;
    dfv_batch *b = new dfv_batch();
    b->count = count;
    b->precision = precision;
    b->opt = *opt;
    b->nmat_opt = opt->nmat;
    b->seed_opt = (opt->normal_method == 1 ? 1 : 0) | (opt->seed_variant == 1 ? 2 : 0);
    b->desc.assign(desc, desc + count);
    if (!plan_batch(count, desc, precision, opt->nmat, opt->gas_rows, b->plan)) {
        delete b;
        return DFV_ERR_ARG;
    }
    const Plan &P = b->plan;
    if (!workspace || workspace_bytes < P.total || ((uintptr_t)workspace & 255u)) {
        delete b;
        return DFV_ERR_WORKSPACE;
    }
    for (int i = 0; i < count; i++)
        for (int d = 0; d < 2; d++)
            if (!(desc[i].hi[d] > desc[i].lo[d]) ||
                ((desc[i].bc[2 * d] == DFV_BC_PERIODIC) != (desc[i].bc[2 * d + 1] == DFV_BC_PERIODIC)) ||
                desc[i].bc[2 * d] < DFV_BC_TRANSMISSIVE || desc[i].bc[2 * d] > DFV_BC_REFLECTIVE ||
                desc[i].bc[2 * d + 1] < DFV_BC_TRANSMISSIVE || desc[i].bc[2 * d + 1] > DFV_BC_REFLECTIVE) {
                delete b;
                return DFV_ERR_ARG;
            }
    b->ops = dfv::ops_for(precision == DFV_FP32 ? 1 : 0, 2, opt->nmat, 0);
    b->kern = kernels_for(precision, opt->nmat);
    b->stream = (cudaStream_t)stream;
    b->ws = (char *)workspace;
    b->d_inst = (BatchInst *)(b->ws + P.off_inst);
    b->d_items[0] = (int2 *)(b->ws + P.off_items0);
    b->d_items[1] = (int2 *)(b->ws + P.off_items1);
    b->d_ctl = (Ctl *)(b->ws + P.off_ctl);
    b->d_ctl_bak = (Ctl *)(b->ws + P.off_ctlbak);
    b->d_part = (double *)(b->ws + P.off_part);
    b->d_queue = (unsigned int *)(b->ws + P.off_queue);
    if (cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned int) * 8, b->stream) != cudaSuccess) {
        delete b;
        return DFV_ERR_CUDA;
    }
    b->d_vbody = (double *)(b->ws + P.off_vbody);
    b->U = b->ws + P.off_U;
    b->U1 = b->ws + P.off_U1;
    b->U3 = b->ws + P.off_U3;
    b->Ubak = b->ws + P.off_Ubak;
    b->staging = (double *)(b->ws + P.off_stage);
    b->fields_set.assign(count, 0);

    // instance records (materials are filled by dfv_batch_add_material)
    b->hinst.resize(count);
    for (int i = 0; i < count; i++) {
        BatchInst &I = b->hinst[i];
        memset(&I, 0, sizeof(I));
        GridP &p = I.g;
        p.dim = 2;
        p.ncell = 1;
        p.dxmin = 1e300;
        p.dV = 1.0;
        for (int d = 0; d < 3; d++) {
            p.n[d] = d < 2 ? desc[i].n[d] : 1;
            p.periodic[d] = d < 2 ? (desc[i].bc[2 * d] == DFV_BC_PERIODIC) : 0;
            for (int s = 0; s < 2; s++) p.wall[d][s] = d < 2 ? (desc[i].bc[2 * d + s] == DFV_BC_REFLECTIVE) : 0;
            p.lo[d] = d < 2 ? desc[i].lo[d] : 0.0;
            p.dx[d] = d < 2 ? (desc[i].hi[d] - desc[i].lo[d]) / p.n[d] : 1.0;
            p.inv_dx[d] = 1.0 / p.dx[d];
            p.ncell *= p.n[d];
            if (d < 2) {
                p.dxmin = std::fmin(p.dxmin, p.dx[d]);
                p.dV *= p.dx[d];
            }
        }
        p.pitch = (p.ncell + 63) / 64 * 64;
        dfv::apply_options(p, opt->use_thinc, opt->thinc_beta, opt->hllc_lm, opt->seed_variant,
                       opt->normal_method, opt->probe_mode);
        I.off = P.inst_off[i];
        I.part0 = P.inst_part0[i];
        I.tiles_x = P.tiles_x[i];
        I.tiles_y = P.tiles_y[i];
        I.ntiles = P.tiles_x[i] * P.tiles_y[i];
        I.ctl = b->d_ctl + i;
    }
    // work lists: instance order, and largest instances first
    std::vector<int2> items0, items1;
    items0.reserve(P.nitems);
    for (int i = 0; i < count; i++)
        for (int t = 0; t < b->hinst[i].ntiles; t++) items0.push_back(make_int2(i, t));
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->hinst[x].ntiles > b->hinst[y].ntiles; });
    for (int i : order)
        for (int t = 0; t < b->hinst[i].ntiles; t++) items1.push_back(make_int2(i, t));
    std::vector<double> vb(3 * count);
    for (int i = 0; i < count; i++)
        for (int d = 0; d < 3; d++) vb[3 * i + d] = d < 2 ? desc[i].v_body[d] : 0.0;

    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    // the gas stage kernel (dfv_gasw.cuh): one FP32 gas, no HLLC-LM, every
    // instance with a static body and no periodic side
    b->d_ginst = (dfv::GasInst *)(b->ws + P.off_ginst);
    b->d_gitems[0] = (int2 *)(b->ws + P.off_gitems0);
    b->d_gitems[1] = (int2 *)(b->ws + P.off_gitems1);
    bool gas = !opt->general_stage && precision == DFV_FP32 && opt->nmat == 1 && !opt->hllc_lm;
    for (int i = 0; i < count && gas; i++) {
        const int per[3] = {b->hinst[i].g.periodic[0], b->hinst[i].g.periodic[1], 0};
        const bool moving = desc[i].v_body[0] != 0.0 || desc[i].v_body[1] != 0.0 || desc[i].v_body[2] != 0.0;
        gas = dfv::gas_eligible(1, 2, 1, 0, DFV_MAT_IDEAL, per, 0, moving);
    }
    std::vector<dfv::GasInst> ginst;
    std::vector<int2> gitems0, gitems1;
    if (gas) {
        ginst.resize(count);
        for (int i = 0; i < count; i++) {
            const GridP &p = b->hinst[i].g;
            dfv::GasInst &G = ginst[i];
            memset(&G, 0, sizeof(G));
            G.n0 = p.n[0];
            G.n1 = p.n[1];
            G.rows = P.gas_rows;
            G.strips = dfv::gasw_strips(p.n[0]);
            G.nitems = G.strips * ((p.n[1] + G.rows - 1) / G.rows);
            G.off = b->hinst[i].off;
            G.pitch = p.pitch;
            G.idx = (float)p.inv_dx[0];
            G.idy = (float)p.inv_dx[1];
            G.wall_x0 = p.wall[0][0];
            G.wall_x1 = p.wall[0][1];
            G.wall_y0 = p.wall[1][0];
            G.wall_y1 = p.wall[1][1];
            G.ctl = b->d_ctl + i;
        }
        {
            for (int i = 0; i < count; i++)
                for (int t = 0; t < ginst[i].nitems; t++) gitems0.push_back(make_int2(i, t));
            std::vector<int> gord(count);
            std::iota(gord.begin(), gord.end(), 0);
            std::stable_sort(gord.begin(), gord.end(),
                             [&](int x, int y) { return ginst[x].nitems > ginst[y].nitems; });
            for (int i : gord)
                for (int t = 0; t < ginst[i].nitems; t++) gitems1.push_back(make_int2(i, t));
        }
    }
    cudaError_t e = b->kern.prepare();
    if (e == cudaSuccess) {
        b->max_ctas = b->kern.max_ctas_per_sm();
        b->ctas_per_sm = b->max_ctas;
        e = cudaMemcpyAsync(b->d_items[0], items0.data(), sizeof(int2) * items0.size(), cudaMemcpyHostToDevice,
                            b->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_items[1], items1.data(), sizeof(int2) * items1.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_vbody, vb.data(), sizeof(double) * vb.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && gas) {
        e = cudaMemcpyAsync(b->d_ginst, ginst.data(), sizeof(dfv::GasInst) * count, cudaMemcpyHostToDevice,
                            b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_gitems[0], gitems0.data(), sizeof(int2) * gitems0.size(),
                                cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_gitems[1], gitems1.data(), sizeof(int2) * gitems1.size(),
                                cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) {
            b->gas = true;
            b->gas_max_ctas = dfv::gasw_max_ctas_per_sm();
        }
    }
    if (e == cudaSuccess) {
        dfv::k_batch_init_ctl<<<(count + 255) / 256, 256, 0, b->stream>>>(b->d_ctl, count, b->d_vbody);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        delete b;
        return DFV_ERR_CUDA;
    }
    *out = b;
    return DFV_OK;
}

dfv_status dfv_batch_add_material(dfv_batch *b, int kind, const dfv_material_params *m)
{
    if (!b) return DFV_ERR_ARG;
    if (!m || b->nmat >= b->nmat_opt) return bfail(b, DFV_ERR_ARG, "dfv_batch_add_material: too many materials");
    if (kind != DFV_MAT_IDEAL && kind != DFV_MAT_STIFFENED)
        return bfail(b, DFV_ERR_UNSUPPORTED, "dfv_batch_add_material: batches are fluid-only");
    if (!(m->gamma > 1.0)) return bfail(b, DFV_ERR_ARG, "dfv_batch_add_material: gamma <= 1");
    for (auto &I : b->hinst) {
        dfv::MatP &p = I.g.mat[b->nmat];
        p.kind = kind;
        p.gamma = m->gamma;
        p.pinf = m->pinf;
        p.rho0 = m->rho0;
        p.sigY = m->sigma_y;
    }
    b->nmat++;
    b->uploaded = false;
    return DFV_OK;
}

}  // extern "C"

namespace {

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

// The copy and conversion of one instance's fields, issued on the batch's
// stream (the staging buffer is reused in stream order: no synchronisation
// between instances is needed).  Page-locked host fields are converted in
// place, without the staging copy.
dfv_status set_one(dfv_batch *b, int i, const double *prim, int on_device)
{
    const GridP &g = b->hinst[i].g;
    const int w = b->precision == DFV_FP32 ? 4 : 8;
    const size_t bytes = sizeof(double) * b->ops->nvar * (size_t)g.ncell;
    const double *src = on_device ? prim : static_cast<const double *>(mapped_host(prim));
    if (!src) {
        B_CU(b, cudaMemcpyAsync(b->staging, prim, bytes, cudaMemcpyHostToDevice, b->stream), "set_fields copy");
        src = b->staging;
    }
    B_CU(b, b->ops->prim_to_cons(g, src, g.ncell, (char *)b->U + (size_t)w * b->hinst[i].off, b->stream),
         "prim_to_cons");
    b->launches++;
    // new r: the instance's rigid box is unknown until its next stage 3
    B_CU(b, cudaMemsetAsync(&b->d_ctl[i].rbox_valid, 0, sizeof(int), b->stream), "set_fields box");
    b->fields_set[i] = 1;
    b->dt_valid = false;
    return DFV_OK;
}

dfv_status get_one(dfv_batch *b, int i, double *outp, int which, int on_device)
{
    const GridP &g = b->hinst[i].g;
    const int w = b->precision == DFV_FP32 ? 4 : 8;
    const void *Ui = (const char *)b->U + (size_t)w * b->hinst[i].off;
    double *dst = on_device ? outp : static_cast<double *>(const_cast<void *>(mapped_host(outp)));
    const bool staged = dst == nullptr;
    if (staged) dst = b->staging;
    if (which == DFV_FIELDS_PRIMITIVE) {
        B_CU(b, b->ops->cons_to_prim(g, Ui, dst, g.ncell, b->stream), "cons_to_prim");
    } else {
        B_CU(b, b->ops->cons_to_f64(g, Ui, dst, g.ncell, b->ops->nvar, b->stream), "cons_to_f64");
    }
    b->launches++;
    if (staged) {
        const size_t bytes = sizeof(double) * b->ops->nvar * (size_t)g.ncell;
        B_CU(b, cudaMemcpyAsync(outp, b->staging, bytes, cudaMemcpyDeviceToHost, b->stream), "get_fields copy");
    }
    return DFV_OK;
}

dfv_status set_ready(dfv_batch *b)
{
    if (b->nmat != b->nmat_opt) return bfail(b, DFV_ERR_ARG, "dfv_batch_set_fields: materials missing");
    return upload(b);
}

}  // namespace

extern "C" {

dfv_status dfv_batch_set_fields(dfv_batch *b, int i, const double *prim, int on_device)
{
    if (!b) return DFV_ERR_ARG;
    if (i < 0 || i >= b->count || !prim) return bfail(b, DFV_ERR_ARG, "dfv_batch_set_fields: bad arguments");
    dfv_status s = set_ready(b);
    if (s == DFV_OK) s = set_one(b, i, prim, on_device);
    if (s != DFV_OK) return s;
    if (!on_device) B_CU(b, cudaStreamSynchronize(b->stream), "set_fields sync");
    return DFV_OK;
}

dfv_status dfv_batch_set_all_fields(dfv_batch *b, const double *const *prim, int on_device)
{
    if (!b) return DFV_ERR_ARG;
    if (!prim) return bfail(b, DFV_ERR_ARG, "dfv_batch_set_all_fields: bad arguments");
    for (int i = 0; i < b->count; i++)
        if (!prim[i]) return bfail(b, DFV_ERR_ARG, "dfv_batch_set_all_fields: bad arguments");
    dfv_status s = set_ready(b);
    for (int i = 0; i < b->count && s == DFV_OK; i++) s = set_one(b, i, prim[i], on_device);
    if (s != DFV_OK) return s;
    if (!on_device) B_CU(b, cudaStreamSynchronize(b->stream), "set_all_fields sync");
    return DFV_OK;
}

dfv_status dfv_batch_get_fields(dfv_batch *b, int i, double *outp, int which, int on_device)
{
    if (!b) return DFV_ERR_ARG;
    if (i < 0 || i >= b->count || !outp || !b->fields_set[i])
        return bfail(b, DFV_ERR_ARG, "dfv_batch_get_fields: bad arguments");
    dfv_status s = get_one(b, i, outp, which, on_device);
    if (s != DFV_OK) return s;
    if (!on_device) B_CU(b, cudaStreamSynchronize(b->stream), "get_fields sync");
    return DFV_OK;
}

dfv_status dfv_batch_get_all_fields(dfv_batch *b, double *const *out, int which, int on_device)
{
    if (!b) return DFV_ERR_ARG;
    if (!out) return bfail(b, DFV_ERR_ARG, "dfv_batch_get_all_fields: bad arguments");
    for (int i = 0; i < b->count; i++)
        if (!out[i] || !b->fields_set[i]) return bfail(b, DFV_ERR_ARG, "dfv_batch_get_all_fields: bad arguments");
    for (int i = 0; i < b->count; i++) {
        dfv_status s = get_one(b, i, out[i], which, on_device);
        if (s != DFV_OK) return s;
    }
    if (!on_device) B_CU(b, cudaStreamSynchronize(b->stream), "get_all_fields sync");
    return DFV_OK;
}

dfv_status dfv_batch_run(dfv_batch *b, int steps, double cfl, double t_end)
{
    if (!b) return DFV_ERR_ARG;
    if (steps < 0 || !(cfl > 0.0)) return bfail(b, DFV_ERR_ARG, "dfv_batch_run: bad arguments");
    for (int i = 0; i < b->count; i++)
        if (!b->fields_set[i]) return bfail(b, DFV_ERR_ARG, "dfv_batch_run: fields of an instance not set");
    dfv_status s = upload(b);
    if (s != DFV_OK) return s;
    if ((s = ensure_dt(b, cfl, t_end)) != DFV_OK) return s;
    const bool use_graph = b->stream != nullptr && steps > 0 && !b->prof;
    if (use_graph && !b->graph_ready) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaGraph_t graph = nullptr;
        B_CU(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        const long long before = b->launches;
        dfv_status cs = batch_step(b, true);
        cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        b->graph_launches = b->launches - before;   // kernels of one replay
        b->launches = before;
        if (cs != DFV_OK) return cs;
        if (e != cudaSuccess) return bfail(b, DFV_ERR_CUDA, "dfv_batch_run: end capture failed");
        e = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bfail(b, DFV_ERR_CUDA, "dfv_batch_run: graph instantiate failed");
        b->graph_ready = true;
    }
    for (int k = 0; k < steps; k++) {
        if (use_graph) {
            B_CU(b, cudaGraphLaunch(b->graph, b->stream), "graph launch");
            b->launches += b->graph_launches;
        } else if ((s = batch_step(b, false)) != DFV_OK) {
            return s;
        }
    }
    return DFV_OK;
}

dfv_status dfv_batch_autotune(dfv_batch *b, int trial_steps, double cfl, int choice_out[2])
{
    if (!b) return DFV_ERR_ARG;
    if (trial_steps < 1 || !(cfl > 0.0)) return bfail(b, DFV_ERR_ARG, "dfv_batch_autotune: bad arguments");
    for (int i = 0; i < b->count; i++)
        if (!b->fields_set[i]) return bfail(b, DFV_ERR_ARG, "dfv_batch_autotune: fields of an instance not set");
    dfv_status s = upload(b);
    if (s != DFV_OK) return s;
    if ((s = ensure_dt(b, cfl, b->run_tend > 0 ? b->run_tend : 0.0)) != DFV_OK) return s;
    const int w = b->precision == DFV_FP32 ? 4 : 8;
    const size_t ubytes = (size_t)w * b->plan.elems;
    B_CU(b, cudaMemcpyAsync(b->Ubak, b->U, ubytes, cudaMemcpyDeviceToDevice, b->stream), "backup");
    B_CU(b, cudaMemcpyAsync(b->d_ctl_bak, b->d_ctl, sizeof(Ctl) * b->count, cudaMemcpyDeviceToDevice, b->stream),
         "backup ctl");
    cudaEvent_t e0 = take_ev(b), e1 = take_ev(b);
    float best = 1e30f;
    int best_c = b->ctas_per_sm, best_s = b->schedule;
    const bool prof = b->prof;
    b->prof = false;
    const int cmax = b->gas ? b->gas_max_ctas : b->max_ctas;
    for (int sched = 0; sched < 3; sched++)
        for (int c = 0; c <= cmax; c++) {
            b->schedule = sched;
            b->ctas_per_sm = c;
            batch_step(b, false);   // warm
            B_CU(b, cudaEventRecord(e0, b->stream), "event");
            for (int k = 0; k < trial_steps; k++)
                if ((s = batch_step(b, false)) != DFV_OK) return s;
            B_CU(b, cudaEventRecord(e1, b->stream), "event");
            B_CU(b, cudaEventSynchronize(e1), "event sync");
            float ms = 0.f;
            B_CU(b, cudaEventElapsedTime(&ms, e0, e1), "elapsed");
            if (ms < best) {
                best = ms;
                best_c = c;
                best_s = sched;
            }
            B_CU(b, cudaMemcpyAsync(b->U, b->Ubak, ubytes, cudaMemcpyDeviceToDevice, b->stream), "restore");
            B_CU(b, cudaMemcpyAsync(b->d_ctl, b->d_ctl_bak, sizeof(Ctl) * b->count, cudaMemcpyDeviceToDevice,
                                    b->stream),
                 "restore ctl");
        }
    b->ev_free.push_back(e0);
    b->ev_free.push_back(e1);
    b->prof = prof;
    b->schedule = best_s;
    b->ctas_per_sm = best_c;
    b->graph_ready = false;
    B_CU(b, cudaStreamSynchronize(b->stream), "autotune sync");
    if (choice_out) {
        choice_out[0] = best_c;
        choice_out[1] = best_s;
    }
    return DFV_OK;
}

dfv_status dfv_batch_set_schedule(dfv_batch *b, int ctas_per_sm, int schedule)
{
    if (!b) return DFV_ERR_ARG;
    if (ctas_per_sm < 0 || schedule < 0 || schedule > 2)
        return bfail(b, DFV_ERR_ARG, "dfv_batch_set_schedule: bad arguments");
    b->ctas_per_sm = std::min(ctas_per_sm, b->gas ? b->gas_max_ctas : b->max_ctas);
    b->schedule = schedule;
    b->graph_ready = false;
    return DFV_OK;
}

dfv_status dfv_batch_get_time(dfv_batch *b, int i, double *t, double *dt)
{
    if (!b) return DFV_ERR_ARG;
    if (i < 0 || i >= b->count) return bfail(b, DFV_ERR_ARG, "dfv_batch_get_time: bad index");
    Ctl h;
    B_CU(b, cudaMemcpyAsync(&h, b->d_ctl + i, sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream), "read ctl");
    B_CU(b, cudaStreamSynchronize(b->stream), "read ctl sync");
    if (t) *t = h.t;
    if (dt) *dt = h.dt;
    if (h.err) return bfail(b, DFV_ERR_NONPHYSICAL, "dfv_batch: non-physical state in this instance");
    return DFV_OK;
}

dfv_status dfv_batch_profile(dfv_batch *b, int enable, double ms_out[4], long long *steps_out)
{
    if (!b) return DFV_ERR_ARG;
    double ms[4] = {0, 0, 0, 0};
    long long n = 0;
    if (!b->ev_steps.empty()) {
        B_CU(b, cudaStreamSynchronize(b->stream), "profile sync");
        for (auto &ev : b->ev_steps) {
            for (int k = 0; k < 4; k++) {
                float t = 0.f;
                B_CU(b, cudaEventElapsedTime(&t, ev[k], ev[k + 1]), "elapsed");
                ms[k] += t;
            }
            for (auto x : ev) b->ev_free.push_back(x);
            n++;
        }
        b->ev_steps.clear();
    }
    if (ms_out)
        for (int k = 0; k < 4; k++) ms_out[k] = ms[k];
    if (steps_out) *steps_out = n;
    b->prof = enable != 0;
    return DFV_OK;
}

dfv_status dfv_batch_launch_count(const dfv_batch *b, long long *count)
{
    if (!b || !count) return DFV_ERR_ARG;
    *count = b->launches;
    return DFV_OK;
}

dfv_status dfv_batch_destroy(dfv_batch *b)
{
    if (!b) return DFV_ERR_ARG;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (auto &ev : b->ev_steps)
        for (auto x : ev) b->ev_free.push_back(x);
    for (auto x : b->ev_free) cudaEventDestroy(x);
    delete b;
    return DFV_OK;
}

const char *dfv_batch_last_error(const dfv_batch *b)
{
    if (!b) return "dfv_batch: null batch";
    return b->err.c_str();
}

}  // extern "C"
