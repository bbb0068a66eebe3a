// dfv_noalloc.cu -- dfv_compute_dt_noalloc: the CFL time step of a conserved
// state that the caller already holds on the device, computed without any
// device allocation, for callers that cannot call cudaMalloc (a solver
// embedded in a host code whose device memory is owned and pooled elsewhere,
// or one that must not allocate while other work runs on the device).
//
// It runs the library's CFL reduction kernel (one block of 256 threads per 256
// cells, one partial maximum per block) followed by the one-block finalize,
// with the per-block partials and the small control block in a file-scope
// device array instead of the grid workspace.  The array has a fixed maximum
// size: DFV_NOALLOC_MAX_CELLS cells (2 MiB of partials).  Every GPU that loads
// the library holds the array until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/dfvrb.h"
#include "dfv_kernels.cuh"
#include "dfv_ops.h"

namespace {

constexpr long long kMaxBlocks = DFV_NOALLOC_MAX_CELLS / 256;
constexpr size_t kCtlDoubles = 32;   // room for the control block (sizeof(Ctl) <= 256 bytes)
static_assert(sizeof(dfv::Ctl) <= kCtlDoubles * sizeof(double), "control block does not fit its slot");

// Scratch shared by every call on a device: [control block][4 doubles per block].
static __device__ __align__(256) double g_noalloc_scratch[kCtlDoubles + 4 * kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up once per
// device: the host-side name of a __device__ array is not a device address).
cudaError_t scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

__global__ void k_noalloc_init_ctl(dfv::Ctl *c, double v0, double v1, double v2)
{
    memset(c, 0, sizeof(dfv::Ctl));
    dfv::ctl_box_reset(c);
    c->v[0] = v0;
    c->v[1] = v1;
    c->v[2] = v2;
    dfv::ctl_sync_v(c);
}

}  // namespace

extern "C" dfv_status dfv_compute_dt_noalloc(int dim, const int n[3], const double lo[3], const double hi[3],
                                             int precision, const dfv_options *opt, const int kinds[],
                                             const dfv_material_params params[], const void *cons,
                                             long long plane_pitch, const double v_body[3], double cfl,
                                             void *stream, double *dt_out)
{
    if (!n || !lo || !hi || !opt || !kinds || !params || !cons || !dt_out || !(cfl > 0.0)) return DFV_ERR_ARG;
    if (dim < 1 || dim > 3 || opt->nmat < 1 || opt->nmat > 3) return DFV_ERR_ARG;
    if (precision != DFV_FP64 && precision != DFV_FP32) return DFV_ERR_ARG;
    const dfv::Ops *ops = dfv::ops_for(precision == DFV_FP32 ? 1 : 0, dim, opt->nmat,
                                       opt->solid == 2 ? 2 : (opt->solid ? 1 : 0));
    if (!ops) return DFV_ERR_UNSUPPORTED;

    dfv::GridP p;
    memset(&p, 0, sizeof(p));
    p.dim = dim;
    p.ncell = 1;
    p.dxmin = 1e300;
    p.dV = 1.0;
    for (int d = 0; d < 3; d++) {
        const int nd = d < dim ? n[d] : 1;
        if (nd < 1 || (d < dim && !(hi[d] > lo[d]))) return DFV_ERR_ARG;
        p.n[d] = nd;
        p.lo[d] = d < dim ? lo[d] : 0.0;
        p.dx[d] = d < dim ? (hi[d] - lo[d]) / nd : 1.0;
        p.inv_dx[d] = 1.0 / p.dx[d];
        p.ncell *= nd;
        if (d < dim) {
            p.dxmin = std::fmin(p.dxmin, p.dx[d]);
            p.dV *= p.dx[d];
        }
    }
    if (p.ncell > DFV_NOALLOC_MAX_CELLS) return DFV_ERR_TOO_LARGE;
    if (plane_pitch < p.ncell) return DFV_ERR_ARG;
    p.pitch = plane_pitch;
    dfv::apply_options(p, opt->use_thinc, opt->thinc_beta, opt->hllc_lm, opt->seed_variant,
                       opt->normal_method, opt->probe_mode);
    for (int l = 0; l < opt->nmat; l++) {
        const dfv_material_params &q = params[l];
        if (dfv::material_problem(kinds[l], q.gamma, q.rho0, q.Gamma0, q.alpha, q.jc_c1, q.jc_c2, q.jc_n, q.jc_tmelt,
                                  q.jc_cv))
            return DFV_ERR_ARG;
        dfv::set_material(p.mat[l], kinds[l], q);
    }
    dfv::finish_params(p);

    double *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return DFV_ERR_CUDA;
    dfv::Ctl *ctl = reinterpret_cast<dfv::Ctl *>(scratch);
    double *partials = scratch + kCtlDoubles;
    const long long nblocks = (p.ncell + 255) / 256;
    cudaStream_t st = (cudaStream_t)stream;
    const double v0 = v_body && dim > 0 ? v_body[0] : 0.0, v1 = v_body && dim > 1 ? v_body[1] : 0.0,
                 v2 = v_body && dim > 2 ? v_body[2] : 0.0;
    k_noalloc_init_ctl<<<1, 1, 0, st>>>(ctl, v0, v1, v2);
    if (cudaGetLastError() != cudaSuccess) return DFV_ERR_CUDA;
    if (ops->cfl(p, cons, partials, (int)nblocks, st) != cudaSuccess) return DFV_ERR_CUDA;
    dfv::k_finalize<<<1, 1024, 0, st>>>(ctl, partials, nblocks, 0, 1, dim, p.dx[0], p.dx[1], p.dx[2]);
    if (cudaGetLastError() != cudaSuccess) return DFV_ERR_CUDA;
    double smax = 0.0;
    if (cudaMemcpyAsync(&smax, &ctl->smax, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return DFV_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DFV_ERR_CUDA;
    if (!(smax > 0.0) || std::isinf(smax)) return DFV_ERR_NONPHYSICAL;
    *dt_out = cfl / smax;
    return DFV_OK;
}
