// dfv_device.cuh -- device-side physics of the diffuse rigid-body
// finite-volume update (arXiv:2111.11806), written for sm_103a.
//
// Everything here is a __device__ function templated on the compute type T
// (double for the plain FP64 form, float for the FP32 bulk form) and on the
// system shape (dimension, number of materials, solid or fluid), so that every
// index into the per-cell state is a compile-time constant and lives in
// registers.  The stretch-tensor logarithm and the plastic return are always
// evaluated in FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace dfv {

// ------------------------------------------------------------------ params

struct MatP {
    int kind;                 // 0 ideal, 1 stiffened, 2 Romenskii
    double gamma, pinf;
    double rho0, K0, G0, alpha, beta, Gamma0;
    double sigY;
    int jc;                   // 1: Johnson-Cook flow stress instead of sigY
    double jc_c1, jc_c2, jc_c3, jc_n, jc_m, jc_tmelt, jc_cv;
};

// Material and grid constants in the compute precision, derived on the host
// (finish_params) so that the FP32 form does no double-precision arithmetic
// or conversion in its face and cell loops.
template <class T>
struct MatC {
    int kind;
    T Gam;          // Grueneisen coefficient (gamma - 1 for the gases)
    T invGam;       // 1 / Gam
    T pref0;        // constant p_ref of the gases (-gamma p_inf, 0)
    T rho0, K0, G0, alpha, beta, sigY;
    int has_rho0;
};

template <class T>
struct GridC {
    T lo[3], dx[3], inv_dx[3];
    T dxmin, dV;
    T beta, cosh_b, sinh_b, tanh_b;   // THINC constants
    T inv_sinh_b;
    T phi_guard;
};

struct GridP {
    int dim;
    int n[3];
    int periodic[3];
    double lo[3], dx[3], inv_dx[3];
    long long ncell, pitch;   // cells, elements between planes
    double dV, dxmin;
    MatP mat[3];
    int use_thinc;
    int hllc_lm;        // 1: low-Mach HLLC-LM dissipation in the star regions
    int seed_variant;   // 0: reflected state (Sec. 3.2), 1: Riemann-problem star state
    int normal_method;  // 0: Youngs, 1: ELVIRA (2-D) (Sec. 3.3)
    int probe_mode;     // 0: stepped probe 1.0..4.0 dx, 1: fixed 1.5 dx (Sec. 3.2)
    int wall[3][2];     // reflective wall on the low / high side of direction d
    double beta, cosh_b, sinh_b, tanh_b;   // THINC constants
    double phi_guard;
    MatC<double> mc_d[3];
    MatC<float> mc_f[3];
    GridC<double> gc_d;
    GridC<float> gc_f;
    int any_jc;         // some material has a Johnson-Cook flow stress
};

template <class T>
__host__ inline void fill_consts(const GridP &g, MatC<T> *mc, GridC<T> &gc)
{
    for (int l = 0; l < 3; l++) {
        const MatP &m = g.mat[l];
        mc[l].kind = m.kind;
        mc[l].Gam = (T)(m.kind == 2 ? m.Gamma0 : m.gamma - 1.0);
        mc[l].invGam = (T)(1.0 / (m.kind == 2 ? m.Gamma0 : m.gamma - 1.0));
        mc[l].pref0 = (m.kind == 1) ? (T)(-m.gamma * m.pinf) : T(0);
        mc[l].rho0 = (T)m.rho0;
        mc[l].K0 = (T)m.K0;
        mc[l].G0 = (T)m.G0;
        mc[l].alpha = (T)m.alpha;
        mc[l].beta = (T)m.beta;
        mc[l].sigY = (T)m.sigY;
        mc[l].has_rho0 = m.rho0 > 0.0;
    }
    for (int d = 0; d < 3; d++) {
        gc.lo[d] = (T)g.lo[d];
        gc.dx[d] = (T)g.dx[d];
        gc.inv_dx[d] = (T)g.inv_dx[d];
    }
    gc.dxmin = (T)g.dxmin;
    gc.dV = (T)g.dV;
    gc.beta = (T)g.beta;
    gc.cosh_b = (T)g.cosh_b;
    gc.sinh_b = (T)g.sinh_b;
    gc.tanh_b = (T)g.tanh_b;
    gc.inv_sinh_b = (T)(1.0 / g.sinh_b);
    gc.phi_guard = (T)g.phi_guard;
}

// The scheme options of a grid: THINC on/off and its steepness (default 1.6),
// the HLLC-LM flux, the seeding variant, the normal method and the probe.
__host__ inline void apply_options(GridP &g, int use_thinc, double thinc_beta, int hllc_lm, int seed_variant,
                                   int normal_method, int probe_mode)
{
    g.normal_method = normal_method == 1 ? 1 : 0;
    g.probe_mode = probe_mode == 1 ? 1 : 0;
    g.use_thinc = use_thinc ? 1 : 0;
    g.beta = thinc_beta > 0.0 ? thinc_beta : 1.6;
    g.cosh_b = std::cosh(g.beta);
    g.sinh_b = std::sinh(g.beta);
    g.tanh_b = std::tanh(g.beta);
    g.hllc_lm = hllc_lm ? 1 : 0;
    g.seed_variant = seed_variant == 1 ? 1 : 0;
    g.phi_guard = 1e-14;
}

// The checks of one material's parameters (kind 0 ideal, 1 stiffened, 2
// Romenskii), shared by every entry point that takes materials: nullptr when
// valid, else what is wrong.  Gases need gamma > 1 (Gamma = gamma - 1 > 0);
// the Romenskii solid needs rho0 > 0, Gamma0 > 0 and alpha != 0 (Sec. 2.1.3,
// eq:Romenskii divides by both).
__host__ inline const char *material_problem(int kind, double gamma, double rho0, double Gamma0, double alpha,
                                             double jc_c1 = 0.0, double jc_c2 = 0.0, double jc_n = 0.0,
                                             double jc_tmelt = 0.0, double jc_cv = 0.0)
{
    if (kind < 0 || kind > 2) return "bad material kind";
    if (kind != 2 && !(gamma > 1.0)) return "gamma <= 1";
    if (kind == 2 && !(rho0 > 0.0 && Gamma0 > 0.0 && alpha != 0.0)) return "bad Romenskii parameters";
    if ((jc_c1 > 0.0 || jc_c2 > 0.0) && !(jc_tmelt > 298.0 && jc_cv > 0.0 && jc_n >= 0.0 && jc_c1 >= 0.0 &&
                                         jc_c2 >= 0.0))
        return "bad Johnson-Cook parameters";
    return nullptr;
}

// Copy the caller's material parameters (dfvrb.h) into a MatP.
template <class P>
__host__ inline void set_material(MatP &m, int kind, const P &p)
{
    m.kind = kind;
    m.gamma = p.gamma;
    m.pinf = p.pinf;
    m.rho0 = p.rho0;
    m.K0 = p.K0;
    m.G0 = p.G0;
    m.alpha = p.alpha;
    m.beta = p.beta;
    m.Gamma0 = p.Gamma0;
    m.sigY = p.sigma_y;
    m.jc = (p.jc_c1 > 0.0 || p.jc_c2 > 0.0) ? 1 : 0;
    m.jc_c1 = p.jc_c1;
    m.jc_c2 = p.jc_c2;
    m.jc_c3 = p.jc_c3;
    m.jc_n = p.jc_n;
    m.jc_m = p.jc_m;
    m.jc_tmelt = p.jc_tmelt;
    m.jc_cv = p.jc_cv;
}

// Derive the per-precision constants from the double parameters; call after
// every change of the grid or of a material.
__host__ inline void finish_params(GridP &g)
{
    fill_consts<double>(g, g.mc_d, g.gc_d);
    fill_consts<float>(g, g.mc_f, g.gc_f);
    g.any_jc = 0;
    for (int l = 0; l < 3; l++) g.any_jc |= g.mat[l].jc;
}

template <class T>
__device__ __forceinline__ const MatC<T> &matc(const GridP &g, int l);
template <>
__device__ __forceinline__ const MatC<double> &matc<double>(const GridP &g, int l) { return g.mc_d[l]; }
template <>
__device__ __forceinline__ const MatC<float> &matc<float>(const GridP &g, int l) { return g.mc_f[l]; }

template <class T>
__device__ __forceinline__ const GridC<T> &gridc(const GridP &g);
template <>
__device__ __forceinline__ const GridC<double> &gridc<double>(const GridP &g) { return g.gc_d; }
template <>
__device__ __forceinline__ const GridC<float> &gridc<float>(const GridP &g) { return g.gc_f; }

// Device-resident control block: time step, time, body state and the error
// word.  Kernels read dt and the body velocity from here so that a whole step
// can be replayed from a CUDA graph without host involvement.
struct Ctl {
    double dt, t, t_end, cfl;
    double smax;              // max_cells sum_d (|u_d|+c)/dx_d of the last reduction
    unsigned long long smax_acc;  // running maximum of the tiles of a stage-3 launch, as
                                  // the bits of a non-negative double (0 between launches)
    double force[3];
    double v[3];
    double x[3];
    double mass;
    int dynamic;
    int auto_dt;              // 1: the finalize kernel sets the next dt from cfl
    unsigned int err;         // bit 0: rho<=0/NaN in an update, bit 1: c^2<=0/NaN
    int steps;
    unsigned int ticket;      // blocks of the last stage that have written their partials
    float dtf, vf[3];         // dt and v in single precision, kept equal to (float)dt, (float)v
    int rbox_valid;           // 1: rbox bounds every cell with r > 0.5 of the stored state
    int rbox[6];              // inclusive cell-index box lo x, y, z, hi x, y, z (empty: lo > hi)
    int rnext[6];             // the same for the state stage 3 produces (atomic min / max)
};

// Empty box for rnext, and a fresh control block's fields that are not 0.
__host__ __device__ inline void ctl_box_reset(Ctl *c)
{
    for (int d = 0; d < 3; d++) {
        c->rnext[d] = 0x7fffffff;
        c->rnext[3 + d] = -1;
    }
}

// dt and body velocity in the compute precision
template <class T>
__device__ __forceinline__ T ctl_dt(const Ctl *c);
template <>
__device__ __forceinline__ double ctl_dt<double>(const Ctl *c) { return c->dt; }
template <>
__device__ __forceinline__ float ctl_dt<float>(const Ctl *c) { return c->dtf; }
template <class T>
__device__ __forceinline__ T ctl_v(const Ctl *c, int d);
template <>
__device__ __forceinline__ double ctl_v<double>(const Ctl *c, int d) { return c->v[d]; }
template <>
__device__ __forceinline__ float ctl_v<float>(const Ctl *c, int d) { return c->vf[d]; }
// the same read from L2 (bypassing a possibly stale L1 line)
template <class T>
__device__ __forceinline__ T ctl_v_cg(const Ctl *c, int d);
template <>
__device__ __forceinline__ double ctl_v_cg<double>(const Ctl *c, int d) { return __ldcg(&c->v[d]); }
template <>
__device__ __forceinline__ float ctl_v_cg<float>(const Ctl *c, int d) { return __ldcg(&c->vf[d]); }

__device__ __forceinline__ void ctl_set_dt(Ctl *c, double dt)
{
    c->dt = dt;
    c->dtf = (float)dt;
}
__device__ __forceinline__ void ctl_sync_v(Ctl *c)
{
    for (int d = 0; d < 3; d++) c->vf[d] = (float)c->v[d];
}

enum { ERR_STATE = 1u, ERR_SOUND = 2u, ERR_TIMEOUT = 4u };   // ERR_TIMEOUT: a bounded device wait ran out

// Programmatic dependent launch: the kernels of a step are launched with
// launch_pdl, so a kernel's CTAs may be scheduled while the previous kernel
// on the stream is still finishing.  Each such kernel first waits for its
// predecessor to complete with its memory visible (griddepcontrol.wait; a
// no-op without a programmatic predecessor), then lets its own successor be
// scheduled (griddepcontrol.launch_dependents): the successor's CTAs take SM
// slots only after every CTA of this grid has started, and they wait in turn.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The two halves, for a kernel that does work not depending on its
// predecessor before it waits.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
__host__ inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                       cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ------------------------------------------------------------------ layout

template <int DIM, int NMAT, int SOLID>
struct Lay {
    static constexpr int NV = SOLID ? (DIM == 1 ? 3 : (DIM == 2 ? 5 : 9)) : 0;
    static constexpr int IPHI = 0;
    static constexpr int IAR = NMAT - 1;
    static constexpr int IMOM = 2 * NMAT - 1;
    static constexpr int IE = IMOM + DIM;
    static constexpr int IV = IE + 1;
    static constexpr int IR = IV + NV;
    static constexpr int NH = SOLID == 2 ? NMAT : 0;   // plastic-strain planes (phi rho eps)_l
    static constexpr int IH = IR + 1;
    static constexpr int NVAR = IR + 1 + NH;
    static constexpr int NB = SOLID ? DIM : 0;   // V*_{d b} entries kept per face
    static constexpr int NF = NVAR + 1 + NB;     // per-face record: fluxes, u*_d, V*_{d.}
};

// stored stretch component c -> tensor indices (a, b)
__host__ __device__ constexpr int v_row(int dim, int c)
{
    return dim == 1 ? c : (dim == 2 ? (c < 2 ? 0 : (c < 4 ? 1 : 2)) : c / 3);
}
__host__ __device__ constexpr int v_col(int dim, int c)
{
    return dim == 1 ? c : (dim == 2 ? (c == 0 ? 0 : (c == 1 ? 1 : (c == 2 ? 0 : (c == 3 ? 1 : 2)))) : c % 3);
}

// ------------------------------------------------------------------ math

__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_sin(double x) { return sin(x); }
// products and sums rounded one by one (never fused into an FMA)
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float m_sin(float x) { return sinf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_pow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float m_pow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double m_abs(double x) { return fabs(x); }
__device__ __forceinline__ float m_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double m_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float m_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double m_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float m_max(float a, float b) { return fmaxf(a, b); }

__device__ __forceinline__ int map_idx(int i, int n, int periodic)
{
    if (periodic) {
        int m = i % n;
        return m < 0 ? m + n : m;
    }
    return i < 0 ? 0 : (i > n - 1 ? n - 1 : i);
}

// Halo index of direction d with reflective walls: a wall side mirrors (cell
// -1-i below, 2n-1-i above, clamped into the grid when n < 3); *flip is set
// when the cell is a mirror image.
__device__ __forceinline__ int halo_idx(const GridP &g, int d, int i, bool *flip)
{
    const int n = g.n[d];
    if ((i < 0 && g.wall[d][0]) || (i > n - 1 && g.wall[d][1])) {
        *flip = true;
        const int m = i < 0 ? -1 - i : 2 * n - 1 - i;
        return m < 0 ? 0 : (m > n - 1 ? n - 1 : m);
    }
    return map_idx(i, n, g.periodic[d]);
}

// ------------------------------------------------------ material closure

template <class T>
struct Ref {
    T Gam, eref, pref, deref, dpref, G;
};

// Mie-Grueneisen reference curves p = p_ref + rho Gamma (e - e_ref) of one
// material (Sec. 2.1.2-2.1.3): ideal gas (p_ref = e_ref = 0), stiffened gas
// (e_ref = 0, p_ref = -gamma p_inf), Romenskii solid (eq:Romenskii, cold term
// K0/(2 rho alpha^2)(x^alpha - 1)^2 as printed, shear energy G J^2/rho with
// G = G0 x^(beta+1), x = rho/rho0, and p_ref = rho^2 de_ref/drho).
template <class T>
__device__ __forceinline__ Ref<T> mat_ref(const MatC<T> &m, T rho, T J2)
{
    Ref<T> r;
    if (m.kind == 2) {
        const T al = m.alpha, be = m.beta, K0 = m.K0, rho0 = m.rho0;
        const T x = rho / rho0;
        const T xa = m_pow(x, al);
        const T xm1 = xa - T(1);
        const T ec = K0 / (T(2) * rho * al * al) * xm1 * xm1;
        const T pc = -K0 / (T(2) * al * al) * xm1 * xm1 + (K0 / al) * xm1 * xa;
        const T dpc = (K0 / rho0) * (xa / x) * (T(2) * xa - T(1) - xm1 / al);
        const T G = m.G0 * m_pow(x, be + T(1));
        const T ps = be * G * J2;
        r.Gam = m.Gam;
        r.eref = ec + G * J2 / rho;
        r.pref = pc + ps;
        r.deref = (pc + ps) / (rho * rho);
        r.dpref = dpc + be * (be + T(1)) * G * J2 / rho;
        r.G = G;
    } else {
        r.Gam = m.Gam;
        r.eref = T(0);
        r.pref = m.pref0;
        r.deref = T(0);
        r.dpref = T(0);
        r.G = T(0);
    }
    return r;
}

// ------------------------------------------------- stretch tensor (FP64)

// dev(H) = ln V with V^2 = A A^T (Sec. 2.1.2), traceless part, and
// J^2 = |dev H|^2.  2-D: A A^T is block diagonal, so the in-plane 2x2 block is
// diagonalised in closed form through the double angle 2 theta of its
// eigenvectors; 1-D: diagonal.  Also returns the data needed to rebuild a
// tensor with the same eigenvectors (plastic return).
struct Eig2 {
    double d[3];       // deviatoric log-stretches (in-plane 1, 2; out-of-plane)
    double c2, s2;     // cos 2 theta, sin 2 theta of the in-plane eigenvectors
};

template <int DIM>
__device__ __forceinline__ void stretch_log(const double A[3][3], double H[3][3], double &J2, Eig2 &e)
{
    double h0, h1, h2;
    if (DIM == 1) {
        h0 = 0.5 * log(A[0][0] * A[0][0]);
        h1 = 0.5 * log(A[1][1] * A[1][1]);
        h2 = 0.5 * log(A[2][2] * A[2][2]);
        e.c2 = 1.0;
        e.s2 = 0.0;
    } else {
        const double b00 = A[0][0] * A[0][0] + A[0][1] * A[0][1];
        const double b01 = A[0][0] * A[1][0] + A[0][1] * A[1][1];
        const double b11 = A[1][0] * A[1][0] + A[1][1] * A[1][1];
        const double b22 = A[2][2] * A[2][2];
        const double mid = 0.5 * (b00 + b11), half = 0.5 * (b00 - b11);
        const double rad = sqrt(half * half + b01 * b01);
        h0 = 0.5 * log(mid + rad);
        h1 = 0.5 * log(mid - rad);
        h2 = 0.5 * log(b22);
        e.c2 = rad > 0.0 ? half / rad : 1.0;
        e.s2 = rad > 0.0 ? b01 / rad : 0.0;
    }
    const double hm = (h0 + h1 + h2) * (1.0 / 3.0);
    e.d[0] = h0 - hm;
    e.d[1] = h1 - hm;
    e.d[2] = h2 - hm;
    J2 = e.d[0] * e.d[0] + e.d[1] * e.d[1] + e.d[2] * e.d[2];
    const double av = 0.5 * (e.d[0] + e.d[1]), df = 0.5 * (e.d[0] - e.d[1]);
    H[0][0] = av + df * e.c2;
    H[1][1] = av - df * e.c2;
    H[0][1] = H[1][0] = df * e.s2;
    H[2][2] = e.d[2];
    H[0][2] = H[2][0] = H[1][2] = H[2][1] = 0.0;
}

// The same in the compute precision T, for the closures (J^2 and dev H at
// every face side and cell): the FP32 form keeps FP64 for the plastic
// update's decomposition (plastic_return) only.  For T = double the
// arithmetic is that of stretch_log.
template <class T, int DIM>
__device__ __forceinline__ void stretch_log_ct(const T A[3][3], T H[3][3], T &J2)
{
    T h0, h1, h2, c2, s2;
    if (DIM == 1) {
        h0 = T(0.5) * m_log(A[0][0] * A[0][0]);
        h1 = T(0.5) * m_log(A[1][1] * A[1][1]);
        h2 = T(0.5) * m_log(A[2][2] * A[2][2]);
        c2 = T(1);
        s2 = T(0);
    } else {
        const T b00 = A[0][0] * A[0][0] + A[0][1] * A[0][1];
        const T b01 = A[0][0] * A[1][0] + A[0][1] * A[1][1];
        const T b11 = A[1][0] * A[1][0] + A[1][1] * A[1][1];
        const T b22 = A[2][2] * A[2][2];
        const T mid = T(0.5) * (b00 + b11), half = T(0.5) * (b00 - b11);
        const T rad = m_sqrt(half * half + b01 * b01);
        h0 = T(0.5) * m_log(mid + rad);
        h1 = T(0.5) * m_log(mid - rad);
        h2 = T(0.5) * m_log(b22);
        c2 = rad > T(0) ? half / rad : T(1);
        s2 = rad > T(0) ? b01 / rad : T(0);
    }
    const T hm = (h0 + h1 + h2) * (T(1) / T(3));
    const T d0 = h0 - hm, d1 = h1 - hm, d2 = h2 - hm;
    J2 = d0 * d0 + d1 * d1 + d2 * d2;
    const T av = T(0.5) * (d0 + d1), df = T(0.5) * (d0 - d1);
    H[0][0] = av + df * c2;
    H[1][1] = av - df * c2;
    H[0][1] = H[1][0] = df * s2;
    H[2][2] = d2;
    H[0][2] = H[2][0] = H[1][2] = H[2][1] = T(0);
}

// ------------------------------------------------------------- thermo

// Closure weight of a transported volume fraction: clipped to [0, 1].
template <class T>
__device__ __forceinline__ T phi_clip(T f)
{
    return f < T(0) ? T(0) : (f > T(1) ? T(1) : f);
}

// Phasic density (phi rho)_l / phi_l (Sec. 2.2); a material whose clipped
// fraction is below 1e-6 is absent from the cell and takes its reference
// density rho0 (when one is given) -- the ratio of two round-off-sized numbers
// would otherwise set the pressure through a stiff cold curve.
template <class T>
__device__ __forceinline__ T phasic_density(const GridP &g, int l, T ar, T phc)
{
    const MatC<T> &m = matc<T>(g, l);
    if (phc < T(1e-6) && m.has_rho0) return m.rho0;
    const T guard = gridc<T>(g).phi_guard;
    return ar / (phc > guard ? phc : guard);
}

template <class T, int DIM, int NMAT, int SOLID>
struct State {
    T phi[NMAT], ar[NMAT];
    T rho, u[DIM], p, rhoE, c2, G, sigY;
    T H[DIM][DIM];     // dev(H), in-plane block
    T eps[NMAT];       // equivalent plastic strain (SOLID == 2)
};

template <class T, int DIM, int NMAT, int SOLID>
__device__ __forceinline__ void unpack_A_ct(const T *w, T A[3][3])
{
    using L = Lay<DIM, NMAT, SOLID>;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) A[a][b] = T(0);
#pragma unroll
    for (int c = 0; c < L::NV; c++) A[v_row(DIM, c)][v_col(DIM, c)] = w[L::IV + c];
}

template <class T, int DIM, int NMAT, int SOLID>
__device__ __forceinline__ void unpack_A(const T *w, double A[3][3])
{
    using L = Lay<DIM, NMAT, SOLID>;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) A[a][b] = 0.0;
#pragma unroll
    for (int c = 0; c < L::NV; c++) A[v_row(DIM, c)][v_col(DIM, c)] = (double)w[L::IV + c];
}

// Full state from primitives w (mixture rules of Sec. 2.2): rho = sum phi_l rho_l,
// rho e = sum [ (phi rho)_l e_ref,l + phi_l (p - p_ref,l)/Gamma_l ],
// G = sum(phi_l G_l/Gamma_l)/sum(phi_l/Gamma_l) (sigma_Y with the same weights),
// c^2 = sum(Y_l c_l^2/Gamma_l)/sum(phi_l/Gamma_l) with c_l^2 = a_l^2 + 4/3 G_l/rho_l.
template <class T, int DIM, int NMAT, int SOLID>
__device__ __forceinline__ void state_from_prim_ct(const GridP &g, const T *w, State<T, DIM, NMAT, SOLID> &s)
{
    using L = Lay<DIM, NMAT, SOLID>;
    T fsum = T(0);
#pragma unroll
    for (int l = 0; l < NMAT - 1; l++) {
        s.phi[l] = w[L::IPHI + l];
        fsum += s.phi[l];
    }
    s.phi[NMAT - 1] = T(1) - fsum;
    T rhol[NMAT];
    s.rho = T(0);
#pragma unroll
    for (int l = 0; l < NMAT; l++) {
        s.phi[l] = phi_clip(s.phi[l]);
        rhol[l] = w[L::IAR + l];
        s.ar[l] = s.phi[l] * rhol[l];
        s.rho += s.ar[l];
    }
#pragma unroll
    for (int a = 0; a < DIM; a++) s.u[a] = w[L::IMOM + a];
    s.p = w[L::IE];
#pragma unroll
    for (int l = 0; l < NMAT; l++) s.eps[l] = T(0);
    if constexpr (SOLID == 2) {
#pragma unroll
        for (int l = 0; l < NMAT; l++) s.eps[l] = w[L::IH + l];
    }
    T J2 = T(0);
    if (SOLID) {
        T A[3][3], H[3][3];
        unpack_A_ct<T, DIM, NMAT, SOLID>(w, A);
        stretch_log_ct<T, DIM>(A, H, J2);
#pragma unroll
        for (int a = 0; a < DIM; a++)
#pragma unroll
            for (int b = 0; b < DIM; b++) s.H[a][b] = H[a][b];
    }
    if constexpr (NMAT == 1) {
        // single material: the mixture rules reduce to the material's own closure
        const MatC<T> &m = matc<T>(g, 0);
        const Ref<T> r = mat_ref<T>(m, rhol[0], J2);
        const T irl = T(1) / rhol[0];
        T ke = T(0);
#pragma unroll
        for (int a = 0; a < DIM; a++) ke += T(0.5) * s.rho * s.u[a] * s.u[a];
        s.rhoE = s.ar[0] * r.eref + (s.p - r.pref) * m.invGam + ke;
        s.G = r.G;
        s.sigY = m.sigY;
        s.c2 = (r.Gam * s.p + (s.p - r.pref)) * irl + r.dpref - r.Gam * rhol[0] * r.deref + T(4) / T(3) * r.G * irl;
        return;
    }
    T rhoe = T(0), den = T(0), Gn = T(0), Sn = T(0), Yn = T(0);
#pragma unroll
    for (int l = 0; l < NMAT; l++) {
        const MatC<T> &m = matc<T>(g, l);
        const Ref<T> r = mat_ref<T>(m, rhol[l], J2);
        const T iG = m.invGam;
        const T irl = T(1) / rhol[l];
        if (s.ar[l] != T(0)) rhoe += s.ar[l] * r.eref;
        rhoe += s.phi[l] * (s.p - r.pref) * iG;
        den += s.phi[l] * iG;
        Gn += s.phi[l] * r.G * iG;
        Sn += s.phi[l] * m.sigY * iG;
        const T a2 = (r.Gam * s.p + (s.p - r.pref)) * irl + r.dpref - r.Gam * rhol[l] * r.deref;
        const T c2l = a2 + T(4) / T(3) * r.G * irl;
        if (s.ar[l] != T(0)) Yn += s.ar[l] * c2l * iG;
    }
    T ke = T(0);
#pragma unroll
    for (int a = 0; a < DIM; a++) ke += T(0.5) * s.rho * s.u[a] * s.u[a];
    const T iden = T(1) / den;
    s.rhoE = rhoe + ke;
    s.G = Gn * iden;
    s.sigY = Sn * iden;
    s.c2 = Yn / s.rho * iden;
}

// The FP32 form's precision rule: the closure of a mixed cell -- at least two
// materials present (fraction >= 1e-6) -- in which another material's fraction
// is below 1e-6 runs in FP64.  A material below 1e-6 is absent (it takes its
// reference density, reading of Sec. 2.2), so with two materials such a cell
// does not exist; the rule acts from three materials on.
template <class T, int NMAT>
__device__ __forceinline__ bool needs_fp64(const T *phi_first)
{
    if (NMAT < 3) return false;
    T fsum = T(0), mn = T(1);
    int present = 0;
#pragma unroll
    for (int l = 0; l < NMAT - 1; l++) {
        mn = m_min(mn, phi_first[l]);
        fsum += phi_first[l];
        present += phi_first[l] >= T(1e-6);
    }
    const T last = T(1) - fsum;
    mn = m_min(mn, last);
    present += last >= T(1e-6);
    return present >= 2 && mn < T(1e-6);
}

// State from primitives in the compute type T; the FP32 form switches to FP64
// for cells whose smallest volume fraction is below 1e-6.
template <class T, int DIM, int NMAT, int SOLID>
__device__ __forceinline__ void state_from_prim(const GridP &g, const T *w, State<T, DIM, NMAT, SOLID> &s)
{
    using L = Lay<DIM, NMAT, SOLID>;
    if (sizeof(T) == 4 && needs_fp64<T, NMAT>(w + L::IPHI)) {
        double wd[L::NVAR];
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) wd[v] = (double)w[v];
        State<double, DIM, NMAT, SOLID> sd;
        state_from_prim_ct<double, DIM, NMAT, SOLID>(g, wd, sd);
#pragma unroll
        for (int l = 0; l < NMAT; l++) {
            s.phi[l] = (T)sd.phi[l];
            s.ar[l] = (T)sd.ar[l];
        }
        s.rho = (T)sd.rho;
#pragma unroll
        for (int a = 0; a < DIM; a++) s.u[a] = (T)sd.u[a];
        s.p = (T)sd.p;
        s.rhoE = (T)sd.rhoE;
        s.c2 = (T)sd.c2;
        s.G = (T)sd.G;
        s.sigY = (T)sd.sigY;
#pragma unroll
        for (int l = 0; l < NMAT; l++) s.eps[l] = (T)sd.eps[l];
        if (SOLID) {
#pragma unroll
            for (int a = 0; a < DIM; a++)
#pragma unroll
                for (int b = 0; b < DIM; b++) s.H[a][b] = (T)sd.H[a][b];
        }
        return;
    }
    state_from_prim_ct<T, DIM, NMAT, SOLID>(g, w, s);
}

// Conserved -> primitive (Sec. 2.2): rho_l = (phi rho)_l / max(phi_l, guard),
// u = (rho u)/rho and the mixture pressure
// p = (rho E - rho|u|^2/2 - sum[(phi rho)_l e_ref,l - phi_l p_ref,l/Gamma_l]) / sum phi_l/Gamma_l.
template <class T, int DIM, int NMAT, int SOLID>
__device__ __forceinline__ void cons_to_prim_ct(const GridP &g, const T *q, T *w)
{
    using L = Lay<DIM, NMAT, SOLID>;
    T phi[NMAT], ar[NMAT], rho = T(0), fsum = T(0);
#pragma unroll
    for (int l = 0; l < NMAT - 1; l++) {
        phi[l] = q[L::IPHI + l];
        fsum += phi[l];
    }
    phi[NMAT - 1] = T(1) - fsum;
#pragma unroll
    for (int l = 0; l < NMAT; l++) {
        ar[l] = q[L::IAR + l];
        rho += ar[l];
    }
    T u[DIM];
    const T irho = T(1) / rho;
#pragma unroll
    for (int a = 0; a < DIM; a++) u[a] = q[L::IMOM + a] * irho;
    T J2 = T(0);
    if (SOLID) {
        T A[3][3], H[3][3];
        unpack_A_ct<T, DIM, NMAT, SOLID>(q, A);
        stretch_log_ct<T, DIM>(A, H, J2);
    }
    T ke = T(0);
#pragma unroll
    for (int a = 0; a < DIM; a++) ke += T(0.5) * rho * u[a] * u[a];
    T num = q[L::IE] - ke, den = T(0);
    T rhol[NMAT];
    if constexpr (NMAT == 1) {
        const MatC<T> &m = matc<T>(g, 0);
        const Ref<T> r = mat_ref<T>(m, rho, J2);
#pragma unroll
        for (int a = 0; a < DIM; a++) w[L::IMOM + a] = u[a];
        w[L::IAR] = rho;
        // p = p_ref + Gamma (rho e - rho e_ref)   (eq:MieGruneisenEOS)
        w[L::IE] = r.pref + r.Gam * (num - rho * r.eref);
#pragma unroll
        for (int c = 0; c < L::NV; c++) w[L::IV + c] = q[L::IV + c];
        w[L::IR] = q[L::IR];
        if constexpr (SOLID == 2) w[L::IH] = rho != T(0) ? q[L::IH] / rho : T(0);
        return;
    }
#pragma unroll
    for (int l = 0; l < NMAT; l++) {
        const T phc = phi_clip(phi[l]);
        rhol[l] = (NMAT == 1) ? rho : phasic_density<T>(g, l, ar[l], phc);
        const MatC<T> &m = matc<T>(g, l);
        const Ref<T> r = mat_ref<T>(m, rhol[l], J2);
        if (ar[l] != T(0)) num -= ar[l] * r.eref;
        num += phc * r.pref * m.invGam;
        den += phc * m.invGam;
    }
#pragma unroll
    for (int l = 0; l < NMAT - 1; l++) w[L::IPHI + l] = phi[l];
#pragma unroll
    for (int l = 0; l < NMAT; l++) w[L::IAR + l] = rhol[l];
#pragma unroll
    for (int a = 0; a < DIM; a++) w[L::IMOM + a] = u[a];
    w[L::IE] = num / den;
#pragma unroll
    for (int c = 0; c < L::NV; c++) w[L::IV + c] = q[L::IV + c];
    w[L::IR] = q[L::IR];
    // history: specific eps_l = (phi rho eps)_l / (phi rho)_l, 0 without mass
    if constexpr (SOLID == 2) {
#pragma unroll
        for (int l = 0; l < NMAT; l++) w[L::IH + l] = ar[l] != T(0) ? q[L::IH + l] / ar[l] : T(0);
    }
}

template <class T, int DIM, int NMAT, int SOLID>
__device__ __forceinline__ void cons_to_prim(const GridP &g, const T *q, T *w)
{
    using L = Lay<DIM, NMAT, SOLID>;
    if (sizeof(T) == 4 && needs_fp64<T, NMAT>(q + L::IPHI)) {
        double qd[L::NVAR], wd[L::NVAR];
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) qd[v] = (double)q[v];
        cons_to_prim_ct<double, DIM, NMAT, SOLID>(g, qd, wd);
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) w[v] = (T)wd[v];
        return;
    }
    cons_to_prim_ct<T, DIM, NMAT, SOLID>(g, q, w);
}

template <class T, int DIM, int NMAT, int SOLID>
__device__ __forceinline__ void prim_to_cons(const GridP &g, const T *w, T *q)
{
    using L = Lay<DIM, NMAT, SOLID>;
    State<T, DIM, NMAT, SOLID> s;
    state_from_prim<T, DIM, NMAT, SOLID>(g, w, s);
#pragma unroll
    for (int l = 0; l < NMAT - 1; l++) q[L::IPHI + l] = s.phi[l];
#pragma unroll
    for (int l = 0; l < NMAT; l++) q[L::IAR + l] = s.ar[l];
#pragma unroll
    for (int a = 0; a < DIM; a++) q[L::IMOM + a] = s.rho * s.u[a];
    q[L::IE] = s.rhoE;
#pragma unroll
    for (int c = 0; c < L::NV; c++) q[L::IV + c] = w[L::IV + c];
    q[L::IR] = w[L::IR];
    if constexpr (SOLID == 2) {
#pragma unroll
        for (int l = 0; l < NMAT; l++) q[L::IH + l] = s.ar[l] * s.eps[l];
    }
}

// ------------------------------------------------------- reconstruction

template <class T>
__device__ __forceinline__ T vanleer(T a, T b)
{
    return (a * b <= T(0)) ? T(0) : T(2) * a * b / (a + b);
}

// THINC face values of a cell (Sec. 3.1, MUSCL-BVD-THINC): the tanh profile
// q_min + dq/2 (1 + theta tanh(beta (x - x_c))) on [0,1] whose cell average is
// q0 has tanh(beta x_c) = (cosh beta - exp(theta beta (2C-1)))/sinh beta with
// C = (q0 - q_min)/dq; its end values are returned.  Only monotone cells with
// 1e-8 < C < 1 - 1e-8.
template <class T>
__device__ __forceinline__ bool thinc(const GridP &g, T qm, T q0, T qp, T &fm, T &fp)
{
    if ((qp - q0) * (q0 - qm) <= T(0)) return false;
    const T qmin = m_min(qm, qp), qmax = m_max(qm, qp);
    const T dq = qmax - qmin;
    const T th = (qp - qm) >= T(0) ? T(1) : T(-1);
    const T C = (q0 - qmin) / dq;
    if (!(C > T(1e-8) && C < T(1) - T(1e-8))) return false;
    const GridC<T> &gc = gridc<T>(g);
    const T B = m_exp(th * gc.beta * (T(2) * C - T(1)));
    const T ty = (gc.cosh_b - B) * gc.inv_sinh_b;
    const T tb = gc.tanh_b;
    const T t1 = (tb - ty) / (T(1) - tb * ty);
    fm = qmin + T(0.5) * dq * (T(1) - th * ty);
    fp = qmin + T(0.5) * dq * (T(1) + th * t1);
    return true;
}

// Left and right states at the face between cells f-1 and f of a pencil,
// s[0..5] = q_{f-3} .. q_{f+2}.  MUSCL (van Leer) for every primitive; for a
// volume fraction (frac = true) the BVD rule keeps a cell's THINC face values
// only where its total boundary variation is strictly below MUSCL's.
template <class T>
__device__ __forceinline__ void recon_face(const GridP &g, const T *s, bool frac, T &qL, T &qR)
{
    const T slB = vanleer(s[2] - s[1], s[3] - s[2]);
    const T slC = vanleer(s[3] - s[2], s[4] - s[3]);
    const T Bp = s[2] + T(0.5) * slB, Cm = s[3] - T(0.5) * slC;
    qL = Bp;
    qR = Cm;
    if (!frac || !g.use_thinc) return;
    const T slA = vanleer(s[1] - s[0], s[2] - s[1]);
    const T slE = vanleer(s[4] - s[3], s[5] - s[4]);
    const T Ap = s[1] + T(0.5) * slA, Bm = s[2] - T(0.5) * slB;
    const T Cp = s[3] + T(0.5) * slC, Em = s[4] - T(0.5) * slE;
    T tAm = s[1] - T(0.5) * slA, tAp = Ap, tBm = Bm, tBp = Bp, tCm = Cm, tCp = Cp, tEm = Em, tEp = s[4] + T(0.5) * slE;
    thinc<T>(g, s[0], s[1], s[2], tAm, tAp);
    thinc<T>(g, s[1], s[2], s[3], tBm, tBp);
    thinc<T>(g, s[2], s[3], s[4], tCm, tCp);
    thinc<T>(g, s[3], s[4], s[5], tEm, tEp);
    const T tbvBM = m_abs(Ap - Bm) + m_abs(Bp - Cm);
    const T tbvBT = m_abs(tAp - tBm) + m_abs(tBp - tCm);
    const T tbvCM = m_abs(Bp - Cm) + m_abs(Cp - Em);
    const T tbvCT = m_abs(tBp - tCm) + m_abs(tCp - tEm);
    if (tbvBT < tbvBM) qL = tBp;
    if (tbvCT < tbvCM) qR = tCm;
}

// ------------------------------------------------------------- Riemann

// Left value for w = 1, right value for w = 0, the mean for w = 1/2 (exactly
// xl or xr in the first two cases).
template <class T>
__device__ __forceinline__ T upwind_mix(T w, T xl, T xr)
{
    return w == T(1) ? xl : (w == T(0) ? xr : T(0.5) * (xl + xr));
}

// out += a (U*_K - U_K) on the partial densities, momenta and energy, for the
// HLLC star state of side K (wave speed SK, normal traction TK, contact Ss).
template <class T, int DIM, int NMAT, int SOLID, int D>
__device__ __forceinline__ void star_jump(const State<T, DIM, NMAT, SOLID> &K, T SK, T TK, T Ss, T a, T *out)
{
    using L = Lay<DIM, NMAT, SOLID>;
    const T uK = K.u[D];
    const T chi = (SK - uK) / (SK - Ss);
#pragma unroll
    for (int l = 0; l < NMAT; l++) out[L::IAR + l] += a * (K.ar[l] * chi - K.ar[l]);
    if constexpr (SOLID == 2) {
#pragma unroll
        for (int l = 0; l < NMAT; l++) out[L::IH + l] += a * (K.ar[l] * K.eps[l] * chi - K.ar[l] * K.eps[l]);
    }
#pragma unroll
    for (int b = 0; b < DIM; b++) out[L::IMOM + b] += a * (K.rho * chi * (b == D ? Ss : K.u[b]) - K.rho * K.u[b]);
    const T EK = K.rhoE / K.rho;
    out[L::IE] += a * (K.rho * chi * (EK + (Ss - uK) * (Ss + TK / (K.rho * (SK - uK)))) - K.rhoE);
}

// HLLC flux across a face normal to direction D (Sec. 3.1: Toro's HLLC; the
// fluid pressure replaced by the normal traction T = p - 2G devH_DD for solids;
// Davis wave speeds; partial densities scaled like the mixture density).
// out[0..NVAR-1]: flux of every plane (r: upwind with the body velocity vr),
// out[NVAR]: face velocity u*_D, out[NVAR+1+b]: V*_{D b} (upwind by S*).
template <class T, int DIM, int NMAT, int SOLID, int D>
__device__ __forceinline__ void riemann(const GridP &g, const T *wL, const T *wR, T vr, T *out)
{
    using L = Lay<DIM, NMAT, SOLID>;
    State<T, DIM, NMAT, SOLID> sl, sr;
    state_from_prim<T, DIM, NMAT, SOLID>(g, wL, sl);
    state_from_prim<T, DIM, NMAT, SOLID>(g, wR, sr);
    const T cL = m_sqrt(sl.c2), cR = m_sqrt(sr.c2);
    const T uL = sl.u[D], uR = sr.u[D];
    const T TL = SOLID ? sl.p - T(2) * sl.G * sl.H[D][D] : sl.p;
    const T TR = SOLID ? sr.p - T(2) * sr.G * sr.H[D][D] : sr.p;
    const T SL = m_min(uL - cL, uR - cR);
    const T SR = m_max(uL + cL, uR + cR);
    // contact speed; the numerator's products are rounded one by one and
    // summed left to right, so that mirror-image states (a wall face) give
    // S* = 0 exactly
    const T num = add_rn(add_rn(TR - TL, mul_rn(mul_rn(sl.rho, uL), SL - uL)),
                         -mul_rn(mul_rn(sr.rho, uR), SR - uR));
    const T Ss = num / (sl.rho * (SL - uL) - sr.rho * (SR - uR));
    int region;
    if (SL >= T(0)) region = 0;
    else if (Ss >= T(0)) region = 1;
    else if (SR > T(0)) region = 2;
    else region = 3;
    const State<T, DIM, NMAT, SOLID> &K = (region <= 1) ? sl : sr;
    const T SK = (region <= 1) ? SL : SR;
    const T TK = (region <= 1) ? TL : TR;
    const T uK = K.u[D];
    const bool star = (region == 1 || region == 2);
    // quantities carried by the contact take the left value for S* > 0, the
    // right one for S* < 0 and the mean of both at S* = 0 (mirror-symmetric
    // at a wall face)
    const T wlf = Ss > T(0) ? T(1) : (Ss < T(0) ? T(0) : T(0.5));
    // Tangential traction and velocity at the face: the linear shear-wave
    // Riemann problem (sigma -/+ Z u constant along the shear characteristics,
    // Z = sqrt(rho G)); a gas (Z = 0) transmits no shear.  Without shear
    // stiffness on either side the tangential velocity is upwind by S*.
    T sig_t[DIM], ut[DIM];
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        sig_t[a] = T(0);
        ut[a] = upwind_mix(wlf, sl.u[a], sr.u[a]);
    }
    if (SOLID) {
        const T ZL = m_sqrt(sl.rho * sl.G), ZR = m_sqrt(sr.rho * sr.G);
#pragma unroll
        for (int a = 0; a < DIM; a++) {
            if (a == D) continue;
            const T sL = T(2) * sl.G * sl.H[a][D], sR = T(2) * sr.G * sr.H[a][D];
            if (ZL + ZR > T(0)) {
                sig_t[a] = (ZR * sL + ZL * sR + ZL * ZR * (sr.u[a] - sl.u[a])) / (ZL + ZR);
                ut[a] = (ZL * sl.u[a] + ZR * sr.u[a] + sR - sL) / (ZL + ZR);
            }
        }
    }
    // physical flux of the selected side; in the star regions the tangential
    // stress is replaced by its face value
    T sig[DIM];
#pragma unroll
    for (int a = 0; a < DIM; a++) sig[a] = (a == D ? -K.p : T(0)) + (SOLID ? T(2) * K.G * K.H[a][D] : T(0));
    T work = T(0), work_n = T(0), work_s = T(0);
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        work += K.u[a] * sig[a];
        if (a == D) work_n += K.u[a] * sig[a];
        else work_s += ut[a] * sig_t[a];
    }
    const T chi = star ? (SK - uK) / (SK - Ss) : T(0);
#pragma unroll
    for (int l = 0; l < NMAT; l++) {
        const T F = K.ar[l] * uK;
        out[L::IAR + l] = star ? F + SK * (K.ar[l] * chi - K.ar[l]) : F;
    }
    if constexpr (SOLID == 2) {
        // plastic-strain planes: carried like the partial densities
#pragma unroll
        for (int l = 0; l < NMAT; l++) {
            const T m = K.ar[l] * K.eps[l];
            out[L::IH + l] = star ? m * uK + SK * (m * chi - m) : m * uK;
        }
    }
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        const T m = K.rho * K.u[a];
        const T Us = K.rho * chi * (a == D ? Ss : K.u[a]);
        if (star) {
            const T Fa = m * uK - (a == D ? sig[a] : T(0));
            out[L::IMOM + a] = Fa + SK * (Us - m) - (a == D ? T(0) : sig_t[a]);
        } else {
            out[L::IMOM + a] = m * uK - sig[a];
        }
    }
    {
        const T EK = K.rhoE / K.rho;
        const T Us = K.rho * chi * (EK + (Ss - uK) * (Ss + TK / (K.rho * (SK - uK))));
        out[L::IE] = star ? (K.rhoE * uK - work_n) + SK * (Us - K.rhoE) - work_s : K.rhoE * uK - work;
    }
    if (star && g.hllc_lm) {
        // HLLC-LM (the published low-Mach form): the centred flux
        // (F_L + F_R)/2 + [phi S_L (U*_L - U_L) + |S*| (U*_L - U*_R) + phi S_R (U*_R - U_R)]/2
        // with phi = sin(min(1, Ma/0.1) pi/2), Ma the larger face-normal Mach
        // number.  With the jump conditions across the three waves this is
        // the HLLC flux above minus (1 - phi)/2 [S_L (U*_L - U_L) + S_R (U*_R - U_R)]
        // on the partial densities, momenta and energy.
        const T Ma = m_max(m_abs(uL) / cL, m_abs(uR) / cR);
        const T ph = m_sin(m_min(T(1), Ma / T(0.1)) * T(3.14159265358979323846) / T(2));
        const T k = T(-0.5) * (T(1) - ph);
        star_jump<T, DIM, NMAT, SOLID, D>(sl, SL, TL, Ss, k * SL, out);
        star_jump<T, DIM, NMAT, SOLID, D>(sr, SR, TR, Ss, k * SR, out);
    }
    // interface state at x/t = 0
    T us[DIM];
#pragma unroll
    for (int a = 0; a < DIM; a++) us[a] = star ? ut[a] : K.u[a];
    us[D] = (region == 0) ? uL : ((region == 3) ? uR : Ss);
#pragma unroll
    for (int l = 0; l < NMAT - 1; l++) out[L::IPHI + l] = upwind_mix(wlf, wL[L::IPHI + l], wR[L::IPHI + l]) * us[D];
#pragma unroll
    for (int c = 0; c < L::NV; c++) {
        const int a = v_row(DIM, c), b = v_col(DIM, c);
        // F(V_ab) = V*_ab u*_D - V*_Db u*_a ; V*_Db is stored whenever b < DIM or (D,b) = (2,2)
        T vdb = T(0);
#pragma unroll
        for (int cc = 0; cc < L::NV; cc++)
            if (v_row(DIM, cc) == D && v_col(DIM, cc) == b) vdb = upwind_mix(wlf, wL[L::IV + cc], wR[L::IV + cc]);
        const T ua = (a < DIM) ? us[a] : T(0);
        out[L::IV + c] = upwind_mix(wlf, wL[L::IV + c], wR[L::IV + c]) * us[D] - vdb * ua;
    }
    out[L::IR] = (vr > T(0)) ? wL[L::IR] * vr : ((vr < T(0)) ? wR[L::IR] * vr : T(0));
    out[L::NVAR] = us[D];
#pragma unroll
    for (int b = 0; b < L::NB; b++) {
        T vdb = T(0);
#pragma unroll
        for (int cc = 0; cc < L::NV; cc++)
            if (v_row(DIM, cc) == D && v_col(DIM, cc) == b) vdb = upwind_mix(wlf, wL[L::IV + cc], wR[L::IV + cc]);
        out[L::NVAR + 1 + b] = vdb;
    }
}

// -------------------------------------------------------- plastic return

// Perfect plasticity by instantaneous radial return, in FP64: the stored A is
// replaced by its symmetric unimodular stretch Q diag(exp(s d_k)) Q^T with d_k
// the deviatoric log-stretches and s = min(1, sigma_Y/sigma_vm),
// sigma_vm = sqrt(3/2) 2 G |d| (mixture G and sigma_Y).  Energy, masses and
// momenta are untouched.  Returns the equivalent plastic strain increment
// sqrt(2/3) (1 - s) |d| (0 below yield).
// yield(svm, |d|, J2) gives the yield stress for the trial von Mises stress
// svm and deviatoric log-stretch norm |d| (Johnson-Cook: plastic strain,
// temperature and rate); the constant-sigma_Y form ignores its arguments.
template <int DIM, class Y>
__device__ __forceinline__ double plastic_return_y(double A[3][3], double G, Y yield)
{
    double H[3][3], J2;
    Eig2 e;
    stretch_log<DIM>(A, H, J2, e);
    const double svm = sqrt(1.5) * 2.0 * G * sqrt(J2);
    const double sigY = yield(svm, sqrt(J2), J2);
    const double sc = (svm > sigY) ? sigY / svm : 1.0;
    // equivalent plastic strain of the removed deviatoric log-strain (1 - s)|d|
    const double deps = sc < 1.0 ? sqrt(2.0 / 3.0) * (1.0 - sc) * sqrt(J2) : 0.0;
    const double e0 = exp(sc * e.d[0]), e1 = exp(sc * e.d[1]), e2 = exp(sc * e.d[2]);
    const double av = 0.5 * (e0 + e1), df = 0.5 * (e0 - e1);
    A[0][0] = av + df * e.c2;
    A[1][1] = av - df * e.c2;
    A[0][1] = A[1][0] = df * e.s2;
    A[2][2] = e2;
    A[0][2] = A[2][0] = A[1][2] = A[2][1] = 0.0;
    if (DIM == 1) {
        A[0][0] = e0;
        A[1][1] = e1;
        A[0][1] = A[1][0] = 0.0;
    }
    return deps;
}

template <int DIM>
__device__ __forceinline__ double plastic_return(double A[3][3], double G, double sigY)
{
    return plastic_return_y<DIM>(A, G, [sigY](double, double, double) { return sigY; });
}

// Johnson-Cook flow stress of material m (the law, the reference temperature
// 298 K and rate 1/s are readings of Table 2, which lists the constants only):
// (c1 + c2 eps^n)(1 + c3 ln max(rate, 1))(1 - T*^m), T* = (T - 298)/(T_melt - 298)
// clipped to [0, 1].
__device__ __forceinline__ double jc_yield(const MatP &m, double eps, double rate, double T)
{
    double ts = (T - 298.0) / (m.jc_tmelt - 298.0);
    ts = ts < 0.0 ? 0.0 : (ts > 1.0 ? 1.0 : ts);
    const double e = eps > 0.0 ? eps : 0.0;
    return (m.jc_c1 + m.jc_c2 * pow(e, m.jc_n)) * (1.0 + m.jc_c3 * log(rate > 1.0 ? rate : 1.0)) *
           (1.0 - pow(ts, m.jc_m));
}

// Mixture yield stress of a cell with Johnson-Cook materials (weights
// phi_l/Gamma_l, Sec. 2.2), each at its plastic strain and at the temperature
// of its Mie-Grueneisen thermal energy, 298 K + (p - p_ref)/(rho_l Gamma_l C_V);
// w: the cell's primitives, J2: its |dev ln V|^2.
template <class R, int DIM, int NMAT, int SOLID>
__device__ __forceinline__ double jc_mixture_yield(const GridP &g, const R *w, double J2, double rate)
{
    using L = Lay<DIM, NMAT, SOLID>;
    double fsum = 0.0, phi[NMAT];
#pragma unroll
    for (int l = 0; l < NMAT - 1; l++) {
        phi[l] = (double)w[L::IPHI + l];
        fsum += phi[l];
    }
    phi[NMAT - 1] = 1.0 - fsum;
    double num = 0.0, den = 0.0;
    const double p = (double)w[L::IE];
#pragma unroll
    for (int l = 0; l < NMAT; l++) {
        const double ph = phi_clip(phi[l]);
        const double rl = (double)w[L::IAR + l];
        const Ref<double> r = mat_ref<double>(g.mc_d[l], rl, J2);
        double sy = g.mat[l].sigY;
        if (g.mat[l].jc) {
            double eps = 0.0;
            if constexpr (SOLID == 2) eps = (double)w[L::IH + l];
            sy = jc_yield(g.mat[l], eps, rate, 298.0 + (p - r.pref) / (rl * r.Gam * g.mat[l].jc_cv));
        }
        num += ph * sy / r.Gam;
        den += ph / r.Gam;
    }
    return num / den;
}

}  // namespace dfv
