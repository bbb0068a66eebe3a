// dfv_kernels.cuh -- the kernels of one time step (arXiv:2111.11806, Sec. 3):
//   k_seed      rigid interface seeding (Sec. 3.2), in place, band cells only
//               (queued per block, seeded by groups of 8 lanes); optionally
//               with the previous step's finalize in one extra block
//   k_stage<S>  one SSP-RK3 stage (Sec. 3.1): halo-3 tile of primitives in
//               shared memory, per-face MUSCL-BVD-THINC + HLLC, divergence,
//               non-conservative terms, rigid mask, RK combination; stage 1
//               also sums the pressure force, stage 3 applies the plastic
//               return and reduces the CFL wave speed of the new state
//   k_cfl       CFL wave-speed reduction of a stored state
//   k_finalize  one block: deterministic sums of the per-block partials,
//               body update, next dt (k_finalize_lite: one warp, no partials)
//   k_prim_to_cons / k_cons_to_prim / k_cons_to_f64   field conversion
// The 3-D FP32 single-material stages march along z instead (dfv_kernels_z.cuh).
#pragma once

#include "dfv_device.cuh"

namespace dfv {

// ------------------------------------------------------------ tiling

// Tile of one CTA: TX x TY x TZ cells, with one thread per face of the
// largest face sweep (the extra warp covers the tile's closing faces).  2-D
// tiles are 32 x 8 in both precisions: measured on the cylinder at 512^2 to
// 2048^2, FP32 steps are 6-8 % shorter than with 32 x 16 tiles (more, smaller
// CTAs balance better over the SMs than the taller tile saves in halo).
template <int DIM, int W>
struct Tile;
template <int W>
struct Tile<1, W> {
    static constexpr int TX = 256, TY = 1, TZ = 1, THREADS = 288;
};
template <int W>
struct Tile<2, W> {
    static constexpr int TX = 32, TY = 8, TZ = 1, THREADS = 288;
};
template <int W>
struct Tile<3, W> {
    static constexpr int TX = 32, TY = 4, TZ = 2, THREADS = 384;
};

template <int DIM, int W>
struct Box {
    using TL = Tile<DIM, W>;
    static constexpr int HX = 3, HY = DIM >= 2 ? 3 : 0, HZ = DIM >= 3 ? 3 : 0;
    static constexpr int BX = TL::TX + 2 * HX, BY = TL::TY + 2 * HY, BZ = TL::TZ + 2 * HZ;
    static constexpr int N = BX * BY * BZ;
    static constexpr int CELLS = TL::TX * TL::TY * TL::TZ;
    static constexpr int FX = (TL::TX + 1) * TL::TY * TL::TZ;
    static constexpr int FY = TL::TX * (TL::TY + 1) * TL::TZ;
    static constexpr int FZ = TL::TX * TL::TY * (TL::TZ + 1);
    static constexpr int MAXF = FX > FY ? (FX > FZ ? FX : FZ) : (FY > FZ ? FY : FZ);
    __host__ __device__ static constexpr int stride(int d) { return d == 0 ? 1 : (d == 1 ? BX : BX * BY); }
};

template <class R, int DIM, int NMAT, int SOLID>
struct StageSmem {
    using L = Lay<DIM, NMAT, SOLID>;
    using B = Box<DIM, (int)sizeof(R)>;
    // 2-D fluid tiles compute the faces of both directions before one
    // barrier, so they keep one face array per direction (solids keep one:
    // their larger face records would cost occupancy)
    static constexpr int NSF = (DIM == 2 && SOLID == 0) ? 2 : 1;
    static constexpr size_t floats = (size_t)L::NVAR * B::N + (size_t)NSF * L::NF * B::MAXF;
    static constexpr size_t bytes = ((sizeof(R) * floats + 7) & ~(size_t)7) + 4 * 32 * sizeof(double);
};

// ---------------------------------------------------- compensated sums

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Accumulator: plain in FP64, (hi, lo) pair with TwoSum in FP32.
template <class R>
struct Acc {
    R hi, lo;
    __device__ __forceinline__ void zero() { hi = R(0); lo = R(0); }
    // first term: exact, no compensation needed
    __device__ __forceinline__ void set(R x) { hi = x; lo = R(0); }
    __device__ __forceinline__ void add(R x)
    {
        if (sizeof(R) == 8) {
            hi += x;
        } else {
            float s, e;
            two_sum((float)hi, (float)x, s, e);
            hi = (R)s;
            lo += (R)e;
        }
    }
};

// out = ca*un + cb*(in - dt*D), D = hi + lo the compensated (TwoSum) flux
// divergence.  FP32: y = in - dt*lo - dt*hi as two fused multiply-adds (the
// low part first), then ca*un rounded and cb*y added in a third fused
// multiply-add -- three roundings, against the one of storing the result in
// FP32; no error-free product is formed.  FP64: plain evaluation.
template <class R>
__device__ __forceinline__ R rk_combine(int stage, R un, R in, const Acc<R> &D, R dt, R ca, R cb)
{
    if (sizeof(R) == 8) {
        const R y = in - dt * D.hi;
        return stage == 1 ? y : ca * un + cb * y;
    } else {
        // y = in - dt*(hi + lo) with a single rounding of the product and sum
        // (fused multiply-add), the low part of the compensated sum folded in
        const float fdt = (float)dt;
        const float y = fmaf(-fdt, (float)D.hi, fmaf(-fdt, (float)D.lo, (float)in));
        if (stage == 1) return (R)y;
        return (R)fmaf((float)cb, y, (float)ca * (float)un);
    }
}

// --------------------------------------------------- block reductions

// Fixed-order block reduction of up to 4 doubles (max for k = 0, sum for the
// rest): warp shuffles, then warp leaders in index order.
template <int THREADS>
__device__ __forceinline__ void block_reduce4(double v[4], double *scratch /* 4*32 */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double m = __shfl_down_sync(0xffffffffu, v[0], o);
        v[0] = fmax(v[0], m);
#pragma unroll
        for (int k = 1; k < 4; k++) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0)
        for (int k = 0; k < 4; k++) scratch[k * 32 + warp] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        constexpr int NW = (THREADS + 31) / 32;
        double r[4] = {scratch[0], scratch[32], scratch[64], scratch[96]};
        for (int w = 1; w < NW; w++) {
            r[0] = fmax(r[0], scratch[w]);
            for (int k = 1; k < 4; k++) r[k] += scratch[k * 32 + w];
        }
        for (int k = 0; k < 4; k++) v[k] = r[k];
    }
}

// Fixed-order compensated block sum of three FP32 values per thread: TwoSum
// at every addition with the low parts summed alongside, over the warp by
// shuffles and then over the warp leaders in index order; the result (hi +
// lo, widened) in thread 0.  The FP32 form's pressure-force partials: no FP64
// arithmetic in the bulk.
template <int THREADS>
__device__ __forceinline__ void block_sum3_f32(const float v[3], float *scratch /* 6*32 */, double out[3])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float hi[3], lo[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        hi[k] = v[k];
        lo[k] = 0.f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float oh = __shfl_down_sync(0xffffffffu, hi[k], o), ol = __shfl_down_sync(0xffffffffu, lo[k], o);
            float s, e;
            two_sum(hi[k], oh, s, e);
            hi[k] = s;
            lo[k] = lo[k] + (ol + e);
        }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            scratch[k * 32 + warp] = hi[k];
            scratch[(3 + k) * 32 + warp] = lo[k];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        constexpr int NW = (THREADS + 31) / 32;
        for (int k = 0; k < 3; k++) {
            float h = scratch[k * 32], l = scratch[(3 + k) * 32];
            for (int w = 1; w < NW; w++) {
                float s, e;
                two_sum(h, scratch[k * 32 + w], s, e);
                h = s;
                l = l + (scratch[(3 + k) * 32 + w] + e);
            }
            out[k] = (double)h + (double)l;
        }
    }
}

// Block maximum of one value per thread (fixed order; result in thread 0).
template <int THREADS, class T>
__device__ __forceinline__ T block_max(T v, T *scratch /* 32 */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = m_max(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        constexpr int NW = (THREADS + 31) / 32;
        T r = scratch[0];
        for (int w = 1; w < NW; w++) r = m_max(r, scratch[w]);
        v = r;
    }
    return v;
}

// ------------------------------------------------------------ finalize

__device__ __forceinline__ void finalize_apply(Ctl *ctl, Ctl &sc, const double red[4], int mode, int dim,
                                               const double dxs[3], bool reset_box);

// mode bit 0: reduce the CFL partials (nb_cfl blocks) into ctl->smax
// mode bit 1: reduce the force partials (nb_force blocks) into ctl->force
// mode bit 2: end of a step: body update with ctl->dt, t += dt
// mode bit 3: set the next dt from ctl->cfl (and t_end when > 0)
// Executed by one whole block of THREADS threads; the sums run in a fixed order.
template <int THREADS>
__device__ __forceinline__ void finalize_block(Ctl *ctl, const double *partials, long long nb_cfl, long long nb_force,
                                               int mode, int dim, double dx0, double dx1, double dx2,
                                               double *sred)
{
    // the control block is read once, word by word in parallel, so that the
    // serial update below works on a shared copy instead of a chain of
    // dependent global loads
    __shared__ Ctl sc;
    constexpr int NWORD = (int)(sizeof(Ctl) / sizeof(unsigned long long));
    for (int k = threadIdx.x; k < NWORD; k += THREADS)
        reinterpret_cast<unsigned long long *>(&sc)[k] = reinterpret_cast<const unsigned long long *>(ctl)[k];
    double red[4] = {0.0, 0.0, 0.0, 0.0};
    // tiles of a stage-3 launch fold their maximum into ctl->smax_acc instead
    // of a partial (nb_cfl = 0 then): read it and leave it at 0
    if ((mode & 1) && threadIdx.x == 0) red[0] = __longlong_as_double((long long)atomicExch(&ctl->smax_acc, 0ull));
    if (mode & 1)
        for (long long b = threadIdx.x; b < nb_cfl; b += THREADS) red[0] = fmax(red[0], partials[4 * b]);
    if (mode & 2) {
        for (long long b = threadIdx.x; b < nb_force; b += THREADS) {
            red[1] += partials[4 * b + 1];
            red[2] += partials[4 * b + 2];
            red[3] += partials[4 * b + 3];
        }
        block_reduce4<THREADS>(red, sred);
    } else {
        red[0] = block_max<THREADS, double>(red[0], sred);
    }
    __syncthreads();     // the shared copy is complete
    if (threadIdx.x != 0) return;
    const double dxs[3] = {dx0, dx1, dx2};
    finalize_apply(ctl, sc, red, mode, dim, dxs, true);
}

// The serial part of the finalize (one thread): sc is a copy of *ctl, red
// the reduced maxima / sums.  reset_box = false leaves ctl->rnext as it is
// (other blocks of the launch still read it; stage 1 resets it).
__device__ __forceinline__ void finalize_apply(Ctl *ctl, Ctl &sc, const double red[4], int mode, int dim,
                                               const double dxs[3], bool reset_box)
{
    if (mode & 2)
        for (int d = 0; d < 3; d++) sc.force[d] = ctl->force[d] = red[1 + d];
    if (mode & 4) {
        if (sc.dynamic && sc.mass > 0.0) {
            for (int d = 0; d < 3; d++) {
                sc.v[d] += sc.dt * sc.force[d] / sc.mass;
                sc.x[d] += sc.dt * sc.v[d];
                ctl->v[d] = sc.v[d];
                ctl->x[d] = sc.x[d];
                ctl->vf[d] = (float)sc.v[d];
            }
        }
        ctl->t = sc.t + sc.dt;
        ctl->steps = sc.steps + 1;
        sc.t += sc.dt;
        // the rigid box of the state just produced becomes the seeding box
        for (int k = 0; k < 6; k++) ctl->rbox[k] = sc.rnext[k];
        ctl->rbox_valid = 1;
        if (reset_box) ctl_box_reset(ctl);
    }
    if (mode & 1) {
        double sb = 0.0;
        for (int d = 0; d < dim; d++) sb += fabs(sc.v[d]) / dxs[d];
        sc.smax = fmax(red[0], sb);
        ctl->smax = sc.smax;
    }
    if (mode & 8) {
        double dt = sc.cfl / sc.smax;
        if (sc.t_end > 0.0) dt = fmin(dt, fmax(sc.t_end - sc.t, 0.0));
        if (!(dt == dt)) dt = 0.0;
        ctl_set_dt(ctl, dt);
    }
}

// The finalize without partial sums (CFL maximum folded into ctl->smax_acc by
// the stage-3 tiles; mode bit 1 not allowed), executed by one warp: the lanes
// copy the control block, lane 0 applies the update.
__device__ __forceinline__ void finalize_warp(Ctl *ctl, int mode, int dim, const double dxs[3], bool reset_box)
{
    __shared__ Ctl sc;
    constexpr int NWORD = (int)(sizeof(Ctl) / sizeof(unsigned long long));
    const int lane = threadIdx.x & 31;
    for (int k = lane; k < NWORD; k += 32)
        reinterpret_cast<unsigned long long *>(&sc)[k] = reinterpret_cast<const unsigned long long *>(ctl)[k];
    __syncwarp();
    if (lane != 0) return;
    double red[4] = {0.0, 0.0, 0.0, 0.0};
    if (mode & 1) red[0] = __longlong_as_double((long long)atomicExch(&ctl->smax_acc, 0ull));
    finalize_apply(ctl, sc, red, mode, dim, dxs, reset_box);
}

static __global__ void __launch_bounds__(32) k_finalize_lite(Ctl *ctl, int mode, int dim, double dx0, double dx1,
                                                             double dx2)
{
    pdl_enter();
    const double dxs[3] = {dx0, dx1, dx2};
    finalize_warp(ctl, mode, dim, dxs, true);
}

static __global__ void __launch_bounds__(1024) k_finalize(Ctl *ctl, const double *partials, long long nb_cfl,
                                                   long long nb_force, int mode, int dim, double dx0, double dx1,
                                                   double dx2)
{
    pdl_enter();
    __shared__ double sred[4 * 32];
    finalize_block<1024>(ctl, partials, nb_cfl, nb_force, mode, dim, dx0, dx1, dx2, sred);
}

// --------------------------------------------------------------- seeding

// ------------------------------------------------------ ELVIRA (Sec. 3.3)

// Fraction of the rectangle [x0, x0+hx] x [y0, y0+hy] on the side
// nx x + ny y <= alpha: coefficients made non-negative by reflecting the
// rectangle, scaled to the unit square, then the piecewise closed form of the
// area of {m1 s + m2 t <= a} (m1 >= m2 >= 0): triangle, trapezoid, square less
// a triangle.
__device__ __forceinline__ double cut_area(double nx, double ny, double alpha, double x0, double y0, double hx,
                                           double hy)
{
    double a = alpha - nx * x0 - ny * y0;
    double m1 = nx * hx, m2 = ny * hy;
    if (m1 < 0.0) {
        a -= m1;
        m1 = -m1;
    }
    if (m2 < 0.0) {
        a -= m2;
        m2 = -m2;
    }
    if (m1 < m2) {
        const double t = m1;
        m1 = m2;
        m2 = t;
    }
    if (a <= 0.0) return 0.0;
    if (a >= m1 + m2) return 1.0;
    if (a < m2) return a * a / (2.0 * m1 * m2);
    if (a <= m1) return (a - 0.5 * m2) / m1;
    const double b = m1 + m2 - a;
    return 1.0 - b * b / (2.0 * m1 * m2);
}

// The line position alpha that leaves the fraction f of the rectangle on the
// side n.x <= alpha: the inverse of the closed form above.
__device__ __forceinline__ double cut_alpha(double nx, double ny, double f, double x0, double y0, double hx,
                                            double hy)
{
    double m1 = nx * hx, m2 = ny * hy;
    double shift = nx * x0 + ny * y0;
    if (m1 < 0.0) {
        shift += m1;
        m1 = -m1;
    }
    if (m2 < 0.0) {
        shift += m2;
        m2 = -m2;
    }
    if (m1 < m2) {
        const double t = m1;
        m1 = m2;
        m2 = t;
    }
    double a;
    if (f <= 0.0) a = 0.0;
    else if (f >= 1.0) a = m1 + m2;
    else if (f * 2.0 * m1 <= m2) a = sqrt(2.0 * m1 * m2 * f);
    else if ((1.0 - f) * 2.0 * m1 <= m2) a = m1 + m2 - sqrt(2.0 * m1 * m2 * (1.0 - f));
    else a = f * m1 + 0.5 * m2;
    return a + shift;
}

// ELVIRA outward normal of a cell from the 3x3 block b[3 (l+1) + (k+1)] of r
// (cell (i+k, j+l)), in FP64: six candidates from the column sums (height y
// of x) and row sums (x of y), backward / central / forward differences, each
// oriented away from r = 1; each candidate line holds the centre cell's r and
// the one reproducing the nine values best (least squares) wins, an earlier
// candidate on ties within 1e-12 (central column, central row, backward
// column, forward column, backward row, forward row).
__device__ __forceinline__ void elvira_normal(const double b[9], double hx, double hy, double nrm[2])
{
    double h[3], gs[3];
#pragma unroll
    for (int k = 0; k < 3; k++) h[k] = (b[k] + b[3 + k] + b[6 + k]) * hy;
#pragma unroll
    for (int l = 0; l < 3; l++) gs[l] = (b[3 * l] + b[3 * l + 1] + b[3 * l + 2]) * hx;
    const double sy = (gs[2] > gs[0]) ? -1.0 : 1.0;
    const double sx = (h[2] > h[0]) ? -1.0 : 1.0;
    const double mc0 = (h[2] - h[0]) / (2.0 * hx), mc1 = (h[1] - h[0]) / hx, mc2 = (h[2] - h[1]) / hx;
    const double mr0 = (gs[2] - gs[0]) / (2.0 * hy), mr1 = (gs[1] - gs[0]) / hy, mr2 = (gs[2] - gs[1]) / hy;
    const double cx[6] = {-mc0, sx, -mc1, -mc2, sx, sx};
    const double cy[6] = {sy, -mr0, sy, sy, -mr1, -mr2};
    double best = 0.0;
    for (int c = 0; c < 6; c++) {
        const double len = sqrt(cx[c] * cx[c] + cy[c] * cy[c]);
        const double nx = cx[c] / len, ny = cy[c] / len;
        const double alpha = cut_alpha(nx, ny, b[4], -0.5 * hx, -0.5 * hy, hx, hy);
        double err = 0.0;
#pragma unroll
        for (int l = 0; l < 3; l++)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const double f = cut_area(nx, ny, alpha, (k - 1.5) * hx, (l - 1.5) * hy, hx, hy);
                err += (f - b[3 * l + k]) * (f - b[3 * l + k]);
            }
        if (c == 0 || err < best - 1e-12) {
            best = err;
            nrm[0] = nx;
            nrm[1] = ny;
        }
    }
}

// Riemann-problem seeding (Sec. 3.2, step 5, second option): the conserved
// right star state of the HLLC problem along the normal n between the
// reflected primitives wl (left) and the interpolated primitives wr (right):
// normal velocities u.n, normal tractions T = p - 2G n.devH.n, Davis speeds,
// contact speed S*; the star state keeps the right state's volume fractions,
// tangential velocity, stretch tensor and r, so its normal velocity is S*,
// which the symmetric problem makes the body's v.n.
template <class R, int DIM, int NMAT, int SOLID>
__device__ __forceinline__ void seed_star(const GridP &g, const R nv[3], const R *wl, const R *wr, R *q)
{
    using L = Lay<DIM, NMAT, SOLID>;
    State<R, DIM, NMAT, SOLID> sl, sr;
    state_from_prim<R, DIM, NMAT, SOLID>(g, wl, sl);
    state_from_prim<R, DIM, NMAT, SOLID>(g, wr, sr);
    R unL = R(0), unR = R(0), HnL = R(0), HnR = R(0);
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        unL += sl.u[a] * nv[a];
        unR += sr.u[a] * nv[a];
        if (SOLID) {
#pragma unroll
            for (int b = 0; b < DIM; b++) {
                HnL += nv[a] * sl.H[a][b] * nv[b];
                HnR += nv[a] * sr.H[a][b] * nv[b];
            }
        }
    }
    const R TL = SOLID ? sl.p - R(2) * sl.G * HnL : sl.p;
    const R TR = SOLID ? sr.p - R(2) * sr.G * HnR : sr.p;
    const R cL = m_sqrt(sl.c2), cR = m_sqrt(sr.c2);
    const R SL = m_min(unL - cL, unR - cR), SR = m_max(unL + cL, unR + cR);
    const R Ss = (TR - TL + sl.rho * unL * (SL - unL) - sr.rho * unR * (SR - unR)) /
                 (sl.rho * (SL - unL) - sr.rho * (SR - unR));
    const R chi = (SR - unR) / (SR - Ss);
#pragma unroll
    for (int l = 0; l < NMAT - 1; l++) q[L::IPHI + l] = sr.phi[l];
#pragma unroll
    for (int l = 0; l < NMAT; l++) q[L::IAR + l] = sr.ar[l] * chi;
    const R rs = sr.rho * chi;
#pragma unroll
    for (int a = 0; a < DIM; a++) q[L::IMOM + a] = rs * (Ss * nv[a] + (sr.u[a] - unR * nv[a]));
    const R ER = sr.rhoE / sr.rho;
    q[L::IE] = rs * (ER + (Ss - unR) * (Ss + TR / (sr.rho * (SR - unR))));
#pragma unroll
    for (int c = 0; c < L::NV; c++) q[L::IV + c] = wr[L::IV + c];
    q[L::IR] = wr[L::IR];
    if constexpr (SOLID == 2) {
#pragma unroll
        for (int l = 0; l < NMAT; l++) q[L::IH + l] = sr.ar[l] * chi * sr.eps[l];
    }
}

// Rigid seeding (Sec. 3.2), one thread per cell: cells with r > 0.5 and
// |grad r| dx_min > 1e-10 get the outward normal n = -grad r/|grad r| (Youngs,
// Sec. 3.3) or the ELVIRA normal; the stepped probe tries points at 1.0, 1.5,
// ..., 4.0 dx_min along n and takes the first whose 2^dim enclosing cell
// centres are in the domain (wrapped if periodic) with r < 0.5 (corners of
// weight 0 excepted: probe_point), the fixed probe
// takes 1.5 dx_min; the primitives are interpolated multilinearly there and
// u <- (I - 2nn^T) u + 2 (v_r.n) n, V <- (I - 2nn^T) V (I - 2nn^T); the cell
// gets that state (original variant) or the right HLLC star state between it
// and the interpolated state (Riemann variant).  With the stepped probe only
// r < 0.5 cells are read and only r > 0.5 cells written, so the update runs in
// place independently of thread order.  Evaluated in the storage precision
// (FP64 closures below phi = 1e-6 as everywhere in the FP32 form).
// The seeded conserved state of rigid cell c (Sec. 3.2), computed from the
// fluid (r < 0.5) cells of U only; false when the cell is not seeded (r <= 0.5,
// no gradient, or no valid probe point).
// OPT: bit 0 ELVIRA normals (2-D), bit 1 Riemann-problem variant; each option
// set is its own kernel so that the plain seeding keeps its small footprint.
// Executed by a group of SEED_G aligned lanes of one warp for the same cell:
// every lane forms the normal, lane k tests step k of the probe ladder, the
// group takes the first valid step, lane m fetches enclosing cell m of the
// probe point, and lane 0 interpolates (in the order of the cells), reflects
// and returns the state (the other lanes return false).
constexpr int SEED_G = 8;

// Probe point of step `step` of the ladder (s = 1.0 + step/2 dx_min along n):
// base cell and fractions of the multilinear stencil.  A point within
// PROBE_SNAP cell widths of a cell-centre line is taken to lie on it, so the
// corners beyond the line get weight 0 exactly: on a symmetry axis of the body
// the normal is axis-aligned, the steps are whole and half cells and the point
// falls on the line, where a zero-weight corner would otherwise decide the step
// by the sign of a rounding error (FP32 against FP64, or one contraction of the
// arithmetic against another).
#define PROBE_SNAP 1e-3

template <class R, int DIM>
__device__ __forceinline__ void probe_point(const GridC<R> &gc, const int ijk[3], const R nv[3], int step, int base[3],
                                            R fr[3])
{
    const R sd = (R(1) + R(0.5) * (R)step) * gc.dxmin;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        base[d] = 0;
        fr[d] = R(0);
    }
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        const R xp = gc.lo[d] + ((R)ijk[d] + R(0.5)) * gc.dx[d] + sd * nv[d];
        const R fi = (xp - gc.lo[d]) / gc.dx[d] - R(0.5);
        R fl = floor(fi);
        R f = fi - fl;
        if (f < R(PROBE_SNAP)) {
            f = R(0);
        } else if (f > R(1) - R(PROBE_SNAP)) {
            f = R(0);
            fl += R(1);
        }
        base[d] = (int)fl;
        fr[d] = f;
    }
}

// A band cell: rigid (r > 0.5) with a non-zero central-difference gradient of
// r (Youngs); r of the cell and of its 2 DIM neighbours in one round of loads.
template <class R, int DIM, int NMAT, int SOLID>
__device__ __forceinline__ bool seed_band_test(const R *U, const GridP &g, const int ijk[3], long long c, R &rc,
                                               R gr[3], R &gn)
{
    using L = Lay<DIM, NMAT, SOLID>;
    const GridC<R> &gc = gridc<R>(g);
    const long long P = g.pitch;
    R rn[3][2];
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        int lo[3] = {ijk[0], ijk[1], ijk[2]}, hi[3] = {ijk[0], ijk[1], ijk[2]};
        lo[d] = map_idx(ijk[d] - 1, g.n[d], g.periodic[d]);
        hi[d] = map_idx(ijk[d] + 1, g.n[d], g.periodic[d]);
        const long long cl = lo[0] + (long long)g.n[0] * (lo[1] + (long long)g.n[1] * lo[2]);
        const long long ch = hi[0] + (long long)g.n[0] * (hi[1] + (long long)g.n[1] * hi[2]);
        rn[d][0] = U[L::IR * P + cl];
        rn[d][1] = U[L::IR * P + ch];
    }
    rc = U[L::IR * P + c];
    gr[0] = gr[1] = gr[2] = R(0);
    gn = R(0);
    if (!(rc > R(0.5))) return false;
#pragma unroll
    for (int d = 0; d < DIM; d++) gr[d] = (rn[d][1] - rn[d][0]) / (R(2) * gc.dx[d]);
    gn = m_sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    return gn * gc.dxmin > R(1e-10);
}

template <class R, int DIM, int NMAT, int SOLID, int OPT>
// rc, gr, gn: r of the band cell, its central-difference gradient and the
// gradient's norm (seed_band_test, true for this cell).
__device__ __forceinline__ bool seed_compute(const R *U, const Ctl *ctl, const GridP &g, const int ijk[3], long long c,
                                             R rc, const R gr[3], R gn, R *q)
{
    using L = Lay<DIM, NMAT, SOLID>;
    const GridC<R> &gc = gridc<R>(g);
    const long long P = g.pitch;
    const int lane = threadIdx.x & 31, sub = lane & (SEED_G - 1), gbase = lane & ~(SEED_G - 1);
    const unsigned gm = ((1u << SEED_G) - 1u) << gbase;
    {
        R nv[3] = {-gr[0] / gn, -gr[1] / gn, -gr[2] / gn};
        if constexpr (DIM == 2 && (OPT & 1)) {
            double blk[9], n2[2];
#pragma unroll
            for (int l = -1; l <= 1; l++)
#pragma unroll
                for (int k = -1; k <= 1; k++) {
                    const int ii = map_idx(ijk[0] + k, g.n[0], g.periodic[0]);
                    const int jj = map_idx(ijk[1] + l, g.n[1], g.periodic[1]);
                    blk[3 * (l + 1) + (k + 1)] = (double)U[L::IR * P + ii + (long long)g.n[0] * jj];
                }
            elvira_normal(blk, g.dx[0], g.dx[1], n2);
            nv[0] = (R)n2[0];
            nv[1] = (R)n2[1];
            nv[2] = R(0);
        }
        // Probe steps s = 1.0, 1.5, ..., 4.0 dx_min: lane k of the group tests
        // step k (its enclosing cells in one round of loads), then the group
        // takes the first valid step.
        constexpr int NC = 1 << DIM;
        int first = -1;
        unsigned int valid = 0u;
        const bool fixed = g.probe_mode == 1;
        if (!fixed) {
            // a step is valid when its 2^DIM enclosing cells lie in the grid
            // (or wrap, in a periodic direction) and all have r < 0.5; corners
            // of weight 0 (a probe point on a cell-centre line, see
            // probe_point) are not part of the stencil
            bool ok = sub < 7;
            if (ok) {
                int base[3];
                R fr[3];
                probe_point<R, DIM>(gc, ijk, nv, sub, base, fr);
#pragma unroll
                for (int m = 0; m < NC; m++) {
                    int ci[3] = {0, 0, 0};
                    bool inside = true;
                    R wt = R(1);
#pragma unroll
                    for (int d = 0; d < DIM; d++) {
                        const int bit = (m >> d) & 1;
                        const int ii = base[d] + bit;
                        if (!g.periodic[d] && (ii < 0 || ii > g.n[d] - 1)) inside = false;
                        ci[d] = map_idx(ii, g.n[d], g.periodic[d]);
                        wt *= bit ? fr[d] : (R(1) - fr[d]);
                    }
                    if (wt > R(0)) {
                        const R rv =
                            U[L::IR * P + ci[0] + (long long)g.n[0] * (ci[1] + (long long)g.n[1] * ci[2])];
                        ok = ok && inside && rv < R(0.5);
                    }
                }
            }
            valid = (__ballot_sync(gm, ok) >> gbase) & 0x7fu;
        }
        if (!fixed && !valid) return false;
        first = fixed ? 1 : __ffs(valid) - 1;     // step 1 of the ladder is the fixed 1.5 dx_min
        // interpolation at the chosen probe point (corner cells clamped into
        // the grid, wrapped if periodic: the fixed probe reads them whatever
        // their r)
        R wi[L::NVAR];
        {
            int base[3];
            R fr[3];
            probe_point<R, DIM>(gc, ijk, nv, first, base, fr);
            // lane m: enclosing cell m and its weight (a corner of weight 0 is
            // not read: it may be a rigid cell that another group is seeding)
            R wt = R(1), w[L::NVAR];
#pragma unroll
            for (int v = 0; v < L::NVAR; v++) w[v] = R(0);
            if (sub < NC) {
                const int m = sub;
                int ci[3] = {0, 0, 0};
#pragma unroll
                for (int d = 0; d < DIM; d++) {
                    const int bit = (m >> d) & 1;
                    ci[d] = map_idx(base[d] + bit, g.n[d], g.periodic[d]);
                    wt *= bit ? fr[d] : (R(1) - fr[d]);
                }
                if (wt > R(0)) {
                    const long long cc = ci[0] + (long long)g.n[0] * (ci[1] + (long long)g.n[1] * ci[2]);
                    R qc[L::NVAR];
#pragma unroll
                    for (int v = 0; v < L::NVAR; v++) qc[v] = U[v * P + cc];
                    cons_to_prim<R, DIM, NMAT, SOLID>(g, qc, w);
                }
            }
            // lane 0 sums them in the order of the cells
#pragma unroll
            for (int v = 0; v < L::NVAR; v++) wi[v] = R(0);
#pragma unroll
            for (int m = 0; m < NC; m++) {
                const R wm = __shfl_sync(gm, wt, gbase + m);
#pragma unroll
                for (int v = 0; v < L::NVAR; v++) wi[v] += wm * __shfl_sync(gm, w[v], gbase + m);
            }
        }
        if (sub != 0) return false;
        R wr[L::NVAR];      // the interpolated state, kept for the Riemann variant
        if constexpr ((OPT & 2) != 0) {
#pragma unroll
            for (int v = 0; v < L::NVAR; v++) wr[v] = wi[v];
        }
        R Pm[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) Pm[i][j] = (i == j ? R(1) : R(0)) - R(2) * nv[i] * nv[j];
        const R vn = ctl_v<R>(ctl, 0) * nv[0] + ctl_v<R>(ctl, 1) * nv[1] + ctl_v<R>(ctl, 2) * nv[2];
        R u[3] = {R(0), R(0), R(0)}, unew[3];
#pragma unroll
        for (int a = 0; a < DIM; a++) u[a] = wi[L::IMOM + a];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            unew[i] = R(2) * vn * nv[i];
#pragma unroll
            for (int j = 0; j < 3; j++) unew[i] += Pm[i][j] * u[j];
        }
#pragma unroll
        for (int a = 0; a < DIM; a++) wi[L::IMOM + a] = unew[a];
        if (SOLID) {
            double A[3][3], PA[3][3];
            unpack_A<R, DIM, NMAT, SOLID>(wi, A);
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    double sm = 0.0;
#pragma unroll
                    for (int k = 0; k < 3; k++) sm += (double)Pm[i][k] * A[k][j];
                    PA[i][j] = sm;
                }
#pragma unroll
            for (int cc = 0; cc < L::NV; cc++) {
                const int i = v_row(DIM, cc), j = v_col(DIM, cc);
                double sm = 0.0;
#pragma unroll
                for (int k = 0; k < 3; k++) sm += PA[i][k] * (double)Pm[k][j];
                wi[L::IV + cc] = (R)sm;
            }
        }
        wi[L::IR] = rc;
        if constexpr ((OPT & 2) != 0) {
            wr[L::IR] = rc;
            seed_star<R, DIM, NMAT, SOLID>(g, nv, wi, wr, q);
        } else {
            prim_to_cons<R, DIM, NMAT, SOLID>(g, wi, q);
        }
        return true;
    }
}

// Seeding from the step-start state when the probe may read rigid cells
// (fixed probe): the seeded state of a cell goes to the scratch planes S,
// whose r plane flags it (1 seeded, 0 not); seed_apply then copies it into U.
template <class R, int DIM, int NMAT, int SOLID>
__device__ __forceinline__ void seed_apply(R *U, const R *S, const GridP &g, long long c)
{
    using L = Lay<DIM, NMAT, SOLID>;
    if (!(U[L::IR * g.pitch + c] > R(0.5)) || S[L::IR * g.pitch + c] != R(1)) return;
#pragma unroll
    for (int v = 0; v < L::NVAR; v++)
        if (v != L::IR) U[v * g.pitch + c] = S[v * g.pitch + c];
}

// MODE 0: in place (stepped probe: reads only r < 0.5 cells, writes only
// r > 0.5 cells); 1: seeded states into the scratch S; 2: S into U.
// The cells to seed lie in the box of the stored state's rigid cells
// (r > 0.5), which stage 3 of the previous step folded into the control block;
// without one (fields just set) the whole grid.  seed_box returns false when
// the box is empty.
__device__ __forceinline__ bool seed_box(const Ctl *ctl, const GridP &g, int lo[3], int hi[3], bool next)
{
    // next: the box that the last stage 3 folded, not yet published (its
    // finalize runs in this launch)
    const bool valid = next || ctl->rbox_valid != 0;
    const int *box = next ? ctl->rnext : ctl->rbox;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        lo[d] = 0;
        hi[d] = g.n[d] - 1;
        if (valid) {
            lo[d] = max(lo[d], box[d]);
            hi[d] = min(hi[d], box[3 + d]);
        }
    }
    return lo[0] <= hi[0] && lo[1] <= hi[1] && lo[2] <= hi[2];
}

// Threads stride over the cells of the rigid box, x fastest.
// Cell t of the box (x fastest) as grid indices and linear index.
__device__ __forceinline__ long long seed_box_cell(const GridP &g, const int lo[3], long long w, long long h,
                                                   bool small, long long t, int ijk[3])
{
    if (small) {
        // 32-bit index arithmetic (64-bit divisions are software routines)
        const unsigned ut = (unsigned)t, uw = (unsigned)w, uh = (unsigned)h, row = ut / uw;
        ijk[0] = lo[0] + (int)(ut - row * uw);
        ijk[1] = lo[1] + (int)(row % uh);
        ijk[2] = lo[2] + (int)(row / uh);
    } else {
        const long long row = t / w;
        ijk[0] = lo[0] + (int)(t - row * w);
        ijk[1] = lo[1] + (int)(row % h);
        ijk[2] = lo[2] + (int)(row / h);
    }
    return ijk[0] + (long long)g.n[0] * (ijk[1] + (long long)g.n[1] * ijk[2]);
}

// The box cells, by whole blocks of at most 256 threads: block_first is the
// block's first cell, stride the cells all blocks cover in one round.  Each
// thread tests one cell; the band cells go to a queue in shared memory and
// are seeded by groups of SEED_G lanes (seed_compute), lane 0 storing the
// state (MODE 0: into U, except r; MODE 1: into S with the flag).  MODE 2
// copies S into U, one cell per thread.
template <class R, int DIM, int NMAT, int SOLID, int OPT, int MODE>
__device__ __forceinline__ void seed_box_cells(R *U, R *S, const Ctl *ctl, const GridP &g, long long block_first,
                                               long long stride, bool next)
{
    using L = Lay<DIM, NMAT, SOLID>;
    const long long P = g.pitch;
    int lo[3], hi[3];
    if (!seed_box(ctl, g, lo, hi, next)) return;
    const long long w = hi[0] - lo[0] + 1, h = hi[1] - lo[1] + 1;
    const long long total = w * h * (hi[2] - lo[2] + 1);
    const bool small = total + stride < (1LL << 31);
    if constexpr (MODE == 2) {
        for (long long t = block_first + threadIdx.x; t < total; t += stride) {
            int ijk[3];
            seed_apply<R, DIM, NMAT, SOLID>(U, S, g, seed_box_cell(g, lo, w, h, small, t, ijk));
        }
        return;
    }
    // the queue: thread index of a band cell in this round, with its r,
    // gradient and gradient norm from the test
    __shared__ int s_n;
    __shared__ unsigned short s_q[256];
    __shared__ R s_b[5][256];
    const int sub = threadIdx.x & (SEED_G - 1);
    for (long long b0 = block_first; b0 < total; b0 += stride) {     // the same rounds for the whole block
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        const long long t = b0 + threadIdx.x;
        if (t < total) {
            int ijk[3];
            const long long c = seed_box_cell(g, lo, w, h, small, t, ijk);
            R rc, gr[3], gn;
            if (seed_band_test<R, DIM, NMAT, SOLID>(U, g, ijk, c, rc, gr, gn)) {
                const int k = atomicAdd(&s_n, 1);
                s_q[k] = (unsigned short)threadIdx.x;
                s_b[0][k] = rc;
                s_b[1][k] = gr[0];
                s_b[2][k] = gr[1];
                s_b[3][k] = gr[2];
                s_b[4][k] = gn;
            } else if (MODE == 1 && rc > R(0.5))
                S[L::IR * P + c] = R(0);
        }
        __syncthreads();
        const int n = s_n;
        for (int k = threadIdx.x / SEED_G; k < n; k += blockDim.x / SEED_G) {
            int ijk[3];
            const long long c = seed_box_cell(g, lo, w, h, small, b0 + s_q[k], ijk);
            const R gr[3] = {s_b[1][k], s_b[2][k], s_b[3][k]};
            R q[L::NVAR];
            const bool ok = seed_compute<R, DIM, NMAT, SOLID, OPT>(U, ctl, g, ijk, c, s_b[0][k], gr, s_b[4][k], q);
            if (sub == 0) {
                if constexpr (MODE == 0) {
                    if (ok) {
#pragma unroll
                        for (int v = 0; v < L::NVAR; v++)
                            if (v != L::IR) U[v * P + c] = q[v];
                    }
                } else {
                    if (ok) {
#pragma unroll
                        for (int v = 0; v < L::NVAR; v++)
                            if (v != L::IR) S[v * P + c] = q[v];
                    }
                    S[L::IR * P + c] = ok ? R(1) : R(0);
                }
            }
        }
        __syncthreads();     // the queue is refilled in the next round
    }
}

// fin_mode != 0: the finalize of the previous step was deferred to this
// launch (a static body: the seeding needs no result of it but the box,
// read from rnext); its last block runs it while the others seed.
template <class R, int DIM, int NMAT, int SOLID, int OPT, int MODE>
__global__ void __launch_bounds__(256) k_seed(void *Uv, void *Sv, Ctl *ctl, GridP g, int fin_mode)
{
    pdl_enter();
    const int nseed = gridDim.x - (fin_mode ? 1 : 0);
    if (fin_mode && (int)blockIdx.x == nseed) {
        if (threadIdx.x < 32) finalize_warp(ctl, fin_mode, g.dim, g.dx, false);
        return;
    }
    seed_box_cells<R, DIM, NMAT, SOLID, OPT, MODE>(reinterpret_cast<R *>(Uv), reinterpret_cast<R *>(Sv), ctl, g,
                                                   blockIdx.x * (long long)blockDim.x, (long long)nseed * blockDim.x,
                                                   fin_mode != 0);
}

// Launch shape of k_seed: up to 16 CTAs of 256 threads per SM.
__host__ inline void seed_grid(const GridP &g, dim3 &block, dim3 &grid)
{
    const long long b = (g.ncell + 255) / 256;
    block = dim3(256, 1, 1);
    grid = dim3((unsigned)(b < 1 ? 1 : (b > 152LL * 16 ? 152LL * 16 : b)), 1, 1);
}

// The option set of a grid as the OPT template argument of the seeding.
__host__ __device__ inline int seed_opt(const GridP &g)
{
    return (g.normal_method == 1 && g.dim == 2 ? 1 : 0) | (g.seed_variant == 1 ? 2 : 0);
}

// --------------------------------------------------------------- stage

struct StageArgs {
    const void *in;     // U^(s-1) (stage input, read with halo)
    const void *un;     // U^n (read at the cell only)
    void *out;          // U^(s)
    Ctl *ctl;
    double *partials;   // 4 doubles per block
    int want_force;
    int early;          // stage 1 after the seeding launch: of the first `early` tiles (the first wave
                        // of CTAs), those that read no cell of the seeding box load and compute their
                        // faces before waiting for it
    int next;           // ... the seeding box is ctl->rnext (its finalize runs in the seeding launch)
};

// Whether a tile's loaded cells (the tile and its halo of 3, after boundary
// mapping) may include a cell of the seeding box, i.e. a cell the seeding
// of this step writes.  Conservative: a halo that wraps (periodic) or is
// mirrored (wall) counts as touching; a clamped (outflow) halo is clamped.
// Read before the seeding launch has finished: the box words come from L2
// (written by an earlier launch, complete before this one started).
template <int DIM, int W>
__device__ __forceinline__ bool tile_touches_box(const GridP &g, const Ctl *ctl, int ox, int oy, int oz, bool next)
{
    using TL = Tile<DIM, W>;
    using B = Box<DIM, W>;
    const bool valid = next || __ldcg(&ctl->rbox_valid) != 0;
    if (!valid) return true;
    const int *box = next ? ctl->rnext : ctl->rbox;
    const int o[3] = {ox, oy, oz}, t[3] = {TL::TX, TL::TY, TL::TZ}, h[3] = {B::HX, B::HY, B::HZ};
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        const int lo = __ldcg(&box[d]), hi = __ldcg(&box[3 + d]);
        int a = o[d] - h[d], b = o[d] + t[d] + h[d] - 1;
        if (a < 0) {
            if (g.periodic[d] || g.wall[d][0]) return true;
            a = 0;
        }
        if (b > g.n[d] - 1) {
            if (g.periodic[d] || g.wall[d][1]) return true;
            b = g.n[d] - 1;
        }
        if (b < lo || a > hi) return false;
    }
    return true;
}

// Fluxes of every face of direction D of the tile into sF (no barrier).
template <class R, int DIM, int NMAT, int SOLID, int D>
__device__ __forceinline__ void face_pass(const GridP &g, const R *sW, R *sF, R vr)
{
    using L = Lay<DIM, NMAT, SOLID>;
    using B = Box<DIM, (int)sizeof(R)>;
    using TL = Tile<DIM, (int)sizeof(R)>;
    constexpr int EX = TL::TX + (D == 0), EY = TL::TY + (D == 1), EZ = TL::TZ + (D == 2);
    constexpr int NFACE = EX * EY * EZ;
    constexpr int SD = B::stride(D);
    // Faces to threads: with 32-wide tiles every warp takes one row of 32
    // faces (lane = x), and in the x sweep the warps past the last row take
    // the rows' closing faces (x = 32); otherwise a flat index.
    constexpr bool ROWS = TL::TX == 32 && DIM >= 2;
    constexpr int NROW = TL::TY * TL::TZ;                   // rows of the tile
    // warps of work: one per face row, plus (x sweep) the closing faces
    constexpr int WROWS = D == 0 ? NROW + (NROW + 31) / 32 : EY * EZ;
    constexpr int ITEMS = ROWS ? WROWS * 32 : NFACE;
    for (int t = threadIdx.x; t < ITEMS; t += TL::THREADS) {
        int fx, fy, fz;
        if constexpr (ROWS) {
            const int lane = t & 31, warp = t >> 5;
            int row;
            if (D == 0 && warp >= NROW) {
                row = (warp - NROW) * 32 + lane;
                fx = TL::TX;
                if (row >= NROW) continue;
            } else {
                row = warp;
                fx = lane;
                if (row >= EY * EZ) continue;
            }
            fy = row % EY;
            fz = row / EY;
        } else {
            if (t >= NFACE) continue;
            fx = t % EX;
            fy = (t / EX) % EY;
            fz = t / (EX * EY);
        }
        const int item = (fz * EY + fy) * EX + fx;
        // box index of the cell on the right of the face
        const int bc = ((fz + B::HZ) * B::BY + (fy + B::HY)) * B::BX + (fx + B::HX);
        R wL[L::NVAR], wR[L::NVAR];
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) {
            if (v == L::IR && vr == R(0)) {
                // the upwind r flux (Sec. 3.1) vanishes for a body at rest in
                // this direction, whatever the face values of r
                wL[v] = wR[v] = R(0);
                continue;
            }
            R s[6];
#pragma unroll
            for (int k = 0; k < 6; k++) s[k] = sW[v * B::N + bc + (k - 3) * SD];
            const bool frac = (v >= L::IPHI && v < L::IPHI + NMAT - 1) || v == L::IR;
            recon_face<R>(g, s, frac, wL[v], wR[v]);
        }
        R F[L::NF];
        riemann<R, DIM, NMAT, SOLID, D>(g, wL, wR, vr, F);
#pragma unroll
        for (int k = 0; k < L::NF; k++) sF[k * B::MAXF + item] = F[k];
    }
}

// Divergence and non-conservative terms of direction D for the thread's own
// cell, from the face fluxes in sF (no barrier).
template <class R, int DIM, int NMAT, int SOLID, int D>
__device__ __forceinline__ void accum_pass(const GridP &g, const R *sW, const R *sF, bool own, int lx, int ly, int lz,
                                           Acc<R> *Dacc)
{
    using L = Lay<DIM, NMAT, SOLID>;
    using B = Box<DIM, (int)sizeof(R)>;
    using TL = Tile<DIM, (int)sizeof(R)>;
    constexpr int EX = TL::TX + (D == 0), EY = TL::TY + (D == 1);
    if (own) {
        const int fl = (lz * EY + ly) * EX + lx;
        const int fr = fl + (D == 0 ? 1 : (D == 1 ? EX : EX * EY));
        const int bcell = ((lz + B::HZ) * B::BY + (ly + B::HY)) * B::BX + (lx + B::HX);
        const R inv = gridc<R>(g).inv_dx[D];
        const R dus = sF[L::NVAR * B::MAXF + fr] - sF[L::NVAR * B::MAXF + fl];
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) {
            const R div = (sF[v * B::MAXF + fr] - sF[v * B::MAXF + fl]) * inv;
            R snc = R(0);
            if (v >= L::IPHI && v < L::IPHI + NMAT - 1) snc = sW[v * B::N + bcell] * dus * inv;
            if (SOLID && v >= L::IV && v < L::IV + L::NV) {
                const int c = v - L::IV;
                const int a = v_row(DIM, c), b = v_col(DIM, c);
                const R ua = (a < DIM) ? sW[(L::IMOM + a) * B::N + bcell] : R(0);
                const R dv = (b < L::NB) ? sF[(L::NVAR + 1 + b) * B::MAXF + fr] - sF[(L::NVAR + 1 + b) * B::MAXF + fl]
                                         : R(0);
                snc = (R(2) / R(3) * sW[v * B::N + bcell] * dus - ua * dv) * inv;
            }
            if (D == 0) Dacc[v].set(div - snc);
            else Dacc[v].add(div - snc);
        }
    }
}

// One tile of one SSP-RK3 stage, executed by a whole CTA: (tbx, tby, tbz) is
// the tile position in tile units, tile_id its index among the ntiles tiles of
// the grid (partials slot; the last of them to finish runs the finalize).
template <class R, int DIM, int NMAT, int SOLID, int STAGE>
__device__ __forceinline__ void stage_tile(const GridP &g, const StageArgs &a, int tbx, int tby, int tbz,
                                           long long tile_id, long long ntiles)
{
    using L = Lay<DIM, NMAT, SOLID>;
    using B = Box<DIM, (int)sizeof(R)>;
    using TL = Tile<DIM, (int)sizeof(R)>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using SM = StageSmem<R, DIM, NMAT, SOLID>;
    R *sW = reinterpret_cast<R *>(smem_raw);
    R *sF = sW + (size_t)L::NVAR * B::N;
    double *sred = reinterpret_cast<double *>(smem_raw + ((sizeof(R) * SM::floats + 7) & ~(size_t)7));

    const R *in = reinterpret_cast<const R *>(a.in);
    const R *un = reinterpret_cast<const R *>(a.un);
    R *out = reinterpret_cast<R *>(a.out);
    const long long P = g.pitch;
    const int ox = tbx * TL::TX, oy = tby * TL::TY, oz = tbz * TL::TZ;
    // a stage-1 tile whose loaded cells miss the seeding box runs up to its
    // update before waiting for the seeding launch (its reads before the
    // wait bypass L1); the others wait first
    // (only the first wave: later tiles start after the seeding anyway, and
    // their loads keep the L1 hits of the halo shared with earlier tiles)
    const bool early = STAGE == 1 && tile_id < a.early &&
                       !tile_touches_box<DIM, (int)sizeof(R)>(g, a.ctl, ox, oy, oz, a.next);
    if (STAGE == 1 && a.early > 0 && !early) pdl_wait();

    // 1. primitives of the tile and its halo (the corner regions are unused);
    // a tile whose halo lies inside the grid needs no boundary mapping
    const bool interior = ox >= B::HX && ox + TL::TX + B::HX <= g.n[0] &&
                          (DIM < 2 || (oy >= B::HY && oy + TL::TY + B::HY <= g.n[1])) &&
                          (DIM < 3 || (oz >= B::HZ && oz + TL::TZ + B::HZ <= g.n[2]));
    for (int i = threadIdx.x; i < B::N; i += TL::THREADS) {
        const int bx = i % B::BX, by = (i / B::BX) % B::BY, bz = i / (B::BX * B::BY);
        const int lx = bx - B::HX, ly = by - B::HY, lz = bz - B::HZ;
        const int outside = (lx < 0 || lx >= TL::TX) + (ly < 0 || ly >= TL::TY) + (lz < 0 || lz >= TL::TZ);
        if (outside > 1) continue;
        bool fl[3] = {false, false, false};
        int gx = ox + lx, gy = DIM >= 2 ? oy + ly : 0, gz = DIM >= 3 ? oz + lz : 0;
        if (!interior) {
            gx = halo_idx(g, 0, ox + lx, &fl[0]);
            if (DIM >= 2) gy = halo_idx(g, 1, oy + ly, &fl[1]);
            if (DIM >= 3) gz = halo_idx(g, 2, oz + lz, &fl[2]);
        }
        const long long c = gx + (long long)g.n[0] * (gy + (long long)g.n[1] * gz);
        R q[L::NVAR], w[L::NVAR];
        if (early) {
#pragma unroll
            for (int v = 0; v < L::NVAR; v++) q[v] = __ldcg(&in[v * P + c]);
        } else {
#pragma unroll
            for (int v = 0; v < L::NVAR; v++) q[v] = in[v * P + c];
        }
        cons_to_prim<R, DIM, NMAT, SOLID>(g, q, w);
        // mirror image behind a reflective wall: u_d and the stretch
        // components with exactly one index d change sign
#pragma unroll
        for (int d = 0; d < DIM; d++) {
            if (!fl[d]) continue;
            w[L::IMOM + d] = -w[L::IMOM + d];
#pragma unroll
            for (int cc = 0; cc < L::NV; cc++)
                if ((v_row(DIM, cc) == d) != (v_col(DIM, cc) == d)) w[L::IV + cc] = -w[L::IV + cc];
        }
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) sW[v * B::N + i] = w[v];
    }
    __syncthreads();

    const bool own = threadIdx.x < B::CELLS;
    const int lx = threadIdx.x % TL::TX, ly = (threadIdx.x / TL::TX) % TL::TY, lz = threadIdx.x / (TL::TX * TL::TY);
    const int gx = ox + lx, gy = oy + ly, gz = oz + lz;
    const bool inside = own && gx < g.n[0] && gy < g.n[1] && gz < g.n[2];
    // the body velocity: set before the seeding launch (a deferred
    // finalize, the only kind that launch runs, leaves it unchanged)
    R vr[3];
#pragma unroll
    for (int d = 0; d < 3; d++) vr[d] = early ? ctl_v_cg<R>(a.ctl, d) : ctl_v<R>(a.ctl, d);
    // the rigid box that stage 3 folds starts empty (the seeding and stage 1,
    // which read it, have finished)
    if (STAGE == 2 && tile_id == 0 && threadIdx.x == 0) ctl_box_reset(a.ctl);

    Acc<R> Dacc[L::NVAR];
#pragma unroll
    for (int v = 0; v < L::NVAR; v++) Dacc[v].zero();

    if constexpr (SM::NSF == 2) {
        // 2-D fluids: the faces of both directions, one barrier, both divergences
        R *sF1 = sF + (size_t)L::NF * B::MAXF;
        face_pass<R, DIM, NMAT, SOLID, 0>(g, sW, sF, vr[0]);
        face_pass<R, DIM, NMAT, SOLID, 1>(g, sW, sF1, vr[1]);
        __syncthreads();
        accum_pass<R, DIM, NMAT, SOLID, 0>(g, sW, sF, own, lx, ly, lz, Dacc);
        accum_pass<R, DIM, NMAT, SOLID, 1>(g, sW, sF1, own, lx, ly, lz, Dacc);
        __syncthreads();
    } else {
#pragma unroll
        for (int d = 0; d < DIM; d++) {
            if (d == 0) face_pass<R, DIM, NMAT, SOLID, 0>(g, sW, sF, vr[0]);
            if constexpr (DIM >= 2) if (d == 1) face_pass<R, DIM, NMAT, SOLID, 1>(g, sW, sF, vr[1]);
            if constexpr (DIM >= 3) if (d == 2) face_pass<R, DIM, NMAT, SOLID, 2>(g, sW, sF, vr[2]);
            __syncthreads();
            if (d == 0) accum_pass<R, DIM, NMAT, SOLID, 0>(g, sW, sF, own, lx, ly, lz, Dacc);
            if constexpr (DIM >= 2) if (d == 1) accum_pass<R, DIM, NMAT, SOLID, 1>(g, sW, sF, own, lx, ly, lz, Dacc);
            if constexpr (DIM >= 3) if (d == 2) accum_pass<R, DIM, NMAT, SOLID, 2>(g, sW, sF, own, lx, ly, lz, Dacc);
            __syncthreads();
        }
    }

    if (early) pdl_wait();   // Δt and the seeded cells of U^n are final from here on
    const R dt = ctl_dt<R>(a.ctl);
    R fcell[3] = {R(0), R(0), R(0)};   // the cell's pressure-force contribution (stage 1)
    R smax_cell = R(0);
    bool rigid_new = false;
    if (inside) {
        const long long c = gx + (long long)g.n[0] * (gy + (long long)g.n[1] * gz);
        const int bcell = ((lz + B::HZ) * B::BY + (ly + B::HY)) * B::BX + (lx + B::HX);
        const bool masked = un[L::IR * P + c] > R(0.5);
        const R ca = STAGE == 2 ? R(0.75) : (STAGE == 3 ? R(1.0 / 3.0) : R(0));
        const R cb = STAGE == 2 ? R(0.25) : (STAGE == 3 ? R(2.0 / 3.0) : R(1));
        R o[L::NVAR];
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) {
            const R unv = un[v * P + c];
            if (masked && v != L::IR) {
                o[v] = unv;
            } else {
                o[v] = rk_combine<R>(STAGE, unv, in[v * P + c], Dacc[v], dt, ca, cb);
            }
        }
        if (SOLID && STAGE == 3 && !masked) {
            // plastic relaxation on the new state (mixture G, sigma_Y from its primitives)
            R w[L::NVAR];
            cons_to_prim<R, DIM, NMAT, SOLID>(g, o, w);
            State<R, DIM, NMAT, SOLID> s;
            state_from_prim<R, DIM, NMAT, SOLID>(g, w, s);
            double A[3][3];
            unpack_A<R, DIM, NMAT, SOLID>(o, A);
            double deps;
            if (g.any_jc) {
                // Johnson-Cook: the rate is that of a return at the rate-free
                // yield stress over the step (one explicit predictor)
                const double G = (double)s.G, dtd = a.ctl->dt;
                deps = plastic_return_y<DIM>(A, G, [&](double svm, double nd, double J2) {
                    const double sy0 = jc_mixture_yield<R, DIM, NMAT, SOLID>(g, w, J2, 0.0);
                    const double rate = (svm > sy0 && dtd > 0.0) ? sqrt(2.0 / 3.0) * (1.0 - sy0 / svm) * nd / dtd : 0.0;
                    return jc_mixture_yield<R, DIM, NMAT, SOLID>(g, w, J2, rate);
                });
            } else {
                deps = plastic_return<DIM>(A, (double)s.G, (double)s.sigY);
            }
#pragma unroll
            for (int cc = 0; cc < L::NV; cc++) o[L::IV + cc] = (R)A[v_row(DIM, cc)][v_col(DIM, cc)];
            if constexpr (SOLID == 2) {
                // the strain removed by the return, added to every material with a yield stress
#pragma unroll
                for (int l = 0; l < NMAT; l++)
                    if ((matc<R>(g, l).sigY > R(0) || g.mat[l].jc) && deps > 0.0)
                        o[L::IH + l] = (R)((double)o[L::IH + l] + (double)o[L::IAR + l] * deps);
            }
        }
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) out[v * P + c] = o[v];
        if (!(o[L::IAR] + (NMAT > 1 ? o[L::IAR + NMAT - 1] : R(0)) > R(0)) || !(o[L::IE] == o[L::IE]))
            atomicOr(&a.ctl->err, (unsigned)ERR_STATE);
        if (STAGE == 1 && a.want_force) {
            // pressure force: p (grad r) dV with central differences (Youngs)
            const GridC<R> &gc = gridc<R>(g);
            const R p = sW[L::IE * B::N + bcell];
#pragma unroll
            for (int d = 0; d < DIM; d++) {
                const int sd = B::stride(d);
                const R gr = (sW[L::IR * B::N + bcell + sd] - sW[L::IR * B::N + bcell - sd]) / (R(2) * gc.dx[d]);
                fcell[d] = p * gr * gc.dV;
            }
        }
        if (STAGE == 3) rigid_new = o[L::IR] > R(0.5);
        if (STAGE == 3) {
            // CFL wave speed of the new state, in the compute precision
            R w[L::NVAR];
            cons_to_prim<R, DIM, NMAT, SOLID>(g, o, w);
            State<R, DIM, NMAT, SOLID> s;
            state_from_prim<R, DIM, NMAT, SOLID>(g, w, s);
            if (!(s.c2 > R(0))) atomicOr(&a.ctl->err, (unsigned)ERR_SOUND);
            const R cs = m_sqrt(s.c2);
            R sum = R(0);
#pragma unroll
            for (int d = 0; d < DIM; d++) sum += (m_abs(s.u[d]) + cs) / gridc<R>(g).dx[d];
            smax_cell = sum;
        }
    }
    if (STAGE == 3) {
        // box of the new state's rigid cells for the next seeding: warp
        // minima / maxima, one atomic set per warp that holds a rigid cell
        if (__any_sync(0xffffffffu, rigid_new)) {
            const int big = 0x7fffffff;
            const int b[6] = {rigid_new ? gx : big, rigid_new ? gy : big, rigid_new ? gz : big,
                              rigid_new ? gx : -1, rigid_new ? gy : -1, rigid_new ? gz : -1};
            int m[6];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                m[k] = __reduce_min_sync(0xffffffffu, b[k]);
                m[3 + k] = __reduce_max_sync(0xffffffffu, b[3 + k]);
            }
            if ((threadIdx.x & 31) == 0) {
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    atomicMin(&a.ctl->rnext[k], m[k]);
                    atomicMax(&a.ctl->rnext[3 + k], m[3 + k]);
                }
            }
        }
        // block maximum in the compute precision (the per-cell values are R),
        // folded into the launch's running maximum: the bits of non-negative
        // doubles order like the doubles, so an integer atomic max is exact
        // and independent of the order of the tiles
        R *sr = reinterpret_cast<R *>(sred);
        const R m = block_max<TL::THREADS, R>(smax_cell, sr);
        if (threadIdx.x == 0) {
            double md = (double)m;
            if (!(md >= 0.0)) md = __longlong_as_double(0x7ff0000000000000LL);   // NaN -> +inf: dt = 0
            atomicMax(&a.ctl->smax_acc, (unsigned long long)__double_as_longlong(md));
        }
    }
    if (STAGE == 1 && a.want_force) {
        // the block's force partial: a compensated FP32 sum in the FP32 form,
        // an FP64 sum in the FP64 form
        double fs[3];
        if constexpr (sizeof(R) == 4) {
            const float fv[3] = {(float)fcell[0], (float)fcell[1], (float)fcell[2]};
            block_sum3_f32<TL::THREADS>(fv, reinterpret_cast<float *>(sred), fs);
        } else {
            double red[4] = {0.0, (double)fcell[0], (double)fcell[1], (double)fcell[2]};
            block_reduce4<TL::THREADS>(red, sred);
            for (int k = 0; k < 3; k++) fs[k] = red[1 + k];
        }
        if (threadIdx.x == 0) {
            double *pp = a.partials + 4 * tile_id;
            pp[1] = fs[0];
            pp[2] = fs[1];
            pp[3] = fs[2];
        }
    }
}

// Register bound: four CTAs per SM for the 2-D FP32 single-material fluid
// (56 registers without spills; stage 3 would otherwise take 62 and three),
// two for the other 2-D forms (which would otherwise take up to 138
// registers and run one 9-warp CTA per SM).
template <class R, int DIM, int NMAT, int SOLID>
constexpr int stage_min_ctas()
{
    return DIM != 2 ? 1 : ((sizeof(R) == 4 && NMAT == 1 && SOLID == 0) ? 4 : 2);
}

template <class R, int DIM, int NMAT, int SOLID, int STAGE>
__global__ void __launch_bounds__(Tile<DIM, (int)sizeof(R)>::THREADS, stage_min_ctas<R, DIM, NMAT, SOLID>())
    k_stage(StageArgs a, GridP g)
{
    // stage 1 after the seeding waits inside stage_tile (early tiles late)
    if (STAGE == 1 && a.early > 0) pdl_release();
    else pdl_enter();
    const long long tile = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    const long long nt = (long long)gridDim.x * gridDim.y * gridDim.z;
    stage_tile<R, DIM, NMAT, SOLID, STAGE>(g, a, blockIdx.x, blockIdx.y, blockIdx.z, tile, nt);
}

// ------------------------------------------------------------------ CFL

template <class R, int DIM, int NMAT, int SOLID>
__global__ void __launch_bounds__(256) k_cfl(const void *Uv, double *partials, GridP g)
{
    using L = Lay<DIM, NMAT, SOLID>;
    __shared__ double sred[4 * 32];
    const R *U = reinterpret_cast<const R *>(Uv);
    const long long P = g.pitch;
    double red[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        R q[L::NVAR], w[L::NVAR];
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) q[v] = U[v * P + c];
        cons_to_prim<R, DIM, NMAT, SOLID>(g, q, w);
        State<R, DIM, NMAT, SOLID> s;
        state_from_prim<R, DIM, NMAT, SOLID>(g, w, s);
        const R cs = m_sqrt(s.c2);
        R sum = R(0);
#pragma unroll
        for (int d = 0; d < DIM; d++) sum += (m_abs(s.u[d]) + cs) / gridc<R>(g).dx[d];
        double sd = (double)sum;
        if (!(sd == sd)) sd = __longlong_as_double(0x7ff0000000000000LL);   // NaN -> +inf: dt = 0
        red[0] = fmax(red[0], sd);
    }
    block_reduce4<256>(red, sred);
    if (threadIdx.x == 0) partials[4 * blockIdx.x] = red[0];
}

static __global__ void k_set_dt(Ctl *ctl, double dt) { ctl_set_dt(ctl, dt); }

// ------------------------------------------------------------ conversions

template <class R, int DIM, int NMAT, int SOLID>
__global__ void __launch_bounds__(256) k_prim_to_cons(const double *prim, long long ppitch, void *Uv, GridP g)
{
    using L = Lay<DIM, NMAT, SOLID>;
    R *U = reinterpret_cast<R *>(Uv);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        double w[L::NVAR], q[L::NVAR];
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) w[v] = prim[v * ppitch + c];
        prim_to_cons<double, DIM, NMAT, SOLID>(g, w, q);
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) U[v * g.pitch + c] = (R)q[v];
    }
}

template <class R, int DIM, int NMAT, int SOLID>
__global__ void __launch_bounds__(256) k_cons_to_prim(const void *Uv, double *prim, long long ppitch, GridP g)
{
    using L = Lay<DIM, NMAT, SOLID>;
    const R *U = reinterpret_cast<const R *>(Uv);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        double q[L::NVAR], w[L::NVAR];
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) q[v] = (double)U[v * g.pitch + c];
        cons_to_prim_ct<double, DIM, NMAT, SOLID>(g, q, w);
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) prim[v * ppitch + c] = w[v];
    }
}

template <class R>
__global__ void __launch_bounds__(256) k_cons_to_f64(const void *Uv, double *outp, long long ppitch, int nvar, GridP g)
{
    const R *U = reinterpret_cast<const R *>(Uv);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x)
        for (int v = 0; v < nvar; v++) outp[v * ppitch + c] = (double)U[v * g.pitch + c];
}

}  // namespace dfv
