// dfv_kernels_z.cuh -- the 3-D FP32 single-material stage kernel that marches
// along z (2.5-D blocking).  A CTA owns a 32 x 8 column of cells and advances
// through zc planes; the primitives of six planes (z-2 .. z+3, each with
// its x and y halo of 3, corners unused) sit in a ring in shared memory, so
// every plane is converted once per chunk instead of once per tile it halos,
// and the z-face fluxes of a column stay in its thread's registers between
// planes.  Same arithmetic per face and per cell as k_stage (Sec. 3.1).
#pragma once

#include "dfv_kernels.cuh"

namespace dfv {

struct ZGeo {
    static constexpr int TX = 32, TY = 8;                     // column tile
    static constexpr int HX = 3, HY = 3;
    static constexpr int BX = TX + 2 * HX, BY = TY + 2 * HY;  // one plane with halo
    static constexpr int SN = BX * BY;
    static constexpr int RING = 6;                            // planes z-2 .. z+3
    static constexpr int CELLS = TX * TY;
    static constexpr int THREADS = CELLS + 32;                // + a warp for the closing x faces
    static constexpr int FX = (TX + 1) * TY, FY = TX * (TY + 1);
    static constexpr int MAXF = FX > FY ? FX : FY;
};

template <class R, int NMAT>
struct ZSmem {
    using L = Lay<3, NMAT, 0>;
    static constexpr size_t floats = (size_t)ZGeo::RING * L::NVAR * ZGeo::SN + 2 * (size_t)L::NF * ZGeo::MAXF;
    static constexpr size_t bytes = ((sizeof(R) * floats + 7) & ~(size_t)7) + 4 * 32 * sizeof(double);
};

__device__ __forceinline__ int z_slot(int z) { return ((z % ZGeo::RING) + ZGeo::RING) % ZGeo::RING; }

// The conserved values of one plane (with its x, y halo) in the registers
// of the CTA's threads: fetched from global memory one plane ahead, so that
// the loads are in flight while the faces of the current plane are computed,
// then converted to primitives into a ring slot.  Boundary planes and cells
// are mapped as in the tiled kernel (mirror images behind walls).
template <class R, int NMAT>
struct ZPlane {
    static constexpr int K = (ZGeo::SN + ZGeo::THREADS - 1) / ZGeo::THREADS;   // cells per thread
    R q[K][Lay<3, NMAT, 0>::NVAR];
    unsigned flip;   // 3 bits per cell: mirrored in x, y, z
};

template <class R, int NMAT>
__device__ __forceinline__ void z_fetch_plane(const GridP &g, const R *in, ZPlane<R, NMAT> &f, int ox, int oy, int z,
                                              bool interior)
{
    using L = Lay<3, NMAT, 0>;
    using Z = ZGeo;
    bool flz = false;
    const int gz = halo_idx(g, 2, z, &flz);
    f.flip = 0u;
#pragma unroll
    for (int k = 0; k < ZPlane<R, NMAT>::K; k++) {
        const int i = threadIdx.x + k * Z::THREADS;
        if (i >= Z::SN) continue;
        const int lx = i % Z::BX - Z::HX, ly = i / Z::BX - Z::HY;
        if ((lx < 0 || lx >= Z::TX) && (ly < 0 || ly >= Z::TY)) continue;
        bool fx = false, fy = false;
        int gx = ox + lx, gy = oy + ly;
        if (!interior) {
            gx = halo_idx(g, 0, ox + lx, &fx);
            gy = halo_idx(g, 1, oy + ly, &fy);
        }
        f.flip |= ((fx ? 1u : 0u) | (fy ? 2u : 0u) | (flz ? 4u : 0u)) << (3 * k);
        const long long c = gx + (long long)g.n[0] * (gy + (long long)g.n[1] * gz);
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) f.q[k][v] = in[v * g.pitch + c];
    }
}

template <class R, int NMAT>
__device__ __forceinline__ void z_commit_plane(const GridP &g, const ZPlane<R, NMAT> &f, R *dst)
{
    using L = Lay<3, NMAT, 0>;
    using Z = ZGeo;
#pragma unroll
    for (int k = 0; k < ZPlane<R, NMAT>::K; k++) {
        const int i = threadIdx.x + k * Z::THREADS;
        if (i >= Z::SN) continue;
        const int lx = i % Z::BX - Z::HX, ly = i / Z::BX - Z::HY;
        if ((lx < 0 || lx >= Z::TX) && (ly < 0 || ly >= Z::TY)) continue;
        R w[L::NVAR];
        cons_to_prim<R, 3, NMAT, 0>(g, f.q[k], w);
#pragma unroll
        for (int d = 0; d < 3; d++)
            if ((f.flip >> (3 * k + d)) & 1u) w[L::IMOM + d] = -w[L::IMOM + d];
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) dst[v * Z::SN + i] = w[v];
    }
}

// Fluxes of the x (D = 0) or y (D = 1) faces of one plane into sF, one warp
// per face row (the warp past the last row takes the closing x faces).
template <class R, int NMAT, int D>
__device__ __forceinline__ void z_face_pass(const GridP &g, const R *pl, R *sF, R vr)
{
    using L = Lay<3, NMAT, 0>;
    using Z = ZGeo;
    constexpr int EX = Z::TX + (D == 0), EY = Z::TY + (D == 1);
    constexpr int SD = D == 0 ? 1 : Z::BX;
    constexpr int WROWS = D == 0 ? Z::TY + 1 : EY;
    for (int t = threadIdx.x; t < WROWS * 32; t += Z::THREADS) {
        const int lane = t & 31, warp = t >> 5;
        int fx, fy;
        if (D == 0 && warp >= Z::TY) {
            fy = lane;
            fx = Z::TX;
            if (fy >= Z::TY) continue;
        } else {
            fy = warp;
            fx = lane;
        }
        const int item = fy * EX + fx;
        const int bc = (fy + Z::HY) * Z::BX + (fx + Z::HX);
        R wL[L::NVAR], wR[L::NVAR];
#pragma unroll
        for (int v = 0; v < L::NVAR; v++) {
            if (v == L::IR && vr == R(0)) {
                wL[v] = wR[v] = R(0);
                continue;
            }
            R s[6];
#pragma unroll
            for (int k = 0; k < 6; k++) s[k] = pl[v * Z::SN + bc + (k - 3) * SD];
            const bool frac = (v >= L::IPHI && v < L::IPHI + NMAT - 1) || v == L::IR;
            recon_face<R>(g, s, frac, wL[v], wR[v]);
        }
        R F[L::NF];
        riemann<R, 3, NMAT, 0, D>(g, wL, wR, vr, F);
#pragma unroll
        for (int k = 0; k < L::NF; k++) sF[k * Z::MAXF + item] = F[k];
    }
}

// Flux of the z face between planes z and z+1 of the thread's column.
template <class R, int NMAT>
__device__ __forceinline__ void z_face(const GridP &g, const R *ring, int z, int lx, int ly, R vr, R *F)
{
    using L = Lay<3, NMAT, 0>;
    using Z = ZGeo;
    const int bc = (ly + Z::HY) * Z::BX + (lx + Z::HX);
    R wL[L::NVAR], wR[L::NVAR];
#pragma unroll
    for (int v = 0; v < L::NVAR; v++) {
        if (v == L::IR && vr == R(0)) {
            wL[v] = wR[v] = R(0);
            continue;
        }
        R s[6];
#pragma unroll
        for (int k = 0; k < 6; k++) s[k] = ring[((size_t)z_slot(z - 2 + k) * L::NVAR + v) * Z::SN + bc];
        const bool frac = (v >= L::IPHI && v < L::IPHI + NMAT - 1) || v == L::IR;
        recon_face<R>(g, s, frac, wL[v], wR[v]);
    }
    riemann<R, 3, NMAT, 0, 2>(g, wL, wR, vr, F);
}

// Two CTAs per SM (the ring takes 92 KB): the register bound keeps both
// resident (without it the pipelined loads push stages 1-2 to 111 registers
// and 40 % longer launches).
template <class R, int NMAT, int STAGE>
__global__ void __launch_bounds__(ZGeo::THREADS, 2) k_stage_z(StageArgs a, GridP g, int zc)
{
    pdl_enter();
    using L = Lay<3, NMAT, 0>;
    using Z = ZGeo;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *ring = reinterpret_cast<R *>(smem_raw);
    R *sFx = ring + (size_t)Z::RING * L::NVAR * Z::SN;
    R *sFy = sFx + (size_t)L::NF * Z::MAXF;
    double *sred = reinterpret_cast<double *>(smem_raw + ((sizeof(R) * ZSmem<R, NMAT>::floats + 7) & ~(size_t)7));

    const R *in = reinterpret_cast<const R *>(a.in);
    const R *un = reinterpret_cast<const R *>(a.un);
    R *out = reinterpret_cast<R *>(a.out);
    const long long P = g.pitch;
    const int ox = blockIdx.x * Z::TX, oy = blockIdx.y * Z::TY;
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.n[2]);
    const bool interior = ox >= Z::HX && ox + Z::TX + Z::HX <= g.n[0] && oy >= Z::HY && oy + Z::TY + Z::HY <= g.n[1];
    const bool own = threadIdx.x < Z::CELLS;
    const int lx = threadIdx.x % Z::TX, ly = threadIdx.x / Z::TX;
    const int gx = ox + lx, gy = oy + ly;
    const bool col = own && gx < g.n[0] && gy < g.n[1];
    const R dt = ctl_dt<R>(a.ctl);
    const R vr[3] = {ctl_v<R>(a.ctl, 0), ctl_v<R>(a.ctl, 1), ctl_v<R>(a.ctl, 2)};
    const GridC<R> &gc = gridc<R>(g);
    const R ca = STAGE == 2 ? R(0.75) : (STAGE == 3 ? R(1.0 / 3.0) : R(0));
    const R cb = STAGE == 2 ? R(0.25) : (STAGE == 3 ? R(2.0 / 3.0) : R(1));
    // the rigid box that stage 3 folds starts empty
    if (STAGE == 2 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
        ctl_box_reset(a.ctl);

    // planes z0-3 .. z0+2, plane z0+3 into registers, then the z face below
    // the first plane
    ZPlane<R, NMAT> fp;
    for (int z = z0 - 3; z <= z0 + 2; z++) {
        z_fetch_plane<R, NMAT>(g, in, fp, ox, oy, z, interior);
        z_commit_plane<R, NMAT>(g, fp, ring + (size_t)z_slot(z) * L::NVAR * Z::SN);
    }
    z_fetch_plane<R, NMAT>(g, in, fp, ox, oy, z0 + 3, interior);
    __syncthreads();
    R Flo[L::NF];
    if (col) z_face<R, NMAT>(g, ring, z0 - 1, lx, ly, vr[2], Flo);
    __syncthreads();   // plane z0-3 is read above and overwritten below

    R smax_cell = R(0);
    int zlo = 0x7fffffff, zhi = -1;     // rigid cells of the column (new state)
    for (int z = z0; z < z1; z++) {
        // plane z+3 into the slot of plane z-3, which nothing reads any more
        // (its last reader, the z face below plane z-1, is behind a barrier)
        z_commit_plane<R, NMAT>(g, fp, ring + (size_t)z_slot(z + 3) * L::NVAR * Z::SN);
        __syncthreads();
        // loads in flight during the faces: plane z+4 and the cell's own
        // stage input and step-start values
        if (z + 1 < z1) z_fetch_plane<R, NMAT>(g, in, fp, ox, oy, z + 4, interior);
        const long long c = gx + (long long)g.n[0] * (gy + (long long)g.n[1] * z);
        R cin[L::NVAR], cun[L::NVAR];
        if (col) {
#pragma unroll
            for (int v = 0; v < L::NVAR; v++) {
                cin[v] = in[v * P + c];
                cun[v] = un[v * P + c];
            }
        }
        const R *pl = ring + (size_t)z_slot(z) * L::NVAR * Z::SN;
        z_face_pass<R, NMAT, 0>(g, pl, sFx, vr[0]);
        z_face_pass<R, NMAT, 1>(g, pl, sFy, vr[1]);
        R Fhi[L::NF];
        if (col) z_face<R, NMAT>(g, ring, z, lx, ly, vr[2], Fhi);
        __syncthreads();
        if (col) {
            const int bcell = (ly + Z::HY) * Z::BX + (lx + Z::HX);
            Acc<R> Dacc[L::NVAR];
            // x, then y, then z, in the order of the tiled kernel
            {
                const int fl = ly * (Z::TX + 1) + lx, fr = fl + 1;
                const R inv = gc.inv_dx[0];
                const R dus = sFx[L::NVAR * Z::MAXF + fr] - sFx[L::NVAR * Z::MAXF + fl];
#pragma unroll
                for (int v = 0; v < L::NVAR; v++) {
                    const R div = (sFx[v * Z::MAXF + fr] - sFx[v * Z::MAXF + fl]) * inv;
                    R snc = R(0);
                    if (v >= L::IPHI && v < L::IPHI + NMAT - 1) snc = pl[v * Z::SN + bcell] * dus * inv;
                    Dacc[v].set(div - snc);
                }
            }
            {
                const int fl = ly * Z::TX + lx, fr = fl + Z::TX;
                const R inv = gc.inv_dx[1];
                const R dus = sFy[L::NVAR * Z::MAXF + fr] - sFy[L::NVAR * Z::MAXF + fl];
#pragma unroll
                for (int v = 0; v < L::NVAR; v++) {
                    const R div = (sFy[v * Z::MAXF + fr] - sFy[v * Z::MAXF + fl]) * inv;
                    R snc = R(0);
                    if (v >= L::IPHI && v < L::IPHI + NMAT - 1) snc = pl[v * Z::SN + bcell] * dus * inv;
                    Dacc[v].add(div - snc);
                }
            }
            {
                const R inv = gc.inv_dx[2];
                const R dus = Fhi[L::NVAR] - Flo[L::NVAR];
#pragma unroll
                for (int v = 0; v < L::NVAR; v++) {
                    const R div = (Fhi[v] - Flo[v]) * inv;
                    R snc = R(0);
                    if (v >= L::IPHI && v < L::IPHI + NMAT - 1) snc = pl[v * Z::SN + bcell] * dus * inv;
                    Dacc[v].add(div - snc);
                }
            }
            const bool masked = cun[L::IR] > R(0.5);
            R o[L::NVAR];
#pragma unroll
            for (int v = 0; v < L::NVAR; v++)
                o[v] = (masked && v != L::IR) ? cun[v] : rk_combine<R>(STAGE, cun[v], cin[v], Dacc[v], dt, ca, cb);
#pragma unroll
            for (int v = 0; v < L::NVAR; v++) out[v * P + c] = o[v];
            if (!(o[L::IAR] + (NMAT > 1 ? o[L::IAR + NMAT - 1] : R(0)) > R(0)) || !(o[L::IE] == o[L::IE]))
                atomicOr(&a.ctl->err, (unsigned)ERR_STATE);
            if (STAGE == 3) {
                if (o[L::IR] > R(0.5)) {
                    zlo = min(zlo, z);
                    zhi = max(zhi, z);
                }
                R w[L::NVAR];
                cons_to_prim<R, 3, NMAT, 0>(g, o, w);
                State<R, 3, NMAT, 0> s;
                state_from_prim<R, 3, NMAT, 0>(g, w, s);
                if (!(s.c2 > R(0))) atomicOr(&a.ctl->err, (unsigned)ERR_SOUND);
                const R cs = m_sqrt(s.c2);
                R sum = R(0);
#pragma unroll
                for (int d = 0; d < 3; d++) sum += (m_abs(s.u[d]) + cs) / gc.dx[d];
                smax_cell = m_max(smax_cell, sum);
            }
#pragma unroll
            for (int k = 0; k < L::NF; k++) Flo[k] = Fhi[k];
        }
    }
    if (STAGE == 3) {
        // the column's rigid cells into the box of the next seeding, the
        // chunk's CFL maximum into the launch's running maximum
        const bool rig = zhi >= 0;
        if (__any_sync(0xffffffffu, rig)) {
            const int big = 0x7fffffff;
            const int b[6] = {rig ? gx : big, rig ? gy : big, rig ? zlo : big, rig ? gx : -1, rig ? gy : -1,
                              rig ? zhi : -1};
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
        R *sr = reinterpret_cast<R *>(sred);
        const R mx = block_max<Z::THREADS, R>(smax_cell, sr);
        if (threadIdx.x == 0) {
            double md = (double)mx;
            if (!(md >= 0.0)) md = __longlong_as_double(0x7ff0000000000000LL);   // NaN -> +inf: dt = 0
            atomicMax(&a.ctl->smax_acc, (unsigned long long)__double_as_longlong(md));
        }
    }
}

}  // namespace dfv
