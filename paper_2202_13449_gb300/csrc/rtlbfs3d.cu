// rtlbfs3d.cu -- the fused 3D RTLBFS time step on sm_103a (arXiv
// 2202.13449, Section 3.2 with the D3Q19 lattice; Section 4.4), its FP64
// Nusselt reductions and the rtlbfs3d_* C ABI.
//
// Step kernel.  Work unit: a TX x TY tile of columns of one mesh and a chunk
// of z-planes [k0, k1); one thread per column.  The block marches up the
// chunk with a rolling window in shared memory -- the values of planes k,
// k+1, k+2 on the tile plus a 2-cell ring, the Green-Gauss gradients of
// planes k and k+1 on a 1-cell ring -- and per plane:
//   loads plane k+2 (ghost rules applied: mirror at walls, wrap when
//     periodic),
//   the gradients of plane k+1 (Eqs. 55-56; a z-wall ghost plane mirrors its
//     neighbour's),
//   every x- and y-face of plane k into shared memory and the z-face between
//     planes k and k+1 into registers -- face_flux3: D3Q19 nodes (Eq. 29),
//     predictor (Eqs. 46-48), corrector fluxes (Eqs. 57-59),
//   the update of plane k with the Boussinesq source (Eq. 64) and the
//     residual sums; the z-face below the next plane is the one just made.
// The last unit to finish a step turns the sums into (R_u, R_T), advances
// the step counter, flips the state buffer and decides whether the run is
// done, so launches need no host round trip.  HBM sees one read and one
// write of the five fields per cell (halo re-reads hit L2).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "rtlbfs.h"
#include "rtlbfs3d.h"
#include "rtlbfs3d_dev.cuh"
#include "rtlbfs_dev.cuh"
#include "rtlbfs_kernels.h"

namespace rtlbfs {
extern std::atomic<long long> g_launches;
}

namespace rtlbfs3 {

using rtlbfs::CellLine;
using rtlbfs::chain_sync;
using rtlbfs::launch_chained;
using rtlbfs::kAdiabatic;
using rtlbfs::kConverged;
using rtlbfs::kDiverged;
using rtlbfs::kDirichlet;
using rtlbfs::kMaxSteps;
using rtlbfs::kPeriodic;
using rtlbfs::kRunning;
using rtlbfs::StoreD;
using rtlbfs::StoreQ;
using rtlbfs::Vec4;

// fixed-point kind of field q (rho - 1, u, v, w, T): 0 density, 1 velocity, 3 temperature
__host__ __device__ constexpr int kind_of(int q) { return q == 0 ? 0 : (q == 4 ? 3 : 1); }

// Read-only description of one mesh on the device.
struct Desc3 {
    int n[3];
    int kind[6];
    int g_axis;
    int tiles_x, tiles_y, chunks, kchunk, units;
    double beta_g, T_ref, dt, force[3];
    float f_beta_g, f_T_ref, f_dt, f_force[3];
    double bcU[6][3], bcT[6];
    float f_bcU[6][3], f_bcT[6];
    void* rec[2];                // Vec4<S>[cells]: (rho - 1, u, v, w)
    void* tem[2];                // S[cells]: T
    const void* fline[3];        // FaceLine<R>[n[a] + 1]
    const void* cline[3];        // CellLine<R>[n[a] + 4], index c + 2 for c in [-2, n+1]
    const void* fline_d[3];      // FP64 copies for the Nusselt sums
    const void* cline_d[3];
};

// Run control: the two-header record of the 2D solver (the stop test of
// step k is made by the launch of step k + 1; see CavityRun).
using rtlbfs::CavityCtl;
using rtlbfs::CavityRun;

// Constants of a mesh in the arithmetic type R and mirror constants in the
// storage type S of a policy.
template <class P>
struct Cst;
template <>
struct Cst<StoreD> {
    static __device__ __forceinline__ double beta_g(const Desc3& d) { return d.beta_g; }
    static __device__ __forceinline__ double T_ref(const Desc3& d) { return d.T_ref; }
    static __device__ __forceinline__ double dt(const Desc3& d) { return d.dt; }
    static __device__ __forceinline__ double force(const Desc3& d, int a) { return d.force[a]; }
    static __device__ __forceinline__ double uw(const Desc3& d, int s, int c) { return d.bcU[s][c]; }
    static __device__ __forceinline__ double Tw(const Desc3& d, int s) { return d.bcT[s]; }
};
template <>
struct Cst<StoreQ> {
    static __device__ __forceinline__ float beta_g(const Desc3& d) { return d.f_beta_g; }
    static __device__ __forceinline__ float T_ref(const Desc3& d) { return d.f_T_ref; }
    static __device__ __forceinline__ float dt(const Desc3& d) { return d.f_dt; }
    static __device__ __forceinline__ float force(const Desc3& d, int a) { return d.f_force[a]; }
    static __device__ __forceinline__ float uw(const Desc3& d, int s, int c) { return d.f_bcU[s][c]; }
    static __device__ __forceinline__ float Tw(const Desc3& d, int s) { return d.f_bcT[s]; }
};

// Source index of coordinate c on an axis of n cells: wrap when periodic;
// the ghost at -1 / n mirrors cell 0 / n-1 across side lo / hi (mside set);
// anything else outside is never used (false).
__host__ __device__ __forceinline__ bool resolve_1d(int c, int n, bool per, int lo, int hi,
                                                    int& src, int& mside)
{
    mside = -1;
    src = c;
    if (c >= 0 && c < n) return true;
    if (per) {
        src = ((c % n) + n) % n;
        return true;
    }
    if (c == -1) {
        src = 0;
        mside = lo;
        return true;
    }
    if (c == n) {
        src = n - 1;
        mside = hi;
        return true;
    }
    return false;
}

// Ghost values across wall `side` from the partner's working values o =
// (rho - 1, u, v, w, T - Tref): rho even, velocity odd about the wall
// velocity (its normal part is 0), T odd about T_wall on a Dirichlet wall and
// even on an adiabatic one.  Formed in the arithmetic type relative to Tref:
// 2 T_wall - T_P can leave the fixed-point range of a stored temperature (a
// hot wall next to cold fluid) while its deviation from a temperature inside
// the unit does not.
template <class P, typename R>
__device__ __forceinline__ void mirror_values3(const Desc3& d, int side, R Tref, R o[5])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) o[1 + c] = R(2) * Cst<P>::uw(d, side, c) - o[1 + c];
    if (d.kind[side] == kDirichlet) o[4] = R(2) * (Cst<P>::Tw(d, side) - Tref) - o[4];
}

// Sign of gradient component (q, dir) of a ghost across a wall normal to
// axis `ax`: even quantities negate the normal component, odd ones the
// tangential components.
__host__ __device__ __forceinline__ bool grad_flips(int kind, int ax, int q, int dir)
{
    const bool even = q == 0 || (q == 4 && kind != kDirichlet);
    return even == (dir == ax);
}

template <class P, int TX, int TY>
struct Smem3 {
    using R = typename P::R;
    static constexpr int BX = TX + 4, BY = TY + 4, GX = TX + 2, GY = TY + 2, NT = TX * TY;
    R v[3][5][BY][BX];      // (rho - 1, u, v, w, T - Tz) of planes, 2-cell ring
    R g[2][15][GY][GX];     // gradients [q*3 + dir] of planes, 1-cell ring
    R fx[5][TY][TX + 1];    // x-face fluxes of the current plane (global components)
    R fy[5][TY + 1][TX];
    // line constants, one array per field: consecutive threads read
    // consecutive words (an array of the 32-byte structs would put 8 threads
    // on one bank)
    R xl[7][TX + 1];        // FaceLine fields h, cL, cR, m_nu_2h, m_chi_2h, m_tf15, m_tg15
    R yl[7][TY + 1];
    R xisn[BX], xdtw[BX];   // CellLine is_next, dt_w of the ringed tile
    R yisn[BY], ydtw[BY];
    double red[NT / 32][4];
    int plan[3];  // after the stop test: done, cur, sum slot
};

// FaceLine from its per-field arrays
template <typename R, int N>
__device__ __forceinline__ FaceLine<R> get_line(const R (&a)[7][N], int i)
{
    FaceLine<R> f;
    f.h = a[0][i];
    f.cL = a[1][i];
    f.cR = a[2][i];
    f.m_nu_2h = a[3][i];
    f.m_chi_2h = a[4][i];
    f.m_tf15 = a[5][i];
    f.m_tg15 = a[6][i];
    f.pad = R(0);
    return f;
}

template <typename R, int N>
__device__ __forceinline__ void set_line(R (&a)[7][N], int i, const FaceLine<R>& f)
{
    a[0][i] = f.h;
    a[1][i] = f.cL;
    a[2][i] = f.cR;
    a[3][i] = f.m_nu_2h;
    a[4][i] = f.m_chi_2h;
    a[5][i] = f.m_tf15;
    a[6][i] = f.m_tg15;
}

__host__ __device__ constexpr int mod3(int k) { return ((k % 3) + 3) % 3; }
__host__ __device__ constexpr int mod2(int k) { return ((k % 2) + 2) % 2; }

// Cells of a face in its frame (n, t1, t2) from the stored-plane layout:
// frame component f of axis-normal `ax` is global component (ax + f) % 3.
template <typename R, typename Sm>
__device__ __forceinline__ void take3(const Sm& sm, int vs, int gs, int r, int c, int ax,
                                      CellNT3<R>& o, R& tau)
{
    const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
    o.q[0] = sm.v[vs][0][r][c];
    o.q[1] = sm.v[vs][1 + ax][r][c];
    o.q[2] = sm.v[vs][1 + a1][r][c];
    o.q[3] = sm.v[vs][1 + a2][r][c];
    tau = sm.v[vs][4][r][c];
    o.q[4] = tau;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int gq = q == 0 ? 0 : (q == 4 ? 4 : 1 + (ax + q - 1) % 3);
        o.gn[q] = sm.g[gs][gq * 3 + ax][r - 1][c - 1];
        o.g1[q] = sm.g[gs][gq * 3 + a1][r - 1][c - 1];
        o.g2[q] = sm.g[gs][gq * 3 + a2][r - 1][c - 1];
    }
}

// One face between cells L and R (frame of axis ax) with face stage SCH
// (0 RTLBFS, 1 TLBFS), the fluxes in the face frame: F = (mass, n-, t1-,
// t2-momentum, energy), t1 = axis (ax + 1) % 3, t2 = (ax + 2) % 3.  Tz is the
// unit's temperature reference; the face reference is the left cell's
// temperature.
template <class P, typename R, int SCH>
__device__ __forceinline__ void face3_frame(const Desc3& d, CellNT3<R>& L, R tauL,
                                            CellNT3<R>& Rc, R tauR, const FaceLine<R>& fl, R Tz,
                                            int ax, int wside, R F[5])
{
    L.q[4] = R(0);
    Rc.q[4] = tauR - tauL;
    const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
    const R keep = wside >= 0 ? R(0) : R(1);
    const R uw1 = wside >= 0 ? Cst<P>::uw(d, wside, a1) : R(0);
    const R uw2 = wside >= 0 ? Cst<P>::uw(d, wside, a2) : R(0);
    if constexpr (SCH == 1) {
        face_flux3_tlbfs<R>(L, Rc, Tz + tauL, fl, keep, uw1, uw2, F);
    } else if constexpr (sizeof(R) == 4) {  // FP32: the node stage in packed pairs
        R O[5], Pn[3][2][5], En[3][4][5];
        face3_nodes_f32(L, Rc, fl, O, Pn, En);
        face_flux3_nodes<R>(O, Pn, En, Tz + tauL, fl, keep, uw1, uw2, F);
    } else {
        face_flux3<R>(L, Rc, Tz + tauL, fl, keep, uw1, uw2, F);
    }
}

// The same with the fluxes in global components (rho, x, y, z, T).
template <class P, typename R, int SCH>
__device__ __forceinline__ void face3(const Desc3& d, CellNT3<R>& L, R tauL, CellNT3<R>& Rc,
                                      R tauR, const FaceLine<R>& fl, R Tz, int ax, int wside,
                                      R out[5])
{
    R F[5];
    face3_frame<P, R, SCH>(d, L, tauL, Rc, tauR, fl, Tz, ax, wside, F);
    const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
    out[0] = F[0];
    out[1 + ax] = F[1];
    out[1 + a1] = F[2];
    out[1 + a2] = F[3];
    out[4] = F[4];
}

template <class P, int TX, int TY, int SCH>
__global__ void __launch_bounds__(TX* TY) step3_kernel(const Desc3* __restrict__ dp,
                                                       CavityRun* __restrict__ run, int par)
{
    using S = typename P::S;
    using R = typename P::R;
    using Sm = Smem3<P, TX, TY>;
    constexpr int BX = Sm::BX, BY = Sm::BY, GX = Sm::GX, GY = Sm::GY, NT = Sm::NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    Sm& sm = *reinterpret_cast<Sm*>(smraw);

    chain_sync();
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    // the stop test of the previous step (thread 0; unit 0 publishes the
    // header for the next launch)
    if (tid == 0) {
        const CavityCtl dc = rtlbfs::run_head(run, par);
        if (blockIdx.x == 0) rtlbfs::run_publish(run, par, dc);
        sm.plan[0] = dc.done;
        sm.plan[1] = dc.cur;
        sm.plan[2] = (int)(dc.steps % 3);
    }
    __syncthreads();
    if (sm.plan[0]) return;  // uniform
    const int slot3 = sm.plan[2];
    const Desc3& d = *dp;
    const int nx = d.n[0], ny = d.n[1], nz = d.n[2];
    int u = blockIdx.x;
    const int tix = u % d.tiles_x;
    u /= d.tiles_x;
    const int tiy = u % d.tiles_y;
    const int ch = u / d.tiles_y;
    const int i0 = tix * TX, j0 = tiy * TY, k0 = ch * d.kchunk, k1 = min(nz, k0 + d.kchunk);
    const bool xper = d.kind[0] == kPeriodic, yper = d.kind[2] == kPeriodic;
    const bool zper = d.kind[4] == kPeriodic;
    const int cur = sm.plan[1];
    const Vec4<S>* __restrict__ rin = static_cast<const Vec4<S>*>(d.rec[cur]);
    const S* __restrict__ tin = static_cast<const S*>(d.tem[cur]);
    Vec4<S>* __restrict__ rout = static_cast<Vec4<S>*>(d.rec[cur ^ 1]);
    S* __restrict__ tout = static_cast<S*>(d.tem[cur ^ 1]);
    const FaceLine<R>* zl = static_cast<const FaceLine<R>*>(d.fline[2]);
    const CellLine<R>* zc = static_cast<const CellLine<R>*>(d.cline[2]);
    {
        const FaceLine<R>* xl = static_cast<const FaceLine<R>*>(d.fline[0]);
        const FaceLine<R>* yl = static_cast<const FaceLine<R>*>(d.fline[1]);
        const CellLine<R>* xc = static_cast<const CellLine<R>*>(d.cline[0]);
        const CellLine<R>* yc = static_cast<const CellLine<R>*>(d.cline[1]);
        for (int t = tid; t < TX + 1; t += NT) set_line(sm.xl, t, xl[min(i0 + t, nx)]);
        for (int t = tid; t < TY + 1; t += NT) set_line(sm.yl, t, yl[min(j0 + t, ny)]);
        for (int t = tid; t < BX; t += NT) {
            const CellLine<R> c = xc[min(i0 + t, nx + 3)];
            sm.xisn[t] = c.is_next;
            sm.xdtw[t] = c.dt_w;
        }
        for (int t = tid; t < BY; t += NT) {
            const CellLine<R> c = yc[min(j0 + t, ny + 3)];
            sm.yisn[t] = c.is_next;
            sm.ydtw[t] = c.dt_w;
        }
    }
    // temperature reference of this unit: one stored cell value
    const S qTz = tin[((size_t)k0 * ny + min(j0 + TY / 2, ny - 1)) * nx + min(i0 + TX / 2, nx - 1)];
    const R Tz = P::val(qTz, 3);

    // plane kk (ghosts included) into value slot mod3(kk), 2-cell ring
    auto load_plane = [&](int kk) {
        const int vs = mod3(kk);
        int ks, zs;
        const bool zok = resolve_1d(kk, nz, zper, 4, 5, ks, zs);
        for (int t = tid; t < BX * BY; t += NT) {
            const int r = t / BX, c = t % BX;
            int is, xs, js, ys;
            const bool xok = resolve_1d(i0 - 2 + c, nx, xper, 0, 1, is, xs);
            const bool yok = resolve_1d(j0 - 2 + r, ny, yper, 2, 3, js, ys);
            const int nm = (xs >= 0) + (ys >= 0) + (zs >= 0);
            R o[5] = {R(0), R(0), R(0), R(0), R(0)};
            if (zok && xok && yok && nm <= 1) {
                const size_t off = ((size_t)ks * ny + js) * nx + is;
                const Vec4<S> a = rin[off];
                o[0] = P::val(a.x, 0);
                o[1] = P::val(a.y, 1);
                o[2] = P::val(a.z, 1);
                o[3] = P::val(a.w, 1);
                o[4] = P::diff(tin[off], qTz, 3);
                const int ms = xs >= 0 ? xs : (ys >= 0 ? ys : zs);
                if (ms >= 0) mirror_values3<P, R>(d, ms, Tz, o);
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) sm.v[vs][q][r][c] = o[q];
        }
    };

    // gradients of plane kk into gradient slot mod2(kk), 1-cell ring; a
    // z-wall ghost plane mirrors the other slot (its neighbour plane)
    auto grad_plane = [&](int kk) {
        const int gs = mod2(kk);
        int ks, zs;
        resolve_1d(kk, nz, zper, 4, 5, ks, zs);
        if (zs >= 0) {
            const int kind = d.kind[zs];
            for (int t = tid; t < GX * GY; t += NT) {
                const int r = t / GX, c = t % GX;
#pragma unroll
                for (int q = 0; q < 5; ++q)
#pragma unroll
                    for (int dir = 0; dir < 3; ++dir) {
                        const R g = sm.g[gs ^ 1][q * 3 + dir][r][c];
                        sm.g[gs][q * 3 + dir][r][c] = grad_flips(kind, 2, q, dir) ? -g : g;
                    }
            }
            return;
        }
        const int vs = mod3(kk), vm = mod3(kk - 1), vp = mod3(kk + 1);
        const R izn = zc[kk + 2].is_next, izm = zc[kk + 1].is_next;
        for (int t = tid; t < GX * GY; t += NT) {
            const int r = t / GX + 1, c = t % GX + 1;
            int is, xs, js, ys;
            const bool xok = resolve_1d(i0 - 2 + c, nx, xper, 0, 1, is, xs);
            const bool yok = resolve_1d(j0 - 2 + r, ny, yper, 2, 3, js, ys);
            R g[15];
#pragma unroll
            for (int e = 0; e < 15; ++e) g[e] = R(0);
            if (xok && yok && !(xs >= 0 && ys >= 0)) {
                int pr = r, pc = c, ms = -1;
                if (xs >= 0) {
                    pc = xs == 0 ? c + 1 : c - 1;
                    ms = xs;
                }
                if (ys >= 0) {
                    pr = ys == 2 ? r + 1 : r - 1;
                    ms = ys;
                }
                const R ixn = sm.xisn[pc], ixm = sm.xisn[pc - 1];
                const R iyn = sm.yisn[pr], iym = sm.yisn[pr - 1];
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    const R vc = sm.v[vs][q][pr][pc];
                    g[q * 3 + 0] = (sm.v[vs][q][pr][pc + 1] - vc) * ixn + (vc - sm.v[vs][q][pr][pc - 1]) * ixm;
                    g[q * 3 + 1] = (sm.v[vs][q][pr + 1][pc] - vc) * iyn + (vc - sm.v[vs][q][pr - 1][pc]) * iym;
                    g[q * 3 + 2] = (sm.v[vp][q][pr][pc] - vc) * izn + (vc - sm.v[vm][q][pr][pc]) * izm;
                }
                if (ms >= 0) {
                    const int kind = d.kind[ms], ax = ms / 2;
#pragma unroll
                    for (int q = 0; q < 5; ++q)
#pragma unroll
                        for (int dir = 0; dir < 3; ++dir)
                            if (grad_flips(kind, ax, q, dir)) g[q * 3 + dir] = -g[q * 3 + dir];
                }
            }
#pragma unroll
            for (int e = 0; e < 15; ++e) sm.g[gs][e][r - 1][c - 1] = g[e];
        }
    };

    // z-face between planes kk and kk+1 of this thread's column
    const int gi = i0 + tx, gj = j0 + ty;
    const bool mine = gi < nx && gj < ny;
    auto zface = [&](int kk, R out[5]) {
        CellNT3<R> L, Rr;
        R tl, tr;
        take3<R>(sm, mod3(kk), mod2(kk), ty + 2, tx + 2, 2, L, tl);
        take3<R>(sm, mod3(kk + 1), mod2(kk + 1), ty + 2, tx + 2, 2, Rr, tr);
        const int ws = zper ? -1 : (kk + 1 == 0 ? 4 : (kk + 1 == nz ? 5 : -1));
        face3<P, R, SCH>(d, L, tl, Rr, tr, zl[kk + 1], Tz, 2, ws, out);
    };

    // ---- prologue: planes k0-2 .. k0+1, gradients of k0-1 and k0, the
    //      z-face below plane k0
    int ks_, zsm;
    resolve_1d(k0 - 1, nz, zper, 4, 5, ks_, zsm);
    const bool below_is_wall = zsm >= 0;
    load_plane(k0 - 2);
    load_plane(k0 - 1);
    load_plane(k0);
    __syncthreads();
    if (!below_is_wall) grad_plane(k0 - 1);
    __syncthreads();
    load_plane(k0 + 1);
    __syncthreads();
    grad_plane(k0);
    __syncthreads();
    if (below_is_wall) {
        grad_plane(k0 - 1);
        __syncthreads();
    }
    R Fd[5] = {R(0), R(0), R(0), R(0), R(0)};
    if (mine) zface(k0 - 1, Fd);
    __syncthreads();

    R s0 = R(0), s1 = R(0), s2 = R(0), s3 = R(0);  // residual partials in the working precision
    bool bad = false;
    for (int k = k0; k < k1; ++k) {
        load_plane(k + 2);
        __syncthreads();
        grad_plane(k + 1);
        __syncthreads();
        // x- and y-faces of plane k
        const int vs = mod3(k), gs = mod2(k);
        constexpr int NXF = TY * (TX + 1), NYF = (TY + 1) * TX;
        if constexpr (sizeof(R) == 4) {
            // FP32: one loop (face t < NXF an x-face, else a y-face), so the
            // face arithmetic is one copy of code and a thread's rounds cover
            // both kinds; the fluxes come back in the face frame and are
            // stored to their global components.  (FP64 keeps two loops: the
            // shared copy would raise its registers past three blocks per SM.)
            for (int t = tid; t < NXF + NYF; t += NT) {
                const bool isx = t < NXF;
                const int u = isx ? t : t - NXF;
                const int fj = isx ? u / (TX + 1) : u / TX, fi = isx ? u % (TX + 1) : u % TX;
                const int g = isx ? i0 + fi : j0 + fj;  // the face's index along its normal
                if (isx ? (g > nx || j0 + fj >= ny) : (g > ny || i0 + fi >= nx)) continue;
                const int ax = isx ? 0 : 1;
                CellNT3<R> L, Rr;
                R tl, tr;
                take3<R>(sm, vs, gs, isx ? fj + 2 : fj + 1, isx ? fi + 1 : fi + 2, ax, L, tl);
                take3<R>(sm, vs, gs, fj + 2, fi + 2, ax, Rr, tr);
                const bool per = isx ? xper : yper;
                const int n_ax = isx ? nx : ny;
                const int ws = per ? -1 : (g == 0 ? 2 * ax : (g == n_ax ? 2 * ax + 1 : -1));
                R F[5];
                face3_frame<P, R, SCH>(d, L, tl, Rr, tr,
                                       isx ? get_line(sm.xl, fi) : get_line(sm.yl, fj), Tz, ax,
                                       ws, F);
                // frame (rho, n, t1, t2, T) to global (rho, x, y, z, T): x-face
                // n = x, t1 = y, t2 = z; y-face n = y, t1 = z, t2 = x
                R* dst = isx ? &sm.fx[0][fj][fi] : &sm.fy[0][fj][fi];
                const int qs = isx ? NXF : NYF;  // stride between components
                dst[0] = F[0];
                dst[(isx ? 1 : 2) * qs] = F[1];
                dst[(isx ? 2 : 3) * qs] = F[2];
                dst[(isx ? 3 : 1) * qs] = F[3];
                dst[4 * qs] = F[4];
            }
        } else {
            for (int t = tid; t < NXF; t += NT) {
                const int fj = t / (TX + 1), fi = t % (TX + 1);
                const int gx = i0 + fi;
                if (gx > nx || j0 + fj >= ny) continue;
                CellNT3<R> L, Rr;
                R tl, tr;
                take3<R>(sm, vs, gs, fj + 2, fi + 1, 0, L, tl);
                take3<R>(sm, vs, gs, fj + 2, fi + 2, 0, Rr, tr);
                const int ws = xper ? -1 : (gx == 0 ? 0 : (gx == nx ? 1 : -1));
                R F[5];
                face3<P, R, SCH>(d, L, tl, Rr, tr, get_line(sm.xl, fi), Tz, 0, ws, F);
#pragma unroll
                for (int q = 0; q < 5; ++q) sm.fx[q][fj][fi] = F[q];
            }
            for (int t = tid; t < NYF; t += NT) {
                const int fj = t / TX, fi = t % TX;
                const int gy = j0 + fj;
                if (gy > ny || i0 + fi >= nx) continue;
                CellNT3<R> L, Rr;
                R tl, tr;
                take3<R>(sm, vs, gs, fj + 1, fi + 2, 1, L, tl);
                take3<R>(sm, vs, gs, fj + 2, fi + 2, 1, Rr, tr);
                const int ws = yper ? -1 : (gy == 0 ? 2 : (gy == ny ? 3 : -1));
                R F[5];
                face3<P, R, SCH>(d, L, tl, Rr, tr, get_line(sm.yl, fj), Tz, 1, ws, F);
#pragma unroll
                for (int q = 0; q < 5; ++q) sm.fy[q][fj][fi] = F[q];
            }
        }
        R Fu[5] = {R(0), R(0), R(0), R(0), R(0)};
        R c0[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) c0[q] = sm.v[vs][q][ty + 2][tx + 2];
        if (mine) zface(k, Fu);
        __syncthreads();
        if (mine) {
            const R one = R(1);
            const R ax = sm.xdtw[tx + 2], ay = sm.ydtw[ty + 2], az = zc[k + 2].dt_w;
            R div[5];
#pragma unroll
            for (int q = 0; q < 5; ++q)
                div[q] = ax * (sm.fx[q][ty][tx + 1] - sm.fx[q][ty][tx]) +
                         ay * (sm.fy[q][ty + 1][tx] - sm.fy[q][ty][tx]) + az * (Fu[q] - Fd[q]);
            const R dr = c0[0], T = Tz + c0[4];
            const R rho = one + dr;
            const R dtc = Cst<P>::dt(d);
            R src[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) src[a] = rho * Cst<P>::force(d, a);
            src[d.g_axis] = vfma(rho * Cst<P>::beta_g(d), T - Cst<P>::T_ref(d), src[d.g_axis]);
            const R inv = P::rcp(rho - div[0]);
            R du[3], u1[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                du[a] = (c0[1 + a] * div[0] - div[1 + a] + dtc * src[a]) * inv;
                u1[a] = c0[1 + a] + du[a];
            }
            const R dT = (T * div[0] - div[4]) * inv;
            const R T1 = T + dT, dr1 = dr - div[0];
            const size_t off = ((size_t)k * ny + gj) * nx + gi;
            const Vec4<S> qo = rin[off];
            const S qT = tin[off];
            rout[off] = {P::add(qo.x, -div[0], 0), P::add(qo.y, du[0], 1), P::add(qo.z, du[1], 1),
                         P::add(qo.w, du[2], 1)};
            tout[off] = P::add(qT, dT, 3);
            bad = bad || !(P::in_range(dr1, 0) && P::in_range(u1[0], 1) && P::in_range(u1[1], 1) &&
                           P::in_range(u1[2], 1) && P::in_range(T1, 3));
            const R m0 = P::fsqrt(c0[1] * c0[1] + c0[2] * c0[2] + c0[3] * c0[3]);
            const R m1 = P::fsqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
            const R den = m0 + m1;
            const R dm = den > R(0)
                             ? (du[0] * (c0[1] + u1[0]) + du[1] * (c0[2] + u1[1]) + du[2] * (c0[3] + u1[2])) *
                                   P::rcp(den)
                             : R(0);
            s0 += dm * dm;
            s1 += m1 * m1;
            s2 += dT * dT;
            s3 += T1 * T1;
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) Fd[q] = Fu[q];
    }
    if (bad) s0 = R(NAN);
    // residual sums: warp sums in the working precision, warps and units in FP64
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    }
    if ((tid & 31) == 0) {
        sm.red[tid >> 5][0] = (double)s0;
        sm.red[tid >> 5][1] = (double)s1;
        sm.red[tid >> 5][2] = (double)s2;
        sm.red[tid >> 5][3] = (double)s3;
    }
    __syncthreads();
    if (tid == 0) {
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < NT / 32; ++w)
            for (int q = 0; q < 4; ++q) a[q] += sm.red[w][q];
        // the step's residual sums; the next launch tests them
        for (int q = 0; q < 4; ++q) atomicAdd(&run->acc[slot3][q], a[q]);
    }
}

// ---------------------------------------------------------------------------
// FP64 Nusselt sums: one thread per face of a wall (or of the x mid-plane),
// cells and gradients read straight from the state with the ghost rules.
// ---------------------------------------------------------------------------

// value and Green-Gauss gradient of cell (c[0], c[1], c[2]), ghosts
// included (a wall ghost mirrors its partner), as doubles; T absolute
template <class P>
__device__ void cell_at(const Desc3& d, const typename P::S* tin,
                        const Vec4<typename P::S>* rin, const int c[3], double q[5], double g[5][3])
{
    using S = typename P::S;
    const bool per[3] = {d.kind[0] == kPeriodic, d.kind[2] == kPeriodic, d.kind[4] == kPeriodic};
    // the cell itself, or the partner a wall ghost mirrors (ms: its side)
    int p[3];
    int ms = -1;
    for (int a = 0; a < 3; ++a) {
        int side;
        resolve_1d(c[a], d.n[a], per[a], 2 * a, 2 * a + 1, p[a], side);
        if (side >= 0) ms = side;
    }
    // stored values of a cell next to p (at most one wall ghost), as doubles
    auto fetch = [&](const int cc[3], double o[5]) {
        int s[3], side = -1;
        for (int a = 0; a < 3; ++a) {
            int sd;
            resolve_1d(cc[a], d.n[a], per[a], 2 * a, 2 * a + 1, s[a], sd);
            if (sd >= 0) side = sd;
        }
        const size_t off = ((size_t)s[2] * d.n[1] + s[1]) * d.n[0] + s[0];
        const Vec4<S> r = rin[off];
        const S qq[5] = {r.x, r.y, r.z, r.w, tin[off]};
        for (int k = 0; k < 5; ++k) o[k] = P::to_double(qq[k], kind_of(k));
        if (side >= 0) mirror_values3<StoreD, double>(d, side, 0.0, o);  // FP64, T absolute
    };
    double qc[5];
    fetch(p, qc);
    // Eqs. 55-56 at p
    for (int a = 0; a < 3; ++a) {
        const CellLine<double>* cl = static_cast<const CellLine<double>*>(d.cline_d[a]);
        int pp[3] = {p[0], p[1], p[2]}, pm[3] = {p[0], p[1], p[2]};
        pp[a] += 1;
        pm[a] -= 1;
        double qp[5], qm[5];
        fetch(pp, qp);
        fetch(pm, qm);
        const double in = cl[p[a] + 2].is_next, im = cl[p[a] + 1].is_next;
        for (int k = 0; k < 5; ++k) g[k][a] = (qp[k] - qc[k]) * in + (qc[k] - qm[k]) * im;
    }
    if (ms < 0) {
        for (int k = 0; k < 5; ++k) q[k] = qc[k];
        return;
    }
    // a wall ghost: the mirrored values of its partner and mirrored gradient
    for (int k = 0; k < 5; ++k) q[k] = qc[k];
    mirror_values3<StoreD, double>(d, ms, 0.0, q);
    const int kind = d.kind[ms], ax = ms / 2;
    for (int k = 0; k < 5; ++k)
        for (int a = 0; a < 3; ++a)
            if (grad_flips(kind, ax, k, a)) g[k][a] = -g[k][a];
}

// Sum over the faces normal to axis `ax` at face index `pos` with the
// tangential index of axis b1 restricted to [t1lo, t1hi): flux F_E times
// face area (times wgt), into *acc.
template <class P, int SCH>
__global__ void nusselt3_kernel(const Desc3* __restrict__ dp, int cur, int ax, int pos, int t1lo,
                                int t1hi, int wside, double wgt, double* acc)
{
    using S = typename P::S;
    const Desc3& d = *dp;
    const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
    const int n1 = t1hi - t1lo, n2 = d.n[b2];
    const long long nf = (long long)n1 * n2;
    double s = 0.0;
    const Vec4<S>* rin = static_cast<const Vec4<S>*>(d.rec[cur]);
    const S* tin = static_cast<const S*>(d.tem[cur]);
    const CellLine<double>* c1 = static_cast<const CellLine<double>*>(d.cline_d[b1]);
    const CellLine<double>* c2 = static_cast<const CellLine<double>*>(d.cline_d[b2]);
    const FaceLine<double>* fl = static_cast<const FaceLine<double>*>(d.fline_d[ax]);
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf;
         f += (long long)gridDim.x * blockDim.x) {
        const int t1 = t1lo + (int)(f % n1), t2 = (int)(f / n1);
        int cr[3], cl[3];
        cr[ax] = pos;
        cr[b1] = t1;
        cr[b2] = t2;
        cl[ax] = pos - 1;
        cl[b1] = t1;
        cl[b2] = t2;
        double qL[5], gL[5][3], qR[5], gR[5][3];
        cell_at<P>(d, tin, rin, cl, qL, gL);
        cell_at<P>(d, tin, rin, cr, qR, gR);
        CellNT3<double> L, Rr;
        const int comp[5] = {0, 1 + ax, 1 + b1, 1 + b2, 4};
        for (int k = 0; k < 5; ++k) {
            const int qk = comp[k];
            L.q[k] = qL[qk];
            Rr.q[k] = qR[qk];
            L.gn[k] = gL[qk][ax];
            L.g1[k] = gL[qk][b1];
            L.g2[k] = gL[qk][b2];
            Rr.gn[k] = gR[qk][ax];
            Rr.g1[k] = gR[qk][b1];
            Rr.g2[k] = gR[qk][b2];
        }
        const double Tbar = qL[4];
        L.q[4] = 0.0;
        Rr.q[4] = qR[4] - qL[4];
        const double keep = wside >= 0 ? 0.0 : 1.0;
        const double uw1 = wside >= 0 ? d.bcU[wside][b1] : 0.0;
        const double uw2 = wside >= 0 ? d.bcU[wside][b2] : 0.0;
        double F[5];
        if (SCH == 1)
            face_flux3_tlbfs<double>(L, Rr, Tbar, fl[pos], keep, uw1, uw2, F);
        else
            face_flux3<double>(L, Rr, Tbar, fl[pos], keep, uw1, uw2, F);
        s += F[4] * c1[t1 + 2].w * c2[t2 + 2].w;
    }
    s *= wgt;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

constexpr int kTiles[3][2] = {{32, 4}, {16, 8}, {32, 8}};
constexpr int kGraphSteps = 32;

double line_width(const std::vector<double>& f, int i, bool periodic)
{
    const int n = (int)f.size() - 1;
    int k = i;
    if (periodic) {
        k = ((i % n) + n) % n;
    } else {
        if (i < 0) k = -1 - i;
        if (i >= n) k = 2 * n - 1 - i;
        k = std::min(std::max(k, 0), n - 1);
    }
    return f[k + 1] - f[k];
}

template <typename R>
void build_lines(const std::vector<double>& f, bool periodic, double kappa, double nu, double chi,
                 double dt, std::vector<FaceLine<R>>& fl, std::vector<CellLine<R>>& cl)
{
    const int n = (int)f.size() - 1;
    fl.resize(n + 1);
    for (int i = 0; i <= n; ++i) {
        const double wl = line_width(f, i - 1, periodic), wr = line_width(f, i, periodic);
        const double h = kappa * std::min(wl, wr);
        FaceLine<R> x;
        x.h = (R)h;
        x.cL = (R)(0.5 * wl - h);
        x.cR = (R)(h - 0.5 * wr);
        x.pad = (R)0;
        x.m_nu_2h = (R)(-nu / (2.0 * h));
        x.m_chi_2h = (R)(-chi / (2.0 * h));
        x.m_tf15 = (R)(1.0 - 3.0 * nu / h);  // -(tau_f - 1.5), Eq. 9 with cs2 = 1/3
        x.m_tg15 = (R)(1.0 - 3.0 * chi / h);
        fl[i] = x;
    }
    cl.resize(n + 4);
    for (int i = -2; i <= n + 1; ++i) {
        const double w = line_width(f, i, periodic), wn = line_width(f, i + 1, periodic);
        CellLine<R> y;
        y.w = (R)w;
        y.is_next = (R)(1.0 / (w + wn));
        y.dt_w = (R)(dt / w);
        y.pad = (R)0;
        cl[i + 2] = y;
    }
}

template <class P, int TX, int TY>
cudaError_t launch_step(int units, int scheme, cudaStream_t s, const Desc3* d, CavityRun* c,
                        int par)
{
    const size_t sm = sizeof(Smem3<P, TX, TY>);
    if (scheme == 1)
        return launch_chained(step3_kernel<P, TX, TY, 1>, units, TX * TY, sm, s, d, c, par);
    return launch_chained(step3_kernel<P, TX, TY, 0>, units, TX * TY, sm, s, d, c, par);
}

// shared-memory opt-in and resident blocks per SM of both face stages
// (occ[0]: RTLBFS, occ[1]: TLBFS)
template <class P, int TX, int TY>
cudaError_t prepare_kernel(int occ[2])
{
    const size_t sm = sizeof(Smem3<P, TX, TY>);
    cudaError_t e = cudaFuncSetAttribute(step3_kernel<P, TX, TY, 0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step3_kernel<P, TX, TY, 1>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], step3_kernel<P, TX, TY, 0>,
                                                          TX * TY, sm);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], step3_kernel<P, TX, TY, 1>,
                                                          TX * TY, sm);
    return e;
}

}  // namespace rtlbfs3

using namespace rtlbfs3;

struct rtlbfs3d_ctx {
    int precision = RTLBFS_FP64;
    int n[3] = {0, 0, 0};
    std::vector<double> f[3];
    bool from_ra = true;
    double Ra = 1e3, Pr = 0.71, Ma = 0.1, dt_req = -1.0, kappa = 1.0;
    double nu = 0.0, chi = 0.0, beta_g = 0.0, dt = 0.0, T_ref = 0.5, dT = 1.0;
    double force[3] = {0.0, 0.0, 0.0};
    int g_axis = 2;
    int kind[6] = {kDirichlet, kDirichlet, kAdiabatic, kAdiabatic, kAdiabatic, kAdiabatic};
    double bcT[6] = {0.0, 1.0, 0.0, 0.0, 0.0, 0.0};
    double bcU[6][3] = {};
    int tile = 0, kchunk_req = 0;
    int scheme = 0;  // face stage: 0 RTLBFS (Section 3.2), 1 TLBFS (Section 2.2)
    int sms = 0, occ[3][2] = {};
    // device memory
    void* d_state = nullptr;  // 2 x (Vec4<S>[cells] + S[cells])
    void* d_lines = nullptr;
    Desc3* d_desc = nullptr;
    CavityRun* d_ctl = nullptr;
    double* d_acc = nullptr;
    CavityCtl* h_ctl = nullptr;  // pinned: the tested header h[0]
    CavityRun* h_run = nullptr;  // pinned: staging of a new run record
    double* h_acc = nullptr;
    size_t cells = 0, ssize = 0;
    // one state buffer: records (rho - 1, u, v, w) then T, each part
    // starting on a 256-byte boundary so the vector accesses stay aligned
    size_t rec_bytes = 0, tem_bytes = 0, buf_bytes = 0;
    Desc3 desc{};
    bool dirty = true;
    cudaStream_t stream = nullptr, own = nullptr, cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int gunits = 0, gtile = -1, gscheme = -1;
    std::string err;

    int fail(int code, const std::string& m)
    {
        err = m;
        return code;
    }
    int cuda_fail(cudaError_t e, const char* what)
    {
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return RTLBFS_ERR_CUDA;
    }
};

#define CK3(call)                                                   \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return h->cuda_fail(e_, #call);      \
    } while (0)

namespace {

double min_width(const rtlbfs3d_ctx* h)
{
    double w = INFINITY;
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < h->n[a]; ++i) w = std::min(w, h->f[a][i + 1] - h->f[a][i]);
    return w;
}

int resolve(rtlbfs3d_ctx* h)
{
    if (h->from_ra) {
        const double L = h->f[0][h->n[0]] - h->f[0][0];
        const double Vc = h->Ma;
        h->nu = Vc * L * std::sqrt(h->Pr / h->Ra);
        h->chi = h->nu / h->Pr;
        h->beta_g = Vc * Vc / (h->dT * L);
    }
    const double wmin = min_width(h);
    if (h->dt_req > 0.0)
        h->dt = h->dt_req;
    else if (h->dt_req == 0.0)
        h->dt = std::min(0.5 * wmin, 0.13 * wmin * wmin / std::max(h->nu, h->chi));
    else
        h->dt = 0.5 * wmin;
    for (int a = 0; a < 3; ++a)
        if ((h->kind[2 * a] == kPeriodic) != (h->kind[2 * a + 1] == kPeriodic))
            return h->fail(RTLBFS_ERR_ARG, "periodic sides must come in opposite pairs");
    return RTLBFS_OK;
}

// units of the current schedule
void decompose(rtlbfs3d_ctx* h, Desc3& d)
{
    const int TX = kTiles[h->tile][0], TY = kTiles[h->tile][1];
    d.tiles_x = (h->n[0] + TX - 1) / TX;
    d.tiles_y = (h->n[1] + TY - 1) / TY;
    int kc = h->kchunk_req;
    if (kc <= 0) {
        const long long slots =
            (long long)std::max(1, h->sms) * std::max(1, h->occ[h->tile][h->scheme]);
        const long long per_plane = (long long)d.tiles_x * d.tiles_y;
        long long chunks = std::max(1LL, (slots + per_plane - 1) / per_plane);
        kc = (int)std::max(4LL, (h->n[2] + chunks - 1) / chunks);
        // small meshes (a wave holds two planes of columns or more): the
        // shortest chunk of at least 4 planes whose units fit one wave, so
        // that no short second wave follows
        if (2 * per_plane <= slots)
            while (kc < h->n[2] && per_plane * ((h->n[2] + kc - 1) / kc) > slots) ++kc;
    }
    kc = std::min(kc, h->n[2]);
    d.kchunk = kc;
    d.chunks = (h->n[2] + kc - 1) / kc;
    d.units = d.tiles_x * d.tiles_y * d.chunks;
}

int upload(rtlbfs3d_ctx* h)
{
    if (!h->dirty) return RTLBFS_OK;
    int rc = resolve(h);
    if (rc) return rc;
    const bool fp64 = h->precision == RTLBFS_FP64;
    // lines: FP64 copies always; R copies for the step kernel
    std::vector<unsigned char> buf;
    size_t offs[3][4];  // [axis][face R, cell R, face d, cell d]
    auto append = [&](const void* p, size_t bytes) {
        size_t o = (buf.size() + 255) / 256 * 256;
        buf.resize(o + bytes);
        std::memcpy(buf.data() + o, p, bytes);
        return o;
    };
    for (int a = 0; a < 3; ++a) {
        const bool per = h->kind[2 * a] == kPeriodic;
        std::vector<FaceLine<double>> fd;
        std::vector<CellLine<double>> cd;
        build_lines<double>(h->f[a], per, h->kappa, h->nu, h->chi, h->dt, fd, cd);
        offs[a][2] = append(fd.data(), fd.size() * sizeof(fd[0]));
        offs[a][3] = append(cd.data(), cd.size() * sizeof(cd[0]));
        if (fp64) {
            offs[a][0] = offs[a][2];
            offs[a][1] = offs[a][3];
        } else {
            std::vector<FaceLine<float>> ff;
            std::vector<CellLine<float>> cf;
            build_lines<float>(h->f[a], per, h->kappa, h->nu, h->chi, h->dt, ff, cf);
            offs[a][0] = append(ff.data(), ff.size() * sizeof(ff[0]));
            offs[a][1] = append(cf.data(), cf.size() * sizeof(cf[0]));
        }
    }
    if (h->d_lines) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->d_lines);
        h->d_lines = nullptr;
    }
    CK3(cudaMalloc(&h->d_lines, buf.size()));
    CK3(cudaMemcpy(h->d_lines, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    Desc3& d = h->desc;
    unsigned char* base = static_cast<unsigned char*>(h->d_lines);
    for (int a = 0; a < 3; ++a) {
        d.n[a] = h->n[a];
        d.fline[a] = base + offs[a][0];
        d.cline[a] = base + offs[a][1];
        d.fline_d[a] = base + offs[a][2];
        d.cline_d[a] = base + offs[a][3];
    }
    for (int s = 0; s < 6; ++s) {
        d.kind[s] = h->kind[s];
        for (int c = 0; c < 3; ++c) {
            const double uw = (c == s / 2) ? 0.0 : h->bcU[s][c];
            d.bcU[s][c] = uw;
            d.f_bcU[s][c] = (float)uw;
        }
        d.bcT[s] = h->bcT[s];
        d.f_bcT[s] = (float)h->bcT[s];
    }
    d.g_axis = h->g_axis;
    d.beta_g = h->beta_g;
    d.T_ref = h->T_ref;
    d.dt = h->dt;
    d.f_beta_g = (float)h->beta_g;
    d.f_T_ref = (float)h->T_ref;
    d.f_dt = (float)h->dt;
    for (int a = 0; a < 3; ++a) {
        d.force[a] = h->force[a];
        d.f_force[a] = (float)h->force[a];
    }
    unsigned char* st = static_cast<unsigned char*>(h->d_state);
    for (int b = 0; b < 2; ++b) {
        d.rec[b] = st + b * h->buf_bytes;
        d.tem[b] = st + b * h->buf_bytes + h->rec_bytes;
    }
    decompose(h, d);
    CK3(cudaMemcpyAsync(h->d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    h->dirty = false;
    return RTLBFS_OK;
}

cudaError_t launch_one(rtlbfs3d_ctx* h, cudaStream_t s, int par)
{
    const int units = h->desc.units;
    rtlbfs::g_launches++;
    const int sc = h->scheme;
    if (h->precision == RTLBFS_FP64) {
        switch (h->tile) {
        case 0: return launch_step<StoreD, 32, 4>(units, sc, s, h->d_desc, h->d_ctl, par);
        case 1: return launch_step<StoreD, 16, 8>(units, sc, s, h->d_desc, h->d_ctl, par);
        default: return launch_step<StoreD, 32, 8>(units, sc, s, h->d_desc, h->d_ctl, par);
        }
    }
    switch (h->tile) {
    case 0: return launch_step<StoreQ, 32, 4>(units, sc, s, h->d_desc, h->d_ctl, par);
    case 1: return launch_step<StoreQ, 16, 8>(units, sc, s, h->d_desc, h->d_ctl, par);
    default: return launch_step<StoreQ, 32, 8>(units, sc, s, h->d_desc, h->d_ctl, par);
    }
}

// the run record with both headers c and cleared sums (h_ctl becomes c)
int put_run(rtlbfs3d_ctx* h, const CavityCtl& c)
{
    std::memset(h->h_run, 0, sizeof(CavityRun));
    h->h_run->h[0] = c;
    h->h_run->h[1] = c;
    *h->h_ctl = c;
    CK3(cudaMemcpyAsync(h->d_ctl, h->h_run, sizeof(CavityRun), cudaMemcpyHostToDevice, h->stream));
    CK3(cudaStreamSynchronize(h->stream));  // h_run is reused
    return RTLBFS_OK;
}

// arm the run control for up to nsteps more steps (tol < 0: no early stop)
int arm(rtlbfs3d_ctx* h, long long nsteps, double tol)
{
    CK3(cudaMemcpyAsync(h->h_ctl, &h->d_ctl->h[0], sizeof(CavityCtl), cudaMemcpyDeviceToHost,
                        h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    CavityCtl c = *h->h_ctl;
    c.done = 0;
    c.status = kRunning;
    c.pend = 0;
    c.max_steps = c.steps + nsteps;
    c.tol = tol;
    return put_run(h, c);
}

int ensure_graph(rtlbfs3d_ctx* h)
{
    if (h->gexec && h->gunits == h->desc.units && h->gtile == h->tile && h->gscheme == h->scheme)
        return RTLBFS_OK;
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    CK3(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    static_assert(kGraphSteps % 2 == 0, "graphs of an even number of launches");
    for (int i = 0; i < kGraphSteps && le == cudaSuccess; ++i) le = launch_one(h, h->cap, i & 1);
    rtlbfs::g_launches -= kGraphSteps;  // captured, not launched
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(h->cap, &g);
    if (le != cudaSuccess) return h->cuda_fail(le, "capture of the step launches");
    if (ee != cudaSuccess) return h->cuda_fail(ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return h->cuda_fail(ie, "cudaGraphInstantiate");
    h->gunits = h->desc.units;
    h->gtile = h->tile;
    h->gscheme = h->scheme;
    return RTLBFS_OK;
}

// queue `count` step launches (graph replays plus single launches)
int launch_steps(rtlbfs3d_ctx* h, long long count)
{
    nvtxRangePushA("rtlbfs3d: step launches");
    struct Pop {
        ~Pop() { nvtxRangePop(); }
    } pop;
    int rc = ensure_graph(h);
    if (rc) return rc;
    // launch k of the chain has parity k & 1; the chain ends with the stop
    // test of its last step
    int par = 0;
    while (count >= kGraphSteps) {
        CK3(cudaGraphLaunch(h->gexec, h->stream));
        rtlbfs::g_launches += kGraphSteps;
        count -= kGraphSteps;
    }
    for (long long i = 0; i < count; ++i) {
        cudaError_t e = launch_one(h, h->stream, par);
        if (e != cudaSuccess) return h->cuda_fail(e, "step launch");
        par ^= 1;
    }
    CK3(rtlbfs::launch_finalize(h->stream, h->d_ctl, 1, par));
    rtlbfs::g_launches++;
    return RTLBFS_OK;
}

int read_ctl(rtlbfs3d_ctx* h)
{
    CK3(cudaMemcpyAsync(h->h_ctl, &h->d_ctl->h[0], sizeof(CavityCtl), cudaMemcpyDeviceToHost,
                        h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    return RTLBFS_OK;
}

bool bad_handle(rtlbfs3d_t h) { return h == nullptr; }

}  // namespace

extern "C" {

int rtlbfs3d_create(int nx, int ny, int nz, const double* xf, const double* yf, const double* zf,
                    int precision, rtlbfs3d_t* out)
{
    if (!out || !xf || !yf || !zf || nx < 1 || ny < 1 || nz < 1) return RTLBFS_ERR_ARG;
    if (precision != RTLBFS_FP64 && precision != RTLBFS_FP32) return RTLBFS_ERR_ARG;
    if ((double)nx * ny * nz > 2147483647.0) return RTLBFS_ERR_ARG;
    *out = nullptr;
    const double* fs[3] = {xf, yf, zf};
    const int ns[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < ns[a]; ++i)
            if (!(fs[a][i + 1] > fs[a][i])) return RTLBFS_ERR_ARG;
    rtlbfs3d_ctx* h = new (std::nothrow) rtlbfs3d_ctx();
    if (!h) return RTLBFS_ERR_OOM;
    h->precision = precision;
    for (int a = 0; a < 3; ++a) {
        h->n[a] = ns[a];
        h->f[a].assign(fs[a], fs[a] + ns[a] + 1);
    }
    h->cells = (size_t)nx * ny * nz;
    h->ssize = precision == RTLBFS_FP64 ? sizeof(double) : sizeof(int);
    h->rec_bytes = (h->cells * 4 * h->ssize + 255) / 256 * 256;
    h->tem_bytes = (h->cells * h->ssize + 255) / 256 * 256;
    h->buf_bytes = h->rec_bytes + h->tem_bytes;
    auto bail = [&](int code) {
        rtlbfs3d_destroy(h);
        return code;
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return bail(RTLBFS_ERR_CUDA);
    if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(RTLBFS_ERR_CUDA);
    cudaError_t e;
    if (precision == RTLBFS_FP64) {
        e = prepare_kernel<StoreD, 32, 4>(h->occ[0]);
        if (e == cudaSuccess) e = prepare_kernel<StoreD, 16, 8>(h->occ[1]);
        if (e == cudaSuccess) e = prepare_kernel<StoreD, 32, 8>(h->occ[2]);
    } else {
        e = prepare_kernel<StoreQ, 32, 4>(h->occ[0]);
        if (e == cudaSuccess) e = prepare_kernel<StoreQ, 16, 8>(h->occ[1]);
        if (e == cudaSuccess) e = prepare_kernel<StoreQ, 32, 8>(h->occ[2]);
    }
    if (e != cudaSuccess) return bail(RTLBFS_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(RTLBFS_ERR_CUDA);
    h->stream = h->own;
    if (cudaMalloc(&h->d_state, 2 * h->buf_bytes) != cudaSuccess) return bail(RTLBFS_ERR_OOM);
    if (cudaMalloc(&h->d_desc, sizeof(Desc3)) != cudaSuccess ||
        cudaMalloc(&h->d_ctl, sizeof(CavityRun)) != cudaSuccess ||
        cudaMalloc(&h->d_acc, sizeof(double)) != cudaSuccess)
        return bail(RTLBFS_ERR_OOM);
    if (cudaMallocHost(&h->h_ctl, sizeof(CavityCtl)) != cudaSuccess ||
        cudaMallocHost(&h->h_run, sizeof(CavityRun)) != cudaSuccess ||
        cudaMallocHost(&h->h_acc, sizeof(double)) != cudaSuccess)
        return bail(RTLBFS_ERR_OOM);
    std::memset(h->h_run, 0, sizeof(CavityRun));
    std::memset(h->h_ctl, 0, sizeof(CavityCtl));
    if (cudaMemcpy(h->d_ctl, h->h_run, sizeof(CavityRun), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(RTLBFS_ERR_CUDA);
    // default state: rest, rho = 1, T linear in x between the walls
    {
        std::vector<double> one(h->cells, 1.0), zero(h->cells, 0.0), T(h->cells);
        const double x0 = xf[0], L = xf[nx] - xf[0];
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const double xc = 0.5 * (xf[i] + xf[i + 1]);
                    T[((size_t)k * ny + j) * nx + i] =
                        h->bcT[0] + (h->bcT[1] - h->bcT[0]) * (xc - x0) / L;
                }
        int rc = rtlbfs3d_set_state(h, one.data(), zero.data(), zero.data(), zero.data(), T.data());
        if (rc) return bail(rc);
    }
    *out = h;
    return RTLBFS_OK;
}

int rtlbfs3d_set_params(rtlbfs3d_t h, double Ra, double Pr, double Ma, double dt)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    if (!(Ra > 0) || !(Pr > 0) || !(Ma > 0) || !(dt >= 0))
        return h->fail(RTLBFS_ERR_ARG, "Ra, Pr, Ma must be positive and dt >= 0");
    h->from_ra = true;
    h->Ra = Ra;
    h->Pr = Pr;
    h->Ma = Ma;
    h->dt_req = dt;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfs3d_set_physics(rtlbfs3d_t h, double nu, double chi, double beta_g)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    if (!(nu > 0) || !(chi > 0) || !std::isfinite(beta_g))
        return h->fail(RTLBFS_ERR_ARG, "nu and chi must be positive");
    h->from_ra = false;
    h->nu = nu;
    h->chi = chi;
    h->beta_g = beta_g;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfs3d_set_lattice(rtlbfs3d_t h, double kappa)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    if (!(kappa > 0)) return h->fail(RTLBFS_ERR_ARG, "kappa must be positive");
    h->kappa = kappa;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfs3d_set_gravity_axis(rtlbfs3d_t h, int axis)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    if (axis < 0 || axis > 2) return h->fail(RTLBFS_ERR_ARG, "axis must be 0, 1 or 2");
    h->g_axis = axis;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfs3d_set_body_force(rtlbfs3d_t h, double fx, double fy, double fz)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    h->force[0] = fx;
    h->force[1] = fy;
    h->force[2] = fz;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfs3d_set_bc(rtlbfs3d_t h, int side, int kind, double T_wall, const double* u_wall)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    if (side < 0 || side > 5 || kind < 0 || kind > 2)
        return h->fail(RTLBFS_ERR_ARG, "bad side or boundary kind");
    if (kind == kDirichlet && !StoreQ::representable(T_wall, 3))
        return h->fail(RTLBFS_ERR_ARG, "wall temperature out of range");
    h->kind[side] = kind;
    h->bcT[side] = T_wall;
    for (int c = 0; c < 3; ++c) h->bcU[side][c] = u_wall ? u_wall[c] : 0.0;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfs3d_set_state(rtlbfs3d_t h, const double* rho, const double* u, const double* v,
                       const double* w, const double* T)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    if (!rho || !u || !v || !w || !T) return h->fail(RTLBFS_ERR_ARG, "null state array");
    const double* src[5] = {rho, u, v, w, T};
    const size_t n = h->cells;
    std::vector<unsigned char> buf(h->buf_bytes);
    if (h->precision == RTLBFS_FP64) {
        double* rec = reinterpret_cast<double*>(buf.data());
        double* tem = reinterpret_cast<double*>(buf.data() + h->rec_bytes);
        for (size_t c = 0; c < n; ++c) {
            rec[4 * c + 0] = rho[c] - 1.0;
            rec[4 * c + 1] = u[c];
            rec[4 * c + 2] = v[c];
            rec[4 * c + 3] = w[c];
            tem[c] = T[c];
        }
    } else {
        int* rec = reinterpret_cast<int*>(buf.data());
        int* tem = reinterpret_cast<int*>(buf.data() + h->rec_bytes);
        for (size_t c = 0; c < n; ++c) {
            for (int q = 0; q < 5; ++q) {
                const double x = q == 0 ? src[0][c] - 1.0 : src[q][c];
                if (!StoreQ::representable(x, kind_of(q)))
                    return h->fail(RTLBFS_ERR_ARG, "state value outside the FP32 fixed-point range");
            }
            rec[4 * c + 0] = StoreQ::from_double(rho[c] - 1.0, 0);
            rec[4 * c + 1] = StoreQ::from_double(u[c], 1);
            rec[4 * c + 2] = StoreQ::from_double(v[c], 1);
            rec[4 * c + 3] = StoreQ::from_double(w[c], 1);
            tem[c] = StoreQ::from_double(T[c], 3);
        }
    }
    CK3(cudaStreamSynchronize(h->stream));
    CK3(cudaMemcpy(h->d_state, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    CavityCtl z;
    std::memset(&z, 0, sizeof(z));
    z.res[0] = z.res[1] = INFINITY;
    return put_run(h, z);
}

int rtlbfs3d_get_state(rtlbfs3d_t h, double* rho, double* u, double* v, double* w, double* T)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    if (!rho || !u || !v || !w || !T) return h->fail(RTLBFS_ERR_ARG, "null state array");
    int rc = read_ctl(h);
    if (rc) return rc;
    const int cur = h->h_ctl->cur;
    const size_t n = h->cells;
    std::vector<unsigned char> buf(h->buf_bytes);
    CK3(cudaMemcpy(buf.data(), static_cast<unsigned char*>(h->d_state) + cur * h->buf_bytes,
                   h->buf_bytes, cudaMemcpyDeviceToHost));
    if (h->precision == RTLBFS_FP64) {
        const double* rec = reinterpret_cast<const double*>(buf.data());
        const double* tem = reinterpret_cast<const double*>(buf.data() + h->rec_bytes);
        for (size_t c = 0; c < n; ++c) {
            rho[c] = 1.0 + rec[4 * c];
            u[c] = rec[4 * c + 1];
            v[c] = rec[4 * c + 2];
            w[c] = rec[4 * c + 3];
            T[c] = tem[c];
        }
    } else {
        const int* rec = reinterpret_cast<const int*>(buf.data());
        const int* tem = reinterpret_cast<const int*>(buf.data() + h->rec_bytes);
        for (size_t c = 0; c < n; ++c) {
            rho[c] = 1.0 + StoreQ::to_double(rec[4 * c], 0);
            u[c] = StoreQ::to_double(rec[4 * c + 1], 1);
            v[c] = StoreQ::to_double(rec[4 * c + 2], 1);
            w[c] = StoreQ::to_double(rec[4 * c + 3], 1);
            T[c] = StoreQ::to_double(tem[c], 3);
        }
    }
    return RTLBFS_OK;
}

int rtlbfs3d_step(rtlbfs3d_t h, long nsteps)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    if (nsteps < 0) return h->fail(RTLBFS_ERR_ARG, "nsteps < 0");
    int rc = upload(h);
    if (rc) return rc;
    if (nsteps == 0) return RTLBFS_OK;
    rc = arm(h, nsteps, -1.0);
    if (rc) return rc;
    rc = launch_steps(h, nsteps);
    if (rc) return rc;
    rc = read_ctl(h);
    if (rc) return rc;
    if (h->h_ctl->status == kDiverged) return h->fail(RTLBFS_ERR_DIVERGED, "the state diverged");
    return RTLBFS_OK;
}

int rtlbfs3d_run_to_steady(rtlbfs3d_t h, double tol, long max_steps, double timeout_s,
                           long* steps_taken, double* res2)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    if (max_steps < 0 || !(tol >= 0)) return h->fail(RTLBFS_ERR_ARG, "bad tol or max_steps");
    int rc = upload(h);
    if (rc) return rc;
    rc = read_ctl(h);
    if (rc) return rc;
    const long long start = h->h_ctl->steps;
    rc = arm(h, max_steps, tol);
    if (rc) return rc;
    const auto t0 = std::chrono::steady_clock::now();
    long long queued = 0;
    int out = RTLBFS_OK;
    while (true) {
        // keep a few graph replays in flight, then look at the run control
        const long long chunk = 4LL * kGraphSteps;
        const long long left = (long long)max_steps - queued;
        const long long now = std::min(chunk, left);
        if (now > 0) {
            rc = launch_steps(h, now);
            if (rc) return rc;
            queued += now;
        }
        rc = read_ctl(h);
        if (rc) return rc;
        const CavityCtl& c = *h->h_ctl;
        if (c.done || queued >= max_steps) {
            if (c.status == kConverged)
                out = RTLBFS_OK;
            else if (c.status == kDiverged)
                out = h->fail(RTLBFS_ERR_DIVERGED, "the state diverged");
            else
                out = h->fail(RTLBFS_ERR_NOT_CONVERGED, "max_steps reached");
            break;
        }
        if (timeout_s > 0) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > timeout_s) {
                out = h->fail(RTLBFS_ERR_TIMEOUT, "wall-clock limit reached");
                break;
            }
        }
    }
    // stop any remaining armed steps from running later
    rc = read_ctl(h);
    if (rc) return rc;
    {
        CavityCtl c = *h->h_ctl;
        c.done = 1;
        rc = put_run(h, c);
        if (rc) return rc;
    }
    if (steps_taken) *steps_taken = (long)(h->h_ctl->steps - start);
    if (res2) {
        res2[0] = h->h_ctl->res[0];
        res2[1] = h->h_ctl->res[1];
    }
    return out;
}

int rtlbfs3d_residual(rtlbfs3d_t h, double* res2, long* steps)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    int rc = read_ctl(h);
    if (rc) return rc;
    if (res2) {
        res2[0] = h->h_ctl->res[0];
        res2[1] = h->h_ctl->res[1];
    }
    if (steps) *steps = (long)h->h_ctl->steps;
    return RTLBFS_OK;
}

int rtlbfs3d_nusselt(rtlbfs3d_t h, int side, int mid, double* nu)
{
    if (bad_handle(h) || !nu) return RTLBFS_ERR_ARG;
    if (side < 0 || side > 6 || mid < 0 || mid > 1) return h->fail(RTLBFS_ERR_ARG, "bad selector");
    if (side == 6 && (mid || h->n[0] % 2)) return h->fail(RTLBFS_ERR_ARG, "mid-plane needs even nx");
    const int ax = side == 6 ? 0 : side / 2;
    if (side < 6 && h->kind[2 * ax] == kPeriodic) return h->fail(RTLBFS_ERR_ARG, "periodic side");
    int rc = upload(h);
    if (rc) return rc;
    rc = read_ctl(h);
    if (rc) return rc;
    const int cur = h->h_ctl->cur;
    const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
    const int pos = side == 6 ? h->n[0] / 2 : (side % 2 ? h->n[ax] : 0);
    const int wside = side == 6 ? -1 : side;
    double L[3];
    for (int a = 0; a < 3; ++a) L[a] = h->f[a][h->n[a]] - h->f[a][0];
    const double base = L[ax] / (h->chi * h->dT);
    CK3(cudaMemsetAsync(h->d_acc, 0, sizeof(double), h->stream));
    auto run = [&](int lo, int hi, double wgt) -> cudaError_t {
        const long long nf = (long long)(hi - lo) * h->n[b2];
        const int block = 128;
        const int grid = (int)std::min<long long>((nf + block - 1) / block, 4LL * std::max(1, h->sms));
        rtlbfs::g_launches++;
        const bool tl = h->scheme == 1;
        if (h->precision == RTLBFS_FP64) {
            if (tl)
                nusselt3_kernel<StoreD, 1><<<grid, block, 0, h->stream>>>(h->d_desc, cur, ax, pos, lo,
                                                                          hi, wside, wgt, h->d_acc);
            else
                nusselt3_kernel<StoreD, 0><<<grid, block, 0, h->stream>>>(h->d_desc, cur, ax, pos, lo,
                                                                          hi, wside, wgt, h->d_acc);
        } else {
            if (tl)
                nusselt3_kernel<StoreQ, 1><<<grid, block, 0, h->stream>>>(h->d_desc, cur, ax, pos, lo,
                                                                          hi, wside, wgt, h->d_acc);
            else
                nusselt3_kernel<StoreQ, 0><<<grid, block, 0, h->stream>>>(h->d_desc, cur, ax, pos, lo,
                                                                          hi, wside, wgt, h->d_acc);
        }
        return cudaGetLastError();
    };
    cudaError_t e;
    if (!mid) {
        e = run(0, h->n[b1], base / (L[b1] * L[b2]));
    } else {
        // the t1 extent is divided out: the line integral along t2 per unit t1 width
        const int n1 = h->n[b1];
        if (n1 % 2) {
            const int r = n1 / 2;
            const double w1 = h->f[b1][r + 1] - h->f[b1][r];
            e = run(r, r + 1, base / (L[b2] * w1));
        } else {
            const int r0 = n1 / 2 - 1, r1 = n1 / 2;
            const double w0 = h->f[b1][r0 + 1] - h->f[b1][r0], w1 = h->f[b1][r1 + 1] - h->f[b1][r1];
            e = run(r0, r0 + 1, 0.5 * base / (L[b2] * w0));
            if (e == cudaSuccess) e = run(r1, r1 + 1, 0.5 * base / (L[b2] * w1));
        }
    }
    if (e != cudaSuccess) return h->cuda_fail(e, "nusselt3_kernel");
    CK3(cudaMemcpyAsync(h->h_acc, h->d_acc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    *nu = *h->h_acc;
    return RTLBFS_OK;
}

int rtlbfs3d_set_scheme(rtlbfs3d_t h, int scheme)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    if (scheme != 0 && scheme != 1) return h->fail(RTLBFS_ERR_ARG, "scheme must be 0 or 1");
    h->scheme = scheme;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfs3d_set_schedule(rtlbfs3d_t h, int tile, int kchunk)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    if (tile < 0 || tile > 2 || kchunk < 0) return h->fail(RTLBFS_ERR_ARG, "bad schedule");
    h->tile = tile;
    h->kchunk_req = kchunk;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfs3d_autotune(rtlbfs3d_t h, int steps, int* tile, double* ms_per_step)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    if (steps < 1) return h->fail(RTLBFS_ERR_ARG, "steps < 1");
    // snapshot of both buffers and the run control
    const size_t bytes = 2 * h->buf_bytes;
    void* snap = nullptr;
    CK3(cudaStreamSynchronize(h->stream));
    CK3(cudaMalloc(&snap, bytes));
    CavityCtl saved;
    int rc = read_ctl(h);
    if (rc) {
        cudaFree(snap);
        return rc;
    }
    saved = *h->h_ctl;
    cudaMemcpy(snap, h->d_state, bytes, cudaMemcpyDeviceToDevice);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int keep_k = h->kchunk_req;
    int best = h->tile;
    float best_ms = INFINITY;
    for (int t = 0; t < 3 && rc == RTLBFS_OK; ++t) {
        h->tile = t;
        h->kchunk_req = keep_k;
        h->dirty = true;
        rc = upload(h);
        if (rc) break;
        rc = arm(h, 1LL << 40, -1.0);
        if (rc) break;
        rc = launch_steps(h, 2);  // warm-up and graph capture
        if (rc) break;
        cudaEventRecord(e0, h->stream);
        rc = launch_steps(h, steps);
        if (rc) break;
        cudaEventRecord(e1, h->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(h->stream);
    cudaMemcpy(h->d_state, snap, bytes, cudaMemcpyDeviceToDevice);
    cudaFree(snap);
    {
        const int prc = put_run(h, saved);
        if (!rc) rc = prc;
    }
    if (rc) return rc;
    h->tile = best;
    h->dirty = true;
    rc = upload(h);
    if (rc) return rc;
    if (tile) *tile = best;
    if (ms_per_step) *ms_per_step = best_ms / steps;
    return RTLBFS_OK;
}

int rtlbfs3d_set_stream(rtlbfs3d_t h, void* stream)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    CK3(cudaStreamSynchronize(h->stream));
    h->stream = stream ? static_cast<cudaStream_t>(stream) : h->own;
    return RTLBFS_OK;
}

int rtlbfs3d_sync(rtlbfs3d_t h)
{
    if (bad_handle(h)) return RTLBFS_ERR_ARG;
    CK3(cudaStreamSynchronize(h->stream));
    return RTLBFS_OK;
}

const char* rtlbfs3d_last_error(rtlbfs3d_t h) { return h ? h->err.c_str() : "null handle"; }

void rtlbfs3d_destroy(rtlbfs3d_t h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    cudaFree(h->d_state);
    cudaFree(h->d_lines);
    cudaFree(h->d_desc);
    cudaFree(h->d_ctl);
    cudaFree(h->d_acc);
    cudaFreeHost(h->h_ctl);
    cudaFreeHost(h->h_run);
    cudaFreeHost(h->h_acc);
    if (h->own) cudaStreamDestroy(h->own);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
}

}  // extern "C"

// The counting type below is host-only; face_flux3 is instantiated on it
// from host code alone, so the host/device call checks do not apply.
#pragma nv_diag_suppress 20011, 20014

// ---------------------------------------------------------------------------
// Operation count of a cell-update: face_flux3 run on a counting value type
// on the host (the same template the kernels execute).  An add, a multiply
// and a fused multiply-add count one each; subtracting from the literal 0
// is a negated operand and free; reciprocals and square roots apart.
// ---------------------------------------------------------------------------
namespace rtlbfs3 {
namespace {
struct Tally3 {
    long long ops = 0, sfu = 0;
};
Tally3 g_tally3;
struct Cnt3 {
    double v;
    bool zero;
};
Cnt3 operator+(Cnt3 a, Cnt3 b)
{
    if (!a.zero && !b.zero) ++g_tally3.ops;
    return {a.v + b.v, a.zero && b.zero};
}
Cnt3 operator-(Cnt3 a, Cnt3 b)
{
    if (!a.zero && !b.zero) ++g_tally3.ops;
    return {a.v - b.v, a.zero && b.zero};
}
Cnt3 operator*(Cnt3 a, Cnt3 b)
{
    ++g_tally3.ops;
    return {a.v * b.v, false};
}
Cnt3 vfma(Cnt3 a, Cnt3 b, Cnt3 c)
{
    ++g_tally3.ops;
    return {a.v * b.v + c.v, false};
}
}  // namespace
}  // namespace rtlbfs3

namespace rtlbfs {
template <>
struct vtraits<rtlbfs3::Cnt3> {
    static rtlbfs3::Cnt3 bc(double c) { return {c, c == 0.0}; }
    static rtlbfs3::Cnt3 rcp(rtlbfs3::Cnt3 x)
    {
        ++rtlbfs3::g_tally3.sfu;
        return {1.0 / x.v, false};
    }
};
}  // namespace rtlbfs

extern "C" int rtlbfs3d_op_counts(double* face_ops, double* cell_ops, double* sfu_ops)
{
    return rtlbfs3d_op_counts_scheme(0, face_ops, cell_ops, sfu_ops);
}

extern "C" int rtlbfs3d_op_counts_scheme(int scheme, double* face_ops, double* cell_ops,
                                         double* sfu_ops)
{
    if (scheme != 0 && scheme != 1) return RTLBFS_ERR_ARG;
    using rtlbfs3::Cnt3;
    rtlbfs3::g_tally3 = rtlbfs3::Tally3();
    rtlbfs3::CellNT3<Cnt3> L, R;
    for (int k = 0; k < 5; ++k) {
        L.q[k] = {0.01 * (k + 1), false};
        L.gn[k] = {0.002 * (k + 1), false};
        L.g1[k] = {0.003 * (k + 1), false};
        L.g2[k] = {0.001 * (k + 2), false};
        R.q[k] = {0.02 * (k + 1), false};
        R.gn[k] = {0.001 * (k + 1), false};
        R.g1[k] = {0.004 * (k + 1), false};
        R.g2[k] = {0.002 * (k + 2), false};
    }
    rtlbfs::FaceLine<Cnt3> fl;
    fl.h = {0.3, false};
    fl.cL = {-0.2, false};
    fl.cR = {0.25, false};
    fl.m_nu_2h = {-0.01, false};
    fl.m_chi_2h = {-0.01, false};
    fl.m_tf15 = {-0.1, false};
    fl.m_tg15 = {-0.1, false};
    fl.pad = {0.0, true};
    Cnt3 F[5];
    if (scheme == 1)
        rtlbfs3::face_flux3_tlbfs<Cnt3>(L, R, Cnt3{0.5, false}, fl, Cnt3{1.0, false},
                                        Cnt3{0.0, false}, Cnt3{0.0, false}, F);
    else
        rtlbfs3::face_flux3<Cnt3>(L, R, Cnt3{0.5, false}, fl, Cnt3{1.0, false}, Cnt3{0.0, false},
                                  Cnt3{0.0, false}, F);
    const rtlbfs3::Tally3 f = rtlbfs3::g_tally3;
    // Per cell, besides its three faces (the -x, -y, -z faces it owns):
    //   working values from the stored state                 5
    //   face frames: Tbar and the right cell's tau, 3 faces    6
    //   Green-Gauss gradients, Eq. 55, 3 x 5 fields           60  (2 differences,
    //                                                              a product, an FMA)
    //   flux divergence, 5 fields                             30
    //   rho, T, body force and buoyancy (Eq. 64)               8
    //   rho^{n+1}, increments of u, v, w, T, new values       21
    //   fixed-point increments                                 5
    //   residual terms of |u| and T (FP32 part)               23
    //   ------------------------------------------------------------
    //                                                        158  (+ 4 SFU: the
    //   reciprocal of rho^{n+1}, two square roots, one reciprocal)
    const double other = 158.0, other_sfu = 4.0;
    if (face_ops) *face_ops = (double)f.ops;
    if (cell_ops) *cell_ops = 3.0 * (double)f.ops + other;
    if (sfu_ops) *sfu_ops = 3.0 * (double)f.sfu + other_sfu;
    return RTLBFS_OK;
}
