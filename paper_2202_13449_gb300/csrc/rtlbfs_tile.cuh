// rtlbfs_tile.cuh -- one tile of the fused RTLBFS time step (arXiv
// 2202.13449, Section 3.2) on a structured 2D mesh: the shared-memory tile
// buffers, ghost resolution and mirror rules, Green-Gauss gradients and the
// tile_step() body shared by the launch-per-step tile kernel
// (rtlbfs_step.cu) and the persistent tile kernel (rtlbfs_persist.cu).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "rtlbfs_dev.cuh"
#include "rtlbfs_kernels.h"

namespace rtlbfs {

template <class P, int TX, int TY, int NT>
struct TileSmem {
    using S = typename P::S;
    using R = typename P::R;
    static constexpr int BX = TX + 4, BY = TY + 4;  // tile + 2-cell halo
    static constexpr int GX = TX + 2, GY = TY + 2;  // gradient ring
    // (rho - 1, u, v, T - T_tile) of the haloed tile; T_tile is one cell's
    // stored temperature, so the in-tile deviations keep their bits in FP32
    Vec4<R> val[BY][BX];
    Vec4<R> gx[GY][GX];
    Vec4<R> gy[GY][GX];
    Vec4<R> fx[TY][TX + 1];
    Vec4<R> fy[TY + 1][TX];
    // the stored records of the tile's own cells, as loaded: the update
    // adds its increments to them instead of reading the state again.  Only
    // where the 16-byte records leave room for four resident blocks per SM
    // (FP32 tiles up to 14 rows); elsewhere the update re-reads them (L2).
    static constexpr bool kRaw = sizeof(S) == 4 && TY <= 14;
    Vec4<S> raw[kRaw ? TY : 1][kRaw ? TX : 1];
    FaceLine<R> xl[TX + 1];
    FaceLine<R> yl[TY + 1];
    CellLine<R> xc[BX];
    CellLine<R> yc[BY];
    R red[NT / 32][4];  // per-warp residual partials (tile_sums adds them)
    CavityDesc desc;  // the tile's cavity, staged by stage_tile
    int plan[3];      // the tile's step after its cavity's stop test: done, cur, sum slot
    int last;         // persistent kernel: this block finalises the step
};

// Resolve global cell (gi, gj) of a cavity, ghosts included: the source
// cell (si, sj) to read, and the wall side whose mirror rule applies
// (-1: none).  Returns false for positions no stencil uses (corner ghosts,
// cells beyond the ghost layer of a wall).
// With halo sides (south: hlo, north: hhi) rows -2, -1 (ny, ny + 1) are
// stored rows of the strip's buffers (sj outside [0, ny)).
__device__ __forceinline__ bool resolve_cell(int nx, int ny, bool xper, bool yper, bool hlo,
                                             bool hhi, int gi, int gj, int& si, int& sj,
                                             int& mside)
{
    si = gi;
    sj = gj;
    mside = -1;
    if (gi < 0 || gi >= nx) {
        if (xper) {
            si = ((gi % nx) + nx) % nx;
        } else if (gi == -1) {
            si = 0;
            mside = kSideW;
        } else if (gi == nx) {
            si = nx - 1;
            mside = kSideE;
        } else {
            return false;
        }
    }
    if (gj < 0 || gj >= ny) {
        if ((gj < 0 && hlo && gj >= -2) || (gj >= ny && hhi && gj <= ny + 1)) {
            sj = gj;  // a halo row (a wall ghost of it keeps its x mirror)
        } else if (yper) {
            sj = ((gj % ny) + ny) % ny;
        } else if ((gj == -1 || gj == ny) && mside < 0) {
            sj = gj < 0 ? 0 : ny - 1;
            mside = gj < 0 ? kSideS : kSideN;
        } else {
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ bool resolve_cell(const CavityDesc& d, int gi, int gj, int& si,
                                             int& sj, int& mside)
{
    return resolve_cell(d.nx, d.ny, d.kind[kSideW] == kPeriodic, d.kind[kSideS] == kPeriodic,
                        d.kind[kSideS] == kHalo, d.kind[kSideN] == kHalo, gi, gj, si, sj, mside);
}

// Ghost values across wall `side` from the partner's working values y =
// (rho - 1, u, v, T - Tref): rho even, velocity odd about the wall velocity
// (normal component about 0), T odd about T_wall on a Dirichlet wall and
// even on an adiabatic one.  Formed in the arithmetic type relative to
// Tref: 2 T_wall - T_P can leave the fixed-point range of a stored
// temperature (a hot wall next to cold fluid) while its deviation from a
// temperature inside the tile does not.
template <class P>
__device__ __forceinline__ Vec4<typename P::R> mirror_values(const CavityDesc& d, int side,
                                                             Vec4<typename P::R> y,
                                                             typename P::R Tref)
{
    using R = typename P::R;
    const bool xn = (side == kSideW || side == kSideE);
    const R ut2 = R(2) * P::bcU(&d, side);
    if (xn) {
        y.y = -y.y;
        y.z = ut2 - y.z;
    } else {
        y.z = -y.z;
        y.y = ut2 - y.y;
    }
    if (d.kind[side] == kDirichlet) y.w = R(2) * (P::Tw(&d, side) - Tref) - y.w;
    return y;
}

// Ghost gradient across wall `side`: even quantities negate the normal
// component, odd ones the tangential component.
template <typename R>
__device__ __forceinline__ void mirror_grad(const CavityDesc& d, int side, Vec4<R>& gx,
                                            Vec4<R>& gy)
{
    const bool nx_ = (side == kSideW || side == kSideE);
    R* ax = &gx.x;
    R* ay = &gy.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool even = wall_parity(d.kind[side], k) > 0;
        if (nx_) {
            if (even) ax[k] = -ax[k];
            else ay[k] = -ay[k];
        } else {
            if (even) ay[k] = -ay[k];
            else ax[k] = -ax[k];
        }
    }
}

template <class P>
__device__ __forceinline__ typename P::S comp(const Vec4<typename P::S>& v, int k)
{
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// Eqs. 55-56: Green-Gauss gradient from the four neighbour differences
// (storage values; exact differences for the fixed-point state).
template <class P>
__device__ __forceinline__ void gg_gradient(const Vec4<typename P::S>& p,
                                            const Vec4<typename P::S>& e,
                                            const Vec4<typename P::S>& w,
                                            const Vec4<typename P::S>& n,
                                            const Vec4<typename P::S>& s, typename P::R ixe,
                                            typename P::R ixw, typename P::R iyn,
                                            typename P::R iys, Vec4<typename P::R>& gx,
                                            Vec4<typename P::R>& gy)
{
    using R = typename P::R;
    R* ax = &gx.x;
    R* ay = &gy.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const auto pk = comp<P>(p, k);
        ax[k] = P::diff(comp<P>(e, k), pk, k) * ixe + P::diff(pk, comp<P>(w, k), k) * ixw;
        ay[k] = P::diff(comp<P>(n, k), pk, k) * iyn + P::diff(pk, comp<P>(s, k), k) * iys;
    }
}

// The same from working values (rho - 1, u, v, T - T_tile) in R.
template <typename R>
__device__ __forceinline__ void gg_gradient_r(const Vec4<R>& p, const Vec4<R>& e,
                                              const Vec4<R>& w, const Vec4<R>& n,
                                              const Vec4<R>& s, R ixe, R ixw, R iyn, R iys,
                                              Vec4<R>& gx, Vec4<R>& gy)
{
    gx.x = (e.x - p.x) * ixe + (p.x - w.x) * ixw;
    gx.y = (e.y - p.y) * ixe + (p.y - w.y) * ixw;
    gx.z = (e.z - p.z) * ixe + (p.z - w.z) * ixw;
    gx.w = (e.w - p.w) * ixe + (p.w - w.w) * ixw;
    gy.x = (n.x - p.x) * iyn + (p.x - s.x) * iys;
    gy.y = (n.y - p.y) * iyn + (p.y - s.y) * iys;
    gy.z = (n.z - p.z) * iyn + (p.z - s.z) * iys;
    gy.w = (n.w - p.w) * iyn + (p.w - s.w) * iys;
}

// The same in FP32, two components per packed FP32x2 instruction.
__device__ __forceinline__ void gg_gradient_r(const Vec4<float>& p, const Vec4<float>& e,
                                              const Vec4<float>& w, const Vec4<float>& n,
                                              const Vec4<float>& s, float ixe, float ixw,
                                              float iyn, float iys, Vec4<float>& gx,
                                              Vec4<float>& gy)
{
    gg_gradient_f32(p, e, w, n, s, ixe, ixw, iyn, iys, gx, gy);
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Build the two cells of a face in the face frame (normal along x for an
// x-face, along y for a y-face) from working values (rho - 1, u, v, T - Tz);
// T enters as a deviation from Tbar = T_L.
template <typename R>
__device__ __forceinline__ void face_cells(bool isx, const Vec4<R>& vl, const Vec4<R>& vr,
                                           R Tz, const Vec4<R>& gxl, const Vec4<R>& gyl,
                                           const Vec4<R>& gxr, const Vec4<R>& gyr, CellNT<R>& L,
                                           CellNT<R>& Rr, R& Tbar)
{
    Tbar = Tz + vl.w;
    const R tR = vr.w - vl.w;
    if (isx) {
        L = {{vl.x, vl.y, vl.z, R(0)}, {gxl.x, gxl.y, gxl.z, gxl.w}, {gyl.x, gyl.y, gyl.z, gyl.w}};
        Rr = {{vr.x, vr.y, vr.z, tR}, {gxr.x, gxr.y, gxr.z, gxr.w}, {gyr.x, gyr.y, gyr.z, gyr.w}};
    } else {
        L = {{vl.x, vl.z, vl.y, R(0)}, {gyl.x, gyl.z, gyl.y, gyl.w}, {gxl.x, gxl.z, gxl.y, gxl.w}};
        Rr = {{vr.x, vr.z, vr.y, tR}, {gyr.x, gyr.z, gyr.y, gyr.w}, {gxr.x, gxr.z, gxr.y, gxr.w}};
    }
}

// Resident blocks per SM to compile for: FP32 aims at 64 registers a thread
// (the tile buffers then bound occupancy); FP64 takes what it needs.
template <class P, int NT>
struct MinBlocks {
    static constexpr int value = 1;
};
template <int NT>
struct MinBlocks<StoreQ, NT> {
    static constexpr int value = 65536 / (NT * 64);
};

// The state record at p: through L2 only (LDCG, for a kernel whose blocks
// read what other blocks of the same launch wrote; L1 is not coherent) or
// by the default path.
template <bool LDCG, typename T>
__device__ __forceinline__ T ld_state(const T* p)
{
    if constexpr (LDCG) {
        static_assert(sizeof(T) % 16 == 0, "16-byte records");
        T v;
        const int4* src = reinterpret_cast<const int4*>(p);
        int4* dst = reinterpret_cast<int4*>(&v);
#pragma unroll
        for (int k = 0; k < (int)(sizeof(T) / 16); ++k) dst[k] = __ldcg(src + k);
        return v;
    } else {
        return *p;
    }
}

// The mesh lines of a tile and its halo into shared memory.
template <class P, int TX, int TY, int NT>
__device__ __forceinline__ void stage_lines(TileSmem<P, TX, TY, NT>& sm, const CavityDesc* gdp,
                                            int i0, int j0)
{
    using Sm = TileSmem<P, TX, TY, NT>;
    using R = typename P::R;
    constexpr int BX = Sm::BX, BY = Sm::BY;
    const int tid = threadIdx.x;
    const int nx = gdp->nx, ny = gdp->ny;
    const CellLine<R>* xc = static_cast<const CellLine<R>*>(gdp->xcell);
    const CellLine<R>* yc = static_cast<const CellLine<R>*>(gdp->ycell);
    const FaceLine<R>* xl = static_cast<const FaceLine<R>*>(gdp->xline);
    const FaceLine<R>* yl = static_cast<const FaceLine<R>*>(gdp->yline);
    for (int k = tid; k < BX; k += NT) sm.xc[k] = xc[min(i0 + k, nx + 3)];
    for (int k = tid; k < BY; k += NT) sm.yc[k] = yc[min(j0 + k, ny + 3)];
    for (int k = tid; k < TX + 1; k += NT) sm.xl[k] = xl[min(i0 + k, nx)];
    for (int k = tid; k < TY + 1; k += NT) sm.yl[k] = yl[min(j0 + k, ny)];
}

// What a tile needs that no time step changes: a copy of its cavity's
// descriptor (sm.desc) and the mesh lines of the tile and its halo.  Kernels
// call it before they wait for the previous step, so these loads overlap
// that step's tail instead of heading this step's chain of dependent loads;
// a barrier must separate it from tile_step (called with lines_staged).
template <class P, int TX, int TY, int NT>
__device__ __forceinline__ void stage_tile(TileSmem<P, TX, TY, NT>& sm, const CavityDesc* gdp,
                                           int i0, int j0)
{
    static_assert(sizeof(CavityDesc) % 8 == 0, "descriptor of 8-byte words");
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(gdp);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sm.desc);
    for (int k = threadIdx.x; k < (int)(sizeof(CavityDesc) / 8); k += NT) dst[k] = src[k];
    stage_lines(sm, gdp, i0, j0);
}

// The tile's four residual sums from the per-warp partials in sm.red:
// warp 0 adds them in the arithmetic type (shuffles; on GB300 an FP64
// instruction occupies the narrow FP64 pipe for 16 cycles, so a serial FP64
// loop here lengthened every block's tail) and returns them in FP64, the
// precision of the sums across tiles.  Call from all of warp 0, after the
// barrier that follows tile_step.
template <class P, int TX, int TY, int NT>
__device__ __forceinline__ void tile_sums(const TileSmem<P, TX, TY, NT>& sm, double a[4])
{
    using R = typename P::R;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        R v = lane < NT / 32 ? sm.red[lane][q] : R(0);
        v = warp_sum(v);
        a[q] = (double)v;
    }
}

// One tile of one time step on cavity *dp, tile origin (i0, j0): phases 1-4
// below read the state from fin and write the new state to fout; the
// tile's four residual sums are left in sm.red (a row per warp) for the
// caller to add (tile_sums) after a barrier.  lines_staged: stage_tile has put the
// tile's mesh lines in shared memory (dp may then point at its copy of the
// descriptor); otherwise phase 1 loads them beside the state.
//
// Work of a thread.  The tile's TX x TY cells are split into CPT = TX*TY/NT
// cells per thread at fixed places: thread (c, r) = (tid % CW, tid / CW),
// CW = TX / CPT, owns cells (c + m CW, r), m < CPT.  In every phase a thread
// first works on its own cells (and their west and south faces), whose
// shared-memory places are fixed offsets from one base, then on a share of
// the phase's remainder: the halo ring of the load, the gradient ring, the
// east face column and north face row of the tile.  The remainders go to the
// lowest threads, so they keep as few warps as possible busy for the extra
// round; the north face row starts on the warp after the east column's, so
// no warp computes two faces more than the others.  With CW = 16 or 32
// lanes of a warp read consecutive records: no bank conflicts.
template <class P, int TX, int TY, int NT, int SCHEME, bool LDCG>
__device__ __forceinline__ void tile_step(TileSmem<P, TX, TY, NT>& sm, const CavityDesc* dp,
                                          int i0, int j0,
                                          const Vec4<typename P::S>* __restrict__ fin,
                                          Vec4<typename P::S>* __restrict__ fout,
                                          bool lines_staged)
{
    using Sm = TileSmem<P, TX, TY, NT>;
    using S = typename P::S;
    using R = typename P::R;
    constexpr int BX = Sm::BX, BY = Sm::BY, GX = Sm::GX, GY = Sm::GY;
    constexpr int CPT = TX * TY / NT;
    constexpr int CW = TX / CPT;
    static_assert(CPT * NT == TX * TY && CW * CPT == TX && CW * TY == NT, "thread layout");
    // the gradient and face loops unrolled where that stays within the
    // register budget of four resident blocks (FP32 tiles of 4+ rows)
    constexpr int UNROLL = (sizeof(R) == 4 && TY >= 4) ? 8 : 1;
    const int tid = threadIdx.x;
    const int tc = tid % CW, tr = tid / CW;
    const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch;
    const bool xper = dp->kind[kSideW] == kPeriodic, yper = dp->kind[kSideS] == kPeriodic;
    const bool hlo = dp->kind[kSideS] == kHalo, hhi = dp->kind[kSideN] == kHalo;
    // temperature reference of this tile: its (clamped) centre cell
    const int ic = min(i0 + TX / 2, nx - 1), jc = min(j0 + TY / 2, ny - 1);
    const S qTz = ld_state<LDCG>(&fin[(size_t)jc * pitch + ic]).w;
    const R Tz = P::val(qTz, 3);

    // A tile whose halo lies inside the mesh touches no boundary: no
    // ghost resolution, no mirror rules, no wall faces (block-uniform).
    const bool interior = i0 >= 2 && j0 >= 2 && i0 + TX + 2 <= nx && j0 + TY + 2 <= ny;

    // ---- 1. mesh lines (unless staged) and the haloed tile -------------
    if (!lines_staged) stage_lines(sm, dp, i0, j0);
    {
        // box positions (column, row) of load k: own cells, then the ring
        // (the two rows below, the two above, two columns each side)
        constexpr int NRING = BX * BY - TX * TY;
        constexpr int RQ = (NRING + NT - 1) / NT;
        constexpr int NL = CPT + RQ;
        auto place = [&](int k, int& bc, int& br) -> bool {
            if (k < CPT) {
                bc = tc + k * CW + 2;
                br = tr + 2;
                return true;
            }
            const int t = tid + (k - CPT) * NT;
            if (t < 2 * BX) {
                br = t >= BX;
                bc = t - br * BX;
            } else if (t < 4 * BX) {
                const int u = t - 2 * BX;
                br = BY - 2 + (u >= BX);
                bc = u - (u >= BX) * BX;
            } else {
                const int u = t - 4 * BX;
                br = 2 + (u >> 2);
                bc = (u & 1) + ((u & 2) ? BX - 2 : 0);
            }
            return t < NRING;
        };
        Vec4<S> v[NL];
        int ms[NL];
        bool ok[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {  // issue every load first
            int bc = 0, br = 0;
            ok[k] = place(k, bc, br);
            ms[k] = -1;
            v[k] = {S(0), S(0), S(0), S(0)};
            if (interior) {
                if (ok[k])
                    v[k] = ld_state<LDCG>(&fin[(size_t)(j0 - 2 + br) * pitch + (i0 - 2 + bc)]);
            } else {
                int si = 0, sj = 0;
                ok[k] = ok[k] && resolve_cell(nx, ny, xper, yper, hlo, hhi, i0 - 2 + bc,
                                              j0 - 2 + br, si, sj, ms[k]);
                if (ok[k]) v[k] = ld_state<LDCG>(&fin[(long long)sj * pitch + si]);
            }
        }
        if constexpr (Sm::kRaw) {
#pragma unroll
            for (int k = 0; k < CPT; ++k) sm.raw[tr][tc + k * CW] = v[k];
        }
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            int bc = 0, br = 0;
            if (!place(k, bc, br)) continue;
            const Vec4<S> x = v[k];
            Vec4<R> y = {R(0), R(0), R(0), R(0)};
            if (ok[k]) {
                y = {P::val(x.x, 0), P::val(x.y, 1), P::val(x.z, 2), P::diff(x.w, qTz, 3)};
                if (ms[k] >= 0) y = mirror_values<P>(*dp, ms[k], y, Tz);
            }
            sm.val[br][bc] = y;
        }
    }
    __syncthreads();

    // ---- 2. gradients on the tile plus a 1-cell ring ----------------
    {
        constexpr int NGR = GX * GY - TX * TY;
        constexpr int GQ = CPT + (NGR + NT - 1) / NT;
#pragma unroll(UNROLL)
        for (int k = 0; k < GQ; ++k) {
            int gc, gr;
            if (k < CPT) {
                gc = tc + k * CW + 1;
                gr = tr + 1;
            } else {
                const int t = tid + (k - CPT) * NT;
                if (t >= NGR) break;
                if (t < 2 * GX) {
                    gr = t >= GX ? GY - 1 : 0;
                    gc = t - (t >= GX) * GX;
                } else {
                    const int u = t - 2 * GX;
                    gr = 1 + (u >> 1);
                    gc = (u & 1) ? GX - 1 : 0;
                }
            }
            int c = gc + 1, r = gr + 1;  // box position
            int si, sj, ms = -1;
            Vec4<R> gxv = {R(0), R(0), R(0), R(0)}, gyv = gxv;
            if (interior ||
                resolve_cell(nx, ny, xper, yper, hlo, hhi, i0 - 2 + c, j0 - 2 + r, si, sj, ms)) {
                // a wall ghost takes its partner's gradient, mirrored
                if (ms == kSideW) c += 1;
                else if (ms == kSideE) c -= 1;
                else if (ms == kSideS) r += 1;
                else if (ms == kSideN) r -= 1;
                gg_gradient_r(sm.val[r][c], sm.val[r][c + 1], sm.val[r][c - 1], sm.val[r + 1][c],
                              sm.val[r - 1][c], sm.xc[c].is_next, sm.xc[c - 1].is_next,
                              sm.yc[r].is_next, sm.yc[r - 1].is_next, gxv, gyv);
                if (ms >= 0) mirror_grad(*dp, ms, gxv, gyv);
            }
            sm.gx[gr][gc] = gxv;
            sm.gy[gr][gc] = gyv;
        }
    }
    __syncthreads();

    // ---- 3. faces ----------------------------------------------------
    // x-face (fc, fr) between cells fc - 1 and fc of row fr; y-face (fc, fr)
    // between rows fr - 1 and fr of column fc.  Own: the west and south faces
    // of the thread's cells; then the tile's east column (threads 0..TY-1)
    // and north row (threads TY..TY+TX-1) of faces.
    auto face = [&](auto isx_c, int fc, int fr) {
        constexpr bool isx = decltype(isx_c)::value;
        const int gi = i0 + fc, gj = j0 + fr;
        const bool valid = interior || (isx ? (gi <= nx && gj < ny) : (gi < nx && gj <= ny));
        Vec4<R> out = {R(0), R(0), R(0), R(0)};
        if (valid) {
            const int lc = isx ? fc + 1 : fc + 2, lr = isx ? fr + 2 : fr + 1;
            const int rc = fc + 2, rr = fr + 2;
            CellNT<R> L, Rr;
            R Tbar;
            face_cells<R>(isx, sm.val[lr][lc], sm.val[rr][rc], Tz, sm.gx[lr - 1][lc - 1],
                          sm.gy[lr - 1][lc - 1], sm.gx[rr - 1][rc - 1], sm.gy[rr - 1][rc - 1],
                          L, Rr, Tbar);
            const FaceLine<R> fl = isx ? sm.xl[fc] : sm.yl[fr];
            int wside = -1;
            if (!interior) {
                if (isx && !xper) wside = gi == 0 ? kSideW : (gi == nx ? kSideE : -1);
                if (!isx && !yper)
                    wside = (gj == 0 && !hlo) ? kSideS : ((gj == ny && !hhi) ? kSideN : -1);
            }
            const R uw = wside >= 0 ? P::bcU(dp, wside) : R(0);
            R F[4];
            if constexpr (SCHEME == 1) {
                face_flux_tlbfs<R>(L, Rr, Tbar, fl, wside >= 0 ? R(0) : R(1), uw, F);
            } else if constexpr (sizeof(R) == 4) {
                // FP32: the column stage in packed pairs of the storage order
                const Vec4<R> gl = isx ? sm.gx[lr - 1][lc - 1] : sm.gy[lr - 1][lc - 1];
                const Vec4<R> tl = isx ? sm.gy[lr - 1][lc - 1] : sm.gx[lr - 1][lc - 1];
                const Vec4<R> gr = isx ? sm.gx[rr - 1][rc - 1] : sm.gy[rr - 1][rc - 1];
                const Vec4<R> tr = isx ? sm.gy[rr - 1][rc - 1] : sm.gx[rr - 1][rc - 1];
                R A[4], Sa[4], M[4], Sm[4], B[4], Sb[4];
                face_columns_f32<isx>(sm.val[lr][lc], sm.val[rr][rc], gl, tl, gr, tr, fl, A, Sa, M,
                                      Sm, B, Sb);
                face_flux_columns<R>(A, Sa, M, Sm, B, Sb, Tbar, fl, wside >= 0 ? R(0) : R(1), uw, F);
            } else {
                face_flux<R>(L, Rr, Tbar, fl, wside >= 0 ? R(0) : R(1), uw, F);
            }
            if (isx) out = {F[0], F[1], F[2], F[3]};
            else out = {F[0], F[2], F[1], F[3]};
        }
        if (isx) sm.fx[fr][fc] = out;
        else sm.fy[fr][fc] = out;
    };
    {
        using XF = std::true_type;
        using YF = std::false_type;
        constexpr int TQ = (TX + TY + NT - 1) / NT;  // rounds of the east/north faces
        // the north row starts at the first warp past the east column where
        // the rounds leave room: the two remainders then fall on different
        // warps, and no warp computes two faces more than the others
        constexpr int EW = (TY + 31) / 32 * 32;
        constexpr int YOFF = EW + TX <= TQ * NT ? EW : TY;
#pragma unroll(UNROLL)
        for (int k = 0; k < CPT + TQ; ++k) {
            int fc = tc + k * CW, fr = tr;
            if (k >= CPT) {
                const int t = tid + (k - CPT) * NT;
                if (t >= TY) break;
                fc = TX;
                fr = t;
            }
            face(XF(), fc, fr);
        }
#pragma unroll(UNROLL)
        for (int k = 0; k < CPT + TQ; ++k) {
            int fc = tc + k * CW, fr = tr;
            if (k >= CPT) {
                const int t = tid + (k - CPT) * NT - YOFF;
                if (t >= TX) break;
                if (t < 0) continue;
                fc = t;
                fr = TY;
            }
            face(YF(), fc, fr);
        }
    }
    __syncthreads();

    // ---- 4. update (increment form), 5. residual sums ---------------
    R s0 = R(0), s1 = R(0), s2 = R(0), s3 = R(0);
    {
        const R one = rconst<R>(1.0);
        const R dt = P::dt(dp), bg = P::beta_g(dp), Tr = P::T_ref(dp);
        const R fxb = P::fx(dp), fyb = P::fy(dp);
        bool bad = false;
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            const int cc = tc + m * CW;
            const int gi = i0 + cc, gj = j0 + tr;
            if (gi >= nx || gj >= ny) continue;
            const size_t o = (size_t)gj * pitch + gi;
            Vec4<S> q;
            if constexpr (Sm::kRaw) q = sm.raw[tr][cc];
            else q = ld_state<LDCG>(&fin[o]);
            const Vec4<R> p = sm.val[tr + 2][cc + 2];
            const Vec4<R> Fw = sm.fx[tr][cc], Fe = sm.fx[tr][cc + 1];
            const Vec4<R> Fs = sm.fy[tr][cc], Fn = sm.fy[tr + 1][cc];
            const R ax = sm.xc[cc + 2].dt_w, ay = sm.yc[tr + 2].dt_w;
            const R dr = p.x, u = p.y, v = p.z, T = Tz + p.w;
            const R rho = one + dr;
            // Dt/dV sum_k F_k dS_k for mass, momentum, energy
            R div0, div1, div2, div3;
            if constexpr (sizeof(R) == 4) {
                flux_div_f32(Fw, Fe, Fs, Fn, ax, ay, div0, div1, div2, div3);
            } else {
                div0 = ax * (Fe.x - Fw.x) + ay * (Fn.x - Fs.x);
                div1 = ax * (Fe.y - Fw.y) + ay * (Fn.y - Fs.y);
                div2 = ax * (Fe.z - Fw.z) + ay * (Fn.z - Fs.z);
                div3 = ax * (Fe.w - Fw.w) + ay * (Fn.w - Fs.w);
            }
            // Boussinesq source (Eq. 64, hot fluid rises) and body force
            const R src_x = rho * fxb;
            const R src_y = rho * (bg * (T - Tr) + fyb);
            // rho^{n+1} = rho - div0; q^{n+1} - q = (q div0 - div_q + dt src) / rho^{n+1}
            const R inv = P::rcp(rho - div0);
            const R du = (u * div0 - div1 + dt * src_x) * inv;
            const R dv = (v * div0 - div2 + dt * src_y) * inv;
            const R dT = (T * div0 - div3) * inv;
            const R dr1 = dr - div0, u1 = u + du, v1 = v + dv, T1 = T + dT;
            fout[o] = {P::add(q.x, -div0, 0), P::add(q.y, du, 1), P::add(q.z, dv, 2),
                       P::add(q.w, dT, 3)};
            bad = bad || !(P::in_range(dr1, 0) && P::in_range(u1, 1) && P::in_range(v1, 2) &&
                           P::in_range(T1, 3));
            // |u|^{n+1} - |u|^n without cancellation
            const R m0 = P::fsqrt(u * u + v * v), m1 = P::fsqrt(u1 * u1 + v1 * v1);
            const R den = m0 + m1;
            const R dm = den > R(0) ? (du * (u + u1) + dv * (v + v1)) * P::rcp(den) : R(0);
            s0 += dm * dm;
            s1 += m1 * m1;
            s2 += dT * dT;
            s3 += T1 * T1;
        }
        if (bad) s0 = R(NAN);
    }
    // warp sums in R, then FP64 across warps and tiles
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    s3 = warp_sum(s3);
    if ((tid & 31) == 0) {
        sm.red[tid >> 5][0] = s0;
        sm.red[tid >> 5][1] = s1;
        sm.red[tid >> 5][2] = s2;
        sm.red[tid >> 5][3] = s3;
    }
}

// Threads of a tile block: two cells per thread in the update; one cell per
// thread for the small FP64 tiles, whose point is to spread the narrow FP64
// units' work over as many SM sub-partitions as possible.
template <class P, int TY>
struct TileThreads {
    static constexpr int value = 16 * TY;
};
template <int TY>
struct TileThreads<StoreD, TY> {
    static constexpr int value = TY <= 8 ? 32 * TY : 16 * TY;
};

}  // namespace rtlbfs
