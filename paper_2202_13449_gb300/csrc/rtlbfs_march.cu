// rtlbfs_march.cu -- the RTLBFS step as a warp-marching stencil.
//
// Work unit: one warp, a strip of kStrip = 28 interior columns and a chunk
// of rows [j0, j1) of one cavity.  Lane l holds column c0 - 2 + l: lanes 0-1
// and 30-31 are the 2-cell halo, lanes 2-29 the interior.  The warp walks up
// the chunk keeping a rolling window in registers -- values of rows j, j+1,
// j+2, gradients of rows j and j+1, the flux through the face below row j --
// and per row:
//   loads row j+2 (one coalesced 128-byte line per field),
//   x-faces of row j: each lane computes its west face; the left cell's
//     values and gradients come from lane l-1 by shuffles,
//   Green-Gauss gradients of row j+1 (Eqs. 55-56; x-neighbours by shuffles),
//   the y-face between rows j and j+1 (both cells in the lane's registers),
//   the update of row j (east face from lane l+1) and the residual sums.
// No shared memory, no block barriers; every face is computed once (plus the
// strip-edge halo); HBM sees one read and one write of the state per cell.
// Boundary ghosts follow the same mirror rules as the tiled kernel.
#include <cuda_runtime.h>

#include <cmath>

#include "rtlbfs_dev.cuh"
#include "rtlbfs_kernels.h"

namespace rtlbfs {

namespace {

// Source index of cell coordinate c on a line of n cells with the given
// ends: wrap when periodic; the ghost at -1 / n mirrors cell 0 / n-1 (mside
// set); anything else outside is unused (returns false).
// (halo_lo / halo_hi: the two cells beyond that end are stored ones, see
// kHalo.)
__device__ __forceinline__ bool resolve_1d(int c, int n, bool per, int side_lo, int side_hi,
                                           int& src, int& mside, bool halo_lo = false,
                                           bool halo_hi = false)
{
    mside = -1;
    src = c;
    if (c >= 0 && c < n) return true;
    if ((c < 0 && halo_lo && c >= -2) || (c >= n && halo_hi && c <= n + 1)) return true;
    if (per) {
        src = ((c % n) + n) % n;
        return true;
    }
    if (c == -1) {
        src = 0;
        mside = side_lo;
        return true;
    }
    if (c == n) {
        src = n - 1;
        mside = side_hi;
        return true;
    }
    return false;
}

// Ghost values across wall `side` from the partner's working values (rho - 1,
// u, v, T - Tref), formed in the arithmetic type: rho even, velocity odd
// about the wall velocity (normal component about 0), T odd about T_wall on
// a Dirichlet wall, even on an adiabatic one.  The mirror temperature
// 2 T_wall - T_P can leave the fixed-point range of a stored value; its
// deviation from the unit's reference does not.
template <class P>
__device__ __forceinline__ Vec4<typename P::R> mirror_values_m(const CavityDesc* d, int side,
                                                               Vec4<typename P::R> y,
                                                               typename P::R Tref)
{
    using R = typename P::R;
    const bool xn = (side == kSideW || side == kSideE);
    const R ut2 = R(2) * P::bcU(d, side);
    if (xn) {
        y.y = -y.y;
        y.z = ut2 - y.z;
    } else {
        y.z = -y.z;
        y.y = ut2 - y.y;
    }
    if (d->kind[side] == kDirichlet) y.w = R(2) * (P::Tw(d, side) - Tref) - y.w;
    return y;
}

template <typename R>
__device__ __forceinline__ void mirror_grad_m(int kind, int side, Vec4<R>& gx, Vec4<R>& gy)
{
    const bool xn = (side == kSideW || side == kSideE);
    R* ax = &gx.x;
    R* ay = &gy.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool even = wall_parity(kind, k) > 0;
        if (xn) {
            if (even) ax[k] = -ax[k];
            else ay[k] = -ay[k];
        } else {
            if (even) ay[k] = -ay[k];
            else ax[k] = -ax[k];
        }
    }
}

template <typename T>
__device__ __forceinline__ T shfl_up1(T v)
{
    return __shfl_up_sync(0xffffffffu, v, 1);
}
template <typename T>
__device__ __forceinline__ T shfl_dn1(T v)
{
    return __shfl_down_sync(0xffffffffu, v, 1);
}
template <typename R>
__device__ __forceinline__ Vec4<R> shfl_up1(const Vec4<R>& v)
{
    return {shfl_up1(v.x), shfl_up1(v.y), shfl_up1(v.z), shfl_up1(v.w)};
}
template <typename R>
__device__ __forceinline__ Vec4<R> shfl_dn1(const Vec4<R>& v)
{
    return {shfl_dn1(v.x), shfl_dn1(v.y), shfl_dn1(v.z), shfl_dn1(v.w)};
}

template <typename R>
__device__ __forceinline__ R wsum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class P>
struct MarchMin {
    static constexpr int value = 2;
};
template <>
struct MarchMin<StoreQ> {
    static constexpr int value = kMarchMinBlocksFP32;
};

}  // namespace

template <class P>
__global__ void __launch_bounds__(kMarchThreads, MarchMin<P>::value)
march_kernel(const CavityDesc* __restrict__ descs, CavityRun* __restrict__ runs,
             const int4* __restrict__ units, const int* __restrict__ nunits_ptr, int par)
{
    using S = typename P::S;
    using R = typename P::R;
    using V2 = typename P::V2;
    const int lane = threadIdx.x & 31;
    const int wpb = kMarchThreads / 32;
    chain_sync();
    const int nunits = *nunits_ptr;

    for (int ui = blockIdx.x * wpb + (threadIdx.x >> 5); ui < nunits; ui += gridDim.x * wpb) {
        const int4 wu = units[ui];
        const int slot = wu.x, c0 = wu.y, j0 = wu.z, j1 = wu.w;
        const CavityDesc* dp = descs + slot;
        CavityRun* run = runs + slot;
        // the stop test of the cavity's previous step (lane 0; the cavity's
        // first unit also publishes the header for the next launch)
        int plan = 0;
        if (lane == 0) {
            const CavityCtl d = run_head(run, par);
            if (ui == dp->tile_begin) run_publish(run, par, d);
            plan = d.done | (d.cur << 1) | ((int)(d.steps % 3) << 2);
        }
        plan = __shfl_sync(0xffffffffu, plan, 0);
        if (plan & 1) continue;  // warp-uniform
        const int cur = (plan >> 1) & 1, slot3 = plan >> 2;
        const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch;
        const bool xper = dp->kind[kSideW] == kPeriodic, yper = dp->kind[kSideS] == kPeriodic;
        const bool hlo = dp->kind[kSideS] == kHalo, hhi = dp->kind[kSideN] == kHalo;
        // south / north sides that are walls (not periodic, not a strip's halo)
        const bool wall_s = !yper && !hlo, wall_n = !yper && !hhi;
        const Vec4<S>* __restrict__ fin = static_cast<const Vec4<S>*>(dp->f[cur][0]);
        Vec4<S>* __restrict__ fout = static_cast<Vec4<S>*>(dp->f[cur ^ 1][0]);
        const CellLine<R>* xc = static_cast<const CellLine<R>*>(dp->xcell);
        const CellLine<R>* yc = static_cast<const CellLine<R>*>(dp->ycell);
        const FaceLine<R>* xl = static_cast<const FaceLine<R>*>(dp->xline);
        const FaceLine<R>* yl = static_cast<const FaceLine<R>*>(dp->yline);

        // this lane's column
        const int g = c0 - 2 + lane;
        int gs, xms;
        const bool colok = resolve_1d(g, nx, xper, kSideW, kSideE, gs, xms);
        const R isx_e = xc[min(max(g + 2, 0), nx + 3)].is_next;
        const R isx_w = xc[min(max(g + 1, 0), nx + 3)].is_next;
        const FaceLine<R> flx = xl[min(max(g, 0), nx)];
        const bool upd_lane = lane >= 2 && lane <= 29 && g < nx;
        const int wsx = (!xper && g == 0) ? kSideW : ((!xper && g == nx) ? kSideE : -1);
        const bool xghosts = !xper && (c0 == 0 || c0 + 29 >= nx);  // warp-uniform

        // temperature reference of this unit
        const S qTz = fin[(size_t)min(j0, ny - 1) * pitch + min(c0 + 14, nx - 1)].w;
        const R Tz = P::val(qTz, 3);

        // raw row r of this lane's column (ghost rule applied later in conv)
        auto fetch = [&](int r, Vec4<S>& q) {
            int rs, yms;
            const bool rowok = resolve_1d(r, ny, yper, kSideS, kSideN, rs, yms, hlo, hhi);
            q = {S(0), S(0), S(0), S(0)};
            if (colok && rowok && !(xms >= 0 && yms >= 0)) q = fin[(long long)rs * pitch + gs];
        };
        auto conv = [&](int r, Vec4<S> q) -> Vec4<R> {
            int rs, yms;
            const bool rowok = resolve_1d(r, ny, yper, kSideS, kSideN, rs, yms, hlo, hhi);
            if (!(colok && rowok && !(xms >= 0 && yms >= 0))) return {R(0), R(0), R(0), R(0)};
            Vec4<R> y = {P::val(q.x, 0), P::val(q.y, 1), P::val(q.z, 2), P::diff(q.w, qTz, 3)};
            if (xms >= 0) y = mirror_values_m<P>(dp, xms, y, Tz);
            if (yms >= 0) y = mirror_values_m<P>(dp, yms, y, Tz);
            return y;
        };
        // Green-Gauss gradient of row r from its value v, the rows below (vs)
        // and above (vn); x-neighbours by shuffles.  Wall ghost lanes mirror
        // their partner lane.
        auto grad = [&](int r, const Vec4<R>& vs, const Vec4<R>& v, const Vec4<R>& vn,
                        Vec4<R>& gx, Vec4<R>& gy) {
            const Vec4<R> vw = shfl_up1(v), ve = shfl_dn1(v);
            const int ri = min(max(r + 2, 1), ny + 3);
            const R isy_n = yc[ri].is_next, isy_s = yc[ri - 1].is_next;
            if constexpr (sizeof(R) == 4) {
                gg_gradient_f32(v, ve, vw, vn, vs, isx_e, isx_w, isy_n, isy_s, gx, gy);
            } else {
                gx.x = (ve.x - v.x) * isx_e + (v.x - vw.x) * isx_w;
                gx.y = (ve.y - v.y) * isx_e + (v.y - vw.y) * isx_w;
                gx.z = (ve.z - v.z) * isx_e + (v.z - vw.z) * isx_w;
                gx.w = (ve.w - v.w) * isx_e + (v.w - vw.w) * isx_w;
                gy.x = (vn.x - v.x) * isy_n + (v.x - vs.x) * isy_s;
                gy.y = (vn.y - v.y) * isy_n + (v.y - vs.y) * isy_s;
                gy.z = (vn.z - v.z) * isy_n + (v.z - vs.z) * isy_s;
                gy.w = (vn.w - v.w) * isy_n + (v.w - vs.w) * isy_s;
            }
            if (xghosts) {
                const Vec4<R> gxd = shfl_dn1(gx), gyd = shfl_dn1(gy);
                const Vec4<R> gxu = shfl_up1(gx), gyu = shfl_up1(gy);
                if (xms >= 0) {
                    gx = xms == kSideW ? gxd : gxu;
                    gy = xms == kSideW ? gyd : gyu;
                    mirror_grad_m(dp->kind[xms], xms, gx, gy);
                }
            }
        };
        // One packed call for two faces: component x = the x-face west of this
        // lane's column in row jx (left cell from lane l-1), component y = the
        // y-face between rows jf-1 and jf of this lane's column.
        auto faces = [&](const Vec4<R>& vxl, const Vec4<R>& gxxl, const Vec4<R>& gyxl,
                         const Vec4<R>& vxr, const Vec4<R>& gxxr, const Vec4<R>& gyxr, int jf,
                         const Vec4<R>& vyl, const Vec4<R>& gxyl, const Vec4<R>& gyyl,
                         const Vec4<R>& vyr, const Vec4<R>& gxyr, const Vec4<R>& gyyr,
                         Vec4<R>& Fxo, Vec4<R>& Fyo) {
            const FaceLine<R> fly = yl[min(max(jf, 0), ny)];
            const int ws = (wall_s && jf == 0) ? kSideS : ((wall_n && jf == ny) ? kSideN : -1);
            const R uwy = ws >= 0 ? P::bcU(dp, ws) : R(0);
            const R uwx = wsx >= 0 ? P::bcU(dp, wsx) : R(0);
            CellNT<V2> L, Rr;
            // x-face frame (n = x, t = y) in .x, y-face frame (n = y, t = x) in .y
            L.q[0] = {vxl.x, vyl.x};
            L.q[1] = {vxl.y, vyl.z};
            L.q[2] = {vxl.z, vyl.y};
            L.q[3] = {R(0), R(0)};
            L.gn[0] = {gxxl.x, gyyl.x};
            L.gn[1] = {gxxl.y, gyyl.z};
            L.gn[2] = {gxxl.z, gyyl.y};
            L.gn[3] = {gxxl.w, gyyl.w};
            L.gt[0] = {gyxl.x, gxyl.x};
            L.gt[1] = {gyxl.y, gxyl.z};
            L.gt[2] = {gyxl.z, gxyl.y};
            L.gt[3] = {gyxl.w, gxyl.w};
            Rr.q[0] = {vxr.x, vyr.x};
            Rr.q[1] = {vxr.y, vyr.z};
            Rr.q[2] = {vxr.z, vyr.y};
            Rr.q[3] = {vxr.w - vxl.w, vyr.w - vyl.w};
            Rr.gn[0] = {gxxr.x, gyyr.x};
            Rr.gn[1] = {gxxr.y, gyyr.z};
            Rr.gn[2] = {gxxr.z, gyyr.y};
            Rr.gn[3] = {gxxr.w, gyyr.w};
            Rr.gt[0] = {gyxr.x, gxyr.x};
            Rr.gt[1] = {gyxr.y, gxyr.z};
            Rr.gt[2] = {gyxr.z, gxyr.y};
            Rr.gt[3] = {gyxr.w, gxyr.w};
            FaceLine<V2> fl;
            fl.h = {flx.h, fly.h};
            fl.cL = {flx.cL, fly.cL};
            fl.cR = {flx.cR, fly.cR};
            fl.m_nu_2h = {flx.m_nu_2h, fly.m_nu_2h};
            fl.m_chi_2h = {flx.m_chi_2h, fly.m_chi_2h};
            fl.m_tf15 = {flx.m_tf15, fly.m_tf15};
            fl.m_tg15 = {flx.m_tg15, fly.m_tg15};
            const V2 Tbar = {Tz + vxl.w, Tz + vyl.w};
            const V2 keep = {wsx >= 0 ? R(0) : R(1), ws >= 0 ? R(0) : R(1)};
            const V2 uw = {uwx, uwy};
            V2 F[4];
            face_flux<V2>(L, Rr, Tbar, fl, keep, uw, F);
            Fxo = {F[0].x, F[1].x, F[2].x, F[3].x};
            Fyo = {F[0].y, F[2].y, F[1].y, F[3].y};
        };

        // The same two faces as two scalar evaluations.
        auto face1 = [&](const Vec4<R>& vxl, const Vec4<R>& gxxl, const Vec4<R>& gyxl,
                         const Vec4<R>& vxr, const Vec4<R>& gxxr, const Vec4<R>& gyxr, int jf,
                         const Vec4<R>& vyl, const Vec4<R>& gxyl, const Vec4<R>& gyyl,
                         const Vec4<R>& vyr, const Vec4<R>& gxyr, const Vec4<R>& gyyr,
                         Vec4<R>& Fxo, Vec4<R>& Fyo) {
            {
                R F[4];
                if constexpr (sizeof(R) == 4) {  // FP32: packed column stage
                    R A[4], Sa[4], M[4], Sm[4], B[4], Sb[4];
                    face_columns_f32<true>(vxl, vxr, gxxl, gyxl, gxxr, gyxr, flx, A, Sa, M, Sm, B, Sb);
                    face_flux_columns<R>(A, Sa, M, Sm, B, Sb, Tz + vxl.w, flx, wsx >= 0 ? R(0) : R(1),
                                         wsx >= 0 ? P::bcU(dp, wsx) : R(0), F);
                } else {
                    CellNT<R> L = {{vxl.x, vxl.y, vxl.z, R(0)}, {gxxl.x, gxxl.y, gxxl.z, gxxl.w},
                                   {gyxl.x, gyxl.y, gyxl.z, gyxl.w}};
                    CellNT<R> Rr = {{vxr.x, vxr.y, vxr.z, vxr.w - vxl.w},
                                    {gxxr.x, gxxr.y, gxxr.z, gxxr.w}, {gyxr.x, gyxr.y, gyxr.z, gyxr.w}};
                    face_flux<R>(L, Rr, Tz + vxl.w, flx, wsx >= 0 ? R(0) : R(1),
                                 wsx >= 0 ? P::bcU(dp, wsx) : R(0), F);
                }
                Fxo = {F[0], F[1], F[2], F[3]};
            }
            {
                const FaceLine<R> fly = yl[min(max(jf, 0), ny)];
                const int ws = (wall_s && jf == 0) ? kSideS : ((wall_n && jf == ny) ? kSideN : -1);
                R F[4];
                if constexpr (sizeof(R) == 4) {
                    R A[4], Sa[4], M[4], Sm[4], B[4], Sb[4];
                    face_columns_f32<false>(vyl, vyr, gyyl, gxyl, gyyr, gxyr, fly, A, Sa, M, Sm, B, Sb);
                    face_flux_columns<R>(A, Sa, M, Sm, B, Sb, Tz + vyl.w, fly, ws >= 0 ? R(0) : R(1),
                                         ws >= 0 ? P::bcU(dp, ws) : R(0), F);
                } else {
                    CellNT<R> L = {{vyl.x, vyl.z, vyl.y, R(0)}, {gyyl.x, gyyl.z, gyyl.y, gyyl.w},
                                   {gxyl.x, gxyl.z, gxyl.y, gxyl.w}};
                    CellNT<R> Rr = {{vyr.x, vyr.z, vyr.y, vyr.w - vyl.w},
                                    {gyyr.x, gyyr.z, gyyr.y, gyyr.w}, {gxyr.x, gxyr.z, gxyr.y, gxyr.w}};
                    face_flux<R>(L, Rr, Tz + vyl.w, fly, ws >= 0 ? R(0) : R(1),
                                 ws >= 0 ? P::bcU(dp, ws) : R(0), F);
                }
                Fyo = {F[0], F[2], F[1], F[3]};
            }
        };

        // ---- prologue: rows j0-2 .. j0+1, gradients of j0-1 and j0,
        //      the face between rows j0-1 and j0, prefetch of row j0+2
        Vec4<R> v0, v1, v2;
        Vec4<R> gx0, gy0, gx1, gy1;
        Vec4<S> qpre;
        {
            Vec4<S> qa, qb, qc, qd;
            fetch(j0 - 2, qa);
            fetch(j0 - 1, qb);
            fetch(j0, qc);
            fetch(j0 + 1, qd);
            fetch(j0 + 2, qpre);
            const Vec4<R> vm2 = conv(j0 - 2, qa), vm1 = conv(j0 - 1, qb);
            v0 = conv(j0, qc);
            v1 = conv(j0 + 1, qd);
            Vec4<R> gxm1, gym1;
            grad(j0 - 1, vm2, vm1, v0, gxm1, gym1);
            grad(j0, vm1, v0, v1, gx0, gy0);
            if (wall_s && j0 == 0) {  // row -1 is the south ghost: mirror row 0
                gxm1 = gx0;
                gym1 = gy0;
                mirror_grad_m(dp->kind[kSideS], kSideS, gxm1, gym1);
            }
            gx1 = gxm1;  // the face below row j0 is computed from (j0-1, j0)
            gy1 = gym1;
            v2 = vm1;
        }
        // the face below row j0 (paired with a throw-away copy of itself)
        Vec4<R> Fs, Fdummy;
        faces(v2, gx1, gy1, v0, gx0, gy0, j0, v2, gx1, gy1, v0, gx0, gy0, Fdummy, Fs);

        R s0 = R(0), s1 = R(0), s2 = R(0), s3 = R(0);
        bool bad = false;

        for (int j = j0; j < j1; ++j) {
            v2 = conv(j + 2, qpre);
            fetch(j + 3, qpre);  // in flight during this row's work
            Vec4<S> qo = {S(0), S(0), S(0), S(0)};
            if (upd_lane) qo = fin[(size_t)j * pitch + g];  // raw state of the updated cell (L1)
            // gradients of row j+1 (a north ghost row mirrors row j)
            grad(j + 1, v0, v1, v2, gx1, gy1);
            if (wall_n && j + 1 == ny) {
                gx1 = gx0;
                gy1 = gy0;
                mirror_grad_m(dp->kind[kSideN], kSideN, gx1, gy1);
            }
            // x-face west of this lane's column in row j and the y-face
            // between rows j and j+1
            Vec4<R> Fx, Fn;
            {
                const Vec4<R> vl = shfl_up1(v0), gxl = shfl_up1(gx0), gyl = shfl_up1(gy0);
#if RTLBFS_PAIR_FACES
                faces(vl, gxl, gyl, v0, gx0, gy0, j + 1, v0, gx0, gy0, v1, gx1, gy1, Fx, Fn);
#else
                face1(vl, gxl, gyl, v0, gx0, gy0, j + 1, v0, gx0, gy0, v1, gx1, gy1, Fx, Fn);
#endif
            }
            const Vec4<R> Fe = shfl_dn1(Fx);
            // update row j
            if (upd_lane) {
                const R one = rconst<R>(1.0);
                const R ax = xc[g + 2].dt_w;
                const R ay = yc[j + 2].dt_w;
                const R dr = v0.x, u = v0.y, v = v0.z, T = Tz + v0.w;
                const R rho = one + dr;
                R div0, div1, div2, div3;
                if constexpr (sizeof(R) == 4) {
                    flux_div_f32(Fx, Fe, Fs, Fn, ax, ay, div0, div1, div2, div3);
                } else {
                    div0 = ax * (Fe.x - Fx.x) + ay * (Fn.x - Fs.x);
                    div1 = ax * (Fe.y - Fx.y) + ay * (Fn.y - Fs.y);
                    div2 = ax * (Fe.z - Fx.z) + ay * (Fn.z - Fs.z);
                    div3 = ax * (Fe.w - Fx.w) + ay * (Fn.w - Fs.w);
                }
                const R src_x = rho * P::fx(dp);
                const R src_y = rho * (P::beta_g(dp) * (T - P::T_ref(dp)) + P::fy(dp));
                const R dtc = P::dt(dp);
                const R inv = P::rcp(rho - div0);
                const R du = (u * div0 - div1 + dtc * src_x) * inv;
                const R dv = (v * div0 - div2 + dtc * src_y) * inv;
                const R dT = (T * div0 - div3) * inv;
                const R dr1 = dr - div0, u1 = u + du, v1n = v + dv, T1 = T + dT;
                fout[(size_t)j * pitch + g] = {P::add(qo.x, -div0, 0), P::add(qo.y, du, 1),
                                               P::add(qo.z, dv, 2), P::add(qo.w, dT, 3)};
                bad = bad || !(P::in_range(dr1, 0) && P::in_range(u1, 1) && P::in_range(v1n, 2) &&
                               P::in_range(T1, 3));
                const R m0 = P::fsqrt(u * u + v * v), m1 = P::fsqrt(u1 * u1 + v1n * v1n);
                const R den = m0 + m1;
                const R dm = den > R(0) ? (du * (u + u1) + dv * (v + v1n)) * P::rcp(den) : R(0);
                s0 += dm * dm;
                s1 += m1 * m1;
                s2 += dT * dT;
                s3 += T1 * T1;
            }
            // roll the window
            Fs = Fn;
            v0 = v1;
            v1 = v2;
            gx0 = gx1;
            gy0 = gy1;
        }
        if (bad) s0 = R(NAN);
        s0 = wsum(s0);
        s1 = wsum(s1);
        s2 = wsum(s2);
        s3 = wsum(s3);
        // the step's residual sums; the next launch tests them
        if (lane == 0) {
            double* acc = run->acc[slot3];
            atomicAdd(&acc[0], (double)s0);
            atomicAdd(&acc[1], (double)s1);
            atomicAdd(&acc[2], (double)s2);
            atomicAdd(&acc[3], (double)s3);
        }
        __syncwarp();
    }
}

cudaError_t march_prepare(int precision)
{
    (void)precision;
    return cudaSuccess;
}

cudaError_t march_occupancy(int precision, int* blocks_per_sm)
{
    if (precision == 0)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, march_kernel<StoreD>,
                                                             kMarchThreads, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, march_kernel<StoreQ>,
                                                         kMarchThreads, 0);
}

cudaError_t launch_march(int precision, int grid, cudaStream_t s, const CavityDesc* descs,
                         CavityRun* runs, const int4* units, const int* nunits, int par)
{
    if (precision == 0)
        return launch_chained(march_kernel<StoreD>, grid, kMarchThreads, 0, s, descs, runs, units,
                              nunits, par);
    return launch_chained(march_kernel<StoreQ>, grid, kMarchThreads, 0, s, descs, runs, units,
                          nunits, par);
}

}  // namespace rtlbfs
