// rtlbfs_curv.cu -- the fused 2D RTLBFS time step on structured curvilinear
// (body-fitted) meshes on sm_103a (arXiv 2202.13449, Section 3.2 with the
// unit lattice of each face in its local frame; the O-meshes of Section
// 4.3), its FP64 wall-heat sums and the rtlbfsc_* C ABI.
//
// Geometry is precomputed on the host in FP64 (cell centres, areas, ghost
// centres mirrored across wall faces).  The step kernel reads two records:
// per face, its unit normal and length, the tangential offsets of the two
// centres, the lattice spacing with their normal offsets and the transport
// coefficients of Eqs. 9-10 (FaceRec); per cell, the four Green-Gauss
// coefficients w_f S_f / A of Eqs. 55-56 (CellGrad).
//
// Step kernel.  Work unit: a TX x TY tile of cells.  Before it waits for the
// previous step's grid, a block starts asynchronous copies of the tile's
// geometry into shared memory (it never changes between steps); then:
//   1. the tile plus a 2-cell ring of (rho - 1, u, v, T - Tz), ghosts
//      materialised (wall mirror, free stream, periodic seam);
//   2. Green-Gauss gradients (Eqs. 55-56) on the tile plus a 1-cell ring,
//      written over the cell's staged coefficients; a wall ghost takes its
//      partner's gradient reflected in the face normal;
//   3. every face of the tile: the cells' values and gradients rotated into
//      the face frame (n, t), the tangential offsets of the centres folded
//      into the values, then the rectilinear face template face_flux (Eq. 29
//      nodes, Eqs. 46-48, Eqs. 57-59) and the fluxes rotated back;
//   4. the update with the face lengths and areas, the Boussinesq source
//      along the gravity direction, and the residual sums; the last unit
//      finalises the step (residual, step counter, buffer flip, stop test).
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
#include "rtlbfs_curv.h"
#include "rtlbfs_dev.cuh"
#include "rtlbfs_kernels.h"

namespace rtlbfs {
extern std::atomic<long long> g_launches;
}

namespace rtlbfsc {

using rtlbfs::CellNT;
using rtlbfs::chain_sync;
using rtlbfs::launch_chained;
using rtlbfs::FaceLine;
using rtlbfs::face_flux;
using rtlbfs::face_flux_columns;
using rtlbfs::kConverged;
using rtlbfs::kDiverged;
using rtlbfs::kMaxSteps;
using rtlbfs::kRunning;
using rtlbfs::StoreD;
using rtlbfs::StoreQ;
using rtlbfs::Vec4;
using rtlbfs::vfma;

constexpr int kDir = 0, kAdia = 1, kPer = 2, kFar = 3;

// Geometry of one face (16 values, host side and the FP64 wall sums).
template <typename R>
struct __align__(16) FaceGeo {
    R Sx, Sy;   // face vector: length times the unit normal, from the low- to the high-index cell
    R wR;       // Eq. 56: phi_S = phi_L + wR (phi_R - phi_L)
    R pad;
    R nx, ny;   // unit normal
    R tL, tR;   // tangential offsets (x_L - x_S).t, (x_R - x_S).t, t = (-n_y, n_x)
    R h, cL, cR, m_nu_2h, m_chi_2h, m_tf15, m_tg15;  // FaceLine fields
    R len;      // face length
};

// What the face stage of the step kernel reads of a face (12 values).
template <typename R>
struct __align__(16) FaceRec {
    R nx, ny, tL, tR;
    R h, cL, cR, m_nu_2h;
    R m_chi_2h, m_tf15, m_tg15, len;
};

template <typename R>
__host__ __device__ __forceinline__ FaceRec<R> face_rec(const FaceGeo<double>& a)
{
    FaceRec<R> b;
    b.nx = (R)a.nx;
    b.ny = (R)a.ny;
    b.tL = (R)a.tL;
    b.tR = (R)a.tR;
    b.h = (R)a.h;
    b.cL = (R)a.cL;
    b.cR = (R)a.cR;
    b.m_nu_2h = (R)a.m_nu_2h;
    b.m_chi_2h = (R)a.m_chi_2h;
    b.m_tf15 = (R)a.m_tf15;
    b.m_tg15 = (R)a.m_tg15;
    b.len = (R)a.len;
    return b;
}

// Green-Gauss coefficients of a cell (Eqs. 55-56 with the weights and the
// area folded in): grad phi = sum_f c_f (phi_f - phi_P) over the east, west,
// north and south neighbours, c_f = +-w_f S_f / A.
template <typename R>
struct __align__(16) CellGrad {
    R c[8];  // (x, y) of east, west, north, south
};

// A 16-byte aligned record by 16-byte vector loads (the unused groups are
// not loaded).
template <typename T>
__device__ __forceinline__ T ld_vec(const T* p)
{
    static_assert(sizeof(T) % 16 == 0 && alignof(T) >= 16, "16-byte records");
    T v;
    const uint4* src = reinterpret_cast<const uint4*>(p);
    uint4* dst = reinterpret_cast<uint4*>(&v);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(T) / 16); ++k) dst[k] = src[k];
    return v;
}

struct DescC {
    int ni, nj, per, tiles_x, tiles_y, units;
    int kind[4];
    double gdir[2], force[2], beta_g, T_ref, dt;
    float f_gdir[2], f_force[2], f_beta_g, f_T_ref, f_dt;
    double bcU[4][2], bcT[4];
    float f_bcU[4][2], f_bcT[4];
    double d_inf[4];  // free stream (rho - 1, u, v, T)
    float f_inf[4];
    void* rec[2];                          // Vec4<S>[cells]
    const void* fri;                       // FaceRec<R>[nj][ni+1]
    const void* frj;                       // FaceRec<R>[nj+1][ni]
    const void* cg;                        // CellGrad<R>[cells]
    const void* dta;                       // R[cells]: dt / area
    const void* gi_d;                      // FP64 copies for the wall sums
    const void* gj_d;
    const void* ia_d;
};

// Run control: the two-header record of the rectilinear solver (the stop
// test of step k is made by the launch of step k + 1; see CavityRun).
using rtlbfs::CavityCtl;
using rtlbfs::CavityRun;

template <class P>
struct CstC;
template <>
struct CstC<StoreD> {
    static __device__ __forceinline__ double gdir(const DescC& d, int a) { return d.gdir[a]; }
    static __device__ __forceinline__ double force(const DescC& d, int a) { return d.force[a]; }
    static __device__ __forceinline__ double beta_g(const DescC& d) { return d.beta_g; }
    static __device__ __forceinline__ double T_ref(const DescC& d) { return d.T_ref; }
    static __device__ __forceinline__ double dt(const DescC& d) { return d.dt; }
    static __device__ __forceinline__ double uw(const DescC& d, int s, int c) { return d.bcU[s][c]; }
    static __device__ __forceinline__ double Tw(const DescC& d, int s) { return d.bcT[s]; }
    static __device__ __forceinline__ double inf(const DescC& d, int q) { return d.d_inf[q]; }
};
template <>
struct CstC<StoreQ> {
    static __device__ __forceinline__ float gdir(const DescC& d, int a) { return d.f_gdir[a]; }
    static __device__ __forceinline__ float force(const DescC& d, int a) { return d.f_force[a]; }
    static __device__ __forceinline__ float beta_g(const DescC& d) { return d.f_beta_g; }
    static __device__ __forceinline__ float T_ref(const DescC& d) { return d.f_T_ref; }
    static __device__ __forceinline__ float dt(const DescC& d) { return d.f_dt; }
    static __device__ __forceinline__ float uw(const DescC& d, int s, int c) { return d.f_bcU[s][c]; }
    static __device__ __forceinline__ float Tw(const DescC& d, int s) { return d.f_bcT[s]; }
    static __device__ __forceinline__ float inf(const DescC& d, int q) { return d.f_inf[q]; }
};

// Resolve a cell index along i (periodic or bounded by sides 0, 1) or j
// (bounded by sides 2, 3): source index and the ghost's side (-1: none);
// false for positions no stencil uses.
__host__ __device__ __forceinline__ bool resolve_c(int c, int n, bool per, int lo, int hi, int& src,
                                                   int& side)
{
    side = -1;
    src = c;
    if (c >= 0 && c < n) return true;
    if (per) {
        src = ((c % n) + n) % n;
        return true;
    }
    if (c == -1) {
        src = 0;
        side = lo;
        return true;
    }
    if (c == n) {
        src = n - 1;
        side = hi;
        return true;
    }
    return false;
}

// Ghost values across side s from the partner's working values o =
// (rho - 1, u, v, T - Tref): a wall mirrors the partner (rho even, velocity
// odd about the wall velocity, T odd about T_wall or even); a far-field
// side holds the free stream.  Formed in the arithmetic type relative to
// Tref: 2 T_wall - T_P can leave the fixed-point range of a stored
// temperature (a hot wall next to cold fluid) while its deviation from a
// reference inside the tile does not.
template <class P, typename R>
__device__ __forceinline__ void ghost_values(const DescC& d, int s, R Tref, R o[4])
{
    if (d.kind[s] == kFar) {
        o[0] = CstC<P>::inf(d, 0);
        o[1] = CstC<P>::inf(d, 1);
        o[2] = CstC<P>::inf(d, 2);
        o[3] = CstC<P>::inf(d, 3) - Tref;
        return;
    }
    o[1] = R(2) * CstC<P>::uw(d, s, 0) - o[1];
    o[2] = R(2) * CstC<P>::uw(d, s, 1) - o[2];
    if (d.kind[s] == kDir) o[3] = R(2) * (CstC<P>::Tw(d, s) - Tref) - o[3];
}

// Reflect the gradients g[8] (d/dx, d/dy of rho, u, v, T) of a wall
// ghost's partner in the face normal (nx, ny): even quantities keep the
// tangential and negate the normal part, odd quantities the reverse.
template <typename R>
__host__ __device__ __forceinline__ void mirror_grad_c(int kind, R nx, R ny, R g[8])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const R gx = g[2 * q], gy = g[2 * q + 1];
        const R gn = gx * nx + gy * ny;
        R rx = gx - R(2) * gn * nx, ry = gy - R(2) * gn * ny;
        const bool odd = (q == 1 || q == 2) || (q == 3 && kind == kDir);
        if (odd) {
            rx = -rx;
            ry = -ry;
        }
        g[2 * q] = rx;
        g[2 * q + 1] = ry;
    }
}

// face_columns in FP32 on face-frame cells whose components were formed
// in registers (a curvilinear face's rotated values): pairs (rho, u_n) and
// (u_t, T) in packed FP32x2 instructions, the same operations bit for bit.
__device__ __forceinline__ void face_columns_nt_f32(const rtlbfs::CellNT<float>& L, const rtlbfs::CellNT<float>& Rc,
                                                    const FaceLine<float>& fl, float A[4],
                                                    float Sa[4], float M[4], float Sm[4],
                                                    float B[4], float Sb[4])
{
    const float h = fl.h;
    const float wL = fl.cL + h, mwR = fl.cR - h, hh = h * 0.5f;
    const float2 cL2 = make_float2(fl.cL, fl.cL), cR2 = make_float2(fl.cR, fl.cR);
    const float2 wL2 = make_float2(wL, wL), mwR2 = make_float2(mwR, mwR);
    const float2 h2 = make_float2(h, h), hh2 = make_float2(hh, hh), half2 = make_float2(0.5f, 0.5f);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int k = 2 * i;
        const float2 ql = make_float2(L.q[k], L.q[k + 1]), qr = make_float2(Rc.q[k], Rc.q[k + 1]);
        const float2 nl = make_float2(L.gn[k], L.gn[k + 1]), nr = make_float2(Rc.gn[k], Rc.gn[k + 1]);
        const float2 tl = make_float2(L.gt[k], L.gt[k + 1]), tr = make_float2(Rc.gt[k], Rc.gt[k + 1]);
        const float2 a = __ffma2_rn(nl, cL2, ql), sa = __fmul2_rn(tl, h2);
        const float2 b = __ffma2_rn(nr, cR2, qr), sb = __fmul2_rn(tr, h2);
        const float2 m = __fmul2_rn(half2, __fadd2_rn(__ffma2_rn(nl, wL2, ql), __ffma2_rn(nr, mwR2, qr)));
        const float2 sm = __fmul2_rn(hh2, __fadd2_rn(tl, tr));
        A[k] = a.x, A[k + 1] = a.y;
        Sa[k] = sa.x, Sa[k + 1] = sa.y;
        B[k] = b.x, B[k + 1] = b.y;
        Sb[k] = sb.x, Sb[k + 1] = sb.y;
        M[k] = m.x, M[k + 1] = m.y;
        Sm[k] = sm.x, Sm[k + 1] = sm.y;
    }
}

// One face: values v[4] = (rho - 1, u, v, T - Tz) and gradients g[8] of the
// two cells, the face geometry, the wall flag and tangential wall velocity.
// Returns the fluxes times the face length in x, y components.
template <typename R>
__host__ __device__ __forceinline__ void face_c(const R vL[4], const R gL[8], const R vR[4],
                                                const R gR[8], const FaceRec<R>& fg, R keep,
                                                R uwx, R uwy, R Tz, R out[4])
{
    const R nx = fg.nx, ny = fg.ny, tx = -ny, ty = nx;
    CellNT<R> L, Rr;
    auto frame = [&](const R v[4], const R g[8], R toff, CellNT<R>& c) {
        const R gnu = g[2] * nx + g[3] * ny, gtu = g[2] * tx + g[3] * ty;
        const R gnv = g[4] * nx + g[5] * ny, gtv = g[4] * tx + g[5] * ty;
        c.gn[0] = g[0] * nx + g[1] * ny;
        c.gt[0] = g[0] * tx + g[1] * ty;
        c.gn[1] = nx * gnu + ny * gnv;  // u_n = n.u
        c.gt[1] = nx * gtu + ny * gtv;
        c.gn[2] = tx * gnu + ty * gnv;  // u_t = t.u
        c.gt[2] = tx * gtu + ty * gtv;
        c.gn[3] = g[6] * nx + g[7] * ny;
        c.gt[3] = g[6] * tx + g[7] * ty;
        const R un = nx * v[1] + ny * v[2], ut = tx * v[1] + ty * v[2];
        // values on the face's normal line: the centre's tangential offset folded in
        c.q[0] = v[0] - c.gt[0] * toff;
        c.q[1] = un - c.gt[1] * toff;
        c.q[2] = ut - c.gt[2] * toff;
        c.q[3] = v[3] - c.gt[3] * toff;
    };
    frame(vL, gL, fg.tL, L);
    frame(vR, gR, fg.tR, Rr);
    const R tauL = L.q[3];
    L.q[3] = R(0);
    Rr.q[3] = Rr.q[3] - tauL;
    FaceLine<R> fl;
    fl.h = fg.h;
    fl.cL = fg.cL;
    fl.cR = fg.cR;
    fl.m_nu_2h = fg.m_nu_2h;
    fl.m_chi_2h = fg.m_chi_2h;
    fl.m_tf15 = fg.m_tf15;
    fl.m_tg15 = fg.m_tg15;
    fl.pad = R(0);
    const R uwt = uwx * tx + uwy * ty;
    R F[4];
#ifdef __CUDA_ARCH__
    constexpr bool packed = sizeof(R) == 4;  // FP32 on the device: packed column stage
#else
    constexpr bool packed = false;
#endif
    if constexpr (packed) {
        R A[4], Sa[4], M[4], Sm[4], B[4], Sb[4];
        face_columns_nt_f32(L, Rr, fl, A, Sa, M, Sm, B, Sb);
        face_flux_columns<R>(A, Sa, M, Sm, B, Sb, Tz + tauL, fl, keep, uwt, F);
    } else {
        face_flux<R>(L, Rr, Tz + tauL, fl, keep, uwt, F);
    }
    out[0] = F[0] * fg.len;
    out[1] = (F[1] * nx + F[2] * tx) * fg.len;
    out[2] = (F[1] * ny + F[2] * ty) * fg.len;
    out[3] = F[3] * fg.len;
}

// Asynchronous global -> shared copies (completed by cp_async_wait_all).
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_n(void* sdst, const void* gsrc, float*)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(a), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_n(void* sdst, const void* gsrc, double*)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(a), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <class P, int TX, int TY>
struct SmemC {
    using R = typename P::R;
    static constexpr int BX = TX + 4, BY = TY + 4, GX = TX + 2, GY = TY + 2, NT = TX * TY;
    FaceRec<R> fi[TY][TX + 1];  // face records; each face's flux is written over its own
    FaceRec<R> fj[TY + 1][TX];
    CellGrad<R> g[GY][GX];      // coefficients, overwritten by the gradients
    R v[4][BY][BX];
    R dta[TY][TX];
    R red[NT / 32][4];  // per-warp residual partials
    int plan[3];        // after the stop test: done, cur, sum slot
};

template <class P, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) curv_step_kernel(const DescC* __restrict__ dp,
                                                           CavityRun* __restrict__ run, int par)
{
    using S = typename P::S;
    using R = typename P::R;
    using Sm = SmemC<P, TX, TY>;
    constexpr int BX = Sm::BX, BY = Sm::BY, GX = Sm::GX, GY = Sm::GY, NT = Sm::NT;
    constexpr int FC = sizeof(FaceRec<R>) / 16, GC = sizeof(CellGrad<R>) / 16;
    extern __shared__ __align__(16) unsigned char smraw[];
    Sm& sm = *reinterpret_cast<Sm*>(smraw);
    const DescC& d = *dp;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int ni = d.ni, nj = d.nj;
    const bool per = d.per != 0;
    const int i0 = (blockIdx.x % d.tiles_x) * TX, j0 = (blockIdx.x / d.tiles_x) * TY;
    const FaceRec<R>* fI = static_cast<const FaceRec<R>*>(d.fri);
    const FaceRec<R>* fJ = static_cast<const FaceRec<R>*>(d.frj);
    const CellGrad<R>* cG = static_cast<const CellGrad<R>*>(d.cg);
    const R* dta = static_cast<const R*>(d.dta);

    // 0. the tile's geometry (constant across steps) into shared memory
    for (int t = tid; t < TY * (TX + 1) * FC; t += NT) {
        const int f = t / FC, k = t % FC, fj = f / (TX + 1), fi = f % (TX + 1);
        const int gx = i0 + fi, gy = j0 + fj;
        if (gx <= ni && gy < nj)
            cp_async16(reinterpret_cast<unsigned char*>(&sm.fi[fj][fi]) + 16 * k,
                       reinterpret_cast<const unsigned char*>(&fI[(size_t)gy * (ni + 1) + gx]) + 16 * k);
    }
    for (int t = tid; t < (TY + 1) * TX * FC; t += NT) {
        const int f = t / FC, k = t % FC, fj = f / TX, fi = f % TX;
        const int gx = i0 + fi, gy = j0 + fj;
        if (gx < ni && gy <= nj)
            cp_async16(reinterpret_cast<unsigned char*>(&sm.fj[fj][fi]) + 16 * k,
                       reinterpret_cast<const unsigned char*>(&fJ[(size_t)gy * ni + gx]) + 16 * k);
    }
    for (int t = tid; t < GY * GX * GC; t += NT) {
        const int e = t / GC, k = t % GC, r = e / GX, c = e % GX;
        int is, xs, js, ys;
        const bool iok = resolve_c(i0 - 1 + c, ni, per, 0, 1, is, xs);
        const bool jok = resolve_c(j0 - 1 + r, nj, false, 2, 3, js, ys);
        if (iok && jok && xs < 0 && ys < 0)
            cp_async16(reinterpret_cast<unsigned char*>(&sm.g[r][c]) + 16 * k,
                       reinterpret_cast<const unsigned char*>(&cG[(size_t)js * ni + is]) + 16 * k);
    }
    if (i0 + tx < ni && j0 + ty < nj)
        cp_async_n(&sm.dta[ty][tx], &dta[(size_t)(j0 + ty) * ni + i0 + tx], (R*)nullptr);
    cp_async_commit();

    chain_sync();
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
    if (sm.plan[0]) {  // uniform
        cp_async_wait_all();
        return;
    }
    const int cur = sm.plan[1], slot3 = sm.plan[2];
    const Vec4<S>* __restrict__ rin = static_cast<const Vec4<S>*>(d.rec[cur]);
    Vec4<S>* __restrict__ rout = static_cast<Vec4<S>*>(d.rec[cur ^ 1]);
    const S qTz = rin[(size_t)min(j0 + TY / 2, nj - 1) * ni + min(i0 + TX / 2, ni - 1)].w;
    const R Tz = P::val(qTz, 3);

    // 1. values on the tile and a 2-cell ring
    for (int t = tid; t < BX * BY; t += NT) {
        const int r = t / BX, c = t % BX;
        int is, xs, js, ys;
        const bool iok = resolve_c(i0 - 2 + c, ni, per, 0, 1, is, xs);
        const bool jok = resolve_c(j0 - 2 + r, nj, false, 2, 3, js, ys);
        R o[4] = {R(0), R(0), R(0), R(0)};
        if (iok && jok && !(xs >= 0 && ys >= 0)) {
            const Vec4<S> q = rin[(size_t)js * ni + is];
            o[0] = P::val(q.x, 0);
            o[1] = P::val(q.y, 1);
            o[2] = P::val(q.z, 2);
            o[3] = P::diff(q.w, qTz, 3);
            const int s = xs >= 0 ? xs : ys;
            if (s >= 0) ghost_values<P, R>(d, s, Tz, o);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) sm.v[q][r][c] = o[q];
    }
    cp_async_wait_all();
    __syncthreads();

    // 2. gradients on the tile and a 1-cell ring
    for (int t = tid; t < GX * GY; t += NT) {
        const int r = t / GX + 1, c = t % GX + 1;
        int is, xs, js, ys;
        const bool iok = resolve_c(i0 - 2 + c, ni, per, 0, 1, is, xs);
        const bool jok = resolve_c(j0 - 2 + r, nj, false, 2, 3, js, ys);
        CellGrad<R> g;
#pragma unroll
        for (int e = 0; e < 8; ++e) g.c[e] = R(0);
        const int side = xs >= 0 ? xs : ys;
        if (iok && jok && !(xs >= 0 && ys >= 0) && !(side >= 0 && d.kind[side] == kFar)) {
            // the cell itself, or the partner (is, js) a wall ghost mirrors,
            // whose coefficients a ghost reads from global memory
            int pr = r, pc = c;
            if (xs >= 0) pc = xs == 0 ? c + 1 : c - 1;
            if (ys >= 0) pr = ys == 2 ? r + 1 : r - 1;
            const CellGrad<R> k = side >= 0 ? ld_vec(&cG[(size_t)js * ni + is]) : sm.g[r - 1][c - 1];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const R vc = sm.v[q][pr][pc];
                const R de = sm.v[q][pr][pc + 1] - vc, dw = sm.v[q][pr][pc - 1] - vc;
                const R dn = sm.v[q][pr + 1][pc] - vc, ds = sm.v[q][pr - 1][pc] - vc;
                g.c[2 * q] = vfma(k.c[0], de, vfma(k.c[2], dw, vfma(k.c[4], dn, k.c[6] * ds)));
                g.c[2 * q + 1] = vfma(k.c[1], de, vfma(k.c[3], dw, vfma(k.c[5], dn, k.c[7] * ds)));
            }
            if (side >= 0) {
                // the boundary face of the partner
                const FaceRec<R> fb = ld_vec(side == 0   ? &fI[(size_t)js * (ni + 1)]
                                             : side == 1 ? &fI[(size_t)js * (ni + 1) + ni]
                                             : side == 2 ? &fJ[is]
                                                         : &fJ[(size_t)nj * ni + is]);
                mirror_grad_c<R>(d.kind[side], fb.nx, fb.ny, g.c);
            }
        }
        sm.g[r - 1][c - 1] = g;
    }
    __syncthreads();

    // 3. faces of the tile; each face's flux replaces its record
    auto cell = [&](int r, int c, R v[4], R g[8]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = sm.v[q][r][c];
        const CellGrad<R> k = sm.g[r - 1][c - 1];
#pragma unroll
        for (int e = 0; e < 8; ++e) g[e] = k.c[e];
    };
    for (int t = tid; t < TY * (TX + 1); t += NT) {
        const int fj = t / (TX + 1), fi = t % (TX + 1);
        const int gx = i0 + fi, gy = j0 + fj;
        if (gx > ni || gy >= nj) continue;
        R vL[4], gL[8], vR[4], gR[8];
        cell(fj + 2, fi + 1, vL, gL);
        cell(fj + 2, fi + 2, vR, gR);
        const int ws = per ? -1 : (gx == 0 ? 0 : (gx == ni ? 1 : -1));
        const bool wall = ws >= 0 && d.kind[ws] != kFar;
        const FaceRec<R> fr = sm.fi[fj][fi];
        R F[4];
        face_c<R>(vL, gL, vR, gR, fr, wall ? R(0) : R(1), wall ? CstC<P>::uw(d, ws, 0) : R(0),
                  wall ? CstC<P>::uw(d, ws, 1) : R(0), Tz, F);
        sm.fi[fj][fi].nx = F[0];
        sm.fi[fj][fi].ny = F[1];
        sm.fi[fj][fi].tL = F[2];
        sm.fi[fj][fi].tR = F[3];
    }
    for (int t = tid; t < (TY + 1) * TX; t += NT) {
        const int fj = t / TX, fi = t % TX;
        const int gx = i0 + fi, gy = j0 + fj;
        if (gy > nj || gx >= ni) continue;
        R vL[4], gL[8], vR[4], gR[8];
        cell(fj + 1, fi + 2, vL, gL);
        cell(fj + 2, fi + 2, vR, gR);
        const int ws = gy == 0 ? 2 : (gy == nj ? 3 : -1);
        const bool wall = ws >= 0 && d.kind[ws] != kFar;
        const FaceRec<R> fr = sm.fj[fj][fi];
        R F[4];
        face_c<R>(vL, gL, vR, gR, fr, wall ? R(0) : R(1), wall ? CstC<P>::uw(d, ws, 0) : R(0),
                  wall ? CstC<P>::uw(d, ws, 1) : R(0), Tz, F);
        sm.fj[fj][fi].nx = F[0];
        sm.fj[fj][fi].ny = F[1];
        sm.fj[fj][fi].tL = F[2];
        sm.fj[fj][fi].tR = F[3];
    }
    __syncthreads();

    // 4. update
    R s0 = R(0), s1 = R(0), s2 = R(0), s3 = R(0);
    bool bad = false;
    const int gi = i0 + tx, gj = j0 + ty;
    if (gi < ni && gj < nj) {
        const size_t off = (size_t)gj * ni + gi;
        const R a = sm.dta[ty][tx];
        const FaceRec<R>&fw = sm.fi[ty][tx], &fe = sm.fi[ty][tx + 1];
        const FaceRec<R>&fs = sm.fj[ty][tx], &fn = sm.fj[ty + 1][tx];
        R div[4];
        div[0] = a * ((fe.nx - fw.nx) + (fn.nx - fs.nx));
        div[1] = a * ((fe.ny - fw.ny) + (fn.ny - fs.ny));
        div[2] = a * ((fe.tL - fw.tL) + (fn.tL - fs.tL));
        div[3] = a * ((fe.tR - fw.tR) + (fn.tR - fs.tR));
        const R one = R(1);
        const R dr = sm.v[0][ty + 2][tx + 2], u = sm.v[1][ty + 2][tx + 2];
        const R v = sm.v[2][ty + 2][tx + 2], T = Tz + sm.v[3][ty + 2][tx + 2];
        const R rho = one + dr;
        const R b = rho * CstC<P>::beta_g(d) * (T - CstC<P>::T_ref(d));
        const R srcx = vfma(b, CstC<P>::gdir(d, 0), rho * CstC<P>::force(d, 0));
        const R srcy = vfma(b, CstC<P>::gdir(d, 1), rho * CstC<P>::force(d, 1));
        const R dtc = CstC<P>::dt(d);
        const R inv = P::rcp(rho - div[0]);
        const R du = (u * div[0] - div[1] + dtc * srcx) * inv;
        const R dv = (v * div[0] - div[2] + dtc * srcy) * inv;
        const R dT = (T * div[0] - div[3]) * inv;
        const R dr1 = dr - div[0], u1 = u + du, v1 = v + dv, T1 = T + dT;
        const Vec4<S> qo = rin[off];
        rout[off] = {P::add(qo.x, -div[0], 0), P::add(qo.y, du, 1), P::add(qo.z, dv, 2),
                     P::add(qo.w, dT, 3)};
        bad = !(P::in_range(dr1, 0) && P::in_range(u1, 1) && P::in_range(v1, 2) &&
                P::in_range(T1, 3));
        const R m0 = P::fsqrt(u * u + v * v), m1 = P::fsqrt(u1 * u1 + v1 * v1);
        const R den = m0 + m1;
        const R dm = den > R(0) ? (du * (u + u1) + dv * (v + v1)) * P::rcp(den) : R(0);
        s0 = dm * dm;
        s1 = m1 * m1;
        s2 = dT * dT;
        s3 = T1 * T1;
    }
    if (bad) s0 = R(NAN);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    }
    if ((tid & 31) == 0) {
        sm.red[tid >> 5][0] = s0;
        sm.red[tid >> 5][1] = s1;
        sm.red[tid >> 5][2] = s2;
        sm.red[tid >> 5][3] = s3;
    }
    __syncthreads();
    // warp 0 adds the warp partials in the arithmetic type (a serial FP64
    // loop would hold GB300's narrow FP64 pipe at the tail of every block);
    // the tile sums go to the FP64 sums across tiles
    double acc4[4];
    if (tid < 32) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            R v = tid < NT / 32 ? sm.red[tid][q] : R(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc4[q] = (double)v;
        }
    }
    // the step's residual sums; the next launch tests them
    if (tid == 0)
        for (int q = 0; q < 4; ++q) atomicAdd(&run->acc[slot3][q], acc4[q]);
}

// ---------------------------------------------------------------------------
// FP64 heat through side 2 or 3, one thread per face.
// ---------------------------------------------------------------------------

// value (T absolute) and gradient of cell (ci, cj) in FP64, ghosts included
template <class P>
__device__ void cell_c(const DescC& d, const Vec4<typename P::S>* rin, int ci, int cj, double v[4],
                       double g[8])
{
    using S = typename P::S;
    const bool per = d.per != 0;
    const FaceGeo<double>* gI = static_cast<const FaceGeo<double>*>(d.gi_d);
    const FaceGeo<double>* gJ = static_cast<const FaceGeo<double>*>(d.gj_d);
    const double* ia = static_cast<const double*>(d.ia_d);
    auto fetch = [&](int i, int j, double o[4]) {
        int is, xs, js, ys;
        resolve_c(i, d.ni, per, 0, 1, is, xs);
        resolve_c(j, d.nj, false, 2, 3, js, ys);
        const Vec4<S> q = rin[(size_t)js * d.ni + is];
        o[0] = P::to_double(q.x, 0);
        o[1] = P::to_double(q.y, 1);
        o[2] = P::to_double(q.z, 2);
        o[3] = P::to_double(q.w, 3);
        const int s = xs >= 0 ? xs : ys;
        if (s >= 0) ghost_values<StoreD, double>(d, s, 0.0, o);  // FP64, T absolute
    };
    int is, xs, js, ys;
    resolve_c(ci, d.ni, per, 0, 1, is, xs);
    resolve_c(cj, d.nj, false, 2, 3, js, ys);
    const int side = xs >= 0 ? xs : ys;
    fetch(ci, cj, v);
    for (int e = 0; e < 8; ++e) g[e] = 0.0;
    if (side >= 0 && d.kind[side] == kFar) return;
    // partner (the cell itself unless a wall ghost)
    int pi_ = ci, pj = cj;
    if (xs >= 0) pi_ = xs == 0 ? ci + 1 : ci - 1;
    if (ys >= 0) pj = ys == 2 ? cj + 1 : cj - 1;
    double c0[4], ce[4], cw[4], cn[4], cs[4];
    fetch(pi_, pj, c0);
    fetch(pi_ + 1, pj, ce);
    fetch(pi_ - 1, pj, cw);
    fetch(pi_, pj + 1, cn);
    fetch(pi_, pj - 1, cs);
    const FaceGeo<double>& fw = gI[(size_t)js * (d.ni + 1) + is];
    const FaceGeo<double>& fe = gI[(size_t)js * (d.ni + 1) + is + 1];
    const FaceGeo<double>& fs = gJ[(size_t)js * d.ni + is];
    const FaceGeo<double>& fn = gJ[(size_t)(js + 1) * d.ni + is];
    const double iA = ia[(size_t)js * d.ni + is];
    for (int q = 0; q < 4; ++q) {
        const double de = (ce[q] - c0[q]) * fe.wR, dw = (cw[q] - c0[q]) * (1.0 - fw.wR);
        const double dn = (cn[q] - c0[q]) * fn.wR, ds = (cs[q] - c0[q]) * (1.0 - fs.wR);
        g[2 * q] = iA * ((de * fe.Sx - dw * fw.Sx) + (dn * fn.Sx - ds * fs.Sx));
        g[2 * q + 1] = iA * ((de * fe.Sy - dw * fw.Sy) + (dn * fn.Sy - ds * fs.Sy));
    }
    if (side >= 0) {
        const FaceGeo<double>& fb = side == 0 ? fw : (side == 1 ? fe : (side == 2 ? fs : fn));
        mirror_grad_c<double>(d.kind[side], fb.nx, fb.ny, g);
    }
}

template <class P>
__global__ void curv_heat_kernel(const DescC* __restrict__ dp, int cur, int jface, double* acc)
{
    const DescC& d = *dp;
    const Vec4<typename P::S>* rin = static_cast<const Vec4<typename P::S>*>(d.rec[cur]);
    const FaceGeo<double>* gJ = static_cast<const FaceGeo<double>*>(d.gj_d);
    const int side = jface == 0 ? 2 : 3;
    const bool wall = d.kind[side] != kFar;
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.ni; i += gridDim.x * blockDim.x) {
        double vL[4], gL[8], vR[4], gR[8];
        cell_c<P>(d, rin, i, jface - 1, vL, gL);
        cell_c<P>(d, rin, i, jface, vR, gR);
        const double TL = vL[3];
        vL[3] = 0.0;
        vR[3] -= TL;
        double F[4];
        face_c<double>(vL, gL, vR, gR, face_rec<double>(gJ[(size_t)jface * d.ni + i]), wall ? 0.0 : 1.0,
                       wall ? d.bcU[side][0] : 0.0, wall ? d.bcU[side][1] : 0.0, TL, F);
        s += F[3];  // already times the face length
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
constexpr int kTileX = 32;
constexpr int kGraphSteps = 32;

template <class P, int TY>
cudaError_t launch_c(int units, cudaStream_t s, const DescC* d, CavityRun* c, int par)
{
    const size_t sm = sizeof(SmemC<P, kTileX, TY>);
    return launch_chained(curv_step_kernel<P, kTileX, TY>, units, kTileX * TY, sm, s, d, c, par);
}

template <class P, int TY>
cudaError_t prepare_c()
{
    const size_t sm = sizeof(SmemC<P, kTileX, TY>);
    cudaError_t e = cudaFuncSetAttribute(curv_step_kernel<P, kTileX, TY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // the staged geometry makes shared memory the resource that bounds
    // resident blocks: all of the unified L1/shared array to shared memory
    return cudaFuncSetAttribute(curv_step_kernel<P, kTileX, TY>,
                                cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

}  // namespace rtlbfsc

using namespace rtlbfsc;

struct rtlbfsc_ctx {
    int precision = RTLBFS_FP64, ni = 0, nj = 0, per = 0;
    std::vector<double> X, Y;
    double nu = 0.01, chi = 0.01, beta_g = 0.0, dt = 0.1, kappa = 1.0, T_ref = 0.5;
    double gdir[2] = {0.0, 1.0}, force[2] = {0.0, 0.0};
    int kind[4] = {kDir, kDir, kDir, kDir};
    double bcT[4] = {0.0, 0.0, 0.0, 0.0}, bcU[4][2] = {};
    double inf[4] = {1.0, 0.0, 0.0, 0.0};
    int tile_rows = 0, sms = 0;
    size_t cells = 0, ssize = 0, buf_bytes = 0;
    void* d_state = nullptr;
    void* d_geo = nullptr;
    DescC* d_desc = nullptr;
    CavityRun* d_ctl = nullptr;
    double* d_acc = nullptr;
    CavityCtl* h_ctl = nullptr;  // pinned: the tested header h[0]
    CavityRun* h_run = nullptr;  // pinned: staging of a new run record
    double* h_acc = nullptr;
    DescC desc{};
    bool dirty = true;
    cudaStream_t stream = nullptr, own = nullptr, cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int gunits = 0, gty = 0;
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

#define CKC(call)                                                  \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return h->cuda_fail(e_, #call);     \
    } while (0)

namespace {

// Host geometry, the same construction as the FP64 oracle's: centres (vertex
// averages), areas (shoelace), ghost centres (mirrored across wall and
// far-field faces; the opposite cell moved by the seam's translation when
// periodic).
struct HostGeo {
    int ni, nj;
    std::vector<double> cx, cy, area;  // padded (ni+2) x (nj+2)
    size_t id(int i, int j) const { return (size_t)(j + 1) * (ni + 2) + (i + 1); }
};

double VX(const rtlbfsc_ctx* h, int i, int j) { return h->X[(size_t)j * (h->ni + 1) + i]; }
double VY(const rtlbfsc_ctx* h, int i, int j) { return h->Y[(size_t)j * (h->ni + 1) + i]; }

void reflect(double px, double py, double ax, double ay, double bx, double by, double& rx, double& ry)
{
    const double dx = bx - ax, dy = by - ay, L2 = dx * dx + dy * dy;
    const double s = ((px - ax) * dx + (py - ay) * dy) / L2;
    const double fx = ax + s * dx, fy = ay + s * dy;
    rx = 2.0 * fx - px;
    ry = 2.0 * fy - py;
}

bool build_geo(const rtlbfsc_ctx* h, HostGeo& g)
{
    const int ni = h->ni, nj = h->nj;
    g.ni = ni;
    g.nj = nj;
    const size_t np = (size_t)(ni + 2) * (nj + 2);
    g.cx.assign(np, 0.0);
    g.cy.assign(np, 0.0);
    g.area.assign(np, 0.0);
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            const double x0 = VX(h, i, j), y0 = VY(h, i, j), x1 = VX(h, i + 1, j), y1 = VY(h, i + 1, j);
            const double x2 = VX(h, i + 1, j + 1), y2 = VY(h, i + 1, j + 1);
            const double x3 = VX(h, i, j + 1), y3 = VY(h, i, j + 1);
            const size_t c = g.id(i, j);
            g.cx[c] = 0.25 * (x0 + x1 + x2 + x3);
            g.cy[c] = 0.25 * (y0 + y1 + y2 + y3);
            g.area[c] = 0.5 * ((x0 * y1 - x1 * y0) + (x1 * y2 - x2 * y1) + (x2 * y3 - x3 * y2) +
                               (x3 * y0 - x0 * y3));
            if (!(g.area[c] > 0.0)) return false;
        }
    for (int j = 0; j < nj; ++j) {
        if (h->per) {
            const double sx = VX(h, ni, j) - VX(h, 0, j), sy = VY(h, ni, j) - VY(h, 0, j);
            g.cx[g.id(-1, j)] = g.cx[g.id(ni - 1, j)] - sx;
            g.cy[g.id(-1, j)] = g.cy[g.id(ni - 1, j)] - sy;
            g.cx[g.id(ni, j)] = g.cx[g.id(0, j)] + sx;
            g.cy[g.id(ni, j)] = g.cy[g.id(0, j)] + sy;
        } else {
            reflect(g.cx[g.id(0, j)], g.cy[g.id(0, j)], VX(h, 0, j), VY(h, 0, j), VX(h, 0, j + 1),
                    VY(h, 0, j + 1), g.cx[g.id(-1, j)], g.cy[g.id(-1, j)]);
            reflect(g.cx[g.id(ni - 1, j)], g.cy[g.id(ni - 1, j)], VX(h, ni, j), VY(h, ni, j),
                    VX(h, ni, j + 1), VY(h, ni, j + 1), g.cx[g.id(ni, j)], g.cy[g.id(ni, j)]);
        }
    }
    for (int i = 0; i < ni; ++i) {
        reflect(g.cx[g.id(i, 0)], g.cy[g.id(i, 0)], VX(h, i, 0), VY(h, i, 0), VX(h, i + 1, 0),
                VY(h, i + 1, 0), g.cx[g.id(i, -1)], g.cy[g.id(i, -1)]);
        reflect(g.cx[g.id(i, nj - 1)], g.cy[g.id(i, nj - 1)], VX(h, i, nj), VY(h, i, nj),
                VX(h, i + 1, nj), VY(h, i + 1, nj), g.cx[g.id(i, nj)], g.cy[g.id(i, nj)]);
    }
    return true;
}

// Geometry of the face with edge A -> B between padded cells L and R;
// kind 0: i-face (S = edge rotated clockwise), 1: j-face (counter-clockwise).
FaceGeo<double> face_geo(const rtlbfsc_ctx* h, const HostGeo& g, int kind, double ax, double ay,
                         double bx, double by, size_t L, size_t R)
{
    FaceGeo<double> f;
    const double dx = bx - ax, dy = by - ay;
    f.Sx = kind == 0 ? dy : -dy;
    f.Sy = kind == 0 ? -dx : dx;
    f.len = std::hypot(f.Sx, f.Sy);
    f.nx = f.Sx / f.len;
    f.ny = f.Sy / f.len;
    const double tx = -f.ny, ty = f.nx;
    const double mx = 0.5 * (ax + bx), my = 0.5 * (ay + by);
    const double dL = std::hypot(g.cx[L] - mx, g.cy[L] - my), dR = std::hypot(g.cx[R] - mx, g.cy[R] - my);
    f.wR = dL / (dL + dR);
    const double dLn = (mx - g.cx[L]) * f.nx + (my - g.cy[L]) * f.ny;
    const double dRn = (g.cx[R] - mx) * f.nx + (g.cy[R] - my) * f.ny;
    f.tL = (g.cx[L] - mx) * tx + (g.cy[L] - my) * ty;
    f.tR = (g.cx[R] - mx) * tx + (g.cy[R] - my) * ty;
    const double wl = 2.0 * std::fabs(dLn), wr = 2.0 * std::fabs(dRn);
    const double hh = h->kappa * std::min(wl, wr);
    f.h = hh;
    f.cL = dLn - hh;
    f.cR = hh - dRn;
    f.m_nu_2h = -h->nu / (2.0 * hh);
    f.m_chi_2h = -h->chi / (2.0 * hh);
    f.m_tf15 = 1.0 - 3.0 * h->nu / hh;  // -(tau_f - 1.5), Eq. 9 with cs2 = 1/3
    f.m_tg15 = 1.0 - 3.0 * h->chi / hh;
    f.pad = 0.0;
    return f;
}

size_t align256(std::vector<unsigned char>& buf)
{
    const size_t o = (buf.size() + 255) / 256 * 256;
    buf.resize(o);
    return o;
}

template <typename T>
size_t append_array(std::vector<unsigned char>& buf, const std::vector<T>& a)
{
    const size_t o = align256(buf);
    buf.resize(o + a.size() * sizeof(T));
    if (!a.empty()) std::memcpy(buf.data() + o, a.data(), a.size() * sizeof(T));
    return o;
}

// The FP64 face geometry and inverse areas of the wall-heat sums.
void append_heat_geo(std::vector<unsigned char>& buf, size_t& off_i, size_t& off_j, size_t& off_ia,
                     const std::vector<FaceGeo<double>>& fi, const std::vector<FaceGeo<double>>& fj,
                     const std::vector<double>& ia)
{
    off_i = append_array(buf, fi);
    off_j = append_array(buf, fj);
    off_ia = append_array(buf, ia);
}

// The step kernel's arrays in precision R: face records, the cells'
// Green-Gauss coefficients (formed in FP64) and dt / area.
template <typename R>
void append_step_geo(std::vector<unsigned char>& buf, size_t& off_i, size_t& off_j, size_t& off_cg,
                     size_t& off_dta, int ni, int nj, const std::vector<FaceGeo<double>>& fi,
                     const std::vector<FaceGeo<double>>& fj, const std::vector<double>& ia, double dt)
{
    std::vector<FaceRec<R>> ri(fi.size()), rj(fj.size());
    for (size_t k = 0; k < fi.size(); ++k) ri[k] = face_rec<R>(fi[k]);
    for (size_t k = 0; k < fj.size(); ++k) rj[k] = face_rec<R>(fj[k]);
    std::vector<CellGrad<R>> cg((size_t)ni * nj);
    std::vector<R> dta((size_t)ni * nj);
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            const size_t c = (size_t)j * ni + i;
            const FaceGeo<double>& fw = fi[(size_t)j * (ni + 1) + i];
            const FaceGeo<double>& fe = fi[(size_t)j * (ni + 1) + i + 1];
            const FaceGeo<double>& fs = fj[(size_t)j * ni + i];
            const FaceGeo<double>& fn = fj[(size_t)(j + 1) * ni + i];
            const double a = ia[c];
            const double we = a * fe.wR, ww = -a * (1.0 - fw.wR);
            const double wn = a * fn.wR, ws = -a * (1.0 - fs.wR);
            const double k[8] = {we * fe.Sx, we * fe.Sy, ww * fw.Sx, ww * fw.Sy,
                                 wn * fn.Sx, wn * fn.Sy, ws * fs.Sx, ws * fs.Sy};
            for (int e = 0; e < 8; ++e) cg[c].c[e] = (R)k[e];
            dta[c] = (R)(dt * a);
        }
    off_i = append_array(buf, ri);
    off_j = append_array(buf, rj);
    off_cg = append_array(buf, cg);
    off_dta = append_array(buf, dta);
}

int tile_rows_of(const rtlbfsc_ctx* h)
{
    if (h->tile_rows == 8 || h->tile_rows == 16) return h->tile_rows;
    // 32 x 8 by default: four resident blocks per SM against two of the
    // 32 x 16 tile (measured faster on small and large O-meshes alike)
    return 8;
}

int upload(rtlbfsc_ctx* h)
{
    if (!h->dirty) return RTLBFS_OK;
    HostGeo g;
    if (!build_geo(h, g)) return h->fail(RTLBFS_ERR_ARG, "a cell has a non-positive area");
    const int ni = h->ni, nj = h->nj;
    std::vector<FaceGeo<double>> fi((size_t)nj * (ni + 1)), fj((size_t)(nj + 1) * ni);
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i <= ni; ++i)
            fi[(size_t)j * (ni + 1) + i] = face_geo(h, g, 0, VX(h, i, j), VY(h, i, j), VX(h, i, j + 1),
                                                    VY(h, i, j + 1), g.id(i - 1, j), g.id(i, j));
    for (int j = 0; j <= nj; ++j)
        for (int i = 0; i < ni; ++i)
            fj[(size_t)j * ni + i] = face_geo(h, g, 1, VX(h, i, j), VY(h, i, j), VX(h, i + 1, j),
                                              VY(h, i + 1, j), g.id(i, j - 1), g.id(i, j));
    std::vector<double> ia((size_t)ni * nj);
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) ia[(size_t)j * ni + i] = 1.0 / g.area[g.id(i, j)];
    std::vector<unsigned char> buf;
    size_t oi_d, oj_d, oia_d, oi, oj, ocg, odta;
    append_heat_geo(buf, oi_d, oj_d, oia_d, fi, fj, ia);
    if (h->precision == RTLBFS_FP64)
        append_step_geo<double>(buf, oi, oj, ocg, odta, ni, nj, fi, fj, ia, h->dt);
    else
        append_step_geo<float>(buf, oi, oj, ocg, odta, ni, nj, fi, fj, ia, h->dt);
    if (h->d_geo) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->d_geo);
        h->d_geo = nullptr;
    }
    CKC(cudaMalloc(&h->d_geo, buf.size()));
    CKC(cudaMemcpy(h->d_geo, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    unsigned char* base = static_cast<unsigned char*>(h->d_geo);
    DescC& d = h->desc;
    d.ni = ni;
    d.nj = nj;
    d.per = h->per;
    const int ty = tile_rows_of(h);
    d.tiles_x = (ni + kTileX - 1) / kTileX;
    d.tiles_y = (nj + ty - 1) / ty;
    d.units = d.tiles_x * d.tiles_y;
    d.fri = base + oi;
    d.frj = base + oj;
    d.cg = base + ocg;
    d.dta = base + odta;
    d.gi_d = base + oi_d;
    d.gj_d = base + oj_d;
    d.ia_d = base + oia_d;
    double gl = std::hypot(h->gdir[0], h->gdir[1]);
    for (int a = 0; a < 2; ++a) {
        d.gdir[a] = h->gdir[a] / gl;
        d.f_gdir[a] = (float)d.gdir[a];
        d.force[a] = h->force[a];
        d.f_force[a] = (float)h->force[a];
    }
    d.beta_g = h->beta_g;
    d.f_beta_g = (float)h->beta_g;
    d.T_ref = h->T_ref;
    d.f_T_ref = (float)h->T_ref;
    d.dt = h->dt;
    d.f_dt = (float)h->dt;
    for (int s = 0; s < 4; ++s) {
        d.kind[s] = h->kind[s];
        for (int c = 0; c < 2; ++c) {
            d.bcU[s][c] = h->bcU[s][c];
            d.f_bcU[s][c] = (float)h->bcU[s][c];
        }
        d.bcT[s] = h->bcT[s];
        d.f_bcT[s] = (float)h->bcT[s];
    }
    const double infs[4] = {h->inf[0] - 1.0, h->inf[1], h->inf[2], h->inf[3]};
    for (int q = 0; q < 4; ++q) {
        d.d_inf[q] = infs[q];
        d.f_inf[q] = (float)infs[q];
    }
    unsigned char* st = static_cast<unsigned char*>(h->d_state);
    d.rec[0] = st;
    d.rec[1] = st + h->buf_bytes;
    CKC(cudaMemcpyAsync(h->d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, h->stream));
    CKC(cudaStreamSynchronize(h->stream));
    h->dirty = false;
    return RTLBFS_OK;
}

cudaError_t launch_one(rtlbfsc_ctx* h, cudaStream_t s, int par)
{
    rtlbfs::g_launches++;
    const int ty = tile_rows_of(h);
    if (h->precision == RTLBFS_FP64)
        return ty == 16 ? launch_c<StoreD, 16>(h->desc.units, s, h->d_desc, h->d_ctl, par)
                        : launch_c<StoreD, 8>(h->desc.units, s, h->d_desc, h->d_ctl, par);
    return ty == 16 ? launch_c<StoreQ, 16>(h->desc.units, s, h->d_desc, h->d_ctl, par)
                    : launch_c<StoreQ, 8>(h->desc.units, s, h->d_desc, h->d_ctl, par);
}

int read_ctl(rtlbfsc_ctx* h)
{
    CKC(cudaMemcpyAsync(h->h_ctl, &h->d_ctl->h[0], sizeof(CavityCtl), cudaMemcpyDeviceToHost,
                        h->stream));
    CKC(cudaStreamSynchronize(h->stream));
    return RTLBFS_OK;
}

// the run record with both headers c and cleared sums (h_ctl becomes c)
int put_run(rtlbfsc_ctx* h, const CavityCtl& c)
{
    std::memset(h->h_run, 0, sizeof(CavityRun));
    h->h_run->h[0] = c;
    h->h_run->h[1] = c;
    *h->h_ctl = c;
    CKC(cudaMemcpyAsync(h->d_ctl, h->h_run, sizeof(CavityRun), cudaMemcpyHostToDevice, h->stream));
    CKC(cudaStreamSynchronize(h->stream));  // h_run is reused
    return RTLBFS_OK;
}

int arm(rtlbfsc_ctx* h, long long nsteps, double tol)
{
    int rc = read_ctl(h);
    if (rc) return rc;
    CavityCtl c = *h->h_ctl;
    c.done = 0;
    c.status = kRunning;
    c.pend = 0;
    c.max_steps = c.steps + nsteps;
    c.tol = tol;
    return put_run(h, c);
}

int launch_steps(rtlbfsc_ctx* h, long long count)
{
    nvtxRangePushA("rtlbfsc: step launches");
    struct Pop {
        ~Pop() { nvtxRangePop(); }
    } pop;
    const int ty = tile_rows_of(h);
    if (!h->gexec || h->gunits != h->desc.units || h->gty != ty) {
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        CKC(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = cudaSuccess;
        static_assert(kGraphSteps % 2 == 0, "graphs of an even number of launches");
        for (int i = 0; i < kGraphSteps && le == cudaSuccess; ++i) le = launch_one(h, h->cap, i & 1);
        rtlbfs::g_launches -= kGraphSteps;
        cudaGraph_t g = nullptr;
        cudaError_t ee = cudaStreamEndCapture(h->cap, &g);
        if (le != cudaSuccess) return h->cuda_fail(le, "capture of the step launches");
        if (ee != cudaSuccess) return h->cuda_fail(ee, "cudaStreamEndCapture");
        cudaError_t ie = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return h->cuda_fail(ie, "cudaGraphInstantiate");
        h->gunits = h->desc.units;
        h->gty = ty;
    }
    // launch k of the chain has parity k & 1; the chain ends with the stop
    // test of its last step
    int par = 0;
    while (count >= kGraphSteps) {
        CKC(cudaGraphLaunch(h->gexec, h->stream));
        rtlbfs::g_launches += kGraphSteps;
        count -= kGraphSteps;
    }
    for (long long i = 0; i < count; ++i) {
        cudaError_t e = launch_one(h, h->stream, par);
        if (e != cudaSuccess) return h->cuda_fail(e, "step launch");
        par ^= 1;
    }
    CKC(rtlbfs::launch_finalize(h->stream, h->d_ctl, 1, par));
    rtlbfs::g_launches++;
    return RTLBFS_OK;
}

}  // namespace

extern "C" {

int rtlbfsc_create(int ni, int nj, const double* X, const double* Y, int periodic_i, int precision,
                   rtlbfsc_t* out)
{
    if (!out || !X || !Y || ni < 1 || nj < 1) return RTLBFS_ERR_ARG;
    if (precision != RTLBFS_FP64 && precision != RTLBFS_FP32) return RTLBFS_ERR_ARG;
    if ((double)ni * nj > 2147483647.0) return RTLBFS_ERR_ARG;
    *out = nullptr;
    rtlbfsc_ctx* h = new (std::nothrow) rtlbfsc_ctx();
    if (!h) return RTLBFS_ERR_OOM;
    h->precision = precision;
    h->ni = ni;
    h->nj = nj;
    h->per = periodic_i ? 1 : 0;
    const size_t nv = (size_t)(ni + 1) * (nj + 1);
    h->X.assign(X, X + nv);
    h->Y.assign(Y, Y + nv);
    if (h->per) h->kind[0] = h->kind[1] = kPer;
    auto bail = [&](int code) {
        rtlbfsc_destroy(h);
        return code;
    };
    {
        HostGeo g;
        if (!build_geo(h, g)) return bail(RTLBFS_ERR_ARG);
    }
    h->cells = (size_t)ni * nj;
    h->ssize = precision == RTLBFS_FP64 ? sizeof(double) : sizeof(int);
    h->buf_bytes = (h->cells * 4 * h->ssize + 255) / 256 * 256;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(RTLBFS_ERR_CUDA);
    cudaError_t e = precision == RTLBFS_FP64 ? prepare_c<StoreD, 8>() : prepare_c<StoreQ, 8>();
    if (e == cudaSuccess) e = precision == RTLBFS_FP64 ? prepare_c<StoreD, 16>() : prepare_c<StoreQ, 16>();
    if (e != cudaSuccess) return bail(RTLBFS_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(RTLBFS_ERR_CUDA);
    h->stream = h->own;
    if (cudaMalloc(&h->d_state, 2 * h->buf_bytes) != cudaSuccess ||
        cudaMalloc(&h->d_desc, sizeof(DescC)) != cudaSuccess ||
        cudaMalloc(&h->d_ctl, sizeof(CavityRun)) != cudaSuccess ||
        cudaMalloc(&h->d_acc, sizeof(double)) != cudaSuccess)
        return bail(RTLBFS_ERR_OOM);
    if (cudaMallocHost(&h->h_ctl, sizeof(CavityCtl)) != cudaSuccess ||
        cudaMallocHost(&h->h_run, sizeof(CavityRun)) != cudaSuccess ||
        cudaMallocHost(&h->h_acc, sizeof(double)) != cudaSuccess)
        return bail(RTLBFS_ERR_OOM);
    std::vector<double> one(h->cells, 1.0), zero(h->cells, 0.0);
    int rc = rtlbfsc_set_state(h, one.data(), zero.data(), zero.data(), zero.data());
    if (rc) return bail(rc);
    *out = h;
    return RTLBFS_OK;
}

int rtlbfsc_set_physics(rtlbfsc_t h, double nu, double chi, double beta_g, double dt)
{
    if (!h) return RTLBFS_ERR_ARG;
    if (!(nu > 0) || !(chi > 0) || !(dt > 0) || !std::isfinite(beta_g))
        return h->fail(RTLBFS_ERR_ARG, "nu, chi and dt must be positive");
    h->nu = nu;
    h->chi = chi;
    h->beta_g = beta_g;
    h->dt = dt;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfsc_set_lattice(rtlbfsc_t h, double kappa)
{
    if (!h) return RTLBFS_ERR_ARG;
    if (!(kappa > 0)) return h->fail(RTLBFS_ERR_ARG, "kappa must be positive");
    h->kappa = kappa;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfsc_set_gravity(rtlbfsc_t h, double gx, double gy, double T_ref)
{
    if (!h) return RTLBFS_ERR_ARG;
    if (!(std::hypot(gx, gy) > 0)) return h->fail(RTLBFS_ERR_ARG, "zero gravity direction");
    h->gdir[0] = gx;
    h->gdir[1] = gy;
    h->T_ref = T_ref;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfsc_set_body_force(rtlbfsc_t h, double fx, double fy)
{
    if (!h) return RTLBFS_ERR_ARG;
    h->force[0] = fx;
    h->force[1] = fy;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfsc_set_bc(rtlbfsc_t h, int side, int kind, double T_wall, double ux, double uy)
{
    if (!h) return RTLBFS_ERR_ARG;
    if (side < 0 || side > 3 || !(kind == kDir || kind == kAdia || kind == kFar))
        return h->fail(RTLBFS_ERR_ARG, "bad side or kind");
    if (h->per && side < 2) return h->fail(RTLBFS_ERR_ARG, "sides 0 and 1 are the periodic seam");
    if (!StoreQ::representable(T_wall, 3)) return h->fail(RTLBFS_ERR_ARG, "T_wall out of range");
    h->kind[side] = kind;
    h->bcT[side] = T_wall;
    h->bcU[side][0] = ux;
    h->bcU[side][1] = uy;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfsc_set_farfield(rtlbfsc_t h, double rho, double u, double v, double T)
{
    if (!h) return RTLBFS_ERR_ARG;
    if (!StoreQ::representable(rho - 1.0, 0) || !StoreQ::representable(u, 1) ||
        !StoreQ::representable(v, 1) || !StoreQ::representable(T, 3))
        return h->fail(RTLBFS_ERR_ARG, "free stream out of range");
    h->inf[0] = rho;
    h->inf[1] = u;
    h->inf[2] = v;
    h->inf[3] = T;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfsc_set_state(rtlbfsc_t h, const double* rho, const double* u, const double* v,
                      const double* T)
{
    if (!h) return RTLBFS_ERR_ARG;
    if (!rho || !u || !v || !T) return h->fail(RTLBFS_ERR_ARG, "null state array");
    const size_t n = h->cells;
    std::vector<unsigned char> buf(h->buf_bytes);
    if (h->precision == RTLBFS_FP64) {
        double* r = reinterpret_cast<double*>(buf.data());
        for (size_t c = 0; c < n; ++c) {
            r[4 * c] = rho[c] - 1.0;
            r[4 * c + 1] = u[c];
            r[4 * c + 2] = v[c];
            r[4 * c + 3] = T[c];
        }
    } else {
        int* r = reinterpret_cast<int*>(buf.data());
        for (size_t c = 0; c < n; ++c) {
            const double x[4] = {rho[c] - 1.0, u[c], v[c], T[c]};
            const int k[4] = {0, 1, 2, 3};
            for (int q = 0; q < 4; ++q) {
                if (!StoreQ::representable(x[q], k[q]))
                    return h->fail(RTLBFS_ERR_ARG, "state value outside the FP32 fixed-point range");
                r[4 * c + q] = StoreQ::from_double(x[q], k[q]);
            }
        }
    }
    CKC(cudaStreamSynchronize(h->stream));
    CKC(cudaMemcpy(h->d_state, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    CavityCtl z;
    std::memset(&z, 0, sizeof(z));
    z.res[0] = z.res[1] = INFINITY;
    return put_run(h, z);
}

int rtlbfsc_get_state(rtlbfsc_t h, double* rho, double* u, double* v, double* T)
{
    if (!h) return RTLBFS_ERR_ARG;
    if (!rho || !u || !v || !T) return h->fail(RTLBFS_ERR_ARG, "null state array");
    int rc = read_ctl(h);
    if (rc) return rc;
    std::vector<unsigned char> buf(h->buf_bytes);
    CKC(cudaMemcpy(buf.data(), static_cast<unsigned char*>(h->d_state) + h->h_ctl->cur * h->buf_bytes,
                   h->buf_bytes, cudaMemcpyDeviceToHost));
    for (size_t c = 0; c < h->cells; ++c) {
        double x[4];
        if (h->precision == RTLBFS_FP64) {
            const double* r = reinterpret_cast<const double*>(buf.data());
            for (int q = 0; q < 4; ++q) x[q] = r[4 * c + q];
        } else {
            const int* r = reinterpret_cast<const int*>(buf.data());
            for (int q = 0; q < 4; ++q) x[q] = StoreQ::to_double(r[4 * c + q], q);
        }
        rho[c] = 1.0 + x[0];
        u[c] = x[1];
        v[c] = x[2];
        T[c] = x[3];
    }
    return RTLBFS_OK;
}

int rtlbfsc_step(rtlbfsc_t h, long nsteps)
{
    if (!h) return RTLBFS_ERR_ARG;
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

int rtlbfsc_run_to_steady(rtlbfsc_t h, double tol, long max_steps, double timeout_s,
                          long* steps_taken, double* res2)
{
    if (!h) return RTLBFS_ERR_ARG;
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
        const long long now = std::min<long long>(8LL * kGraphSteps, (long long)max_steps - queued);
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
        if (timeout_s > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > timeout_s) {
            out = h->fail(RTLBFS_ERR_TIMEOUT, "wall-clock limit reached");
            break;
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

int rtlbfsc_residual(rtlbfsc_t h, double* res2, long* steps)
{
    if (!h) return RTLBFS_ERR_ARG;
    int rc = read_ctl(h);
    if (rc) return rc;
    if (res2) {
        res2[0] = h->h_ctl->res[0];
        res2[1] = h->h_ctl->res[1];
    }
    if (steps) *steps = (long)h->h_ctl->steps;
    return RTLBFS_OK;
}

int rtlbfsc_wall_heat(rtlbfsc_t h, int side, double* heat, double* perimeter)
{
    if (!h || !heat) return RTLBFS_ERR_ARG;
    if (side != 2 && side != 3) return h->fail(RTLBFS_ERR_ARG, "side must be 2 or 3");
    int rc = upload(h);
    if (rc) return rc;
    rc = read_ctl(h);
    if (rc) return rc;
    const int jf = side == 2 ? 0 : h->nj;
    CKC(cudaMemsetAsync(h->d_acc, 0, sizeof(double), h->stream));
    const int block = 128, grid = std::max(1, std::min((h->ni + block - 1) / block, 4 * h->sms));
    rtlbfs::g_launches++;
    if (h->precision == RTLBFS_FP64)
        curv_heat_kernel<StoreD><<<grid, block, 0, h->stream>>>(h->d_desc, h->h_ctl->cur, jf, h->d_acc);
    else
        curv_heat_kernel<StoreQ><<<grid, block, 0, h->stream>>>(h->d_desc, h->h_ctl->cur, jf, h->d_acc);
    CKC(cudaGetLastError());
    CKC(cudaMemcpyAsync(h->h_acc, h->d_acc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CKC(cudaStreamSynchronize(h->stream));
    *heat = *h->h_acc;
    if (perimeter) {
        double p = 0.0;
        for (int i = 0; i < h->ni; ++i)
            p += std::hypot(VX(h, i + 1, jf) - VX(h, i, jf), VY(h, i + 1, jf) - VY(h, i, jf));
        *perimeter = p;
    }
    return RTLBFS_OK;
}

int rtlbfsc_set_schedule(rtlbfsc_t h, int tile_rows)
{
    if (!h) return RTLBFS_ERR_ARG;
    if (tile_rows != 0 && tile_rows != 8 && tile_rows != 16)
        return h->fail(RTLBFS_ERR_ARG, "tile rows must be 0, 8 or 16");
    h->tile_rows = tile_rows;
    h->dirty = true;
    return RTLBFS_OK;
}

int rtlbfsc_set_stream(rtlbfsc_t h, void* stream)
{
    if (!h) return RTLBFS_ERR_ARG;
    CKC(cudaStreamSynchronize(h->stream));
    h->stream = stream ? static_cast<cudaStream_t>(stream) : h->own;
    return RTLBFS_OK;
}

int rtlbfsc_sync(rtlbfsc_t h)
{
    if (!h) return RTLBFS_ERR_ARG;
    CKC(cudaStreamSynchronize(h->stream));
    return RTLBFS_OK;
}

const char* rtlbfsc_last_error(rtlbfsc_t h) { return h ? h->err.c_str() : "null handle"; }

void rtlbfsc_destroy(rtlbfsc_t h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    cudaFree(h->d_state);
    cudaFree(h->d_geo);
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

// ---------------------------------------------------------------------------
// Operation count: face_c (the frame rotation plus face_flux) run on a
// counting type on the host; the face template is host-instantiated only.
// ---------------------------------------------------------------------------
#pragma nv_diag_suppress 20011, 20014
namespace rtlbfsc {
namespace {
struct TallyC {
    long long ops = 0, sfu = 0;
};
TallyC g_tc;
struct CntC {
    double v = 0.0;
    bool zero = true;
    CntC() = default;
    CntC(double x) : v(x), zero(x == 0.0) {}  // literals of the templates
    CntC(double x, bool z) : v(x), zero(z) {}
};
CntC operator+(CntC a, CntC b)
{
    if (!a.zero && !b.zero) ++g_tc.ops;
    return {a.v + b.v, a.zero && b.zero};
}
CntC operator-(CntC a, CntC b)
{
    if (!a.zero && !b.zero) ++g_tc.ops;
    return {a.v - b.v, a.zero && b.zero};
}
CntC operator*(CntC a, CntC b)
{
    ++g_tc.ops;
    return {a.v * b.v, false};
}
CntC operator-(CntC a) { return {-a.v, a.zero}; }
CntC vfma(CntC a, CntC b, CntC c)
{
    ++g_tc.ops;
    return {a.v * b.v + c.v, false};
}
}  // namespace
}  // namespace rtlbfsc

namespace rtlbfs {
template <>
struct vtraits<rtlbfsc::CntC> {
    static rtlbfsc::CntC bc(double c) { return {c, c == 0.0}; }
    static rtlbfsc::CntC rcp(rtlbfsc::CntC x)
    {
        ++rtlbfsc::g_tc.sfu;
        return {1.0 / x.v, false};
    }
};
}  // namespace rtlbfs

extern "C" int rtlbfsc_op_counts(double* face_ops, double* cell_ops, double* sfu_ops)
{
    using rtlbfsc::CntC;
    rtlbfsc::g_tc = rtlbfsc::TallyC();
    CntC vL[4], gL[8], vR[4], gR[8];
    for (int k = 0; k < 4; ++k) {
        vL[k] = {0.01 * (k + 1), false};
        vR[k] = {0.02 * (k + 1), false};
    }
    for (int k = 0; k < 8; ++k) {
        gL[k] = {0.001 * (k + 1), false};
        gR[k] = {0.002 * (k + 1), false};
    }
    rtlbfsc::FaceRec<CntC> fg;
    CntC x{0.3, false};
    fg.nx = fg.ny = fg.len = fg.tL = fg.tR = x;
    fg.h = fg.cL = fg.cR = fg.m_nu_2h = fg.m_chi_2h = fg.m_tf15 = fg.m_tg15 = x;
    CntC F[4];
    rtlbfsc::face_c<CntC>(vL, gL, vR, gR, fg, CntC{1.0, false}, CntC{0.0, true}, CntC{0.0, true},
                          CntC{0.5, false}, F);
    const rtlbfsc::TallyC f = rtlbfsc::g_tc;
    // Per cell besides its two faces: working values 4, Green-Gauss gradients
    // with the coefficients w_f S_f / A of each cell precomputed (4 fields x
    // (4 differences, 8 products and FMAs) = 48), flux divergence 4 x 4 = 16,
    // sources 8, increments and new values 15, fixed-point increments 4,
    // residual 16.
    const double other = 111.0, other_sfu = 4.0;
    if (face_ops) *face_ops = (double)f.ops;
    if (cell_ops) *cell_ops = 2.0 * (double)f.ops + other;
    if (sfu_ops) *sfu_ops = 2.0 * (double)f.sfu + other_sfu;
    return RTLBFS_OK;
}
