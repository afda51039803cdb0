// rtlbfs_dev.cuh -- device-side data layout and the per-face arithmetic of
// RTLBFS (arXiv 2202.13449, Section 3.2), templated on the storage type R
// (double for the FP64 path, float for the FP32 bulk path).
//
// Every field is stored as (drho = rho - 1, u, v, T); in FP32 this keeps the
// weakly compressible density perturbation in the mantissa, and the pressure
// part c_s^2 rho of the momentum flux is formed from drho (the constant
// c_s^2 * 1 cancels in every flux difference because the face areas of a
// closed rectilinear cell sum to zero).
#pragma once

#include <cmath>
#include <cstdint>

namespace rtlbfs {

constexpr int kSideW = 0, kSideE = 1, kSideS = 2, kSideN = 3;
constexpr int kDirichlet = 0, kAdiabatic = 1, kPeriodic = 2;

// Status of a cavity's run, written by the device.
constexpr int kRunning = 0, kConverged = 1, kMaxSteps = 2, kDiverged = 3;

// Constants of one line of faces normal to an axis (all faces of an x-face
// column share them): lattice spacing h = kappa*min(wL, wR) (per-face dt of
// the reconstructed lattice), node offsets, transport coefficients.
template <typename R>
struct FaceLine {
    R h;       // lattice spacing dt_f
    R cL;      // wL - h : normal offset of node a = -1 from the left centre
    R cR;      // h - wR : normal offset of node a = +1 from the right centre
    R wL, wR;  // half widths of the two cells (centre-to-face distances)
    R nu_2h;   // nu / (2 h): viscous term with a central difference over 2h
    R chi_2h;  // chi / (2 h)
    R tf15;    // tau_f - 1.5 = nu / (cs2 h) - 1   (Eqs. 9, 58)
    R tg15;    // tau_g - 1.5 = chi / (cs2 h) - 1  (Eqs. 10, 59)
};

// Constants of one line of cells along an axis, ghosts included.
//
// Eqs. 55-56 on a rectilinear mesh: with inverse-distance face values the
// Green-Gauss derivative of cell c along a line is
//   (phi_{c+1} - phi_c) / (w_c + w_{c+1}) + (phi_c - phi_{c-1}) / (w_{c-1} + w_c),
// which is formed from neighbour differences (exact for the fixed-point
// state) with is_next = 1 / (w_c + w_{c+1}).
template <typename R>
struct CellLine {
    R w;        // cell width (ghost: partner's width, periodic: opposite cell's)
    R is_next;  // 1 / (w + w_next)
    R dt_w;     // Delta t / width
    R pad;
};

// Read-only description of one cavity (one mesh) on the device.
struct CavityDesc {
    int nx, ny, pitch, ntiles;    // cells, row stride (elements), tiles of this cavity
    int kind[4];                  // boundary kind per side W,E,S,N
    int tiles_x, tiles_y, tile_begin, pad0;
    double bcT[4], bcU[4];        // wall temperature, tangential wall velocity
    double beta_g, T_ref, fx, fy, dt, dT, nu, chi;
    void* f[2][4];                // two buffers of (drho, u, v, T)
    const void* xline;            // FaceLine<R>[nx+1]
    const void* yline;            // FaceLine<R>[ny+1]
    const void* xcell;            // CellLine<R>[nx+4], index i+2 for cell i in [-2, nx+1]
    const void* ycell;            // CellLine<R>[ny+4]
};

// Mutable per-cavity run control (device-written between steps).
struct CavityCtl {
    int cur;                  // buffer holding the current state
    int done;                 // 1: this cavity takes no more steps
    int status;               // kRunning, kConverged, kMaxSteps, kDiverged
    unsigned int arrive;      // tiles of this cavity finished in this step
    long long steps;          // steps taken since the last state upload
    long long max_steps;      // done when steps reaches this
    double tol;               // done when max(R_u, R_T) < tol (tol < 0: never)
    double res[2];            // (R_u, R_T) of the last step
    double acc[4];            // running sums of this step: sum (d|u|)^2, |u|^2, (dT)^2, T^2
};

template <typename R>
struct Vec4 {
    R x, y, z, w;
};

template <typename R>
__host__ __device__ __forceinline__ R rconst(double v) { return static_cast<R>(v); }

// 1/x: IEEE in FP64; the hardware approximation (a few ulp) in FP32.
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }

// -------------------------------------------------------------------------
// One face in its own frame: normal n (the "x" of a node (a, b)), tangent t.
// q[] = (drho, u_n, u_t, T - Tbar) of a cell, gn/gt its gradients along n
// and t.  Temperatures enter as deviations from a face reference Tbar so
// that the O(1) energy rho*T never has to be differenced in FP32.
// -------------------------------------------------------------------------
template <typename R>
struct CellNT {
    R q[4];
    R gn[4];
    R gt[4];
};

// Eqs. 29, 46-48 and the braces of Eqs. 57-59 for one face.  Output
// F = (mass, normal momentum, tangential momentum, energy) flux through the
// face along +n, with the constant c_s^2 dropped from the normal momentum
// flux (see the file comment).  wall: the face lies on a wall whose
// tangential velocity is u_wall_t.
//
// Node values.  A cell's reconstruction plane restricted to a column of
// nodes a = const is linear in b, so the three columns are c_a + b s_a:
//   a = -1: left plane,  a = +1: right plane,  a = 0: mean of both (Eq. 29).
// Central differences on the 9 nodes, written without the powers of h that
// cancel in Eqs. 46-48 (d_x ~ 2h D_x, d_xx ~ h^2 D_xx, d_xy ~ 4h^2 D_xy).
// The energy rho*T at a node is written Tbar + e with e = tau + drho*T,
// tau = T - Tbar; every difference of rho*T is a difference of e.
template <typename R>
__device__ __forceinline__ void face_flux(const CellNT<R>& L, const CellNT<R>& Rc, R Tbar,
                                          const FaceLine<R>& fl, bool wall, R u_wall_t,
                                          R F[4])
{
    const R half = rconst<R>(0.5);
    const R one = rconst<R>(1.0);
    const R cs2 = rconst<R>(1.0 / 3.0);
    const R hh = fl.h * half;
    R A[4], Sa[4], M[4], Sm[4], B[4], Sb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        A[k] = L.q[k] + L.gn[k] * fl.cL;
        Sa[k] = L.gt[k] * fl.h;
        B[k] = Rc.q[k] + Rc.gn[k] * fl.cR;
        Sb[k] = Rc.gt[k] * fl.h;
        M[k] = half * ((L.q[k] + L.gn[k] * fl.wL) + (Rc.q[k] - Rc.gn[k] * fl.wR));
        Sm[k] = hh * (L.gt[k] + Rc.gt[k]);
    }
    // plus nodes: c = (0,0), w = (-1,0), e = (+1,0), s = (0,-1), n = (0,+1);
    // d* = rho - 1, t* = tangential velocity, a* = T - Tbar
    const R d0 = M[0], n0 = M[1], t0 = M[2], a0 = M[3];
    const R dw = A[0], nw = A[1], tw = A[2], aw = A[3];
    const R de = B[0], ne = B[1], te = B[2], ae = B[3];
    const R ds = M[0] - Sm[0], ns = M[1] - Sm[1], ts = M[2] - Sm[2], as = M[3] - Sm[3];
    const R dn = M[0] + Sm[0], nn = M[1] + Sm[1], tn = M[2] + Sm[2], an = M[3] + Sm[3];
    const R T0 = Tbar + a0, Tw = Tbar + aw, Te = Tbar + ae, Ts = Tbar + as, Tn = Tbar + an;

    // node products (only those the predictor and the flux use)
    const R mn0 = (one + d0) * n0, mt0 = (one + d0) * t0, e0 = a0 + d0 * T0;
    const R Pnn0 = mn0 * n0, Pnt0 = mn0 * t0, Ptt0 = mt0 * t0, Qn0 = mn0 * T0;
    const R mnw = (one + dw) * nw, mtw = (one + dw) * tw, ew = aw + dw * Tw;
    const R Pnnw = mnw * nw, Pntw = mnw * tw, Qnw = mnw * Tw;
    const R mne = (one + de) * ne, mte = (one + de) * te, ee = ae + de * Te;
    const R Pnne = mne * ne, Pnte = mne * te, Qne = mne * Te;
    const R mns = (one + ds) * ns, mts = (one + ds) * ts, es = as + ds * Ts;
    const R Pnts = mns * ts, Ptts = mts * ts, Qts = mts * Ts;
    const R mnn = (one + dn) * nn, mtn = (one + dn) * tn, en = an + dn * Tn;
    const R Pntn = mnn * tn, Pttn = mtn * tn, Qtn = mtn * Tn;
    // corners (a, b): only rho u_n, rho u_t and rho u_n u_t enter (through d_xy)
    R mnc[4], mtc[4], Pntc[4];  // order (-1,-1), (-1,+1), (+1,-1), (+1,+1)
    {
        const R rc[4] = {one + (A[0] - Sa[0]), one + (A[0] + Sa[0]), one + (B[0] - Sb[0]),
                         one + (B[0] + Sb[0])};
        const R nc[4] = {A[1] - Sa[1], A[1] + Sa[1], B[1] - Sb[1], B[1] + Sb[1]};
        const R tc[4] = {A[2] - Sa[2], A[2] + Sa[2], B[2] - Sb[2], B[2] + Sb[2]};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            mnc[k] = rc[k] * nc[k];
            mtc[k] = rc[k] * tc[k];
            Pntc[k] = mnc[k] * tc[k];
        }
    }
    const R two = rconst<R>(2.0);
    // central differences
    const R dx_mn = mne - mnw, dx_mt = mte - mtw, dx_e = ee - ew;
    const R dy_mn = mnn - mns, dy_mt = mtn - mts;
    const R dx_dr = B[0] - A[0];
    const R dy_dr = two * Sm[0];
    const R dxx_dr = (B[0] + A[0]) - two * M[0];
    const R dxx_Pnn = (Pnne + Pnnw) - two * Pnn0;
    const R dyy_Ptt = (Pttn + Ptts) - two * Ptt0;
    const R dxy_Pnt = (Pntc[3] - Pntc[2]) - (Pntc[1] - Pntc[0]);
    const R dxy_mn = (mnc[3] - mnc[2]) - (mnc[1] - mnc[0]);
    const R dxy_mt = (mtc[3] - mtc[2]) - (mtc[1] - mtc[0]);
    const R dxx_mn = (mne + mnw) - two * mn0, dyy_mn = (mnn + mns) - two * mn0;
    const R dxx_mt = (mte + mtw) - two * mt0, dyy_mt = (mtn + mts) - two * mt0;
    const R dxx_e = (ee + ew) - two * e0, dyy_e = (en + es) - two * e0;
    const R quarter = rconst<R>(0.25);
    const R hcs2 = rconst<R>(0.5 / 3.0);  // c_s^2 / 2

    // Eq. 46: rho* (as drho*)
    const R drs = M[0] - half * (dx_mn + dy_mt) +
                  half * (dxx_Pnn + cs2 * dxx_dr + dyy_Ptt) + quarter * dxy_Pnt;
    // Eq. 47: (rho u_n)*, (rho u_t)*
    R mns_ = mn0 - half * ((Pnne - Pnnw) + cs2 * dx_dr + (Pntn - Pnts)) +
             hcs2 * (rconst<R>(3.0) * dxx_mn + dyy_mn + half * dxy_mt);
    R mts_ = mt0 - half * ((Pnte - Pntw) + (Pttn - Ptts) + cs2 * dy_dr) +
             hcs2 * (dxx_mt + rconst<R>(3.0) * dyy_mt + half * dxy_mn);
    // Eq. 48: (rho T)* - Tbar
    const R es_ = e0 - half * ((Qne - Qnw) + (Qtn - Qts)) + hcs2 * (dxx_e + dyy_e);

    const R rho_s = one + drs;
    if (wall) {  // no mass through a wall; the wall's tangential velocity
        mns_ = rconst<R>(0.0);
        mts_ = rho_s * u_wall_t;
    }
    const R inv = fast_rcp(rho_s);
    const R uns = mns_ * inv, uts = mts_ * inv;
    const R as_ = (es_ - drs * Tbar) * inv;  // T* - Tbar

    // Eqs. 57-59 braces along the face normal
    F[0] = mns_;
    const R Xnn0 = Pnn0 + cs2 * d0;
    F[1] = Xnn0 - fl.nu_2h * (rconst<R>(3.0) * dx_mn + dy_mt) -
           fl.tf15 * ((mns_ * uns + cs2 * drs) - Xnn0);
    F[2] = Pnt0 - fl.nu_2h * (dx_mt + dy_mn) - fl.tf15 * (mns_ * uts - Pnt0);
    // (rho u_n T)* - (rho u_n T)^n = Tbar (mn* - mn0) + mn* a* - mn0 a0
    F[3] = Qn0 - fl.chi_2h * dx_e -
           fl.tg15 * (Tbar * (mns_ - mn0) + (mns_ * as_ - mn0 * a0));
}

// Parity of quantity k (0 drho, 1 u, 2 v, 3 T) about a wall of side s:
// +1 even (mirror value), -1 odd about the wall value.
__host__ __device__ __forceinline__ int wall_parity(int kind, int k)
{
    if (k == 0) return +1;
    if (k == 1 || k == 2) return -1;
    return kind == kDirichlet ? -1 : +1;
}

// -------------------------------------------------------------------------
// Storage of the state.  StoreD: FP64 values, FP64 arithmetic.  StoreQ:
// FP32 arithmetic on a 32-bit fixed-point state (value = q * scale): an
// explicit iteration stalls once its increments fall below half a unit of
// the stored value, so the state keeps more bits than an FP32 mantissa for
// these bounded fields at the same 4 bytes; increments are computed in FP32
// and added exactly.  Ranges: rho - 1 in (-0.5, 0.5), u, v in (-1, 1),
// T in (-2, 2); leaving a range is reported as divergence.
// -------------------------------------------------------------------------
struct StoreD {
    using S = double;
    using R = double;
    static __host__ __device__ __forceinline__ R val(S s, int) { return s; }
    static __host__ __device__ __forceinline__ R diff(S a, S b, int) { return a - b; }
    static __host__ __device__ __forceinline__ S add(S s, R d, int) { return s + d; }
    static __host__ __device__ __forceinline__ S from_double(double v, int) { return v; }
    static __host__ __device__ __forceinline__ double to_double(S s, int) { return s; }
    static __host__ __device__ __forceinline__ S mirror_odd(S wall2, S s) { return wall2 - s; }
    static __host__ __device__ __forceinline__ S twice(S s) { return 2.0 * s; }
    static __host__ __device__ __forceinline__ bool representable(double, int) { return true; }
    static __host__ __device__ __forceinline__ bool in_range(R v, int) { return v == v; }
    static __device__ __forceinline__ R rcp(R x) { return 1.0 / x; }
    static __device__ __forceinline__ R fsqrt(R x) { return sqrt(x); }
};

struct StoreQ {
    using S = int;
    using R = float;
    // scale of quantity k: 2^-32 (rho - 1), 2^-31 (u, v), 2^-30 (T)
    static __host__ __device__ __forceinline__ double scale_d(int k)
    {
        return k == 0 ? 2.3283064365386963e-10 : (k == 3 ? 9.313225746154785e-10 : 4.656612873077393e-10);
    }
    static __host__ __device__ __forceinline__ float scale_f(int k) { return (float)scale_d(k); }
    static __host__ __device__ __forceinline__ float limit(int k)
    {
        return k == 0 ? 0.49f : (k == 3 ? 1.98f : 0.99f);
    }
    static __host__ __device__ __forceinline__ R val(S s, int k) { return (float)s * scale_f(k); }
    // exact integer difference (wrap-around subtraction is exact whenever the
    // true difference fits in 32 bits), then one rounding to float
    static __host__ __device__ __forceinline__ R diff(S a, S b, int k)
    {
        return (float)(int)((unsigned)a - (unsigned)b) * scale_f(k);
    }
    static __device__ __forceinline__ S add(S s, R d, int k)
    {
        return (int)((unsigned)s + (unsigned)__float2int_rn(d * (1.0f / scale_f(k))));
    }
    static __host__ __device__ __forceinline__ bool representable(double v, int k)
    {
        return fabs(v) < (double)limit(k);  // false for NaN too
    }
    static __host__ __device__ __forceinline__ S from_double(double v, int k)
    {
        if (!(v == v)) return 0;
        double q = v / scale_d(k);
        q = q > 2147483000.0 ? 2147483000.0 : (q < -2147483000.0 ? -2147483000.0 : q);
        return (int)(q < 0 ? q - 0.5 : q + 0.5);
    }
    static __host__ __device__ __forceinline__ double to_double(S s, int k) { return (double)s * scale_d(k); }
    static __host__ __device__ __forceinline__ S mirror_odd(S wall2, S s)
    {
        return (int)((unsigned)wall2 - (unsigned)s);
    }
    // 2 s with wrap-around: exact for the mirror 2 s - x whenever that fits
    static __host__ __device__ __forceinline__ S twice(S s) { return (int)(2u * (unsigned)s); }
    static __host__ __device__ __forceinline__ bool in_range(R v, int k)
    {
        return fabsf(v) < limit(k);
    }
    // reciprocal and square root at FP32 accuracy (a few ulp), not IEEE rounding
    static __device__ __forceinline__ R rcp(R x) { return __fdividef(1.0f, x); }
    static __device__ __forceinline__ R fsqrt(R x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
};

}  // namespace rtlbfs
