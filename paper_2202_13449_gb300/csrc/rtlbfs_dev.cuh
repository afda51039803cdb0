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

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

namespace rtlbfs {

// Chained time steps.  A step kernel launched with programmatic stream
// serialisation (launch_chained) may become resident while the previous
// step's grid drains; its blocks wait here, before they read anything that
// grid wrote (run control, state), and then allow the next step's grid to
// launch.  In a launch without the attribute both instructions return at
// once.
__device__ __forceinline__ void chain_sync()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch kernel fn on stream s with programmatic stream serialisation: it
// may start before the preceding kernel on s has finished, and must call
// chain_sync() before it touches that kernel's output.
template <typename... K, typename... A>
cudaError_t launch_chained(void (*fn)(K...), unsigned grid, unsigned block, size_t smem,
                           cudaStream_t s, A... args)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, static_cast<K>(args)...);
}

constexpr int kSideW = 0, kSideE = 1, kSideS = 2, kSideN = 3;
constexpr int kDirichlet = 0, kAdiabatic = 1, kPeriodic = 2;
// A south or north side that borders another row strip of the same mesh:
// the two rows beyond it are stored below / above the strip's own rows
// (rows -2, -1 and ny, ny + 1 of its buffers) and filled by a halo
// exchange before each step; no mirror rule, no wall face.
constexpr int kHalo = 3;

// Status of a cavity's run, written by the device.
constexpr int kRunning = 0, kConverged = 1, kMaxSteps = 2, kDiverged = 3;

// Constants of one line of faces normal to an axis (all faces of an x-face
// column share them): lattice spacing h = kappa*min(wL, wR) (per-face dt of
// the reconstructed lattice), node offsets, transport coefficients.
template <typename R>
struct FaceLine {
    R h;        // lattice spacing dt_f
    R cL;       // wL - h : normal offset of node a = -1 from the left centre
    R cR;       // h - wR : normal offset of node a = +1 from the right centre
    R m_nu_2h;  // -nu / (2 h): viscous term with a central difference over 2h
    R m_chi_2h; // -chi / (2 h)
    R m_tf15;   // -(tau_f - 1.5) = 1 - nu / (cs2 h)   (Eqs. 9, 58)
    R m_tg15;   // -(tau_g - 1.5) = 1 - chi / (cs2 h)  (Eqs. 10, 59)
    R pad;
    // wL = cL + h and wR = h - cR are the two centre-to-face distances
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
    int tiles_x, tiles_y, tile_begin;
    int scheme;  // face stage: 0 RTLBFS (Section 3.2), 1 TLBFS (Section 2.2)
    double bcT[4], bcU[4];        // wall temperature, tangential wall velocity
    double beta_g, T_ref, fx, fy, dt, dT, nu, chi;
    // FP32 copies (a double -> float conversion runs on the narrow FP64
    // pipe; the FP32 kernels never convert in their loops)
    float f_beta_g, f_T_ref, f_fx, f_fy, f_dt, f_bcU[4], f_bcT[4];
    // two state buffers; each is an array of ny*pitch cell records
    // (rho - 1, u, v, T) -- Vec4<S>, 16 bytes in FP32 mode, 32 in FP64 --
    // in f[b][0] (f[b][1..3] used only by callers' separate-array layouts)
    void* f[2][4];
    const void* xline;            // FaceLine<R>[nx+1]
    const void* yline;            // FaceLine<R>[ny+1]
    const void* xcell;            // CellLine<R>[nx+4], index i+2 for cell i in [-2, nx+1]
    const void* ycell;            // CellLine<R>[ny+4]
};

// Run control of a cavity: the state of its run after the last step whose
// stop test has been made.
struct CavityCtl {
    int cur;                  // buffer holding the current state
    int done;                 // 1: this cavity takes no more steps
    int status;               // kRunning, kConverged, kMaxSteps, kDiverged
    int pend;                 // 1: step `steps` was taken, its stop test not yet made
    long long steps;          // steps tested since the last state upload
    long long max_steps;      // done when steps reaches this
    double tol;               // done when max(R_u, R_T) < tol (tol < 0: never)
    double res[2];            // (R_u, R_T) of the last tested step (see res_stale)
    double sums[4];           // residual sums of the last tested step
    int res_stale;            // 1: res not yet formed from sums (finalize_run does it)
    int pad;
};

// Device record of a cavity's run.  A step launch never waits for its own
// residual: its units add their sums for step k into acc[k % 3] and the
// stop test of step k is made by every unit of the next launch as it
// starts.  A launch of parity par reads only h[par]; the cavity's first
// unit writes the header after the test (and after this launch's step) to
// h[par ^ 1] and clears acc[(k + 1) % 3] for the step after.  Between
// launches h[0] is the header the host reads (a finalising launch makes
// the last test and copies the result to both headers).
struct CavityRun {
    CavityCtl h[2];
    double acc[3][4];         // per step: sum (d|u|)^2, |u|^2, (dT)^2, T^2
};

// R12 from the residual sums of a step: ||d|u|||_2 / |||u|^{n+1}||_2 (or
// the same for T); a zero denominator gives infinity.
__host__ __device__ inline double r12(double num, double den)
{
    return den > 0.0 ? sqrt(num) / sqrt(den) : INFINITY;
}

// r12(num, den) < tol, decided without the FP64 square roots and division
// unless the ratio lies within 2 % of tol^2: the same outcome as the
// formula (its rounding error is ~1e-16 relative), a fraction of its
// latency on the narrow FP64 units of this GPU.
__host__ __device__ inline bool r12_below(double num, double den, double tol)
{
    if (!(den > 0.0) || !(tol > 0.0)) return false;
    const double q = tol * tol * den;
    if (q >= 2.2250738585072014e-308 && q < 1e300) {
        if (num < 0.98 * q) return true;
        if (num > 1.02 * q) return false;
    }
    return r12(num, den) < tol;
}

// The stop test of the pending step of c (pend = 1), from that step's
// residual sums s: the header after it (res formed later, res_stale set).
// A header without a pending step is returned as is.  Outcomes as with
// R = r12(...): diverged when R_u or R_T is not a number or a sum is not a
// number, converged when max(R_u, R_T) < tol, else capped at max_steps.
__host__ __device__ inline CavityCtl stop_test(CavityCtl c, const double s[4])
{
    if (!c.pend) return c;
    const double su = s[0], du = s[1], sT = s[2], dT = s[3];
    for (int q = 0; q < 4; ++q) c.sums[q] = s[q];
    c.res_stale = 1;
    c.steps += 1;
    c.cur ^= 1;
    c.pend = 0;
    // r12 is NaN exactly when num is NaN or both are infinite (den > 0)
    const bool nan_u = isnan(su) || (du > 0.0 && isinf(su) && isinf(du));
    const bool nan_T = isnan(sT) || (dT > 0.0 && isinf(sT) && isinf(dT));
    int status = kRunning;
    if (nan_u || nan_T) status = kDiverged;
    else if (r12_below(su, du, c.tol) && r12_below(sT, dT, c.tol)) status = kConverged;
    else if (c.steps >= c.max_steps) status = kMaxSteps;
    c.status = status;
    if (status != kRunning) c.done = 1;
    return c;
}

// Header of parity par after the stop test of its pending step (one
// thread; the header and all three sum slots are loaded at once, so this
// is one round trip).
__device__ inline CavityCtl run_head(const CavityRun* r, int par)
{
    const CavityCtl c = r->h[par];
    double a[3][4];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) a[k][q] = r->acc[k][q];
    const int slot = (int)(c.steps % 3);
    double s[4];  // selected by value: no local-memory copy of a
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] = slot == 0 ? a[0][q] : (slot == 1 ? a[1][q] : a[2][q]);
    return stop_test(c, s);
}

// What the cavity's first unit of a launch of parity par writes: the
// tested header d, with the step this launch takes pending unless the
// cavity is done, and the sum slot of the step after cleared.
__device__ inline void run_publish(CavityRun* r, int par, CavityCtl d)
{
    if (!d.done) {
        d.pend = 1;
        double* z = r->acc[(int)((d.steps + 1) % 3)];
#pragma unroll
        for (int q = 0; q < 4; ++q) z[q] = 0.0;
    }
    r->h[par ^ 1] = d;
}

// Four values of one cell; 16-byte aligned for 4-byte R, 32 for double, so
// a cell record moves in one (or two) vector memory instructions.
template <typename R>
struct alignas(4 * sizeof(R)) Vec4 {
    R x, y, z, w;
};

template <typename R>
__host__ __device__ __forceinline__ R rconst(double v) { return static_cast<R>(v); }

// 1/x: IEEE in FP64; the hardware approximation (a few ulp) in FP32.
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }

// -------------------------------------------------------------------------
// Value types of the face arithmetic.  float / double: one face.  f2: two
// faces at once in the packed FP32x2 instructions of sm_100+ (one issue
// slot for two round-to-nearest FP32 operations); d2: the FP64 pair.
// -------------------------------------------------------------------------
struct f2 {
    float x, y;
};
struct d2 {
    double x, y;
};

__device__ __forceinline__ f2 mk(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 fl2(f2 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return mk(__fadd2_rn(fl2(a), fl2(b))); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b)
{
    return mk(__ffma2_rn(fl2(b), make_float2(-1.0f, -1.0f), fl2(a)));
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return mk(__fmul2_rn(fl2(a), fl2(b))); }
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) { return mk(__ffma2_rn(fl2(a), fl2(b), fl2(c))); }

__host__ __device__ __forceinline__ d2 operator+(d2 a, d2 b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ d2 operator-(d2 a, d2 b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ __forceinline__ d2 operator*(d2 a, d2 b) { return {a.x * b.x, a.y * b.y}; }
__device__ __forceinline__ d2 vfma(d2 a, d2 b, d2 c) { return {fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)}; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }

template <typename V>
struct vtraits;
template <>
struct vtraits<float> {
    static __device__ __forceinline__ float bc(double c) { return (float)c; }
    static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
};
template <>
struct vtraits<double> {
    static __device__ __forceinline__ double bc(double c) { return c; }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
};
template <>
struct vtraits<f2> {
    static __device__ __forceinline__ f2 bc(double c) { return {(float)c, (float)c}; }
    static __device__ __forceinline__ f2 rcp(f2 x) { return {__fdividef(1.0f, x.x), __fdividef(1.0f, x.y)}; }
};
template <>
struct vtraits<d2> {
    static __device__ __forceinline__ d2 bc(double c) { return {c, c}; }
    static __device__ __forceinline__ d2 rcp(d2 x) { return {1.0 / x.x, 1.0 / x.y}; }
};

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

// Eqs. 29, 46-48 and the braces of Eqs. 57-59 for one face (V = float,
// double) or two faces (V = f2, d2).  Output F = (mass, normal momentum,
// tangential momentum, energy) flux through the face along +n, with the
// constant c_s^2 dropped from the normal momentum flux (see the file
// comment).  keep = 1 on an interior face, 0 on a wall face, whose
// tangential wall velocity is u_wall (no mass through a wall, (rho u_t)* =
// rho* u_wall: the products with keep and 1 - keep are exact).
//
// Node values.  Node (a, b) sits at x_S + (a, b) h (a along the normal).
// A cell's reconstruction plane restricted to a column a = const is linear
// in b, so every primitive on column a is c_a + b s_a:
//   a = -1: the left plane,  a = +1: the right plane,  a = 0: their mean
// (Eq. 29).  The predictor needs central differences of node products:
//   d_x f  = f(1,0) - f(-1,0)             (= 2h D_x f)
//   d_xx f = f(1,0) - 2 f(0,0) + f(-1,0)  (= h^2 D_xx f)
//   d_y f  = f(0,1) - f(0,-1),  d_yy f = f(0,1) - 2 f(0,0) + f(0,-1)
//   d_xy f = f(1,1) - f(1,-1) - f(-1,1) + f(-1,-1)  (= 4 h^2 D_xy f)
// and the products are polynomials in b on each column, so
//   d_y f = 2 (odd coefficients at a = 0), d_yy f = 2 (b^2 coefficient at a = 0),
//   d_xy f = 2 (odd(a = +1) - odd(a = -1)):
// the same numbers as forming the products at the nine nodes, with fewer
// operations.  The powers of h cancel in Eqs. 46-48.  The energy rho*T at a
// node is written Tbar + e with e = tau + drho*T, tau = T - Tbar, so every
// difference of rho*T is a difference of e.
//
// The first stage, face_columns, forms the column coefficients c_a and s_a
// of the four primitives; face_flux_columns does the rest.
template <typename V>
__host__ __device__ __forceinline__ void face_columns(const CellNT<V>& L, const CellNT<V>& Rc,
                                                      const FaceLine<V>& fl, V A[4], V Sa[4],
                                                      V M[4], V Sm[4], V B[4], V Sb[4])
{
    using T = vtraits<V>;
    const V half = T::bc(0.5);
    const V h = fl.h;
    const V wL = fl.cL + h, mwR = fl.cR - h;  // wL, -wR
    const V hh = h * half;
    // column coefficients: A (a = -1), M (a = 0), B (a = +1); S* slopes in b
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        A[k] = vfma(L.gn[k], fl.cL, L.q[k]);
        Sa[k] = L.gt[k] * h;
        B[k] = vfma(Rc.gn[k], fl.cR, Rc.q[k]);
        Sb[k] = Rc.gt[k] * h;
        M[k] = half * (vfma(L.gn[k], wL, L.q[k]) + vfma(Rc.gn[k], mwR, Rc.q[k]));
        Sm[k] = hh * (L.gt[k] + Rc.gt[k]);
    }
}

template <typename V>
__host__ __device__ __forceinline__ void face_flux_columns(const V A[4], const V Sa[4], const V M[4],
                                                           const V Sm[4], const V B[4],
                                                           const V Sb[4], V Tbar,
                                                           const FaceLine<V>& fl, V keep, V u_wall,
                                                           V F[4])
{
    using T = vtraits<V>;
    const V half = T::bc(0.5), one = T::bc(1.0), two = T::bc(2.0), three = T::bc(3.0);
    const V m2 = T::bc(-2.0), mhalf = T::bc(-0.5);
    const V cs2 = T::bc(1.0 / 3.0), mcs2 = T::bc(-1.0 / 3.0);
    const V hcs2 = T::bc(0.5 / 3.0);  // c_s^2 / 2
    // centres (b = 0) of the three columns: rho u_n, rho u_t, products
    const V TA = Tbar + A[3], TM = Tbar + M[3], TB = Tbar + B[3];
    const V mnA = vfma(A[0], A[1], A[1]), mnM = vfma(M[0], M[1], M[1]), mnB = vfma(B[0], B[1], B[1]);
    const V mtA = vfma(A[0], A[2], A[2]), mtM = vfma(M[0], M[2], M[2]), mtB = vfma(B[0], B[2], B[2]);
    const V PnnA = mnA * A[1], PnnM = mnM * M[1], PnnB = mnB * B[1];
    const V PntA = mnA * A[2], PntM = mnM * M[2], PntB = mnB * B[2];
    const V QnA = mnA * TA, QnM = mnM * TM, QnB = mnB * TB;
    const V eA = vfma(A[0], TA, A[3]), eM = vfma(M[0], TM, M[3]), eB = vfma(B[0], TB, B[3]);
    // column a = 0 in b: rho = rM + b sd, u_n = M1 + b sn, u_t = M2 + b st, T = TM + b sT
    const V rM = one + M[0];
    const V sd = Sm[0], sn = Sm[1], st = Sm[2], sT = Sm[3];
    const V mn_l = vfma(rM, sn, sd * M[1]), mn_q = sd * sn;  // rho u_n: linear, quadratic
    const V mt_l = vfma(rM, st, sd * M[2]), mt_q = sd * st;  // rho u_t
    const V e_q = sd * sT;                                   // e: quadratic
    const V Pnt_o = vfma(mnM, st, vfma(mn_l, M[2], mn_q * st));  // rho u_n u_t: odd part
    const V Ptt_o = vfma(mtM, st, vfma(mt_l, M[2], mt_q * st));  // rho u_t u_t: odd part
    const V Ptt_q = vfma(mt_l, st, mt_q * M[2]);                 //              quadratic
    const V Qt_o = vfma(mtM, sT, vfma(mt_l, TM, mt_q * sT));     // rho u_t T: odd part
    // columns a = -1, +1: odd parts in b (for d_xy)
    const V rA = one + A[0], rB = one + B[0];
    const V mnA_o = vfma(rA, Sa[1], Sa[0] * A[1]), mnB_o = vfma(rB, Sb[1], Sb[0] * B[1]);
    const V mtA_o = vfma(rA, Sa[2], Sa[0] * A[2]), mtB_o = vfma(rB, Sb[2], Sb[0] * B[2]);
    const V PntA_o = vfma(mnA, Sa[2], vfma(mnA_o, A[2], Sa[0] * Sa[1] * Sa[2]));
    const V PntB_o = vfma(mnB, Sb[2], vfma(mnB_o, B[2], Sb[0] * Sb[1] * Sb[2]));
    // differences along the normal (b = 0)
    const V dx_mn = mnB - mnA, dx_mt = mtB - mtA, dx_e = eB - eA, dx_dr = B[0] - A[0];
    const V dxx_mn = vfma(m2, mnM, mnB + mnA), dxx_mt = vfma(m2, mtM, mtB + mtA);
    const V dxx_e = vfma(m2, eM, eB + eA), dxx_dr = vfma(m2, M[0], B[0] + A[0]);
    const V dxx_Pnn = vfma(m2, PnnM, PnnB + PnnA);

    // Eq. 46: drho* = rho* - 1
    const V drs = vfma(half, (dxx_Pnn - dx_mn) + (PntB_o - PntA_o),
                       vfma(hcs2, dxx_dr, (M[0] - mt_l) + Ptt_q));
    // Eq. 47: (rho u_n)*, (rho u_t)*
    V mns_ = vfma(hcs2, vfma(three, dxx_mn, vfma(two, mn_q, mtB_o - mtA_o)),
                  vfma(mhalf, vfma(cs2, dx_dr, PnnB - PnnA), mnM - Pnt_o));
    V mts_ = vfma(hcs2, vfma(T::bc(6.0), mt_q, dxx_mt + (mnB_o - mnA_o)),
                  vfma(mhalf, PntB - PntA, vfma(mcs2, sd, mtM - Ptt_o)));
    // Eq. 48: (rho T)* - Tbar
    const V es_ = vfma(hcs2, vfma(two, e_q, dxx_e), vfma(mhalf, QnB - QnA, eM - Qt_o));

    const V rho_s = one + drs;
    // wall faces: no mass through the wall, the wall's tangential velocity
    mns_ = mns_ * keep;
    mts_ = vfma(keep, mts_, (one - keep) * (rho_s * u_wall));
    const V inv = T::rcp(rho_s);
    const V uns = mns_ * inv, uts = mts_ * inv;
    const V as_ = (es_ - drs * Tbar) * inv;  // T* - Tbar

    // Eqs. 57-59 braces along the face normal; d_y f = 2 (odd part)
    F[0] = mns_;
    const V Xnn0 = vfma(cs2, M[0], PnnM);
    F[1] = vfma(fl.m_nu_2h, vfma(three, dx_mn, two * mt_l),
                vfma(fl.m_tf15, vfma(mns_, uns, cs2 * drs) - Xnn0, Xnn0));
    F[2] = vfma(fl.m_nu_2h, vfma(two, mn_l, dx_mt), vfma(fl.m_tf15, vfma(mns_, uts, T::bc(0.0) - PntM), PntM));
    // (rho u_n T)* - (rho u_n T)^n = Tbar (mn* - mn0) + mn* a* - mn0 a0
    F[3] = vfma(fl.m_chi_2h, dx_e,
                vfma(fl.m_tg15, vfma(Tbar, mns_ - mnM, vfma(mns_, as_, T::bc(0.0) - mnM * M[3])), QnM));
}

template <typename V>
__host__ __device__ __forceinline__ void face_flux(const CellNT<V>& L, const CellNT<V>& Rc, V Tbar,
                                          const FaceLine<V>& fl, V keep, V u_wall, V F[4])
{
    V A[4], Sa[4], M[4], Sm[4], B[4], Sb[4];
    face_columns<V>(L, Rc, fl, A, Sa, M, Sm, B, Sb);
    face_flux_columns<V>(A, Sa, M, Sm, B, Sb, Tbar, fl, keep, u_wall, F);
}

// Green-Gauss gradients of a cell p from its four neighbours in the
// CellLine form of Eqs. 55-56 (ixe = is_next of the cell, ixw that of its
// west neighbour; iyn, iys along y), FP32, two components per packed
// FP32x2 instruction:
//   g_x = (e - p) ixe + (p - w) ixw,  g_y = (n - p) iyn + (p - s) iys.
__device__ __forceinline__ void gg_gradient_f32(const Vec4<float>& p, const Vec4<float>& e,
                                                const Vec4<float>& w, const Vec4<float>& n,
                                                const Vec4<float>& s, float ixe, float ixw,
                                                float iyn, float iys, Vec4<float>& gx,
                                                Vec4<float>& gy)
{
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 xe = make_float2(ixe, ixe), xw = make_float2(ixw, ixw);
    const float2 yn = make_float2(iyn, iyn), ys = make_float2(iys, iys);
    const float2 P[2] = {make_float2(p.x, p.y), make_float2(p.z, p.w)};
    const float2 E[2] = {make_float2(e.x, e.y), make_float2(e.z, e.w)};
    const float2 W[2] = {make_float2(w.x, w.y), make_float2(w.z, w.w)};
    const float2 N[2] = {make_float2(n.x, n.y), make_float2(n.z, n.w)};
    const float2 S[2] = {make_float2(s.x, s.y), make_float2(s.z, s.w)};
    float2 gxp[2], gyp[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        // a - b as fma(b, -1, a): exact, one rounding like the subtraction
        gxp[i] = __ffma2_rn(__ffma2_rn(P[i], m1, E[i]), xe, __fmul2_rn(__ffma2_rn(W[i], m1, P[i]), xw));
        gyp[i] = __ffma2_rn(__ffma2_rn(P[i], m1, N[i]), yn, __fmul2_rn(__ffma2_rn(S[i], m1, P[i]), ys));
    }
    gx = {gxp[0].x, gxp[0].y, gxp[1].x, gxp[1].y};
    gy = {gyp[0].x, gyp[0].y, gyp[1].x, gyp[1].y};
}

// Flux balance of a cell, FP32, in packed pairs (mass, x-momentum) and
// (y-momentum, energy): div = ax (F_e - F_w) + ay (F_n - F_s), ax and ay the
// time step over the cell's widths.
__device__ __forceinline__ void flux_div_f32(const Vec4<float>& Fw, const Vec4<float>& Fe,
                                             const Vec4<float>& Fs, const Vec4<float>& Fn, float ax,
                                             float ay, float& d0, float& d1, float& d2, float& d3)
{
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 ax2 = make_float2(ax, ax), ay2 = make_float2(ay, ay);
    const float2 d01 = __ffma2_rn(
        __ffma2_rn(make_float2(Fw.x, Fw.y), m1, make_float2(Fe.x, Fe.y)), ax2,
        __fmul2_rn(__ffma2_rn(make_float2(Fs.x, Fs.y), m1, make_float2(Fn.x, Fn.y)), ay2));
    const float2 d23 = __ffma2_rn(
        __ffma2_rn(make_float2(Fw.z, Fw.w), m1, make_float2(Fe.z, Fe.w)), ax2,
        __fmul2_rn(__ffma2_rn(make_float2(Fs.z, Fs.w), m1, make_float2(Fn.z, Fn.w)), ay2));
    d0 = d01.x;
    d1 = d01.y;
    d2 = d23.x;
    d3 = d23.y;
}

// face_columns in FP32 from the two cells' working values (rho - 1, u, v,
// T - Tz) and their gradients along the face normal (gn) and tangent (gt),
// all in storage order, two components per packed FP32x2 instruction: the
// pairs (rho, u) and (v, T) of a record sit in adjacent registers.  The
// same operations as face_columns on the face-frame cells of face_cells
// (bit for bit); ISX: x-face (n = x), else y-face (n = y: u_n = v, u_t = u).
template <bool ISX>
__device__ __forceinline__ void face_columns_f32(const Vec4<float>& vl, const Vec4<float>& vr,
                                                 const Vec4<float>& gnl, const Vec4<float>& gtl,
                                                 const Vec4<float>& gnr, const Vec4<float>& gtr,
                                                 const FaceLine<float>& fl, float A[4],
                                                 float Sa[4], float M[4], float Sm[4], float B[4],
                                                 float Sb[4])
{
    const float h = fl.h;
    const float wL = fl.cL + h, mwR = fl.cR - h, hh = h * 0.5f;
    const float2 cL2 = make_float2(fl.cL, fl.cL), cR2 = make_float2(fl.cR, fl.cR);
    const float2 wL2 = make_float2(wL, wL), mwR2 = make_float2(mwR, mwR);
    const float2 h2 = make_float2(h, h), hh2 = make_float2(hh, hh), half2 = make_float2(0.5f, 0.5f);
    // the left cell's temperature is carried by Tbar = Tz + T_L
    const float2 ql[2] = {make_float2(vl.x, vl.y), make_float2(vl.z, 0.0f)};
    const float2 qr[2] = {make_float2(vr.x, vr.y), make_float2(vr.z, vr.w - vl.w)};
    const float2 nl[2] = {make_float2(gnl.x, gnl.y), make_float2(gnl.z, gnl.w)};
    const float2 tl[2] = {make_float2(gtl.x, gtl.y), make_float2(gtl.z, gtl.w)};
    const float2 nr[2] = {make_float2(gnr.x, gnr.y), make_float2(gnr.z, gnr.w)};
    const float2 tr[2] = {make_float2(gtr.x, gtr.y), make_float2(gtr.z, gtr.w)};
    float2 a[2], sa[2], m[2], sm[2], b[2], sb[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        a[i] = __ffma2_rn(nl[i], cL2, ql[i]);
        sa[i] = __fmul2_rn(tl[i], h2);
        b[i] = __ffma2_rn(nr[i], cR2, qr[i]);
        sb[i] = __fmul2_rn(tr[i], h2);
        m[i] = __fmul2_rn(half2, __fadd2_rn(__ffma2_rn(nl[i], wL2, ql[i]), __ffma2_rn(nr[i], mwR2, qr[i])));
        sm[i] = __fmul2_rn(hh2, __fadd2_rn(tl[i], tr[i]));
    }
    // face-frame order: (rho, u_n, u_t, T)
    auto put = [](const float2* v, float* d) {
        d[0] = v[0].x;
        d[1] = ISX ? v[0].y : v[1].x;
        d[2] = ISX ? v[1].x : v[0].y;
        d[3] = v[1].y;
    };
    put(a, A);
    put(sa, Sa);
    put(m, M);
    put(sm, Sm);
    put(b, B);
    put(sb, Sb);
}

// The original TLBFS face stage (Section 2.2), from the same inputs as
// face_flux and in the same frame: (a) D2Q9 equilibria (Eqs. 3-4, c_p = 1)
// at the nodes x_S - e_i h, i.e. node (a, b) = -e_i of the column form
// above (Eq. 29); (b) the predicted variables as their moments (Eqs. 30-32),
// then the wall rule; (c) the fluxes of Eqs. 38-40 from the equilibria of
// the predicted variables and the non-equilibrium parts of Eqs. 33-34.
// Equilibria are carried as deviations f_i - w_i and g_i - w_i Tbar: the
// constants cancel in every moment used except the pressure c_s^2, which is
// dropped from the normal momentum flux as in face_flux.  The Dirichlet
// override of (rho T)* is omitted: it enters no flux (u*_n = 0 there).
template <typename V>
__host__ __device__ __forceinline__ void face_flux_tlbfs(const CellNT<V>& L, const CellNT<V>& Rc,
                                                        V Tbar, const FaceLine<V>& fl, V keep,
                                                        V u_wall, V F[4])
{
    using T = vtraits<V>;
    const V half = T::bc(0.5), one = T::bc(1.0), three = T::bc(3.0);
    const V c45 = T::bc(4.5), c15 = T::bc(1.5);
    // D2Q9 in the face frame (n, t); weights of Eq. 6
    constexpr int en[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int et[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const V w0 = T::bc(4.0 / 9.0), w1 = T::bc(1.0 / 9.0), w2 = T::bc(1.0 / 36.0);
    const V h = fl.h;
    const V wL = fl.cL + h, mwR = fl.cR - h;
    const V hh = h * half;
    // columns a = -1 (left plane), 0 (mean), +1 (right plane): value + b slope
    V C[3][4], Sl[3][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        C[0][k] = vfma(L.gn[k], fl.cL, L.q[k]);
        Sl[0][k] = L.gt[k] * h;
        C[2][k] = vfma(Rc.gn[k], fl.cR, Rc.q[k]);
        Sl[2][k] = Rc.gt[k] * h;
        C[1][k] = half * (vfma(L.gn[k], wL, L.q[k]) + vfma(Rc.gn[k], mwR, Rc.q[k]));
        Sl[1][k] = hh * (L.gt[k] + Rc.gt[k]);
    }
    // (a), (b): equilibria at the nodes and their moments
    V df[9], dg[9];
    V drs = T::bc(0.0), mn = T::bc(0.0), mt = T::bc(0.0), es = T::bc(0.0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int a = 1 - en[i], b = -et[i];  // column index, offset along t
        V q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            q[k] = b == 0 ? C[a][k] : (b > 0 ? C[a][k] + Sl[a][k] : C[a][k] - Sl[a][k]);
        const V w = i == 0 ? w0 : (i < 5 ? w1 : w2);
        V eu = T::bc(0.0);
        if (en[i] > 0) eu = eu + q[1];
        if (en[i] < 0) eu = eu - q[1];
        if (et[i] > 0) eu = eu + q[2];
        if (et[i] < 0) eu = eu - q[2];
        const V usq = vfma(q[1], q[1], q[2] * q[2]);
        const V rho = one + q[0];
        // f_i - w_i = w_i (drho + rho (3 eu + 4.5 eu^2 - 1.5 u^2))
        df[i] = w * vfma(rho, vfma(eu, vfma(c45, eu, three), T::bc(0.0) - c15 * usq), q[0]);
        // rho T - Tbar = tau + drho T at the node; g_i - w_i Tbar
        const V e_node = vfma(q[0], Tbar + q[3], q[3]);
        dg[i] = w * vfma(three * eu, Tbar + e_node, e_node);
        drs = drs + df[i];
        if (en[i] > 0) mn = mn + df[i];
        if (en[i] < 0) mn = mn - df[i];
        if (et[i] > 0) mt = mt + df[i];
        if (et[i] < 0) mt = mt - df[i];
        es = es + dg[i];
    }
    const V rho_s = one + drs;
    mn = mn * keep;
    mt = vfma(keep, mt, (one - keep) * (rho_s * u_wall));
    const V inv = T::rcp(rho_s);
    const V uns = mn * inv, uts = mt * inv;
    const V usq_s = vfma(uns, uns, uts * uts);
    // (c) fluxes along +n with the non-equilibrium parts; 1/2 - tau_f =
    // -3 nu / h = 6 (-nu / 2h), likewise for tau_g (Eqs. 9-10)
    const V six = T::bc(6.0);
    const V cf = six * fl.m_nu_2h, cg = six * fl.m_chi_2h;
    V Fnn = T::bc(0.0), Fnt = T::bc(0.0), Q = T::bc(0.0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if (en[i] == 0) continue;  // no flux along n
        const V w = i < 5 ? w1 : w2;
        V eu = en[i] > 0 ? uns : T::bc(0.0) - uns;
        if (et[i] > 0) eu = eu + uts;
        if (et[i] < 0) eu = eu - uts;
        const V dfs = w * vfma(rho_s, vfma(eu, vfma(c45, eu, three), T::bc(0.0) - c15 * usq_s), drs);
        const V dgs = w * vfma(three * eu, Tbar + es, es);
        const V pf = vfma(cf, dfs - df[i], dfs);  // f* + (1/2 - tau_f)(f* - f_node)
        const V pg = vfma(cg, dgs - dg[i], dgs);
        Fnn = Fnn + pf;  // e_n^2 = 1
        if (et[i] != 0) Fnt = (en[i] * et[i] > 0) ? Fnt + pf : Fnt - pf;
        Q = en[i] > 0 ? Q + pg : Q - pg;
    }
    F[0] = mn;
    F[1] = Fnn;
    F[2] = Fnt;
    F[3] = Q;
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
    using V2 = d2;
    static __host__ __device__ __forceinline__ R val(S s, int) { return s; }
    static __host__ __device__ __forceinline__ R diff(S a, S b, int) { return a - b; }
    static __host__ __device__ __forceinline__ S add(S s, R d, int) { return s + d; }
    static __host__ __device__ __forceinline__ S from_double(double v, int) { return v; }
    static __host__ __device__ __forceinline__ double to_double(S s, int) { return s; }
    static __host__ __device__ __forceinline__ S mirror_odd(S wall2, S s) { return wall2 - s; }
    static __host__ __device__ __forceinline__ bool representable(double, int) { return true; }
    static __host__ __device__ __forceinline__ bool in_range(R v, int) { return v == v; }
    static __device__ __forceinline__ R rcp(R x) { return 1.0 / x; }
    static __device__ __forceinline__ R fsqrt(R x) { return sqrt(x); }
    // constants of a cavity in R, and the wall mirror constants in S
    static __device__ __forceinline__ R dt(const CavityDesc* d) { return d->dt; }
    static __device__ __forceinline__ R beta_g(const CavityDesc* d) { return d->beta_g; }
    static __device__ __forceinline__ R T_ref(const CavityDesc* d) { return d->T_ref; }
    static __device__ __forceinline__ R fx(const CavityDesc* d) { return d->fx; }
    static __device__ __forceinline__ R fy(const CavityDesc* d) { return d->fy; }
    static __device__ __forceinline__ R bcU(const CavityDesc* d, int s) { return d->bcU[s]; }
    static __device__ __forceinline__ R Tw(const CavityDesc* d, int s) { return d->bcT[s]; }
    // cell records of buffer b
    static __device__ __forceinline__ Vec4<S> load4(const CavityDesc* d, int b, size_t o)
    {
        return static_cast<const Vec4<S>*>(d->f[b][0])[o];
    }
    static __device__ __forceinline__ void store4(const CavityDesc* d, int b, size_t o, Vec4<S> v)
    {
        static_cast<Vec4<S>*>(d->f[b][0])[o] = v;
    }
};

struct StoreQ {
    using S = int;
    using R = float;
    using V2 = f2;
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
    static __host__ __device__ __forceinline__ bool in_range(R v, int k)
    {
        return fabsf(v) < limit(k);
    }
    // reciprocal and square root at FP32 accuracy (a few ulp), not IEEE rounding
    static __device__ __forceinline__ R rcp(R x) { return __fdividef(1.0f, x); }
    static __device__ __forceinline__ R fsqrt(R x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
    static __device__ __forceinline__ R dt(const CavityDesc* d) { return d->f_dt; }
    static __device__ __forceinline__ R beta_g(const CavityDesc* d) { return d->f_beta_g; }
    static __device__ __forceinline__ R T_ref(const CavityDesc* d) { return d->f_T_ref; }
    static __device__ __forceinline__ R fx(const CavityDesc* d) { return d->f_fx; }
    static __device__ __forceinline__ R fy(const CavityDesc* d) { return d->f_fy; }
    static __device__ __forceinline__ R bcU(const CavityDesc* d, int s) { return d->f_bcU[s]; }
    static __device__ __forceinline__ R Tw(const CavityDesc* d, int s) { return d->f_bcT[s]; }
    static __device__ __forceinline__ Vec4<S> load4(const CavityDesc* d, int b, size_t o)
    {
        return static_cast<const Vec4<S>*>(d->f[b][0])[o];
    }
    static __device__ __forceinline__ void store4(const CavityDesc* d, int b, size_t o, Vec4<S> v)
    {
        static_cast<Vec4<S>*>(d->f[b][0])[o] = v;
    }
};

}  // namespace rtlbfs
