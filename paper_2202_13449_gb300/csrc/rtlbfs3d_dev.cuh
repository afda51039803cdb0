// rtlbfs3d_dev.cuh -- the per-face arithmetic of 3D RTLBFS (arXiv
// 2202.13449, Section 3.2 with the D3Q19 lattice of Eqs. 5-6), templated on
// the value type V (float, double, or a host counting type).
//
// A face is handled in its own frame: normal n (index 0) and two tangents
// t1, t2 (indices 1, 2).  Cell quantities enter as (drho, u_n, u_t1, u_t2,
// tau) with drho = rho - 1 and tau = T - Tbar, Tbar a face reference
// temperature, so FP32 never differences the O(1) parts of rho and rho T;
// the constant c_s^2 of the normal momentum flux is dropped (it cancels in
// the flux divergence of a closed cell).
#pragma once

#include "rtlbfs_dev.cuh"

namespace rtlbfs3 {

using rtlbfs::FaceLine;
using rtlbfs::vfma;
using rtlbfs::vtraits;

// One cell seen from a face: values and gradients along n, t1, t2.
template <typename V>
struct CellNT3 {
    V q[5];
    V gn[5];
    V g1[5];
    V g2[5];
};

// Eq. 29, Eqs. 46-48 and the braces of Eqs. 57-59 for one face.
//
// Nodes.  Node (a, b, c) of the D3Q19 lattice sits at x_S + (a n + b t1 +
// c t2) h.  A cell's reconstruction plane restricted to a column a = const
// is linear in (b, c), so each primitive on column a is C + b S1 + c S2:
// a = -1 the left plane, a = +1 the right plane, a = 0 their mean (Eq. 29).
// The 19 nodes are the centre, the axis nodes +-e_a and the edge nodes
// +-e_a +-e_b (a < b).  With products formed at the nodes, the lattice
// differences
//   d_a f  = f(+e_a) - f(-e_a)                   = 2 h D_a f
//   dd_a f = f(+e_a) - 2 f(0) + f(-e_a)          = h^2 D_aa f
//   dd_ab f = f(+a+b) - f(+a-b) - f(-a+b) + f(-a-b) = 4 h^2 D_ab f
// turn Eqs. 46-48 into (the powers of h cancel)
//   drho* = drho - 1/2 sum_a d_a m_a + 1/2 sum_a dd_a (m_a u_a + cs2 drho)
//           + 1/4 sum_{a<b} dd_ab (m_a u_b)
//   m_a*  = m_a - 1/2 sum_b d_b X_ab
//           + cs2/2 [sum_b dd_b m_a + 2 dd_a m_a + 1/2 sum_{b!=a} dd_ab m_b]
//   e*    = e - 1/2 sum_a (Tbar d_a m_a + d_a (m_a tau)) + cs2/2 sum_a dd_a e
// with m_a = rho u_a, X_ab = m_a u_b + cs2 drho delta_ab, e = rho T - Tbar.
// keep = 1 on an interior face, 0 on a wall face whose tangential velocity
// is (uw1, uw2): no mass through the wall, (rho u_t)* = rho* u_wall,t.
// F = (mass, n-, t1-, t2-momentum, energy) flux along +n.
//
// The first stage, face3_nodes, forms the 19 node values of the five
// primitives; face_flux3_nodes does the rest.
template <typename V>
__host__ __device__ __forceinline__ void face3_nodes(const CellNT3<V>& L, const CellNT3<V>& Rc,
                                                    const FaceLine<V>& fl, V O[5], V P[3][2][5],
                                                    V E[3][4][5])
{
    using T = vtraits<V>;
    const V half = T::bc(0.5);
    const V h = fl.h;
    const V wL = fl.cL + h, mwR = fl.cR - h;  // wL, -wR: centre-to-face distances
    const V hh = h * half;

    // column coefficients: A (a = -1), M (a = 0), B (a = +1)
    V Ac[5], A1[5], A2[5], Mc[5], M1[5], M2[5], Bc[5], B1[5], B2[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        Ac[k] = vfma(L.gn[k], fl.cL, L.q[k]);
        A1[k] = L.g1[k] * h;
        A2[k] = L.g2[k] * h;
        Bc[k] = vfma(Rc.gn[k], fl.cR, Rc.q[k]);
        B1[k] = Rc.g1[k] * h;
        B2[k] = Rc.g2[k] * h;
        Mc[k] = half * (vfma(L.gn[k], wL, L.q[k]) + vfma(Rc.gn[k], mwR, Rc.q[k]));
        M1[k] = hh * (L.g1[k] + Rc.g1[k]);
        M2[k] = hh * (L.g2[k] + Rc.g2[k]);
    }

    // node values: centre O, axis nodes P[a][s] (s = 0: -e_a, 1: +e_a), edge
    // nodes E[p][c] for the pairs p = (n,t1), (n,t2), (t1,t2) and the
    // corners c = (+,+), (+,-), (-,+), (-,-)
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        O[k] = Mc[k];
        P[0][0][k] = Ac[k];
        P[0][1][k] = Bc[k];
        P[1][0][k] = Mc[k] - M1[k];
        P[1][1][k] = Mc[k] + M1[k];
        P[2][0][k] = Mc[k] - M2[k];
        P[2][1][k] = Mc[k] + M2[k];
        E[0][0][k] = Bc[k] + B1[k];
        E[0][1][k] = Bc[k] - B1[k];
        E[0][2][k] = Ac[k] + A1[k];
        E[0][3][k] = Ac[k] - A1[k];
        E[1][0][k] = Bc[k] + B2[k];
        E[1][1][k] = Bc[k] - B2[k];
        E[1][2][k] = Ac[k] + A2[k];
        E[1][3][k] = Ac[k] - A2[k];
        const V pp = Mc[k] + M1[k], mm = Mc[k] - M1[k];
        E[2][0][k] = pp + M2[k];
        E[2][1][k] = pp - M2[k];
        E[2][2][k] = mm + M2[k];
        E[2][3][k] = mm - M2[k];
    }
}

template <typename V>
__host__ __device__ __forceinline__ void face_flux3_nodes(const V O[5], const V P[3][2][5],
                                                         const V E[3][4][5], V Tbar,
                                                         const FaceLine<V>& fl, V keep, V uw1,
                                                         V uw2, V F[5])
{
    using T = vtraits<V>;
    const V zero = T::bc(0.0), half = T::bc(0.5), quarter = T::bc(0.25), one = T::bc(1.0);
    const V two = T::bc(2.0), m2 = T::bc(-2.0), mhalf = T::bc(-0.5);
    const V cs2 = T::bc(1.0 / 3.0), hcs2 = T::bc(0.5 / 3.0);
    constexpr int PA[3] = {0, 0, 1}, PB[3] = {1, 2, 2};  // axes of the edge pairs

    // momenta m_a = u_a + drho u_a at the centre and the axis nodes
    V mO[3], mP[3][2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) mO[a] = vfma(O[0], O[1 + a], O[1 + a]);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a)
                mP[ax][s][a] = vfma(P[ax][s][0], P[ax][s][1 + a], P[ax][s][1 + a]);

    // differences of the momenta: d_b m_a and dd_b m_a
    V dm[3][3], ddm[3][3];  // [b][a]
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dm[b][a] = mP[b][1][a] - mP[b][0][a];
            ddm[b][a] = vfma(m2, mO[a], mP[b][1][a] + mP[b][0][a]);
        }
    const V divm = dm[0][0] + dm[1][1] + dm[2][2];  // sum_a d_a m_a

    // X_ab at the axis nodes of b (for d_b X_ab) and X_aa + cs2 drho
    V dX[3][3];  // [a][b] = d_b X_ab
    V ddXd[3];   // dd_a (m_a u_a + cs2 drho)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        V Xp[2][3];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const V x = mP[b][s][a] * P[b][s][1 + b];
                Xp[s][a] = a == b ? vfma(cs2, P[b][s][0], x) : x;
            }
#pragma unroll
        for (int a = 0; a < 3; ++a) dX[a][b] = Xp[1][a] - Xp[0][a];
        const V XO = vfma(mO[b], O[1 + b], cs2 * O[0]);
        ddXd[b] = vfma(m2, XO, Xp[1][b] + Xp[0][b]);
    }

    // edge nodes: dd_ab of m_a u_b, m_a and m_b
    V ddX[3], ddma[3], ddmb[3];  // per pair
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int a = PA[p], b = PB[p];
        V ma[4], mb[4], x[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            ma[c] = vfma(E[p][c][0], E[p][c][1 + a], E[p][c][1 + a]);
            mb[c] = vfma(E[p][c][0], E[p][c][1 + b], E[p][c][1 + b]);
            x[c] = ma[c] * E[p][c][1 + b];
        }
        ddX[p] = (x[0] - x[1]) - (x[2] - x[3]);
        ddma[p] = (ma[0] - ma[1]) - (ma[2] - ma[3]);
        ddmb[p] = (mb[0] - mb[1]) - (mb[2] - mb[3]);
    }
    // dd_ab m_b and dd_ab m_a looked up by (axis a, other axis b)
    auto ddcross = [&](int a, int b) -> V {  // dd_ab (m_b)
        const int p = (a + b == 1) ? 0 : ((a + b == 2) ? 1 : 2);
        return (b == PB[p]) ? ddmb[p] : ddma[p];
    };

    // energies e = tau + drho (Tbar + tau) and m_a tau at the axis nodes
    const V eO = vfma(O[0], Tbar + O[4], O[4]);
    V de[3], dde[3], dmt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const V ep = vfma(P[a][1][0], Tbar + P[a][1][4], P[a][1][4]);
        const V em = vfma(P[a][0][0], Tbar + P[a][0][4], P[a][0][4]);
        de[a] = ep - em;
        dde[a] = vfma(m2, eO, ep + em);
        dmt[a] = mP[a][1][a] * P[a][1][4] - mP[a][0][a] * P[a][0][4];
    }

    // Eq. 46: drho*
    V drs = vfma(mhalf, divm, O[0]);
    drs = vfma(half, ddXd[0] + ddXd[1] + ddXd[2], drs);
    drs = vfma(quarter, ddX[0] + ddX[1] + ddX[2], drs);
    // Eq. 47: m_a*
    V ms[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        V br = (ddm[0][a] + ddm[1][a]) + ddm[2][a];
        br = vfma(two, ddm[a][a], br);
        V cr = zero;
#pragma unroll
        for (int b = 0; b < 3; ++b)
            if (b != a) cr = cr + ddcross(a, b);
        br = vfma(half, cr, br);
        const V fo = (dX[a][0] + dX[a][1]) + dX[a][2];
        ms[a] = vfma(hcs2, br, vfma(mhalf, fo, mO[a]));
    }
    // Eq. 48: e* = (rho T)* - Tbar
    V es = vfma(mhalf, vfma(Tbar, divm, (dmt[0] + dmt[1]) + dmt[2]), eO);
    es = vfma(hcs2, (dde[0] + dde[1]) + dde[2], es);

    const V rho_s = one + drs;
    // wall faces: no mass through the wall, the wall's tangential velocity
    ms[0] = ms[0] * keep;
    const V wallr = (one - keep) * rho_s;
    ms[1] = vfma(keep, ms[1], wallr * uw1);
    ms[2] = vfma(keep, ms[2], wallr * uw2);
    const V inv = T::rcp(rho_s);
    const V un_s = ms[0] * inv;
    const V taus = (es - drs * Tbar) * inv;  // T* - Tbar

    // Eqs. 57-59 braces along +n
    F[0] = ms[0];
    {
        // a = n: X_nn = m_n u_n + cs2 drho, viscous 3 d_n m_n + d_t1 m_t1 + d_t2 m_t2
        const V X0 = vfma(mO[0], O[1], cs2 * O[0]);
        const V Xs = vfma(ms[0], un_s, cs2 * drs);
        const V visc = dm[0][0] + dm[0][0] + divm;
        F[1] = vfma(fl.m_nu_2h, visc, vfma(fl.m_tf15, Xs - X0, X0));
    }
#pragma unroll
    for (int a = 1; a < 3; ++a) {
        const V X0 = mO[a] * O[1];
        const V Xs = ms[a] * un_s;
        const V visc = dm[0][a] + dm[a][0];
        F[1 + a] = vfma(fl.m_nu_2h, visc, vfma(fl.m_tf15, Xs - X0, X0));
    }
    {
        // (rho u_n T)* - (rho u_n T)^n = Tbar (m_n* - m_n) + m_n* tau* - m_n tau
        const V Q0 = mO[0] * (Tbar + O[4]);
        const V dQ = vfma(Tbar, ms[0] - mO[0], vfma(ms[0], taus, zero - mO[0] * O[4]));
        F[4] = vfma(fl.m_chi_2h, de[0], vfma(fl.m_tg15, dQ, Q0));
    }
}

template <typename V>
__host__ __device__ __forceinline__ void face_flux3(const CellNT3<V>& L, const CellNT3<V>& Rc,
                                                   V Tbar, const FaceLine<V>& fl, V keep, V uw1,
                                                   V uw2, V F[5])
{
    V O[5], P[3][2][5], E[3][4][5];
    face3_nodes<V>(L, Rc, fl, O, P, E);
    face_flux3_nodes<V>(O, P, E, Tbar, fl, keep, uw1, uw2, F);
}

// face3_nodes in FP32, components (0, 1) and (2, 3) in packed FP32x2 pairs
// (component 4 alone): the same operations, bit for bit (a - b formed as
// fma(b, -1, a), exact like the subtraction).
__device__ __forceinline__ void face3_nodes_f32(const CellNT3<float>& L, const CellNT3<float>& Rc,
                                                const FaceLine<float>& fl, float O[5],
                                                float P[3][2][5], float E[3][4][5])
{
    const float h = fl.h;
    const float wL = fl.cL + h, mwR = fl.cR - h, hh = h * 0.5f;
    const float2 cL2 = make_float2(fl.cL, fl.cL), cR2 = make_float2(fl.cR, fl.cR);
    const float2 wL2 = make_float2(wL, wL), mwR2 = make_float2(mwR, mwR);
    const float2 h2 = make_float2(h, h), hh2 = make_float2(hh, hh);
    const float2 half2 = make_float2(0.5f, 0.5f), m1 = make_float2(-1.0f, -1.0f);
    auto pr = [](const float* a, int i) { return make_float2(a[2 * i], a[2 * i + 1]); };
    auto sub = [&](float2 a, float2 b) { return __ffma2_rn(b, m1, a); };
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float2 q = pr(L.q, i), gn = pr(L.gn, i), g1 = pr(L.g1, i), g2 = pr(L.g2, i);
        const float2 qr = pr(Rc.q, i), gnr = pr(Rc.gn, i), g1r = pr(Rc.g1, i), g2r = pr(Rc.g2, i);
        const float2 Ac = __ffma2_rn(gn, cL2, q), A1 = __fmul2_rn(g1, h2), A2 = __fmul2_rn(g2, h2);
        const float2 Bc = __ffma2_rn(gnr, cR2, qr), B1 = __fmul2_rn(g1r, h2),
                     B2 = __fmul2_rn(g2r, h2);
        const float2 Mc = __fmul2_rn(half2, __fadd2_rn(__ffma2_rn(gn, wL2, q), __ffma2_rn(gnr, mwR2, qr)));
        const float2 M1 = __fmul2_rn(hh2, __fadd2_rn(g1, g1r)), M2 = __fmul2_rn(hh2, __fadd2_rn(g2, g2r));
        const float2 pp = __fadd2_rn(Mc, M1), mm = sub(Mc, M1);
        const float2 v[19] = {Mc,
                              Ac, Bc, mm, pp, sub(Mc, M2), __fadd2_rn(Mc, M2),
                              __fadd2_rn(Bc, B1), sub(Bc, B1), __fadd2_rn(Ac, A1), sub(Ac, A1),
                              __fadd2_rn(Bc, B2), sub(Bc, B2), __fadd2_rn(Ac, A2), sub(Ac, A2),
                              __fadd2_rn(pp, M2), sub(pp, M2), __fadd2_rn(mm, M2), sub(mm, M2)};
        float* dst[19] = {&O[0],
                          &P[0][0][0], &P[0][1][0], &P[1][0][0], &P[1][1][0], &P[2][0][0], &P[2][1][0],
                          &E[0][0][0], &E[0][1][0], &E[0][2][0], &E[0][3][0],
                          &E[1][0][0], &E[1][1][0], &E[1][2][0], &E[1][3][0],
                          &E[2][0][0], &E[2][1][0], &E[2][2][0], &E[2][3][0]};
#pragma unroll
        for (int n = 0; n < 19; ++n) {
            dst[n][2 * i] = v[n].x;
            dst[n][2 * i + 1] = v[n].y;
        }
    }
    {  // component 4
        const float q = L.q[4], gn = L.gn[4], g1 = L.g1[4], g2 = L.g2[4];
        const float qr = Rc.q[4], gnr = Rc.gn[4], g1r = Rc.g1[4], g2r = Rc.g2[4];
        const float Ac = fmaf(gn, fl.cL, q), A1 = g1 * h, A2 = g2 * h;
        const float Bc = fmaf(gnr, fl.cR, qr), B1 = g1r * h, B2 = g2r * h;
        const float Mc = 0.5f * (fmaf(gn, wL, q) + fmaf(gnr, mwR, qr));
        const float M1 = hh * (g1 + g1r), M2 = hh * (g2 + g2r);
        const float pp = Mc + M1, mm = Mc - M1;
        O[4] = Mc;
        P[0][0][4] = Ac;
        P[0][1][4] = Bc;
        P[1][0][4] = mm;
        P[1][1][4] = pp;
        P[2][0][4] = Mc - M2;
        P[2][1][4] = Mc + M2;
        E[0][0][4] = Bc + B1;
        E[0][1][4] = Bc - B1;
        E[0][2][4] = Ac + A1;
        E[0][3][4] = Ac - A1;
        E[1][0][4] = Bc + B2;
        E[1][1][4] = Bc - B2;
        E[1][2][4] = Ac + A2;
        E[1][3][4] = Ac - A2;
        E[2][0][4] = pp + M2;
        E[2][1][4] = pp - M2;
        E[2][2][4] = mm + M2;
        E[2][3][4] = mm - M2;
    }
}

// The original TLBFS face stage (Section 2.2) with D3Q19, from the same
// inputs and in the same frame as face_flux3: (a) equilibria (Eqs. 3-4,
// c_p = 1) at the nodes x_S - e_i h, i.e. node -e_i of the column form
// (Eq. 29); (b) the predicted variables as their moments (Eqs. 30-32), then
// the wall rule; (c) the fluxes of Eqs. 38-40 from the equilibria of the
// predicted variables and the non-equilibrium parts of Eqs. 33-34.
// Equilibria are carried as deviations f_i - w_i and g_i - w_i Tbar; the
// constants cancel in every moment used except the pressure c_s^2 of the
// normal momentum flux, which is dropped as in face_flux3.
template <typename V>
__host__ __device__ __forceinline__ void face_flux3_tlbfs(const CellNT3<V>& L, const CellNT3<V>& Rc,
                                                         V Tbar, const FaceLine<V>& fl, V keep,
                                                         V uw1, V uw2, V F[5])
{
    using T = vtraits<V>;
    const V zero = T::bc(0.0), half = T::bc(0.5), one = T::bc(1.0), three = T::bc(3.0);
    const V c45 = T::bc(4.5), mc15 = T::bc(-1.5), six = T::bc(6.0);
    // D3Q19 (Eq. 5) in the face frame: the set is the same in every frame
    constexpr int en[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    constexpr int e1[19] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
    constexpr int e2[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
    const V w0 = T::bc(1.0 / 3.0), w1 = T::bc(1.0 / 18.0), w2 = T::bc(1.0 / 36.0);
    const V h = fl.h;
    const V wL = fl.cL + h, mwR = fl.cR - h;
    const V hh = h * half;
    // columns a = -1 (left plane), 0 (mean), +1 (right plane): value + slopes in t1, t2
    V C[3][5], S1[3][5], S2[3][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        C[0][k] = vfma(L.gn[k], fl.cL, L.q[k]);
        S1[0][k] = L.g1[k] * h;
        S2[0][k] = L.g2[k] * h;
        C[2][k] = vfma(Rc.gn[k], fl.cR, Rc.q[k]);
        S1[2][k] = Rc.g1[k] * h;
        S2[2][k] = Rc.g2[k] * h;
        C[1][k] = half * (vfma(L.gn[k], wL, L.q[k]) + vfma(Rc.gn[k], mwR, Rc.q[k]));
        S1[1][k] = hh * (L.g1[k] + Rc.g1[k]);
        S2[1][k] = hh * (L.g2[k] + Rc.g2[k]);
    }
    // (a), (b): equilibria at the nodes -e_i and their moments
    V df[19], dg[19];
    V drs = zero, mn = zero, m1 = zero, m2 = zero, es = zero;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int a = 1 - en[i], b = -e1[i], c = -e2[i];  // column, offsets along t1, t2
        V q[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            V x = C[a][k];
            if (b > 0) x = x + S1[a][k];
            if (b < 0) x = x - S1[a][k];
            if (c > 0) x = x + S2[a][k];
            if (c < 0) x = x - S2[a][k];
            q[k] = x;
        }
        const V w = i == 0 ? w0 : (i < 7 ? w1 : w2);
        V eu = zero;
        if (en[i] > 0) eu = eu + q[1];
        if (en[i] < 0) eu = eu - q[1];
        if (e1[i] > 0) eu = eu + q[2];
        if (e1[i] < 0) eu = eu - q[2];
        if (e2[i] > 0) eu = eu + q[3];
        if (e2[i] < 0) eu = eu - q[3];
        const V usq = vfma(q[1], q[1], vfma(q[2], q[2], q[3] * q[3]));
        const V rho = one + q[0];
        // f_i - w_i = w_i (drho + rho (3 eu + 4.5 eu^2 - 1.5 u^2))
        df[i] = w * vfma(rho, vfma(eu, vfma(c45, eu, three), mc15 * usq), q[0]);
        // rho T - Tbar at the node, and g_i - w_i Tbar
        const V e_node = vfma(q[0], Tbar + q[4], q[4]);
        dg[i] = w * vfma(three * eu, Tbar + e_node, e_node);
        drs = drs + df[i];
        if (en[i] > 0) mn = mn + df[i];
        if (en[i] < 0) mn = mn - df[i];
        if (e1[i] > 0) m1 = m1 + df[i];
        if (e1[i] < 0) m1 = m1 - df[i];
        if (e2[i] > 0) m2 = m2 + df[i];
        if (e2[i] < 0) m2 = m2 - df[i];
        es = es + dg[i];
    }
    const V rho_s = one + drs;
    mn = mn * keep;
    const V wallr = (one - keep) * rho_s;
    m1 = vfma(keep, m1, wallr * uw1);
    m2 = vfma(keep, m2, wallr * uw2);
    const V inv = T::rcp(rho_s);
    const V un = mn * inv, u1 = m1 * inv, u2 = m2 * inv;
    const V usq_s = vfma(un, un, vfma(u1, u1, u2 * u2));
    // (c) fluxes along +n; 1/2 - tau = -3 nu / h = 6 (-nu / 2h) (Eqs. 9-10)
    const V cf = six * fl.m_nu_2h, cg = six * fl.m_chi_2h;
    V Fnn = zero, Fn1 = zero, Fn2 = zero, Q = zero;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        if (en[i] == 0) continue;  // no flux along n
        const V w = i < 7 ? w1 : w2;
        V eu = en[i] > 0 ? un : zero - un;
        if (e1[i] > 0) eu = eu + u1;
        if (e1[i] < 0) eu = eu - u1;
        if (e2[i] > 0) eu = eu + u2;
        if (e2[i] < 0) eu = eu - u2;
        const V dfs = w * vfma(rho_s, vfma(eu, vfma(c45, eu, three), mc15 * usq_s), drs);
        const V dgs = w * vfma(three * eu, Tbar + es, es);
        const V pf = vfma(cf, dfs - df[i], dfs);  // f* + (1/2 - tau_f)(f* - f_node)
        const V pg = vfma(cg, dgs - dg[i], dgs);
        Fnn = Fnn + pf;  // e_n^2 = 1
        if (e1[i] != 0) Fn1 = (en[i] * e1[i] > 0) ? Fn1 + pf : Fn1 - pf;
        if (e2[i] != 0) Fn2 = (en[i] * e2[i] > 0) ? Fn2 + pf : Fn2 - pf;
        Q = en[i] > 0 ? Q + pg : Q - pg;
    }
    F[0] = mn;
    F[1] = Fnn;
    F[2] = Fn1;
    F[3] = Fn2;
    F[4] = Q;
}

}  // namespace rtlbfs3
