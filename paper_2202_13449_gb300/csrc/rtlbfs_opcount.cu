// rtlbfs_opcount.cu -- arithmetic of one cell-update of the step, counted
// on the host by running the face arithmetic of the kernels (face_flux,
// the same template the GPU executes) on an operation-counting value type.
//
// This is the work measure of the ALU roofline: the floating-point
// operations the step needs per cell-update with every face and gradient
// evaluated once (no halo recomputation, no address or control arithmetic).
// An add, a multiply and a fused multiply-add each count as one operation
// (one lane-slot of the FP32 pipe); a subtraction from the constant 0 is a
// negated operand in hardware and is not counted.  Reciprocals and square
// roots run on the special-function unit and are counted apart.
#include <cstring>

#include "rtlbfs.h"
#include "rtlbfs_dev.cuh"

namespace rtlbfs {
namespace {

struct Tally {
    long long ops = 0;  // add, multiply, fused multiply-add
    long long sfu = 0;  // reciprocal, reciprocal square root
};
Tally g_tally;

// counted value; `zero` marks the literal 0 (a negation is free)
struct Cnt {
    double v;
    bool zero;
};

Cnt operator+(Cnt a, Cnt b)
{
    if (!a.zero && !b.zero) ++g_tally.ops;  // adding the literal 0 is no operation
    return {a.v + b.v, a.zero && b.zero};
}
Cnt operator-(Cnt a, Cnt b)
{
    if (!a.zero && !b.zero) ++g_tally.ops;
    return {a.v - b.v, a.zero && b.zero};
}
Cnt operator*(Cnt a, Cnt b)
{
    ++g_tally.ops;
    return {a.v * b.v, false};
}
Cnt vfma(Cnt a, Cnt b, Cnt c)
{
    ++g_tally.ops;
    return {a.v * b.v + c.v, false};
}

}  // namespace

template <>
struct vtraits<Cnt> {
    static Cnt bc(double c) { return {c, c == 0.0}; }
    static Cnt rcp(Cnt x)
    {
        ++g_tally.sfu;
        return {1.0 / x.v, false};
    }
};

namespace {

// One face of generic values: every operation of the face templates is
// data-independent (no branches on values), so any inputs give the count.
Tally count_face(int scheme)
{
    g_tally = Tally();
    CellNT<Cnt> L, R;
    for (int k = 0; k < 4; ++k) {
        L.q[k] = {0.01 * (k + 1), false};
        L.gn[k] = {0.002 * (k + 1), false};
        L.gt[k] = {0.003 * (k + 1), false};
        R.q[k] = {0.02 * (k + 1), false};
        R.gn[k] = {0.001 * (k + 1), false};
        R.gt[k] = {0.004 * (k + 1), false};
    }
    FaceLine<Cnt> fl;
    fl.h = {0.3, false};
    fl.cL = {-0.2, false};
    fl.cR = {0.25, false};
    fl.m_nu_2h = {-0.01, false};
    fl.m_chi_2h = {-0.01, false};
    fl.m_tf15 = {-0.1, false};
    fl.m_tg15 = {-0.1, false};
    fl.pad = {0.0, true};
    Cnt F[4];
    if (scheme == 1)
        face_flux_tlbfs<Cnt>(L, R, Cnt{0.5, false}, fl, Cnt{1.0, false}, Cnt{0.0, false}, F);
    else
        face_flux<Cnt>(L, R, Cnt{0.5, false}, fl, Cnt{1.0, false}, Cnt{0.0, false}, F);
    return g_tally;
}

}  // namespace
}  // namespace rtlbfs

extern "C" int rtlbfs_op_counts_scheme(int scheme, double* face_ops, double* cell_ops,
                                       double* sfu_ops)
{
    if (scheme != 0 && scheme != 1) return RTLBFS_ERR_ARG;
    const rtlbfs::Tally f = rtlbfs::count_face(scheme);
    // Per cell, besides its two faces (the west and south faces it owns):
    //   working values from the stored state         4  (scale of each field)
    //   face frames: Tbar and the right cell's T      4  (2 per face)
    //   Green-Gauss gradients, Eq. 55, 2 x 4 fields  32  (2 differences, a
    //                                                     product, an FMA each)
    //   flux divergence, 4 fields                    16
    //   rho, T, buoyancy and body force (Eq. 64)      6
    //   rho^{n+1}, increments of u, v, T, new values 13
    //   fixed-point increments                        4
    //   residual terms of |u| and T (FP32 part)      16
    //   -------------------------------------------------
    //                                                95  (+ 4 SFU: the
    //   reciprocal of rho^{n+1}, two square roots, one reciprocal; range
    //   checks are comparisons and not counted)
    const double other = 95.0, other_sfu = 4.0;
    if (face_ops) *face_ops = (double)f.ops;
    if (cell_ops) *cell_ops = 2.0 * (double)f.ops + other;
    if (sfu_ops) *sfu_ops = 2.0 * (double)f.sfu + other_sfu;
    return RTLBFS_OK;
}

extern "C" int rtlbfs_op_counts(double* face_ops, double* cell_ops, double* sfu_ops)
{
    return rtlbfs_op_counts_scheme(0, face_ops, cell_ops, sfu_ops);
}
