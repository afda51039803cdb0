/*
 * rtlbfs_curv.h -- C ABI of 2D RTLBFS on structured curvilinear (body-fitted)
 * quadrilateral meshes for GB300 (sm_103a): arXiv 2202.13449, Section 3.2 with
 * the unit lattice of each face in its local frame (Fig. 2), as used on the
 * O-type meshes of Section 4.3 (mixed convection from a heated cylinder).
 *
 * One time step is, per face: face values by Eq. 56 (Euclidean centre-to-face
 * distances), Green-Gauss gradients by Eq. 55 over the four face vectors of a
 * cell, the 9-node lattice x_S + (a n + b t) h in the face's frame (unit
 * normal n from the low-index to the high-index cell, t = (-n_y, n_x)) with
 * node values by Eq. 29, the predicted variables of Eqs. 46-48 and the fluxes
 * of Eqs. 57-59 in that frame, rotated back to x, y; per cell: the update
 * with the face lengths and the cell area, the Boussinesq source along the
 * gravity direction (Eq. 64) and the steady residual.
 *
 * Conventions (the status codes, RTLBFS_FP64 / RTLBFS_FP32 and the wall
 * kinds of rtlbfs.h apply):
 *   - Every call returns an int status and never aborts or traps;
 *     rtlbfsc_last_error() explains the last failure on a handle.
 *   - The mesh is (ni, nj) cells with vertices X, Y of (nj+1) x (ni+1)
 *     doubles (row j, column i at j*(ni+1) + i), right-handed: i and j
 *     increase like x and y (every cell area positive).  Cell centres are
 *     the vertex averages, areas the shoelace formula.
 *   - Fields are nj x ni arrays of doubles (cell (i, j) at j*ni + i).
 *   - Sides: 0 i = 0, 1 i = ni, 2 j = 0, 3 j = nj.  The i direction may be
 *     periodic: the seam of an O-mesh (vertex column ni equal to column 0)
 *     or a translation by X[j][ni] - X[j][0].
 *   - The library owns all device memory of a handle; host arrays are used
 *     during the call only.  One host thread per handle at a time.
 */
#ifndef RTLBFS_CURV_H
#define RTLBFS_CURV_H

#include "rtlbfs.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RTLBFSC_FARFIELD 3 /* side held at the free-stream state (zero gradient) */

typedef struct rtlbfsc_ctx* rtlbfsc_t;

/*
 * New solver on the mesh of vertices X, Y ((nj+1) x (ni+1), copied).
 * periodic_i != 0 makes sides 0 and 1 one periodic seam.  precision:
 * RTLBFS_FP64 or RTLBFS_FP32 (FP32 arithmetic on the 32-bit fixed-point
 * state, FP64 residual and wall sums).  Defaults: nu = chi = 0.01, no
 * buoyancy, dt = 0.1, kappa = 1, walls at rest with T = 0 on the bounded
 * sides, the state rho = 1, u = v = 0, T = 0.  ERR_ARG: n < 1, a cell
 * with a non-positive area, null pointers; ERR_OOM / ERR_CUDA otherwise.
 */
int rtlbfsc_create(int ni, int nj, const double* X, const double* Y, int periodic_i,
                   int precision, rtlbfsc_t* out);

/* Transport coefficients nu, chi, buoyancy coefficient beta_g (the product
 * beta g of Eq. 64) and the macroscopic time step dt.  ERR_ARG unless nu,
 * chi, dt > 0. */
int rtlbfsc_set_physics(rtlbfsc_t h, double nu, double chi, double beta_g, double dt);

/* Lattice spacing of every face: h = kappa * min(w_L, w_R), w = twice the
 * normal distance from a cell centre to the face.  ERR_ARG if kappa <= 0. */
int rtlbfsc_set_lattice(rtlbfsc_t h, double kappa);

/* Direction (gx, gy) of the buoyancy + rho beta_g (T - T_ref) (normalised
 * here; hot fluid moves along it) and T_ref.  ERR_ARG for a zero vector. */
int rtlbfsc_set_gravity(rtlbfsc_t h, double gx, double gy, double T_ref);

/* Body acceleration (fx, fy). */
int rtlbfsc_set_body_force(rtlbfsc_t h, double fx, double fy);

/*
 * Boundary condition of a bounded side: RTLBFS_WALL_DIRICHLET (no slip at
 * wall velocity (ux, uy), T = T_wall), RTLBFS_WALL_ADIABATIC, or
 * RTLBFSC_FARFIELD (the ghost layer holds the free-stream state).  A wall
 * ghost is the mirror image of the adjacent cell across the face line: rho
 * even, velocity odd about the wall velocity, T odd about T_wall or even;
 * gradients reflected in the face normal.  ERR_ARG on a periodic side or a
 * bad kind.
 */
int rtlbfsc_set_bc(rtlbfsc_t h, int side, int kind, double T_wall, double ux, double uy);

/* Free-stream state of the far-field sides. */
int rtlbfsc_set_farfield(rtlbfsc_t h, double rho, double u, double v, double T);

/* State upload / download (four nj*ni arrays).  Upload resets the step
 * counter; FP32 rejects values outside the fixed-point ranges (ERR_ARG). */
int rtlbfsc_set_state(rtlbfsc_t h, const double* rho, const double* u, const double* v,
                      const double* T);
int rtlbfsc_get_state(rtlbfsc_t h, double* rho, double* u, double* v, double* T);

/* nsteps explicit steps (one launch each, replayed from CUDA graphs);
 * ERR_DIVERGED on a non-finite residual or an FP32 range overflow. */
int rtlbfsc_step(rtlbfsc_t h, long nsteps);

/* Step until max(R_u, R_T) < tol, max_steps or timeout_s (<= 0: none);
 * returns OK, ERR_NOT_CONVERGED, ERR_TIMEOUT or ERR_DIVERGED. */
int rtlbfsc_run_to_steady(rtlbfsc_t h, double tol, long max_steps, double timeout_s,
                          long* steps_taken, double* res2);

/* (R_u, R_T) of the last step and the steps since the last upload. */
int rtlbfsc_residual(rtlbfsc_t h, double* res2, long* steps);

/*
 * Heat through side 2 (j = 0) or 3 (j = nj), in FP64: the energy flux of
 * Eq. 59 times the face lengths summed over the side's faces, along
 * increasing j; *perimeter (may be null) receives the side's length.  For
 * the cylinder of Section 4.3 (side 2), Eq. 73's mean Nusselt number is
 * *heat * D / (chi (T_h - T_l) *perimeter).  ERR_ARG for other sides.
 */
int rtlbfsc_wall_heat(rtlbfsc_t h, int side, double* heat, double* perimeter);

/* Rows of cells per work unit (tile height 8 or 16; 0: automatic, which is
 * 8). */
int rtlbfsc_set_schedule(rtlbfsc_t h, int tile_rows);

int rtlbfsc_set_stream(rtlbfsc_t h, void* stream);
int rtlbfsc_sync(rtlbfsc_t h);
const char* rtlbfsc_last_error(rtlbfsc_t h);

/* Operation count of a curvilinear cell-update (two faces with their frame
 * rotations plus the cell's own work, each face and gradient once): FP ops
 * per face, per cell-update, SFU ops per cell-update.  Host only. */
int rtlbfsc_op_counts(double* face_ops, double* cell_ops, double* sfu_ops);

void rtlbfsc_destroy(rtlbfsc_t h);

#ifdef __cplusplus
}
#endif

#endif /* RTLBFS_CURV_H */
