/*
 * rtlbfs3d.h -- C ABI of the 3D RTLBFS solver (arXiv 2202.13449, Section 3.2
 * with the D3Q19 lattice of Eqs. 5-6; the 3D cases of Section 4.4) on a
 * structured rectilinear (hexahedral, possibly stretched) mesh, for GB300
 * (sm_103a).
 *
 * One time step is, per face: face values by inverse-distance weighting
 * (Eq. 56), cell gradients by the discrete Gauss theorem over the six faces
 * of a cell (Eq. 55), the 19-node D3Q19 lattice at the face with node values
 * by Eq. 29, the predicted variables of Eqs. 46-48 (second-order central
 * differences on those 19 nodes), and the corrector fluxes of Eqs. 57-59
 * with their (tau - 1.5)(X* - X^n) dissipation terms; per cell: the explicit
 * update with the Boussinesq buoyancy of Eq. 64 along the gravity axis and
 * the steady residual (the L2 analogue of Eq. 65).
 *
 * Conventions (as in rtlbfs.h, whose status codes and precision constants
 * RTLBFS_OK, RTLBFS_ERR_*, RTLBFS_FP64, RTLBFS_FP32 and boundary kinds
 * RTLBFS_WALL_DIRICHLET, RTLBFS_WALL_ADIABATIC, RTLBFS_PERIODIC apply):
 *   - Every call returns an int status and never aborts or traps;
 *     rtlbfs3d_last_error() explains the last failure on a handle.
 *   - Host arrays are read or written during the call only; the library
 *     owns all device memory of a handle and frees it in rtlbfs3d_destroy.
 *   - Fields are nz x ny x nx arrays of doubles, x fastest: cell (i, j, k)
 *     at (k*ny + j)*nx + i.
 *   - Sides: 0 = -x, 1 = +x, 2 = -y, 3 = +y, 4 = -z, 5 = +z.
 *   - Lattice units: c = 1, c_s^2 = 1/3, c_p = 1; reference length L = the
 *     domain length in x.
 *   - A handle is not thread-safe: one host thread at a time.
 */
#ifndef RTLBFS3D_H
#define RTLBFS3D_H

#include "rtlbfs.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RTLBFS3D_XM 0
#define RTLBFS3D_XP 1
#define RTLBFS3D_YM 2
#define RTLBFS3D_YP 3
#define RTLBFS3D_ZM 4
#define RTLBFS3D_ZP 5
#define RTLBFS3D_MID_X 6 /* rtlbfs3d_nusselt: the x-normal face plane at i = nx/2 */

typedef struct rtlbfs3d_ctx* rtlbfs3d_t;

/*
 * New solver on the mesh with face coordinates xf[0..nx], yf[0..ny],
 * zf[0..nz] (strictly ascending; copied).  precision: RTLBFS_FP64, or
 * RTLBFS_FP32 (FP32 arithmetic on a 32-bit fixed-point state, FP64 residual
 * and Nusselt sums).  Defaults: the cubic cavity of Section 4.4 -- cold
 * wall T = 0 at -x, hot wall T = 1 at +x, the other four walls adiabatic,
 * all no-slip, gravity along -z (buoyancy along +z), Ra = 1e3, Pr = 0.71,
 * Ma = 0.1, Delta t = half the smallest cell width, kappa = 1, and the
 * conduction state rho = 1, u = v = w = 0, T linear in x.  *out receives
 * the handle.  ERR_ARG: n < 1 on an axis, a cell count above 2^31, faces
 * not ascending, null pointers; ERR_OOM / ERR_CUDA on device failure.
 */
int rtlbfs3d_create(int nx, int ny, int nz, const double* xf, const double* yf,
                    const double* zf, int precision, rtlbfs3d_t* out);

/*
 * Physical parameters through Eq. 63 with V_c = Ma (c = 1) and L = the
 * domain length in x: nu = V_c L sqrt(Pr/Ra), chi = nu/Pr, beta_g =
 * V_c^2/(dT L).  dt is the macroscopic time step Delta t; dt = 0 picks
 * min(w_min/2, 0.13 w_min^2/max(nu, chi)) (half the smallest cell width,
 * the paper's setting on unit cells, capped by an explicit diffusive limit).
 * ERR_ARG if Ra, Pr, Ma <= 0 or dt < 0.
 */
int rtlbfs3d_set_params(rtlbfs3d_t h, double Ra, double Pr, double Ma, double dt);

/* Transport and buoyancy coefficients directly (overrides set_params'
 * mapping; dt is kept).  ERR_ARG if nu or chi <= 0. */
int rtlbfs3d_set_physics(rtlbfs3d_t h, double nu, double chi, double beta_g);

/* Lattice spacing of every face: delta t_f = kappa * min(width_L, width_R)
 * normal to the face (Eqs. 9-10 then give tau_f, tau_g per face).
 * ERR_ARG if kappa <= 0. */
int rtlbfs3d_set_lattice(rtlbfs3d_t h, double kappa);

/* Axis (0 x, 1 y, 2 z) along which the buoyancy + rho beta_g (T - T_ref)
 * acts (hot fluid moves to +axis); T_ref = 0.5.  ERR_ARG otherwise. */
int rtlbfs3d_set_gravity_axis(rtlbfs3d_t h, int axis);

/* Body acceleration (fx, fy, fz) added to the momentum source. */
int rtlbfs3d_set_body_force(rtlbfs3d_t h, double fx, double fy, double fz);

/*
 * Boundary condition of one side: kind RTLBFS_WALL_DIRICHLET (no slip,
 * T = T_wall), RTLBFS_WALL_ADIABATIC (no slip, no heat flux) or
 * RTLBFS_PERIODIC (must be set on both sides of an axis before stepping).
 * u_wall[3] is the wall velocity (null: at rest); its component normal to
 * the wall is ignored.  Ghost cells mirror the adjacent cell (rho even,
 * velocity odd about the wall velocity, T odd about T_wall or even).
 * ERR_ARG on a bad side or kind.
 */
int rtlbfs3d_set_bc(rtlbfs3d_t h, int side, int kind, double T_wall, const double* u_wall);

/* Upload the state (five host arrays, nz*ny*nx doubles each); resets the
 * step counter.  FP32: values outside the fixed-point ranges (|rho-1| <
 * 0.49, |u|, |v|, |w| < 0.99, |T| < 1.98) or not finite give ERR_ARG. */
int rtlbfs3d_set_state(rtlbfs3d_t h, const double* rho, const double* u, const double* v,
                       const double* w, const double* T);

/* Download the state into five caller-owned arrays (synchronises). */
int rtlbfs3d_get_state(rtlbfs3d_t h, double* rho, double* u, double* v, double* w, double* T);

/* Advance nsteps explicit steps (one kernel launch each, replayed from CUDA
 * graphs).  Synchronises.  ERR_DIVERGED if a residual became non-finite or
 * an FP32 value left its range (the state is then the last one computed). */
int rtlbfs3d_step(rtlbfs3d_t h, long nsteps);

/*
 * Step until max(R_u, R_T) < tol (checked on the device after every step),
 * max_steps or timeout_s seconds of wall time (<= 0: none).  steps_taken and
 * res2 (R_u, R_T of the last step) may be null.  Returns OK,
 * ERR_NOT_CONVERGED, ERR_TIMEOUT or ERR_DIVERGED.
 */
int rtlbfs3d_run_to_steady(rtlbfs3d_t h, double tol, long max_steps, double timeout_s,
                           long* steps_taken, double* res2);

/* Residual (R_u, R_T) of the last step and steps since the last upload. */
int rtlbfs3d_residual(rtlbfs3d_t h, double* res2, long* steps);

/*
 * Nusselt numbers in FP64 from the current state: the energy flux of Eq. 59
 * through the faces of wall `side` (0..5), summed with the face areas,
 * times the domain length normal to the wall, / (chi dT wall area) -- Eq. 76
 * with the conductive flux the scheme puts through the wall; mid = 1: the
 * same flux along the wall's middle line of its first tangential axis
 * (y for x-walls, z for y-walls, x for z-walls), integrated along the
 * second -- Eq. 75 (an even cell count averages the two face rows beside
 * the middle).  side = RTLBFS3D_MID_X (mid = 0, nx even): the face plane
 * x = x_f[nx/2].  Signed along +axis.  Synchronises.  ERR_ARG on a bad
 * selector or a periodic side.
 */
int rtlbfs3d_nusselt(rtlbfs3d_t h, int side, int mid, double* nu);

/*
 * Face stage of every face: 0 = RTLBFS (Section 3.2, the default), 1 = the
 * original TLBFS of Section 2.2 with D3Q19 -- equilibria (Eqs. 3-4) at the
 * nodes x_S - e_i delta t (Eq. 29 values), the predicted variables as their
 * moments (Eqs. 30-32) and the fluxes of Eqs. 38-40 with the
 * non-equilibrium parts of Eqs. 33-34.  The update, boundary conditions,
 * residual and Nusselt sums use the chosen stage.  ERR_ARG otherwise.
 */
int rtlbfs3d_set_scheme(rtlbfs3d_t h, int scheme);

/*
 * Work decomposition of the step kernel: tile 0 = 32 x 4 cells, 1 = 16 x 8,
 * 2 = 32 x 8 in x-y (one thread per column, marching up z); kchunk = planes
 * per work unit (0 = automatic: enough units to fill every SM; on meshes
 * whose tile columns fit a wave of resident blocks twice, the shortest chunk
 * of at least 4 planes whose units fit one wave).
 * ERR_ARG otherwise.
 */
int rtlbfs3d_set_schedule(rtlbfs3d_t h, int tile, int kchunk);

/* Time every tile shape for `steps` steps on a snapshot of the state
 * (restored bit for bit afterwards), keep the fastest; *tile and
 * *ms_per_step may be null. */
int rtlbfs3d_autotune(rtlbfs3d_t h, int steps, int* tile, double* ms_per_step);

/* Run on the given cudaStream_t (null: the library's own stream). */
int rtlbfs3d_set_stream(rtlbfs3d_t h, void* stream);
int rtlbfs3d_sync(rtlbfs3d_t h);
const char* rtlbfs3d_last_error(rtlbfs3d_t h);

/*
 * Operation count of one 3D cell-update with every face and gradient taken
 * once (the ALU roofline's work measure): FP additions, multiplications
 * and fused multiply-adds of one face (*face_ops) and of a cell-update
 * (three faces plus the cell's own work, *cell_ops); reciprocals and
 * square roots apart (*sfu_ops).  Host only; pointers may be null.
 */
int rtlbfs3d_op_counts(double* face_ops, double* cell_ops, double* sfu_ops);

/* The same count for face stage `scheme` (0 RTLBFS, 1 TLBFS); ERR_ARG
 * for any other scheme. */
int rtlbfs3d_op_counts_scheme(int scheme, double* face_ops, double* cell_ops, double* sfu_ops);

void rtlbfs3d_destroy(rtlbfs3d_t h);

#ifdef __cplusplus
}
#endif

#endif /* RTLBFS3D_H */
