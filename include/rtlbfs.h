/*
 * rtlbfs.h -- C ABI of the GB300 (sm_103a) solver for the reconstructed
 * thermal lattice Boltzmann flux solver (RTLBFS) of arXiv 2202.13449, 2D,
 * on a structured rectilinear (tensor-product, possibly stretched) mesh.
 *
 * One time step (Section 3.2 of the paper) is, per face: face values by
 * inverse-distance weighting (Eq. 56), cell gradients by the discrete Gauss
 * theorem (Eq. 55), a 9-node unit lattice at the face with node values by
 * Eq. 29, the predicted variables of Eqs. 46-48, and the corrector fluxes
 * of Eqs. 57-59 with their (tau - 1.5)(X* - X^n) dissipation terms; per
 * cell: the explicit update of Eqs. 57-59 with the Boussinesq buoyancy of
 * Eq. 64 and the steady residual (the L2 analogue of Eq. 65).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an int status (RTLBFS_OK = 0 or a negative
 *     RTLBFS_ERR_*) and never aborts or traps.  rtlbfs_last_error() gives a
 *     human-readable reason for the last failure on a handle.
 *   - Host arrays passed in are read during the call and never retained;
 *     host arrays passed out are written during the call (the call
 *     synchronises the handle's stream before returning).  The library
 *     owns all device memory of a handle and frees it in *_destroy.
 *   - Fields are row-major ny x nx (cell (i, j) at j*nx + i, i along x).
 *   - A handle is not thread-safe: one host thread at a time.
 *   - Lattice units: c = 1, c_s^2 = 1/3, c_p = 1, reference length L = the
 *     domain width in x (for Rayleigh-Benard runs: the height, see
 *     rtlbfs_set_params_ref).
 */
#ifndef RTLBFS_H
#define RTLBFS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RTLBFS_OK 0
#define RTLBFS_ERR_ARG (-1)           /* bad argument (size, range, null) */
#define RTLBFS_ERR_OOM (-2)           /* device or host allocation failed */
#define RTLBFS_ERR_CUDA (-3)          /* a CUDA call failed */
#define RTLBFS_ERR_DIVERGED (-4)      /* the residual became non-finite */
#define RTLBFS_ERR_NOT_CONVERGED (-5) /* max_steps reached before tol */
#define RTLBFS_ERR_TIMEOUT (-6)       /* wall-clock limit reached */
#define RTLBFS_ERR_STATE (-7)         /* call not valid in this state */

/* arithmetic of the bulk step */
#define RTLBFS_FP64 0 /* every stage in FP64 */
#define RTLBFS_FP32 1 /* FP32 bulk on a 32-bit fixed-point state, FP64 residual/Nusselt sums */

/*
 * The FP32 mode's state.  Each cell is stored as four 32-bit fixed-point
 * numbers: rho - 1 in units of 2^-32, u and v in units of 2^-31, and
 * T / T_unit in units of 2^-30.  The step's arithmetic is FP32.  Its
 * increments are added to the stored integers exactly, and gradients use
 * exact integer differences.  Representable ranges:
 *     |rho - 1| < 0.49,  |u|, |v| < 0.99,  |T| < 1.98 T_unit.
 * T_unit is a power of two, at least 1, chosen per handle so that the
 * Dirichlet wall temperatures and T_ref +- dT/2 (rtlbfs_set_params_ref) lie
 * within +-1.5 T_unit, and the state last given to rtlbfs_set_state within
 * +-1.9 T_unit.  With the defaults (walls at 1 and 0) T_unit = 1.  The
 * temperature resolution is 2^-30 T_unit.  A configuration change that
 * needs a larger unit rounds the stored temperatures to it; the unit never
 * shrinks under a running state (rtlbfs_set_state picks it afresh).  The
 * arithmetic stays FP32 on absolute temperatures, so temperatures far from
 * zero compared with dT lose FP32 precision in the face sums.
 * A step whose new values leave a range reports RTLBFS_ERR_DIVERGED, in the
 * same way as a non-finite FP64 residual.  A state outside the ranges is
 * rejected by rtlbfs_set_state with RTLBFS_ERR_ARG.
 */

/* sides and boundary kinds */
#define RTLBFS_WEST 0
#define RTLBFS_EAST 1
#define RTLBFS_SOUTH 2
#define RTLBFS_NORTH 3
#define RTLBFS_WALL_DIRICHLET 0 /* no-slip wall, fixed temperature */
#define RTLBFS_WALL_ADIABATIC 1 /* no-slip wall, zero heat flux */
#define RTLBFS_PERIODIC 2       /* must be set on both opposite sides */
#define RTLBFS_HALO 3           /* a row strip's inner side (rtlbfs_create_strip only) */

/* Nusselt selectors of rtlbfs_nusselt */
#define RTLBFS_NU_WEST 0  /* energy flux through the west wall / (chi dT) */
#define RTLBFS_NU_EAST 1
#define RTLBFS_NU_SOUTH 2
#define RTLBFS_NU_NORTH 3
#define RTLBFS_NU_AVG 4   /* Nu_a of Eq. 69 (Section 4.2) */
#define RTLBFS_NU_HALF 5  /* Nu_1/2: energy flux through the x-face column x = L/2 (Tables 2-3); nx even */

typedef struct rtlbfs_ctx* rtlbfs_t;

/*
 * Face coordinates of the tanh-stretched mesh of Eq. 74 (Section 4.4):
 * out[i] = {tanh(phi) + tanh[2 phi (i/n - 1/2)]} L / (2 tanh(phi)),
 * i = 0..n (out holds n+1 doubles, caller-owned).  phi <= 0 gives the
 * uniform mesh out[i] = i L / n.  Host only.  ERR_ARG if n < 1, L <= 0.
 */
int rtlbfs_tanh_faces(int n, double L, double phi, double* out);

/*
 * Create a solver for an nx x ny cell mesh with face coordinates xf[0..nx],
 * yf[0..ny] (strictly ascending, copied).  precision is RTLBFS_FP64 or
 * RTLBFS_FP32.  Defaults: the differentially heated cavity of Section 3.3
 * (west Dirichlet T = 1, east Dirichlet T = 0, south/north adiabatic, all
 * no-slip at rest), Ra = 1e3, Pr = 0.71, Ma = 0.1, dt = half the smallest
 * cell width, kappa = 1, and the initial state rho = 1, u = v = 0, T linear
 * in x between the wall temperatures.  Allocates the device state
 * (2 buffers x 4 fields) on the current CUDA device.  *out receives the
 * handle.  ERR_ARG on bad sizes or non-ascending faces, ERR_OOM, ERR_CUDA.
 */
int rtlbfs_create_mesh(int nx, int ny, const double* xf, const double* yf, int precision,
                       rtlbfs_t* out);

/*
 * Physical parameters (Eq. 63 with V_c = Ma, c = 1): nu = V_c L sqrt(Pr/Ra),
 * chi = nu / Pr, beta_g = V_c^2 / (dT L) with L = xf[nx] - xf[0] and
 * dT = 1; dt is the macroscopic time step Delta t of Eqs. 41-43 / 57-59;
 * dt = 0 selects the explicit-stability rule
 * dt = min(0.5 w_min, 0.2 w_min^2 / max(nu, chi)) with w_min the smallest
 * cell width (about half the largest stable step, acoustic and diffusive).
 * ERR_ARG unless Ra, Pr, Ma > 0 and dt >= 0.
 */
int rtlbfs_set_params(rtlbfs_t h, double Ra, double Pr, double Ma, double dt);

/*
 * As rtlbfs_set_params with an explicit reference length L (e.g. the
 * height of a Rayleigh-Benard box), temperature difference dT and
 * reference temperature T_ref of the Boussinesq term (Eq. 64).
 */
int rtlbfs_set_params_ref(rtlbfs_t h, double Ra, double Pr, double Ma, double dt, double L,
                          double dT, double T_ref);

/*
 * Lattice spacing of the reconstructed unit lattice (Fig. 2): each face
 * uses dt_f = kappa * min(width of its two cells normal to the face), and
 * tau_f = nu / (c_s^2 dt_f) + 1/2, tau_g = chi / (c_s^2 dt_f) + 1/2
 * (Eqs. 9-10).  kappa = 1 reproduces the paper's dt_f = dx = 1 runs.
 * ERR_ARG unless kappa > 0.
 */
int rtlbfs_set_lattice(rtlbfs_t h, double kappa);

/*
 * Boundary condition of one side (RTLBFS_WEST..NORTH): kind is
 * RTLBFS_WALL_DIRICHLET (wall at temperature T_wall), RTLBFS_WALL_ADIABATIC
 * or RTLBFS_PERIODIC (must be set on both opposite sides before stepping);
 * u_wall is the wall's tangential velocity (0 = no-slip at rest).
 * Walls are ghost cells mirroring the adjacent cell; every wall face
 * carries zero mass flux.  ERR_ARG on a bad side or kind.
 */
int rtlbfs_set_bc(rtlbfs_t h, int side, int kind, double T_wall, double u_wall);

/* Body force per unit mass (fx, fy) added to the momentum source. */
int rtlbfs_set_body_force(rtlbfs_t h, double fx, double fy);

/*
 * Override the parameter mapping: kinematic viscosity nu, thermal
 * diffusivity chi and buoyancy coefficient beta_g (0 switches buoyancy
 * off).  ERR_ARG unless nu > 0, chi > 0.
 */
int rtlbfs_set_physics(rtlbfs_t h, double nu, double chi, double beta_g);

/*
 * Copy a host state in (rho, u, v, T: ny*nx doubles each, caller-owned)
 * and reset the step counter and residual.  In FP32 mode the fields are
 * rounded to the fixed-point storage described at RTLBFS_FP32, after the
 * temperature unit has been picked for this state; ERR_ARG if a value is
 * NaN or outside the representable ranges.
 */
int rtlbfs_set_state(rtlbfs_t h, const double* rho, const double* u, const double* v,
                     const double* T);

/* Copy the current state out to host arrays (ny*nx doubles each). */
int rtlbfs_get_state(rtlbfs_t h, double* rho, double* u, double* v, double* T);

/*
 * The state as the device stores it: ny x nx cell records, row-major
 * without row padding, each record (rho - 1, u, v, T) -- FP64: four
 * doubles (32 bytes); FP32: four 32-bit fixed-point integers (16 bytes)
 * in the units given at RTLBFS_FP32, temperature in units of 2^-30 *T_unit.
 * Exact in both directions (a checkpoint taken with get and restored with
 * set continues bit for bit), half the bytes of the four FP64 planes in
 * FP32, and no conversion kernel.  rtlbfs_state_raw_bytes: the size of
 * `records` (nx * ny * 16 or 32; 0 for a bad handle).  get writes the
 * records and the temperature unit (T_unit may be null); set takes them
 * (T_unit: 1 in FP64, a power of two >= 1 in FP32, else ERR_ARG; a
 * configuration that needs a larger unit rescales the stored temperatures)
 * and, like rtlbfs_set_state, resets the step counter and residual.
 * records: host memory, caller-owned (pinned memory lets the copies run
 * as DMA); both calls return after the copy.
 */
size_t rtlbfs_state_raw_bytes(rtlbfs_t h);
int rtlbfs_get_state_raw(rtlbfs_t h, void* records, double* T_unit);
int rtlbfs_set_state_raw(rtlbfs_t h, const void* records, double T_unit);

/*
 * Advance exactly nsteps explicit steps (no convergence stop).  The steps
 * run as CUDA-graph replays on the handle's stream; the call returns after
 * they complete.  ERR_DIVERGED if the residual became non-finite (the
 * state is then left at the first non-finite step).
 */
int rtlbfs_step(rtlbfs_t h, long nsteps);

/*
 * Step until max(R_u, R_T) < tol, checked after every step on the device,
 * where R_u = ||(|u|^{n+1} - |u|^n)||_2 / ||(|u|^{n+1})||_2 and R_T the
 * same for T (L2 analogue of Eq. 65).  Stops exactly at the first step that
 * meets tol.  max_steps bounds the steps of this call; timeout_s (<= 0: no
 * limit) bounds its wall time, checked between chunks of steps.  Writes
 * the steps taken by this call and the last (R_u, R_T) if the pointers are
 * non-null.  Returns OK, ERR_NOT_CONVERGED, ERR_TIMEOUT or ERR_DIVERGED.
 * In FP32 the residual settles at a floor set by the state's fixed-point
 * quantum over the flow's velocity scale (about 1e-8 for strong flows,
 * above 3e-8 for weak ones): use tol >= 1e-7 there; FP64 reaches 1e-15.
 */
int rtlbfs_run_to_steady(rtlbfs_t h, double tol, long max_steps, double timeout_s,
                         long* steps_taken, double* residual);

/* Residual (R_u, R_T) of the last step and the total step count. */
int rtlbfs_residual(rtlbfs_t h, double* res2, long* steps);

/*
 * Nusselt number of the current state, summed in FP64 on the device:
 * which = RTLBFS_NU_WEST..NORTH: the corrector's energy flux (Eq. 59 brace)
 * through that wall's faces times the face areas, / (chi dT); RTLBFS_NU_AVG:
 * Eq. 69 by the midpoint rule with Green-Gauss dT/dx; RTLBFS_NU_HALF: the
 * energy flux through the x-face column i = nx/2 (requires nx even).
 */
int rtlbfs_nusselt(rtlbfs_t h, int which, double* nu);

/* Face stages (rtlbfs_set_scheme). */
#define RTLBFS_SCHEME_RTLBFS 0
#define RTLBFS_SCHEME_TLBFS 1

/*
 * Face stage of the step.  RTLBFS_SCHEME_RTLBFS (the default): the
 * reconstructed solver of Section 3.2 (Eqs. 46-48, 57-59).
 * RTLBFS_SCHEME_TLBFS: the original TLBFS of Section 2.2 that RTLBFS
 * approximates -- D2Q9 equilibria (Eqs. 3-4) at the nodes x_S - e_i dt_f
 * (Eq. 29 values), predicted variables as their moments (Eqs. 30-32) and
 * fluxes from the equilibria and non-equilibrium parts (Eqs. 33-40); same
 * update, source, boundary and run-control rules.  TLBFS runs on the tile
 * kernel at height 16 (it sets that schedule).  The Nusselt numbers use
 * the energy flux of the chosen stage.  ERR_ARG on another value.
 */
int rtlbfs_set_scheme(rtlbfs_t h, int scheme);

/*
 * Execution schedule of the step (results are the same up to FP rounding
 * order): kernel 0 = warp-marching strips (each warp walks a 28-column strip
 * up a chunk of chunk_rows rows, rolling its stencil window in registers;
 * chunk_rows 0 = chosen from the GPU size), kernel 1 = shared-memory tiles
 * of 32 columns by chunk_rows rows (16, 14, 12, 10, 8, 4 or 2 in FP32; 16,
 * 8, 4 or 2 in FP64; 0 = the height whose tile count fills the SMs most
 * evenly), kernel 2 = the same tiles in one persistent cooperative launch
 * per chunk of steps, each tile waiting only for the eight around it (the
 * RTLBFS stage, every tile resident at once and at least 2 cells wide; the
 * step then fails with ERR_ARG otherwise).  Every kernel stops at the same
 * step under run_to_steady.
 * ERR_ARG on other values, and on anything but the tile kernel at height
 * 16 (or 0) under the TLBFS face stage.
 */
int rtlbfs_set_schedule(rtlbfs_t h, int kernel, int chunk_rows);

/*
 * For tests of the persistent kernel's bounded waits: tile `tile` (>= 0)
 * never reports its progress, so its neighbours' waits run out after about
 * a second and the step returns ERR_CUDA ("stalled"); -1 restores normal
 * running.  Never needed otherwise.
 */
int rtlbfs_debug_withhold_tile(rtlbfs_t h, int tile);

/*
 * Autotuner: time every candidate schedule (the tile kernel at each tile
 * height, the persistent tile kernel at each height it can take, and the
 * marching kernel with 8..256 rows per unit) for `steps` steps each on a
 * device-side snapshot of the current state, restore the state exactly
 * (fields, step counter, residual) and keep the fastest schedule.  Writes
 * the choice and its time per step if the pointers are non-null.  Needs
 * one extra copy of the state in device memory while it runs.
 */
int rtlbfs_autotune(rtlbfs_t h, int steps, int* kernel, int* chunk_rows, double* ms_per_step);

/* Use this CUDA stream (a cudaStream_t, e.g. torch's current stream) for
 * all later work of the handle; NULL restores the handle's own non-blocking
 * stream (pass cudaStreamLegacy to order work with the legacy default
 * stream). */
int rtlbfs_set_stream(rtlbfs_t h, void* stream);

/* Wait for the handle's stream. */
int rtlbfs_sync(rtlbfs_t h);

/* Message of the last failure on h (static storage of the handle). */
const char* rtlbfs_last_error(rtlbfs_t h);

/*
 * Measurement aid (no counterpart in the paper): floating-point operations
 * of one cell-update of the step with every face and gradient evaluated
 * once -- *face_ops per face (the face arithmetic of the kernels run on an
 * operation-counting type), *cell_ops per cell-update (two faces plus the
 * gradients, update and residual terms), *sfu_ops reciprocals and square
 * roots per cell-update.  An add, multiply or fused multiply-add counts 1.
 * Host-only; needs no GPU.  Null pointers are skipped.  Returns RTLBFS_OK.
 */
int rtlbfs_op_counts(double* face_ops, double* cell_ops, double* sfu_ops);

/* The same for a face stage: RTLBFS_SCHEME_RTLBFS or RTLBFS_SCHEME_TLBFS.
 * ERR_ARG on another scheme. */
int rtlbfs_op_counts_scheme(int scheme, double* face_ops, double* cell_ops, double* sfu_ops);

/* Free every device and host resource of h; NULL is ignored. */
void rtlbfs_destroy(rtlbfs_t h);

/*
 * Allocation-free Nusselt number of a caller-owned FP64 state.  The paper
 * has no counterpart: this entry point exists for callers that cannot
 * allocate device memory when they call in -- a real-time loop, where a
 * cudaMalloc may block on the device or fail at an unpredictable moment,
 * and hosts that hand the library only memory they own -- and for fields
 * that live in the caller's buffers rather than in a handle.  It computes
 * what rtlbfs_nusselt computes (same selectors `which`, same FP64
 * arithmetic) and allocates nothing: no cudaMalloc, cudaFree or allocating
 * library call.  bc_kind, bc_T and bc_u are read before the call returns;
 * xf and yf too when they are pageable memory (malloc, new, numpy): the
 * runtime stages such a copy before returning.  From pinned memory the
 * copies read xf and yf when they run on `stream`, so keep pinned arrays
 * unchanged until the stream has passed this call.  The work is queued on
 * `stream`.
 *
 *   nx, ny         cells, each at most 8192 (larger: RTLBFS_ERR_ARG)
 *   xf, yf         host face coordinates (nx+1, ny+1), strictly ascending
 *   rho,u,v,T      device pointers, FP64, row-major ny x nx (rho itself, not rho-1)
 *   nu, chi, kappa transport coefficients and lattice factor (as rtlbfs_set_physics /
 *                  rtlbfs_set_lattice); dT the reference temperature difference
 *   bc_kind, bc_T, bc_u   host arrays of 4 (W, E, S, N) as in rtlbfs_set_bc
 *   nu_out         device pointer to one double, written asynchronously on `stream`
 *   stream         a cudaStream_t (NULL: the legacy default stream)
 *
 * Working memory: one file-scope device array of about 1.8 MB (descriptor,
 * mesh lines, partial sums) that every GPU which loads the library keeps
 * until the process exits.  The first call on a device looks up the array's
 * address (cudaGetSymbolAddress, once per device): make that first call
 * before any stream capture.  Every call reuses the array and the call
 * re-initialises what it needs; two calls whose work overlaps on the GPU
 * (different streams, or different host threads) race on it and must be
 * ordered by the caller.  Returns RTLBFS_OK, RTLBFS_ERR_ARG or
 * RTLBFS_ERR_CUDA.
 */
int rtlbfs_nusselt_noalloc(int nx, int ny, const double* xf, const double* yf,
                           const double* rho, const double* u, const double* v, const double* T,
                           double nu, double chi, double kappa, double dT, const int* bc_kind,
                           const double* bc_T, const double* bc_u, int which, double* nu_out,
                           void* stream);

/*
 * Row strips: one mesh split across GPUs (or processes) by rows.  The
 * explicit step (Section 3.2) reads each cell's neighbours up to two cells
 * away: a face needs the Green-Gauss gradients (Eq. 55) of its two cells,
 * and a gradient needs the values of the cell's neighbours (Eq. 56).  So a
 * strip of rows j0 <= j < j1 can take a step once it holds the two rows
 * beyond each of its inner sides, as they were after the previous step.
 * Exchanging those two rows between neighbouring strips before every step
 * gives exactly the step of the whole mesh.  The paper has no counterpart
 * (it runs serial programs); this is the decomposition of the sweep.
 *
 * rtlbfs_create_strip: a handle for rows j0 <= j < j1 (j1 - j0 >= 2) of
 * an nx x ny_mesh mesh with faces xf[0..nx], yf[0..ny_mesh] (the whole
 * mesh's faces; copied).  Its south side (if j0 > 0) and north side (if
 * j1 < ny_mesh) are halo sides: no wall, the two rows beyond are set by
 * rtlbfs_strip_set_halo (or written to the device addresses of
 * rtlbfs_strip_rows) before each step.  The other sides behave as in
 * rtlbfs_create_mesh (walls by rtlbfs_set_bc); parameters, the dt rule
 * (smallest cell of the whole mesh) and the reference length (the x width)
 * are those of the whole mesh.  Fields of the strip's own rows are (j1 -
 * j0) x nx.  Nusselt numbers of a strip are its share of the whole
 * mesh's (west, east, mid-plane and Eq. 69 sums add over strips; south and
 * north only where that side is a wall); they read the halo rows too, so
 * exchange halos after the last step before taking them.  Stepping takes whole steps; the
 * stop test of rtlbfs_run_to_steady would see one strip only, so a
 * decomposed run sums rtlbfs_residual_sums over the strips instead.
 * ERR_ARG on bad sizes or faces.
 */
int rtlbfs_create_strip(int nx, int ny_mesh, const double* xf, const double* yf, int j0, int j1,
                        int precision, rtlbfs_t* out);

/* The strip's two rows next to side (RTLBFS_SOUTH: rows j0, j0 + 1;
 * RTLBFS_NORTH: rows j1 - 2, j1 - 1) of the current state as four planes
 * rho, u, v, T of 2 x nx doubles each (row-major, southern row first):
 * what the neighbour across that side needs.  rows: host, caller-owned,
 * 8 x nx doubles.  ERR_ARG if side is not a halo side. */
int rtlbfs_strip_get_rows(rtlbfs_t h, int side, double* rows);

/* Set the two halo rows beyond side (RTLBFS_SOUTH: rows j0 - 2, j0 - 1;
 * RTLBFS_NORTH: rows j1, j1 + 1) of the current state from planes in the
 * layout of rtlbfs_strip_get_rows (the neighbour's rows as it returned
 * them).  ERR_ARG if side is not a halo side or (FP32) a value is not
 * representable. */
int rtlbfs_strip_set_halo(rtlbfs_t h, int side, const double* rows);

/* Device address and size (*bytes) of the two rows next to side (halo =
 * 0: the strip's own rows; 1: the halo rows beyond) in state buffer
 * `buffer` (0 or 1), in the device record layout (cell records, row pitch
 * included; the two rows are contiguous).  For exchanges between devices
 * (NCCL send/recv, peer copies) without the host: a step reads buffer
 * rtlbfs_current_buffer() and writes the other one, so before the next
 * step the own rows of the new current buffer go to the neighbour's halo
 * rows of its new current buffer (same record layout and size when both
 * strips have the same nx and precision; in FP32 the strips must also store
 * temperature in the same unit, see RTLBFS_FP32, which holds when their
 * configured temperatures set it).  The library owns the memory. */
int rtlbfs_strip_rows(rtlbfs_t h, int side, int halo, int buffer, void** dev, size_t* bytes);

/* Copy the strip's own two rows next to side in state buffer `buffer` to
 * the device buffer dev (rtlbfs_strip_rows' bytes, caller-owned device
 * memory), or copy dev into the halo rows beyond side of that buffer:
 * device-to-device copies queued on the handle's stream (no host wait, no
 * allocation).  With the strips' steps counted from a state upload, the
 * current buffer after k steps is k % 2, so a caller can exchange halos
 * through its own device buffers (NCCL send/recv or peer copies) without
 * reading the run control.  ERR_ARG if side is not a halo side. */
int rtlbfs_strip_pack(rtlbfs_t h, int side, int buffer, void* dev);
int rtlbfs_strip_unpack(rtlbfs_t h, int side, int buffer, const void* dev);

/* The state buffer (0 or 1) holding the current state. */
int rtlbfs_current_buffer(rtlbfs_t h, int* buffer);

/* The residual sums of the last step (the sums behind R12, Eq. 65's L2
 * analogue): sums[0] = sum (|u|^{n+1} - |u|^n)^2, sums[1] = sum
 * |u|^{n+1}^2, sums[2] = sum (T^{n+1} - T^n)^2, sums[3] = sum T^{n+1}^2
 * over the handle's cells, FP64; summed over the strips of a mesh they give
 * R_u = sqrt(s0 / s1), R_T = sqrt(s2 / s3) of the whole mesh.  *steps: the
 * step count (may be null). */
int rtlbfs_residual_sums(rtlbfs_t h, double* sums, long* steps);

/* Number of kernel launches issued by the library since load (for the
 * benchmark's launch count). */
long long rtlbfs_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* RTLBFS_H */
