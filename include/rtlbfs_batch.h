/*
 * rtlbfs_batch.h -- many independent RTLBFS cavities advanced together, and
 * a continuous-batching request loop on top of them (GB300, sm_103a).
 *
 * The method per cavity is the one of rtlbfs.h (arXiv 2202.13449, Section
 * 3.2: Eqs. 29, 46-48, 55-59, 64).  A batch holds up to max_slots cavities of
 * any mesh size; one kernel launch advances every active cavity by one step
 * (one work list of strips or tiles over all of them), each cavity stopping
 * on its own residual tolerance or step cap (decided on the device after
 * every step).  The paper solves one cavity at a time; batching and serving
 * are systems layers around its per-face arithmetic.
 *
 * Conventions as in rtlbfs.h: status returns, host arrays copied, device
 * memory owned by the batch, not thread-safe per batch.
 */
#ifndef RTLBFS_BATCH_H
#define RTLBFS_BATCH_H

#include <stddef.h>

#include "rtlbfs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rtlbfs_batch_ctx* rtlbfs_batch_t;

/* per-slot status of rtlbfs_batch_poll */
#define RTLBFS_SLOT_EMPTY (-1)
#define RTLBFS_SLOT_RUNNING 0
#define RTLBFS_SLOT_CONVERGED 1
#define RTLBFS_SLOT_MAX_STEPS 2
#define RTLBFS_SLOT_DIVERGED 3

/* Create an empty batch of up to max_slots cavities (precision RTLBFS_FP64
 * or RTLBFS_FP32).  ERR_ARG, ERR_OOM, ERR_CUDA. */
int rtlbfs_batch_create(int precision, int max_slots, rtlbfs_batch_t* out);

/* Device bytes one nx x ny cavity of this precision occupies in a batch
 * (both state buffers and mesh lines); for admission control. */
size_t rtlbfs_batch_bytes(int precision, int nx, int ny);

/* Free and total device memory of the current device (cudaMemGetInfo). */
int rtlbfs_batch_free_bytes(size_t* free_bytes, size_t* total_bytes);

/*
 * Add a cavity with faces xf[0..nx], yf[0..ny] (copied) and parameters as
 * rtlbfs_set_params (Eq. 63 with V_c = Ma, L = domain width; dt = 0: the
 * stability rule of rtlbfs_set_params): the defaults
 * of rtlbfs_create_mesh (differentially heated cavity, conduction initial
 * state).  *slot receives its slot id.  The slot is idle until armed.
 * ERR_STATE when no slot is free, ERR_OOM when device memory is short.
 */
int rtlbfs_batch_add(rtlbfs_batch_t b, int nx, int ny, const double* xf, const double* yf,
                     double Ra, double Pr, double Ma, double dt, int* slot);

/* Boundary condition of one side of a slot (as rtlbfs_set_bc). */
int rtlbfs_batch_set_bc(rtlbfs_batch_t b, int slot, int side, int kind, double T_wall,
                        double u_wall);

/* Lattice parameter of a slot (as rtlbfs_set_lattice: delta t_f = kappa *
 * min(w_L, w_R), Eqs. 9-10).  ERR_ARG unless kappa > 0. */
int rtlbfs_batch_set_lattice(rtlbfs_batch_t b, int slot, double kappa);

/* State in/out of a slot (ny*nx doubles per field, rho/u/v/T). */
int rtlbfs_batch_set_state(rtlbfs_batch_t b, int slot, const double* rho, const double* u,
                           const double* v, const double* T);
int rtlbfs_batch_get_state(rtlbfs_batch_t b, int slot, double* rho, double* u, double* v,
                           double* T);

/*
 * A slot's state as the device stores it (as rtlbfs_get_state_raw /
 * rtlbfs_set_state_raw of include/rtlbfs.h): ny x nx cell records without
 * row padding, 16 bytes in FP32 (fixed point, temperature in units of
 * 2^-30 * T_unit) or 32 in FP64; exact in both directions, half the bytes
 * of the FP64 planes in FP32 and no conversion kernel.
 * rtlbfs_batch_state_raw_bytes: the size of a slot's records (0 for a bad
 * handle or slot).  get writes the records and the temperature unit
 * (T_unit may be null); set takes them (T_unit 1 in FP64, a power of two
 * >= 1 in FP32, else ERR_ARG) and, like rtlbfs_batch_set_state, resets the
 * slot's step counter and run control.  records: caller-owned host memory
 * (pinned memory lets the copies run as DMA); both return after the copy.
 */
size_t rtlbfs_batch_state_raw_bytes(rtlbfs_batch_t b, int slot);
int rtlbfs_batch_get_state_raw(rtlbfs_batch_t b, int slot, void* records, double* T_unit);
int rtlbfs_batch_set_state_raw(rtlbfs_batch_t b, int slot, const void* records, double T_unit);

/*
 * The same for n slots in one call: slots[k]'s records from / to
 * records[k] (each rtlbfs_batch_state_raw_bytes(b, slots[k]) bytes of
 * caller-owned host memory) and its unit T_units[k] (T_units may be null
 * for get).  Every copy is queued on the batch's stream and the call
 * synchronises once, so with pinned buffers the copies run back to back
 * as DMA.  Arguments are checked before any copy: ERR_ARG for n < 0, a
 * null array, a slot not in use, a null record pointer or (set) a bad
 * unit; nothing is copied then.  On ERR_CUDA from set, the states and run
 * records of the listed slots are undefined (some copies may have run);
 * set them again before stepping.  A slot listed twice takes the records
 * of its last entry.
 */
int rtlbfs_batch_get_states_raw(rtlbfs_batch_t b, int n, const int* slots, void* const* records,
                                double* T_units);
int rtlbfs_batch_set_states_raw(rtlbfs_batch_t b, int n, const int* slots,
                                const void* const* records, const double* T_units);

/* Let a slot take up to max_steps more steps, stopping after the first step
 * with max(R_u, R_T) < tol (tol <= 0: never). */
int rtlbfs_batch_arm(rtlbfs_batch_t b, int slot, double tol, long max_steps);

/* rtlbfs_batch_arm for n slots (host array, caller-owned, read before the
 * call returns) in one launch.  ERR_ARG for n < 0, a null array, a slot
 * not in use or max_steps < 0, before any slot is armed. */
int rtlbfs_batch_arm_many(rtlbfs_batch_t b, int n, const int* slots, double tol, long max_steps);

/* Launch nsteps batched steps (asynchronous; slots that are done skip). */
int rtlbfs_batch_step(rtlbfs_batch_t b, long nsteps);

/* Per-slot status, steps since the last state upload and last (R_u, R_T)
 * (arrays of max_slots, 2*max_slots for res2; null pointers skipped).
 * Synchronises. */
int rtlbfs_batch_poll(rtlbfs_batch_t b, int* status, long* steps, double* res2);

/* FP64 Nusselt number of a slot (selectors of rtlbfs_nusselt). */
int rtlbfs_batch_nusselt(rtlbfs_batch_t b, int slot, int which, double* nu);

/* Free a slot and its device memory. */
int rtlbfs_batch_remove(rtlbfs_batch_t b, int slot);

/* Schedule of the batch's step launches, as rtlbfs_set_schedule of
 * include/rtlbfs.h: kernel 0 = warp-marching strips of chunk_rows rows,
 * 1 = shared-memory tiles of height chunk_rows (0: the default of each),
 * 2 is refused for a batch (the persistent kernel takes one cavity).
 * ERR_ARG on other values. */
int rtlbfs_batch_set_schedule(rtlbfs_batch_t b, int kernel, int chunk_rows);

/* Pick the step schedule for the current set of slots (see rtlbfs_autotune). */
int rtlbfs_batch_autotune(rtlbfs_batch_t b, int steps, int* kernel, int* chunk_rows,
                          double* ms_per_step);

/* Stream for all later work of the batch (NULL: its own). */
int rtlbfs_batch_set_stream(rtlbfs_batch_t b, void* stream);

/* Active cells summed over slots, and kernel launches' work units. */
int rtlbfs_batch_info(rtlbfs_batch_t b, long long* active_cells, int* active_slots, int* units);

const char* rtlbfs_batch_last_error(rtlbfs_batch_t b);
void rtlbfs_batch_destroy(rtlbfs_batch_t b);

/* ------------------------------------------------------------------------ */
/* Continuous-batching request loop                                          */
/* ------------------------------------------------------------------------ */

/* One request: a square uniform n x n cavity (L = n, unit cells, dt from
 * the stability rule of rtlbfs_set_params, kappa 1) at Rayleigh number Ra and Prandtl number Pr, arriving t_arrive
 * seconds after the trace starts. */
typedef struct {
    double t_arrive;
    int n;
    double Ra, Pr;
} rtlbfs_request;

/* What became of one request (times in seconds from the trace start; -1:
 * never happened). */
typedef struct {
    double t_admit;   /* admitted to a slot (its work starts on the next launch) */
    double t_finish;  /* converged, capped or diverged, and retired */
    long steps;
    int status;       /* RTLBFS_SLOT_CONVERGED / _MAX_STEPS / _DIVERGED, or -1 not finished */
    double nu_hot, nu_cold;  /* FP64 wall Nusselt numbers (west, east) at the end */
} rtlbfs_result;

typedef struct {
    int max_slots;          /* concurrent cavities */
    double mem_fraction;    /* admit while batch bytes <= this fraction of free memory at start */
    double tol;             /* steady tolerance of every request */
    long max_steps;         /* step cap of every request */
    double Ma;              /* Mach number (V_c) */
    double time_limit_s;    /* wall-clock cap of the whole trace */
    int chunk_steps;        /* batched steps between polls */
    int precision;          /* RTLBFS_FP32 or RTLBFS_FP64 */
} rtlbfs_serve_opts;

/*
 * Replay a request trace in real time: requests are admitted (in arrival
 * order) once they have arrived, a slot is free and the device memory budget
 * allows; all admitted cavities advance together in batched launches of
 * chunk_steps steps; after each chunk finished ones are retired (their
 * Nusselt numbers taken) and their slots and memory reused.  Stops when all
 * requests are finished or time_limit_s has passed.  out[nreq] receives the
 * per-request results; *elapsed_s the wall time.  Returns OK or an error.
 */
int rtlbfs_serve(const rtlbfs_request* reqs, int nreq, const rtlbfs_serve_opts* opts,
                 rtlbfs_result* out, double* elapsed_s);

/* ------------------------------------------------------------------------ */
/* Stability map                                                             */
/* ------------------------------------------------------------------------ */

/*
 * The stability test of Section 3.3 (Figs. 4 and 5) as one batch: case k is
 * the differentially heated cavity of n[k] x n[k] unit cells (L = n[k]) at
 * Rayleigh number Ra[k] with lattice parameter kappa[k] (on unit cells the
 * paper's lattice spacing delta t = kappa[k]) and time step dt[k] (dt null
 * or dt[k] = 0: the stability rule of rtlbfs_set_params), Prandtl number Pr,
 * V_c = Ma, from the conduction state.  All cases advance together in
 * launches of chunk_steps steps until each has converged (max(R_u, R_T) <
 * tol after a step; tol <= 0: never), diverged (a non-finite residual, or in
 * FP32 a value leaving the fixed-point range) or taken max_steps steps.
 * status_out[k] receives RTLBFS_SLOT_CONVERGED, _DIVERGED or _MAX_STEPS and
 * steps_out[k] the steps taken (the diverging step included); *elapsed_s
 * the wall time.  Arrays of ncase; device memory is the library's and freed
 * on return.  ERR_ARG on bad sizes or parameters, ERR_OOM, ERR_CUDA.
 */
int rtlbfs_stability_map(int ncase, const int* n, const double* Ra, const double* kappa,
                         const double* dt, double Pr, double Ma, double tol, long max_steps,
                         int precision, int chunk_steps, int* status_out, long* steps_out,
                         double* elapsed_s);

#ifdef __cplusplus
}
#endif

#endif /* RTLBFS_BATCH_H */
