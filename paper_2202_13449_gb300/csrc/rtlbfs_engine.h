// rtlbfs_engine.h -- host-side engine shared by the single-cavity handle
// and the batch API: device memory of the cavities, the tile list, CUDA
// graphs of step launches and the run control.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rtlbfs_dev.cuh"
#include "rtlbfs_kernels.h"

namespace rtlbfs {

extern std::atomic<long long> g_launches;

// A named NVTX range over a scope (steps, graph replays, reductions, state
// copies), so that a timeline profile shows the library's phases; a no-op
// when no profiler is attached.
struct Nvtx {
    explicit Nvtx(const char* name) { nvtxRangePushA(name); }
    ~Nvtx() { nvtxRangePop(); }
    Nvtx(const Nvtx&) = delete;
    Nvtx& operator=(const Nvtx&) = delete;
};

// Host record of one cavity.
struct Cavity {
    int nx = 0, ny = 0, pitch = 0;
    std::vector<double> xf, yf;
    // parameters
    bool from_ra = true;
    double Ra = 1e3, Pr = 0.71, Ma = 0.1, dt = 0.5, kappa = 1.0;
    bool dt_auto = false;  // dt from the stability rule of resolve_params
    double Lref = 0.0, dT = 1.0, T_ref = 0.5;
    double nu = 0.0, chi = 0.0, beta_g = 0.0, fx = 0.0, fy = 0.0;
    int kind[4] = {kDirichlet, kDirichlet, kAdiabatic, kAdiabatic};
    double bcT[4] = {1.0, 0.0, 0.0, 0.0};
    double bcU[4] = {0.0, 0.0, 0.0, 0.0};
    // FP32: the device state stores T / T_unit in fixed point; T_unit is a
    // power of two >= 1, chosen so the configured temperatures lie within
    // +-1.5 T_unit and the last uploaded state within +-1.9 T_unit (always 1
    // in FP64).  State_Tmax: max |T| of the last state set_state uploaded.
    double T_unit = 1.0, state_Tmax = 0.0;
    // A row strip of a larger mesh (create_strip): halo_rows = 2 extra rows
    // below and above the strip's own rows in every buffer, for the halo
    // sides (kHalo); halo_w[0] = widths of rows -1, -2 and halo_w[1] =
    // widths of rows ny, ny+1 in the whole mesh; wmin_mesh > 0: the
    // smallest cell width of the whole mesh (the dt rule of resolve_params).
    int halo_rows = 0;
    double halo_w[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    double wmin_mesh = 0.0;
    // device memory
    void* d_fields = nullptr;  // 2 buffers x 4 fields x ny x pitch
    void* d_lines = nullptr;   // R lines then FP64 lines
    size_t fields_bytes = 0, lines_bytes = 0;
    size_t off_xl = 0, off_yl = 0, off_xc = 0, off_yc = 0;          // R lines
    size_t off_xld = 0, off_yld = 0, off_xcd = 0, off_ycd = 0;      // FP64 lines
    bool dirty = true;  // parameters changed since the last upload
    bool active = false;
    int first_tile = 0, ntiles = 0;
};

class Engine {
public:
    Engine(int precision, int capacity);
    ~Engine();
    Engine(const Engine&) = delete;
    Engine& operator=(const Engine&) = delete;

    int init();  // device queries, buffers; returns status
    int precision() const { return precision_; }
    int capacity() const { return capacity_; }

    // slots
    int add(int nx, int ny, const double* xf, const double* yf, int* slot, int halo_rows = 0);
    // rows j0 <= j < j1 of an nx x ny_mesh mesh as a cavity whose south /
    // north sides inside the mesh are halo sides (kHalo)
    int add_strip(int nx, int ny_mesh, const double* xf, const double* yf, int j0, int j1,
                  int* slot);
    // the 2 rows next to side S/N (ghost = 0: the strip's own rows; 1: the
    // halo rows beyond it) of buffer b: device address and bytes (contiguous)
    int strip_rows(int slot, int side, int ghost, int buffer, void** ptr, size_t* bytes);
    // the same rows of the current state as FP64 planes rho, u, v, T of
    // 2 x nx values each (host arrays), out of or into the state
    int get_rows(int slot, int side, int ghost, double* host);
    int set_rows(int slot, int side, int ghost, const double* host);
    int remove(int slot);
    Cavity* cavity(int slot);
    static size_t bytes_for(int precision, int nx, int ny);

    // parameters of a slot changed: lines are re-uploaded before the next step
    void touch(int slot);
    int resolve_params(Cavity& c);  // fills nu, chi, beta_g from Ra etc.

    // state I/O (host arrays of ny*nx doubles each)
    int set_state(int slot, const double* rho, const double* u, const double* v,
                  const double* T);
    int get_state(int slot, double* rho, double* u, double* v, double* T);
    int set_conduction_state(int slot);
    // the state as its cell records (ny x nx, no row padding; FP32: the
    // fixed-point records with temperature in units of *T_unit), exact both
    // ways; host memory (pinned memory makes the copies asynchronous DMA)
    int get_records(int slot, void* host, double* T_unit);
    int set_records(int slot, const void* host, double T_unit);
    // several slots at once: every copy queued, one synchronisation
    int get_records_many(int n, const int* slots, void* const* host, double* T_units);
    int set_records_many(int n, const int* slots, const void* const* host, const double* T_units);
    int queue_set_records(int slot, const void* host, double T_unit, CavityRun* run_out = nullptr);
    int arm_many(int n, const int* slots, long long nsteps, double tol);
    size_t record_bytes() const { return 4 * rsize_; }

    // run control: arm a slot for up to nsteps steps (tol < 0: no early stop)
    int arm(int slot, long long nsteps, double tol);
    // launch `launches` step kernels (graph replays where possible)
    int launch_steps(long long launches);
    int read_ctl(int slot, CavityCtl* out);          // synchronises
    int read_ctls(std::vector<CavityCtl>& out);      // all slots, synchronises
    int nusselt(int slot, int which, double* out);   // synchronises

    int sync();
    int set_stream(cudaStream_t s);
    cudaStream_t stream() const { return stream_; }
    const std::string& error() const { return err_; }
    int fail(int code, const std::string& msg);
    int cuda_fail(cudaError_t e, const char* what);
    int active_tiles() const { return ntiles_; }
    int grid() const { return grid_; }
    // step kernel: 0 = warp-marching strips (default), 1 = shared-memory
    // tiles, 2 = the tile kernel in persistent form (one cavity whose tiles
    // all fit on the GPU at once; many steps per launch)
    int set_kernel(int kind);
    // tests only: the persistent kernel's tile that never reports progress
    // (-1: none), to exercise its bounded waits
    void set_withhold(int tile) { withhold_ = tile; }
    int kernel() const { return kernel_; }
    // rows per work unit (0 = automatic): chunk rows of a warp-marching
    // unit, or the tile height of the tile kernel (one of kTileHeights)
    int set_chunk_rows(int rows);
    int chunk_rows() const { return chunk_rows_; }
    // face stage of every cavity: kSchemeRTLBFS or kSchemeTLBFS (the latter
    // runs on the tile kernel at the default height)
    int set_scheme(int scheme);
    int scheme() const { return scheme_; }
    // time every candidate schedule for `steps` steps on a snapshot of the
    // current state (restored afterwards) and keep the fastest
    int autotune(int steps, int* kernel, int* chunk_rows, double* ms_per_step);

private:
    int upload_lines(int slot);
    double temp_unit(const Cavity& c) const;  // the T_unit the configuration asks for
    int rebuild_tiles();
    int prepare_launch();

    int precision_;
    int capacity_;
    size_t rsize_;
    int sms_ = 0, grid_ = 0;
    int occ_tile_[32] = {};  // resident tile blocks per SM, by tile height
    int occ_tlbfs_ = 0;      // the same for the TLBFS tile kernel
    int occ_persist_[32] = {};  // the same for the persistent tile kernel
    int* d_tstep_ = nullptr;    // persistent kernel: last step of each tile
    int tstep_cap_ = 0;
    PersistCtl* d_pctl_ = nullptr;
    int* h_stalled_ = nullptr;  // pinned
    int withhold_ = -1;
    int persist_slot_ = -1;     // the one active cavity, once eligible
    int persist_check();        // sets persist_slot_ or fails with the reason
    int scheme_ = 0;
    int tile_h_ = 16;        // tile height of the current tile list
    int pick_tile_height() const;
    int kernel_ = 0, occ_march_ = 0, chunk_rows_ = 0;
    int launch_one(cudaStream_t s);
    cudaStream_t stream_ = nullptr, own_stream_ = nullptr;
    std::vector<Cavity> slots_;
    std::vector<CavityDesc> h_desc_;
    CavityDesc* d_desc_ = nullptr;
    CavityRun* d_ctl_ = nullptr;       // run control per slot (two headers, sums)
    int put_run(int slot, const CavityCtl& c);  // both headers = c, sums cleared
    int4* d_tiles_ = nullptr;
    int* d_ntiles_ = nullptr;
    int tile_cap_ = 0, ntiles_ = 0;
    bool tiles_dirty_ = true;
    bool desc_dirty_ = false;          // unit ranges changed: re-upload all descriptors
    cudaMemPool_t pool_ = nullptr;     // device memory of the cavities
    double* d_partial_ = nullptr;  // per-block partial sums of the FP64 reductions
    int partial_cap_ = 0;
    double* d_scalar_ = nullptr;
    double* h_scalar_ = nullptr;   // pinned
    double* d_stage_ = nullptr;
    // slot lists and run records of the many-slot calls
    int* d_slot_list_ = nullptr;
    CavityRun* d_run_list_ = nullptr;
    int list_cap_ = 0;
    int grow_lists(int n);
    size_t stage_cap_ = 0;
    cudaGraphExec_t gexec_ = nullptr;
    int gchunk_ = 0;
    cudaStream_t gstream_ = nullptr;
    std::string err_;
};

}  // namespace rtlbfs
