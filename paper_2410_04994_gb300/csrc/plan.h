// Internal definitions shared by the host-side translation units of libshg.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdlib>
#include <string>
#include <vector>

#include "../../include/shg.h"
#include "common.cuh"

namespace shg {

constexpr double kEps0 = 8.8541878128e-12;  // F/m
constexpr double kCLight = 299792458.0;     // m/s
constexpr double kPi = 3.14159265358979323846;
constexpr int kRedBlocks = 64;              // blocks per instance in the FP64 reductions

// Extra per-instance inputs of the initial-field and reduction kernels.
struct InitDesc {
    double x0, dx, y0, dy;
    double w0, zf, kF;      // Eq. (5) at z = 0
    double p1;              // target discrete power
    double cFdxdy;          // (1/2) eps0 c n_F dx dy
    double cSdxdy;          // (1/2) eps0 c n_SH dx dy
    double* red;            // [kRedBlocks][2] partial sums (plan-owned scratch)
    double* pw;             // [2] P_F, P_SH results
    const void* f0;         // custom initial fields [2][ny][nx] or nullptr
};

struct Adjoint;     // adjoint.cu
struct Heat;        // heat.cu
struct HeatDirect;  // heat_direct.cu
struct ThreeWave;   // threewave.cu

}  // namespace shg

struct shg_plan {
    shg_grid_t g;
    shg_crystal_t c;
    shg_beams_t b;
    int flags = 0;
    bool fp64 = false;
    size_t csize = 8;         // bytes per complex element
    int device = 0;

    void* field = nullptr;    // [2][ny][nx] current state
    void* field0 = nullptr;   // [2][ny][nx] custom initial state
    bool custom_init = false;
    void* px = nullptr;       // [2][nx]
    void* py = nullptr;       // [2][ny]
    void* pxc = nullptr;      // conjugate tables for the adjoint
    void* pyc = nullptr;
    void* eph = nullptr;      // [4 nz + 1]
    void* tw = nullptr;       // [1024]
    void* ttab = nullptr;     // [tz][ty][tx] (dT, C) in the plan's precision
    void* umap = nullptr;     // FP32: [tz][ny][nx] (dT, C) at every field point, or nullptr
    size_t umap_bytes = 0;
    float* tmap = nullptr;    // [tz][ty][tx] dT as set
    int tx = 0, ty = 0, tz = 0;
    double tlx = 0, tly = 0;
    void* desc = nullptr;     // device InstDesc<R>[1]
    shg::InitDesc* idesc = nullptr;  // device InitDesc[1]
    double* red = nullptr;
    double* pw = nullptr;
    double pw_host[2] = {0, 0};
    bool has_result = false;
    bool batch_result = false;  // pw_host holds the last batch's powers
    int batch_kst = 0;          // status word of this instance in the last batch
    cudaStream_t last_stream = nullptr;
    // Stream ordering without host synchronisation: `done` is recorded after
    // each propagation (its kernels read the map tables), `ready` after the
    // table rebuild of an asynchronous shg_set_temperature.
    cudaEvent_t done = nullptr, ready = nullptr;
    bool done_valid = false, ready_pending = false;

    // heat grid
    double* Q = nullptr;      // [hz][hy][hx]
    int* hix = nullptr;
    int* hiy = nullptr;
    int* hlz = nullptr;
    double* theat = nullptr;  // [hz][hy][hx] last solved dT
    double* theat_prev = nullptr;
    float* theat_f = nullptr; // dT rounded to float, as installed as the map
    double* hred = nullptr;   // reduction scratch of the heat solve
    int heat_face[6] = {0, 0, 0, 0, 0, 0};  // x-, x+, y-, y+, z-, z+: 0 oven (Eq. 9), 1 convective (Eq. 10)
    double heat_h[6] = {0, 0, 0, 0, 0, 0};  // heat transfer coefficient of each convective face
    double heat_tinf = 0;                    // T_inf - T_oven (K)
    int heat_method = 0;                     // SHG_HEAT_DIRECT or SHG_HEAT_SOR
    DkModel dkm{};                           // Eq. (4) model (dkm.on) or the linearised one
    shg::HeatDirect* hdir = nullptr;         // eigenbases and work buffers of the direct solve
    shg::ThreeWave* w3 = nullptr;            // three-wave plans: their crystal, beams, descriptor

    // tensor map of `field` for the TMA column pass (FP32, supported lengths)
    CUtensorMap cmap;
    void* cmap_dev = nullptr;
    bool has_cmap = false;
    int* status = nullptr;     // device status word written by kernels that give up
    double* mon = nullptr;     // power monitor slots [2 * mon_slots] (shg_set_monitor)
    int mon_every = 0, mon_slots = 0;
    unsigned wait_polls = 1u << 20;  // bound on each device-side wait (shg_set_wait_limit)

    // forward graph
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;
    bool gvalid = false;

    shg::Adjoint* adj = nullptr;
};

namespace shg {

// status helpers
shg_status_t cuda_fail(cudaError_t e, const char* what);
#define SHG_CK(call)                                                 \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return ::shg::cuda_fail(e_, #call);   \
    } while (0)

// Fill host-side descriptors from the plan's current state.
void fill_desc_f32(const shg_plan* p, InstDesc<float>* d);
void fill_desc_f64(const shg_plan* p, InstDesc<double>* d);
void fill_init(const shg_plan* p, InitDesc* d);

// Kernel launchers (passes_f32.cu / passes_f64.cu / aux.cu).
// `variant` selects the kernel flavour: 0 the default FFT shape, 1 the
// alternative shape where it exists; for the column pass 2 is the TMA-staged
// kernel (needs `tmaps`); 3 and 4 are the default shape in 128- and
// 64-thread CTAs (both passes).
// Unavailable choices fall back to 0.
cudaError_t launch_row(bool fp64, int nx, const void* descs, int ninst, int ny, int nz, int s,
                       const void* tw, int hx, cudaStream_t st, int variant = 0);
size_t row_pass_smem(bool fp64, int nx, int hx, int variant = 0);
// `tmaps`: per-instance tensor maps of the fields (CUtensorMap[ninst]) for
// the TMA-staged column pass, or nullptr for the cp.async-staged one.
cudaError_t launch_col(bool fp64, int ny, const void* descs, int ninst, int nx, const void* tw,
                       cudaStream_t st, int variant = 0, const void* tmaps = nullptr);
// The one-pass-per-step schedule (FP32, per-point table, no monitor or
// adjoint state): the row-layout pass s (even s >= 2; Lx, N, Lx) in row
// flavour `variant`, and the column-layout pass s (odd s; Ly, N, Ly); hx, hy:
// the largest heat grid of the group (0 without deposits), for the bins.
cudaError_t launch_row_step(int nx, const void* descs, int ninst, int ny, int nz, int s,
                            const void* tw, int hx, cudaStream_t st, int variant);
cudaError_t launch_col_step(int ny, const void* descs, int ninst, int nx, int nz, int s,
                            const void* tw, int hy, cudaStream_t st, int variant);
bool has_col_step_small(int n);  // the column-layout pass in 128-thread CTAs (flavour 3)
bool has_col_step_wide(int n);   // the column-layout pass in 512-thread CTAs (flavour 5)
bool has_col_step_v1(int n);     // the column-layout pass in the 8-element shape (flavour 1)
int col_tma_tile(bool fp64, int ny);
bool has_fft_variant(bool fp64, int n);
bool has_col_small(bool fp64, int n);  // row and column passes in 128/64-thread CTAs (flavours 3, 4)
bool has_col_wide(bool fp64, int n);   // the column pass in 512-thread CTAs (flavour 5)
// Kernel flavour picked for (precision, length, pass, row-pass table bit) by the autotuner:
// measured once per process on the first group that uses it, unless
// SHG_FFT_VARIANT forces one.  tune_group() must run outside stream capture.
int fft_variant(bool fp64, int n, int pass, int row_bits = 0, int ninst = 1 << 30);
// steps: the group runs one pass per step (the row- and column-layout step
// kernels are tuned then, under keys of their own; hy sizes the deposit bins).
shg_status_t tune_group(bool fp64, int nx, int ny, int nz, const void* descs, int ninst,
                        const void* tw, int hx, cudaStream_t st, const void* tmaps, int row_bits,
                        bool steps = false, int hy = 0);
// Flavour of a one-pass-per-step kernel: which = 0 the row-layout pass, 1 the
// column-layout pass.
int step_variant(bool fp64, int n, int which, int ninst);
// kRowUmap if the row passes of these plans (one grid) read the per-point
// temperature table: every plan with a map keeps one, and one z-step spans
// less than one map layer (so a pass touches at most three layers); else 0.
// With kRowUmap, also kRowLean when no plan deposits heat or monitors power.
int row_umap_bit(const std::vector<shg_plan*>& plans);
cudaError_t launch_init(bool fp64, const InitDesc* idescs, void* const* fields_unused, int ninst,
                        const void* descs, int nx, int ny, cudaStream_t st);
cudaError_t launch_power(bool fp64, const InitDesc* idescs, const void* descs, int ninst, int nx,
                         int ny, cudaStream_t st);
cudaError_t launch_build_ttab(bool fp64, const float* dT, void* ttab, int tx, int ty, int tz,
                              double dZ, const DkModel& dkm, cudaStream_t st);
// One map update of a batched temperature update (device-resident array).
struct TtabJob {
    const float* src;  // the new map [tz][ty][tx]
    float* copy;       // the plan's copy of it
    void* tt;          // the plan's (dT, C) table
    double dZ;         // layer spacing L / (tz - 1)
    DkModel dkm;       // the plan's phase-mismatch model (integrand of C)
};
cudaError_t launch_build_ttab_batch(bool fp64, const TtabJob* jobs, int njobs, int tx, int ty,
                                    int tz, cudaStream_t st);
// Per-point tables of several FP32 plans of one grid: descs[k] and umaps[k]
// are device arrays of the plans' descriptor and table pointers.
cudaError_t launch_upsample_map_batch(const void* const* descs, void* const* umaps, int n, int nx,
                                      int ny, int tz, cudaStream_t st);
cudaError_t setup_pass_attributes();
// Fill the per-point temperature table of an FP32 plan from its uploaded
// descriptor (node table, map geometry): tz layers of ny x nx (dT, C).
cudaError_t launch_upsample_map(const void* desc, void* umap, int nx, int ny, int tz,
                                cudaStream_t st);

// Whether the pass launches of the calling thread use programmatic dependent
// launch; set per enqueue by pdl_scope (SHG_PDL=0|1 overrides the choice).
extern thread_local bool pdl_enabled;
extern thread_local int launch_priority;  // priority attribute of the pass launches (0: none)
struct PdlScope {
    bool prev;
    explicit PdlScope(bool single_group) : prev(pdl_enabled) {
        const char* v = getenv("SHG_PDL");
        pdl_enabled = (v && (v[0] == '0' || v[0] == '1')) ? v[0] == '1' : single_group;
    }
    ~PdlScope() { pdl_enabled = prev; }
};

// Enqueue the whole forward propagation of instances sharing one grid.
shg_status_t enqueue_forward(bool fp64, int nx, int ny, int nz, const void* descs,
                             const InitDesc* idescs, int ninst, const void* tw,
                             const std::vector<shg_plan*>& plans, cudaStream_t st,
                             const void* tmaps = nullptr, int* status_arr = nullptr);

// Cluster-resident propagation of a single small FP32 instance (cluster_f32.cu):
// whether the plans (one plan) take it, the cluster size used for an n x n
// grid (0: none), and the launch of the whole z-march.
bool cluster_path(const std::vector<shg_plan*>& plans);
int cluster_size(int n);
cudaError_t launch_cluster(int n, const void* descs, int ninst, int nz, const void* tw,
                           cudaStream_t st);
// The cluster-resident three-wave propagation (FP32, N = 64, 128; single plans).
bool cluster3_path(const shg_plan* p);
int cluster3_size(int n);
cudaError_t launch_cluster3(int n, const void* q, int nz, const void* tw, cudaStream_t st);

// Three-wave plans (threewave.cu).
shg_status_t three_wave_alloc(shg_plan* p, const shg_crystal3_t* c, const shg_beams3_t* b);
shg_status_t build_prop_tables3(shg_plan* p, void* px, void* py);
shg_status_t upload_desc3(shg_plan* p);
shg_status_t enqueue_forward3(shg_plan* p, cudaStream_t st);
shg_status_t three_wave_powers(shg_plan* p, double out[3]);
double three_wave_input_power(const shg_plan* p);
void free_three_wave(shg_plan* p);

// Lifetime hooks: drop cached batch graphs / adjoint buffers of a plan.
void forget_plan_batches(shg_plan* p);
void free_adjoint(shg_plan* p);
void free_heat_direct(shg_plan* p);
shg_status_t heat_direct_setup(shg_plan* p);
shg_status_t heat_direct_solve(shg_plan* p, int max_iters, double tol, double* resid, int* iters,
                               cudaStream_t st);
shg_status_t adjoint_alloc(shg_plan* p);
// Enqueue the checkpoint copy of the state entering row pass R(s) (adjoint plans).
shg_status_t adjoint_checkpoint(shg_plan* p, int s, cudaStream_t st);
// The plan's phase-mismatch model with its reference temperature set to
// T_oven + T_off (no-op copy for the linearised model).
DkModel plan_dk_model(const shg_plan* p);
// Whether the checkpoints hold the forward pass of the plan's current inputs:
// set by every completed shg_propagate or shg_batch_submit (both write the
// checkpoints of adjoint plans), cleared by every change of beams,
// fields or map (no-op for plans without SHG_FLAG_ADJOINT).
void adjoint_forward_state(shg_plan* p, bool valid);

}  // namespace shg
