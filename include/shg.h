/*
 * shg.h - C ABI of the GB300 split-step Fourier SHG library (libshg.so).
 *
 * The library propagates the coupled fundamental (F) and second-harmonic (SH)
 * envelopes A_F(x,y,z), A_SH(x,y,z) of focused-Gaussian-beam SHG through a
 * chi(2) crystal, as posed in arXiv 2410.04994 ("CUDA-based focused Gaussian
 * beams second-harmonic generation efficiency calculator"):
 *
 *   coupled-wave equations ............ Sec. 2.1, Eqs. (1)-(4)
 *   focused Gaussian input ............ Eqs. (5)-(6)
 *   operator form and split step ...... Sec. 3.1, Eqs. (11)-(15)
 *   K-space diffraction ............... App. A, Eqs. (A.1)-(A.5)
 *   heat equation and its FD form ..... Sec. 2.2 Eqs. (7)-(9), Sec. 3.2 Eq. (16)
 *   self-consistent loop .............. Fig. 2 (Sec. 4.2)
 *   efficiency ........................ Eq. (17)
 *
 * Discrete map (shared with the FP64 oracle that the tests compare against):
 * every z-step of length dz = L/nz is N(dz/2) L(dz) N(dz/2); N(h) is one RK4
 * step of the pointwise three-wave right-hand side
 *     dA_F/dz  = i kF A_SH conj(A_F) e^{-i phi} - (1/2) beta_F I_F A_F + i psi_F A_F
 *     dA_SH/dz = i kS A_F^2 e^{+i phi}          - (1/2) beta_SH I_SH A_SH + i psi_SH A_SH
 * with kF = 2 pi d/(n_F lambda_F), kS = 2 pi d/(n_SH lambda_F), I = eps0 c n |A|^2/2,
 * phi = (dk0 + g T_off) z + g C(x,y,z) (C = cumulative trapezoid integral of the
 * temperature map along z, g = dDk/dT) and psi_j = (2 pi/lambda_j)(dn/dT)(dT + T_off);
 * L(dz) multiplies the 2-D spectrum by exp(-i K^2 dz/(2 k_j)) exp(-alpha_j dz/2)
 * (and by exp(-i tan(rho_j) Kx dz) with a walk-off angle rho_j).
 *
 * Conventions for every entry point:
 *   - Units are SI.  Fields are complex, stored [ny][nx] with x fastest, as
 *     float2 (default) or double2 (SHG_FLAG_FP64) pairs (re, im).
 *   - Pointers named *_dev are device pointers; the caller owns them and they
 *     are only borrowed for the duration of the call, or, for work the call
 *     leaves enqueued (asynchronous map updates, fields), until the stream
 *     has reached it.  Everything else the
 *     plan needs (fields, tables, checkpoints, scratch) is allocated by
 *     shg_plan_create / shg_set_temperature and owned by the plan.
 *   - Work is enqueued on the caller's stream (a cudaStream_t; NULL is the
 *     legacy default stream).  Calls that return host values synchronise that
 *     stream.
 *   - Every call returns a status.  Nothing exits or traps; a failed call
 *     leaves the plan usable (its state is whatever the last successful call
 *     left).
 */
#ifndef SHG_H
#define SHG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *shg_stream_t; /* == cudaStream_t */

typedef enum {
    SHG_OK = 0,
    SHG_ERR_INVALID_ARG = 1,      /* NULL pointer, non-positive size, inconsistent params */
    SHG_ERR_UNSUPPORTED_GRID = 2, /* nx, ny not powers of two in [8, 1024] (FP64: [8, 256]) */
    SHG_ERR_OOM = 3,              /* a device allocation failed */
    SHG_ERR_CUDA = 4,             /* a CUDA runtime call failed (text: shg_last_error) */
    SHG_ERR_TIMEOUT = 5,          /* a bounded device-side wait gave up */
    SHG_ERR_NONFINITE = 6,        /* a power or efficiency came out NaN/Inf */
    SHG_ERR_STATE = 7             /* call out of order (e.g. adjoint before a forward pass) */
} shg_status_t;

/* Transverse grid nx x ny over a window lx x ly (x_m = (m - nx/2) lx/nx),
 * nz steps over the crystal length, and an optional heat grid of hx x hy x hz
 * nodes including the faces (0 = no heat grid) spanning the crystal
 * [-wx/2, wx/2] x [-wy/2, wy/2] x [0, L]. */
typedef struct {
    int nx, ny, nz;
    double lx, ly;
    int hx, hy, hz;
} shg_grid_t;

/* Crystal: length L, pump wavelength lambda_F (SH at lambda_F/2), indices,
 * d_eff, linear (1/m, power) and two-photon (m/W) absorption of each wave,
 * cold mismatch dk0 (1/m), its temperature slope dDk/dT (1/(m K)), the
 * thermo-optic coefficient dn/dT (1/K, both waves), thermal conductivity
 * kappa_th (W/(m K)) and the transverse size wx x wy used by the heat grid. */
typedef struct {
    double L, lambda_f, n_f, n_sh, d_eff;
    double alpha_f, alpha_sh, beta_f, beta_sh;
    double dk0, ddk_dT, dn_dT;
    double kappa_th, wx, wy;
    /* Spatial walk-off angles rho (rad, |rho| < 1.5) of the fundamental and
     * the SH toward +x (Sec. 6 and App. B: the tan(rho) dA/dx term of the propagator,
     * for birefringently phase-matched crystals; 0 for the QPM examples):
     * each step multiplies the field's spectrum by exp(-i tan(rho) Kx dz). */
    double walkoff_f, walkoff_sh;
} shg_crystal_t;

/* Beams: pump power P1 (W), waist w0 (m), focus position z_focus (m from the
 * entrance face), oven offset T_off (K, a uniform dT), and the undepleted-pump
 * switch of Sec. 5.1 (drops only the coupling term of the pump equation). */
typedef struct {
    double p1, w0, z_focus, t_oven_offset;
    int undepleted;
} shg_beams_t;

enum {
    SHG_FLAG_FP64 = 1,    /* fields and arithmetic in double precision */
    SHG_FLAG_THERMAL = 2, /* deposit q_dot (Eq. 8) on the heat grid while propagating */
    SHG_FLAG_ADJOINT = 4, /* keep sqrt(nz)-spaced checkpoints for shg_propagate_adjoint */
    SHG_FLAG_NODE_SAMPLER = 8 /* FP32: sample the temperature map at its nodes in every pass
                                 instead of keeping a per-point table (less memory, slower) */
};

typedef struct shg_plan shg_plan_t;

/* Create a plan (Sec. 4: the field, temperature and phase-matching state of
 * the paper's solver as one object).  Validates the grid, allocates the device state and
 * the twiddle / propagator / phase tables (FP64-computed, rounded once).
 * SHG_ERR_INVALID_ARG for 1 <= nz <= 2^26 violated, for any non-finite
 * double of the three structs, or for a non-positive length, wavelength,
 * index, waist or (THERMAL) heat-grid extent; SHG_ERR_UNSUPPORTED_GRID for
 * nx, ny out of range.  On error *out is NULL. */
shg_status_t shg_plan_create(const shg_grid_t *grid, const shg_crystal_t *crystal,
                             const shg_beams_t *beams, int flags, shg_plan_t **out);

/* Release every device buffer of the plan.  NULL is accepted. */
shg_status_t shg_plan_destroy(shg_plan_t *plan);

/* Bound on the polls of each device-side wait of this plan's kernels (the
 * mbarrier waits of the TMA-staged column pass; default 2^20, about a
 * second).  A wait that runs out makes its CTA skip its tile and the next
 * shg_efficiency / shg_batch_submit return SHG_ERR_TIMEOUT; the context stays
 * usable.  0 makes every such wait give up at once (a test of that path). */
shg_status_t shg_set_wait_limit(shg_plan_t *plan, unsigned polls);

/* Replace the beam parameters (Eq. 5/6 inputs, T_off, undepleted switch) and
 * drop any fields set by shg_set_fields.  Grid and crystal are unchanged.
 * SHG_ERR_INVALID_ARG for a non-finite value, w0 <= 0 or P1 < 0. */
shg_status_t shg_set_beams(shg_plan_t *plan, const shg_beams_t *beams);

/* Temperature map dT (K, relative to the oven) on a node-centred grid
 * dT_dev[tz][ty][tx] (float, device) spanning [-t_lx/2, t_lx/2] x
 * [-t_ly/2, t_ly/2] x [0, L]; t_lx or t_ly <= 0 means the field window.
 * Copied into the plan together with its cumulative z-integral (Eq. 3,
 * trapezoid on the nodes).  tx, ty, tz >= 2.  dT_dev == NULL clears the map
 * (uniform temperature T_off).  A map of the shape and extent already
 * installed is rebuilt asynchronously: the copy from dT_dev and the table
 * kernels are enqueued on `stream`, after the plan's last propagation, and
 * the call returns without waiting (later propagations and map updates on
 * any stream wait for them); dT_dev must stay unchanged until `stream` has
 * reached them.  SHG_ERR_INVALID_ARG (tx, ty or tz < 2, a non-finite
 * extent) leaves the installed map and the adjoint checkpoints untouched.
 * Any other change synchronises.  FP32 plans without SHG_FLAG_NODE_SAMPLER also
 * keep every map layer bilinearly sampled at every field point (tz*ny*nx*8
 * bytes of device memory; the nodes are sampled in the passes instead when
 * that table would exceed 4 GiB). */
shg_status_t shg_set_temperature(shg_plan_t *plan, const float *dT_dev, int tx, int ty,
                                 int tz, double t_lx, double t_ly, shg_stream_t stream);

/* shg_set_temperature for n plans at once, with maps of one shape
 * (dT_devs[k] for plans[k], extents t_lx[k] x t_ly[k]).  The plans whose
 * installed map already has that shape and extent are rebuilt by a few
 * launches for all of them (stream-ordered, no host synchronisation, as the
 * single-plan fast path); the others are set one by one.  The host arrays
 * may be reused once the call returns; the maps must stay unchanged until
 * `stream` has reached the rebuild.  Every argument of every plan (non-NULL
 * plan and map, tx, ty, tz >= 2, finite extents) is checked before any plan
 * changes, so SHG_ERR_INVALID_ARG leaves all maps as they were.  A CUDA
 * failure part-way (SHG_ERR_CUDA / SHG_ERR_OOM) can leave the plans before
 * the failing one with the new map and the rest with the old one. */
shg_status_t shg_set_temperature_batch(shg_plan_t *const *plans, int n, const float *const *dT_devs,
                                       int tx, int ty, int tz, const double *t_lx,
                                       const double *t_ly, shg_stream_t stream);

/* Use the given fields (device, [ny][nx], the plan's precision) as the state
 * at z = 0 instead of the Gaussian pump of Eq. (6) and a zero SH.  Either
 * pointer may be NULL (zero field). */
shg_status_t shg_set_fields(shg_plan_t *plan, const void *a_f_dev, const void *a_sh_dev,
                            shg_stream_t stream);

/* Propagate z = 0 -> L (Eq. 15 marched nz times, Fig. 2 "Compute CWEs"):
 * initial fields, the fused passes and the FP64 power reductions.  The
 * passes are 2 nz + 1 (N with Lx, then Ly, per step), or nz + 1 when Lx and
 * Ly alternate their order so that one pass per step suffices (FP32 plans
 * with the per-point temperature table and no monitor or adjoint state;
 * SHG_STEP_PASSES=0 turns that off); single FP32 64^2 and
 * 128^2 plans run in one cluster-resident launch.  Asynchronous on
 * `stream`. */
shg_status_t shg_propagate(shg_plan_t *plan, shg_stream_t stream);

/* eta = P_SH(L)/P1 and the powers P_F(L), P_SH(L) (W) of the last
 * propagation (Eq. 17 with discrete powers (1/2) eps0 c n sum|A|^2 dx dy).
 * Synchronises the stream of the last propagation.  Any output may be NULL. */
shg_status_t shg_efficiency(shg_plan_t *plan, double *eta, double *p_f, double *p_sh);

/* Copy the current fields (device, [ny][nx], the plan's precision) out. */
shg_status_t shg_get_fields(shg_plan_t *plan, void *a_f_dev, void *a_sh_dev,
                            shg_stream_t stream);

/* Power monitor (Manley-Rowe balance along the crystal).  With every > 0,
 * each later propagation of the plan (single or batched) records the
 * discrete powers P_F(z_s), P_SH(z_s) = (1/2) eps0 c n_j sum |A_j|^2 dx dy
 * (Eq. 17's powers) at z_s = s dz for s = 0, every, 2 every, ... and at
 * s = nz, summed in double precision inside the row pass at the point where
 * the state is exactly at z_s.  Without losses (alpha = beta = 0) the total
 * P_F + P_SH is conserved by Eqs. (1)-(2) (Manley-Rowe), so its drift is the
 * split-step rounding error; with losses it traces the absorbed power.
 * every = 0 turns it off.  Allocates nz/every + 2 pairs of doubles; drops
 * the plan's captured graphs and the result of the last propagation.
 * SHG_ERR_INVALID_ARG for every < 0. */
shg_status_t shg_set_monitor(shg_plan_t *plan, int every);

/* The monitor's samples of the last propagation: z (m), P_F and P_SH (W)
 * for up to max_samples samples (host arrays, any may be NULL);
 * *n_samples = the number recorded.  SHG_ERR_STATE without a monitor or a
 * propagation since it was set.  Synchronises the last propagation's stream. */
shg_status_t shg_get_monitor(shg_plan_t *plan, double *z_out, double *p_f_out, double *p_sh_out,
                             int max_samples, int *n_samples);

/* Temperature model of the phase mismatch, Eq. (4):
 *   Dk(T) = (4 pi / lambda_F) (n_SH(T) - n_F(T)) - 2 pi / Lambda(T),
 *   Lambda(T) = Lambda(25 C) (1 + a_Lambda (T - 25) + b_Lambda (T - 25)^2)
 * (the paper's MgO:sPPLT expansion is a_Lambda = 2.2e-6 /K, b_Lambda =
 * -5.9e-9 /K^2), with n_j(T) = sum_k n_j[k] (T - 25 C)^k supplied by the
 * caller (the paper gives no index data).  The local temperature is
 * T = t_oven + T_off + dT(x,y,z). */
typedef struct {
    double t_oven;            /* oven temperature (deg C) */
    double lambda25;          /* grating period Lambda(25 C) (m), > 0 */
    double a_lambda, b_lambda;
    double n_f[4], n_sh[4];   /* index polynomials in (T - 25 C) */
} shg_qpm_t;

/* Use Eq. (4) for the phase (model != NULL) instead of the linearised
 * dk0 + dDk/dT (dT + T_off), or return to the latter (NULL).  With the model,
 * phi = Dk(T_ref) z + C'(x,y,z), T_ref = t_oven + T_off, where C' is the
 * trapezoid cumulative integral along z of Dk(T_ref + dT) - Dk(T_ref) on the
 * map's nodes (in double precision), interpolated like the map; the crystal's
 * dk0 and dDk/dT are then unused (the thermal lens keeps dn/dT).  The map
 * tables depend on T_off, so shg_set_beams rebuilds them.  The adjoint
 * differentiates the same map (the node gradients carry dDk/dT at each node's
 * temperature).  SHG_ERR_INVALID_ARG for a non-finite value or
 * lambda25 <= 0. */
shg_status_t shg_set_phase_model(shg_plan_t *plan, const shg_qpm_t *model);

/* Reverse sweep of the exact discrete forward map (conjugate propagator,
 * transposed RK4 with Wirtinger calculus), seeded with d_eta = dJ/deta, using
 * the sqrt(nz) checkpoints of the last propagation (shg_propagate or
 * shg_batch_submit; needs SHG_FLAG_ADJOINT).
 * Outputs d_eta * deta/dw0, deta/dz_focus, deta/dT_off (host doubles) and
 * deta/d(dT node) into g_dT_dev[tz][ty][tx] (device float, may be NULL).
 * Grid and window are held fixed.  SHG_ERR_STATE if the plan has no
 * adjoint state, or if its beams, fields or map changed after the last
 * propagation (the checkpoints would belong to other inputs).
 * Synchronises `stream`. */
shg_status_t shg_propagate_adjoint(shg_plan_t *plan, double d_eta, double *g_w0,
                                   double *g_zf, double *g_toven, float *g_dT_dev,
                                   shg_stream_t stream);

/* Propagate n independent plans together (a focusing / power / oven sweep):
 * the plans are grouped by grid, and the whole sweep runs as one CUDA-graph
 * launch (captured on first use of this plan set and reused).  Writes
 * eta_host_out[n] and synchronises `stream`.  SHG_ERR_INVALID_ARG for a
 * NULL or repeated plan (as for shg_set_temperature_batch and
 * shg_pass_times). */
shg_status_t shg_batch_submit(shg_plan_t *const *plans, int n, double *eta_host_out,
                              shg_stream_t stream);

/* Solve kappa lap dT = -q_dot (Eq. 7/16 with the faces of
 * shg_set_heat_boundary) on the heat grid, warm-started from the previous
 * solution, from the q_dot deposited by the last THERMAL propagation, until
 * the largest Jacobi correction is below tol (K) or max_sweeps sweeps
 * (SOR) or refinement passes (direct; see shg_set_heat_method).  The SOR
 * checks the correction every 8 sweeps, so up to 7 sweeps may follow the
 * first converged one.  Installs dT as the plan's temperature map.  Returns
 * the final correction and the sweep or pass count.  Synchronises `stream`. */
shg_status_t shg_heat_solve(shg_plan_t *plan, int max_sweeps, double tol, double *resid,
                            int *sweeps, shg_stream_t stream);

/* Boundary of each face of the heat grid, in the order x-, x+, y-, y+, z-, z+
 * (kinds[6]): SHG_FACE_OVEN holds the face at T_oven (dT = 0, Eq. 9);
 * SHG_FACE_CONVECTIVE cools it by free convection, -kappa dT/dn = h (T - T_inf)
 * (Eq. 10), with h[k] >= 0 (W/(m^2 K); h may be NULL for 0) and the ambient
 * temperature T_inf = T_oven + t_inf.  A convective face node is an unknown
 * whose stencil uses a ghost node beyond the face eliminated by the central
 * difference of Eq. (10); its source density uses its half-size cell.  A node
 * on an oven face is held even where it also lies on a convective face.
 * The paper's arrangements: all faces in the oven, the four side faces in
 * the oven with the end facets in air (setOvenSurrounded), or one oven under
 * the y- face (setBottomOvens).  Default: all oven-held.  Resets the solved
 * dT to 0.  SHG_ERR_INVALID_ARG for another kind, a negative or non-finite h,
 * every face convective with h = 0 (no steady state), or convective faces
 * with the SOR method; SHG_ERR_STATE without SHG_FLAG_THERMAL. */
enum { SHG_FACE_OVEN = 0, SHG_FACE_CONVECTIVE = 1 };
shg_status_t shg_set_heat_boundary(shg_plan_t *plan, const int *kinds, const double *h,
                                   double t_inf);

/* Method of shg_heat_solve and shg_thermal_loop:
 *   SHG_HEAT_DIRECT (default): the operator of Eq. (16) is a Kronecker sum of
 *     three 1-D operators, so it is solved directly: FP32 transforms to the
 *     eigenbases of the x and y operators (computed by Jacobi rotations on
 *     the host when the plan is created and when the boundary changes, tens of
 *     milliseconds at 128 nodes per axis), one tridiagonal solve along z per
 *     transverse mode, transforms back, repeated as FP64 iterative refinement
 *     of dT until the largest Jacobi correction is below tol (max_sweeps
 *     bounds the refinement passes, at most 50; the solves report passes).
 *   SHG_HEAT_SOR: red-black SOR in FP64 (every face oven-held only).
 * Both converge to the same discrete solution. */
enum { SHG_HEAT_DIRECT = 0, SHG_HEAT_SOR = 1 };
shg_status_t shg_set_heat_method(shg_plan_t *plan, int method);

/* The self-consistent loop of Fig. 2 with n_outer fixed iterations:
 * q_dot = 0 -> dT -> (Dk, lens) -> propagate (depositing q_dot) -> ...
 * eta_out[i] and change_out[i] = max|dT_i - dT_{i-1}| per iteration (host
 * arrays of n_outer doubles, may be NULL).  Needs SHG_FLAG_THERMAL. */
shg_status_t shg_thermal_loop(shg_plan_t *plan, int n_outer, int max_sweeps, double tol,
                              double *eta_out, double *change_out, shg_stream_t stream);

/* Heat-grid state for inspection: the deposited heat per node q_dev (W, the
 * sum of q_dot dV, double [hz][hy][hx]) and the last solved dT (solved in
 * double, returned rounded to float).  Either pointer may be NULL. */
shg_status_t shg_get_heat(shg_plan_t *plan, double *q_dev, float *dT_dev,
                          shg_stream_t stream);

/* Profiling aid.  Runs `nsteps` z-steps of the plans' row and column passes
 * eagerly (not from a graph) on `stream`, grouped by grid as in
 * shg_batch_submit, with a CUDA event pair around every launch.  For group g
 * (g < *ngroups <= max_groups) it writes out[5g..5g+4] = {nx, ny, average
 * row-pass ms, average column-pass ms, passes per step (1 or 2)} and
 * inst_out[g] = instances in the
 * group.  The passes timed are those the group's propagation runs: for a
 * group on the one-pass-per-step schedule (FP32, per-point temperature
 * table, no monitor or adjoint state; nz >= 3), the row-layout
 * pass (Lx, N, Lx) and the column-layout pass (Ly, N, Ly); otherwise the
 * row pass (N, Lx) and the column pass (Ly).  A group not tuned yet in this process is tuned first (outside
 * the event pairs).  The plans' fields are advanced (use shg_propagate or
 * shg_batch_submit afterwards for a clean result).  SHG_ERR_INVALID_ARG for
 * n <= 0, nsteps <= 0, max_groups <= 0, NULL outputs, or more groups than
 * max_groups.  Synchronises `stream`. */
shg_status_t shg_pass_times(shg_plan_t *const *plans, int n, int nsteps, double *out,
                            int *inst_out, int max_groups, int *ngroups, shg_stream_t stream);

/* Measurement aid (Sec. 4.3 reports speed-ups only; a roofline needs the
 * device's own ceilings).  Times, with CUDA events on `stream`, best of 5
 * launches after a warm-up:
 *   fp32_tflops: packed two-lane FP32 FMAs (fma.rn.f32x2), 8 independent
 *                chains per thread, 8 CTAs of 256 threads per SM, in TFLOP/s
 *                (an FMA counts 2 flops);
 *   fp32_scalar_tflops: the same with scalar FMAs;
 *   fp64_tflops: scalar double-precision FMAs, 8 chains per thread;
 *   l2_read_gbs: 16 re-reads of a 32 MiB buffer (resident in L2) with
 *                16-byte L2-only loads, in GB/s.
 * Any output may be NULL (not all).  Allocates and frees its buffers on
 * `stream` (stream-ordered allocator); changes no clock or device setting.
 * Synchronises `stream`. */
shg_status_t shg_measure_peaks(double *fp32_tflops, double *l2_read_gbs,
                               double *fp32_scalar_tflops, double *fp64_tflops,
                               shg_stream_t stream);

/* Powers P_F, P_SH = (1/2) eps0 c n_j sum |A_j|^2 dx dy of fields the caller
 * already holds, written to memory the caller already holds, with no device
 * allocation.  This is a library convenience with no counterpart in the
 * paper: it serves callers that may not call cudaMalloc (a host framework
 * with a fixed device-memory budget, or a latency-critical loop where an
 * allocation could wait on the device or fail).
 *   fields_dev: n_inst instances, each [2][ny][nx] (A_F then A_SH), float2, or
 *               double2 if fp64 != 0, contiguous, device.
 *   powers_dev: n_inst x {P_F, P_SH} doubles (W), device.
 *   lx, ly: window (dx = lx/nx, dy = ly/ny); n_f, n_sh: refractive indices.
 * The partial sums live in one static device array of the library
 * (1024 instances x 32 blocks x 2 doubles = 512 KiB), which every GPU that
 * loads the library holds until the process exits; n_inst > 1024 is rejected
 * with SHG_ERR_INVALID_ARG.  Each call overwrites every partial it reads, so
 * nothing carries over between calls, but calls that overlap on the GPU
 * (other streams, other threads) race on the array and must be serialised.
 * The first call on a device looks up the array's device address (and loads
 * the library's device code if that has not happened yet): make that first
 * call before any stream capture.  Asynchronous on `stream`. */
shg_status_t shg_field_powers_noalloc(const void *fields_dev, int nx, int ny, int n_inst,
                                      int fp64, double lx, double ly, double n_f,
                                      double n_sh, double *powers_dev, shg_stream_t stream);

/* ---- Three-wave mixing (sum- and difference-frequency generation) ----
 * The paper closes (Sec. 6) with the coupled-wave model as a starting point
 * for other three-wave processes.  A three-wave plan propagates three fields
 * at omega_3 = omega_1 + omega_2 with the split step of Eq. (15):
 *   dA1/dz = i k1 A3 conj(A2) e^{-i phi} - (1/2) beta1 I1 A1 + i psi1 A1
 *   dA2/dz = i k2 A3 conj(A1) e^{-i phi} - (1/2) beta2 I2 A2 + i psi2 A2
 *   dA3/dz = i k3 A1 A2 e^{+i phi}       - (1/2) beta3 I3 A3 + i psi3 A3
 * with k_j = 2 pi d_eff / (n_j lambda_j), lambda3 = 1 / (1/lambda1 + 1/lambda2),
 * I_j = eps0 c n_j |A_j|^2 / 2, phi and psi_j as for SHG (dk0 + g (T_off + dT),
 * lens (2 pi / lambda_j) dn/dT (dT + T_off)), and each wave's own diffraction,
 * absorption alpha_j and walk-off rho_j in K-space.  Sum-frequency generation
 * starts with P1, P2 > 0 and P3 = 0; difference-frequency generation with a
 * pump at omega_3 and a seed at omega_2 (P1 = 0).  With lambda1 = lambda2,
 * n1 = n2 and A1 = A2 the equations are those of SHG (k3 = 2 k_SH). */
typedef struct {
    double L, lambda1, lambda2;   /* crystal length, input wavelengths (m) */
    double n1, n2, n3, d_eff;
    double alpha[3], beta[3];     /* per wave: 1/m (power), m/W */
    double dk0, ddk_dT, dn_dT;
    double walkoff[3];            /* rad, |rho| < 1.5 */
} shg_crystal3_t;

typedef struct {
    double p[3], w0[3], z_focus[3];  /* per wave: power (W, >= 0), waist, focus (Eq. 5) */
    double t_oven_offset;
    int undepleted;                  /* drop the coupling terms of waves 1 and 2 */
} shg_beams3_t;

/* Create a three-wave plan.  flags: 0 or SHG_FLAG_FP64 (no heat grid,
 * adjoint or sampler flags).  The plan accepts shg_set_temperature (and the
 * batched form), shg_propagate, shg_efficiency (eta = P3(L) / sum of the input
 * powers, *p_f = P1(L), *p_sh = P3(L)), shg_powers, shg_get_field, shg_set_wait_limit
 * and shg_plan_destroy; the calls of the SHG-specific state (beams, fields,
 * monitor, phase model, adjoint, heat, batches, pass timing) return
 * SHG_ERR_INVALID_ARG or SHG_ERR_STATE.  SHG_ERR_INVALID_ARG for a non-finite
 * value, a non-positive length, wavelength, index or waist, a negative
 * power, no input power, or another flag.
 * Propagation: FP32 plans on a 64 x 64 or 128 x 128 grid run the whole
 * z-march in one thread-block-cluster launch (the fields resident in the
 * cluster's shared memory; a map through the per-point table, when one step
 * spans less than one map layer); other plans run a row pass and a column
 * pass per step (the map sampled at its nodes).  SHG_CLUSTER=0 in the
 * environment selects the passes for every plan. */
shg_status_t shg_plan_create_3w(const shg_grid_t *grid, const shg_crystal3_t *crystal,
                                const shg_beams3_t *beams, int flags, shg_plan_t **out);

/* Copy field j (0-based: 0 = A_F, 1 = A_SH of an SHG plan; 0, 1, 2 = A1, A2,
 * A3 of a three-wave plan) of the current state to a device buffer of
 * ny x nx complex values of the plan's precision. */
shg_status_t shg_get_field(shg_plan_t *plan, int j, void *dev, shg_stream_t stream);

/* Discrete powers of the last propagation's fields (W): out[0..n) with n >= 2
 * (SHG: P_F, P_SH) or n >= 3 (three-wave: P1, P2, P3).  Synchronises. */
shg_status_t shg_powers(shg_plan_t *plan, double *out, int n);

/* Static description of a status code. */
const char *shg_status_string(shg_status_t status);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char *shg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SHG_H */
