/*
 * libemt -- EMTP-type electromagnetic-transient time loop on one B300 GPU.
 *
 * C ABI.  All arguments are plain pointers and sizes; no C++ or PyTorch
 * types cross this boundary.  Every call returns an emt_status; no
 * exception or abort crosses it.  One context per host thread.
 *
 * The computation is the fixed-step nodal-analysis loop of the EMTP-type
 * algorithm the CloudPSS paper builds on (Sec. III-A, its four basic
 * processes: update Norton equivalents, update nodal injections, factorise
 * the conductance matrix, solve for the node voltages; formulas from its
 * ref. [2]).  Here the factorisation is an explicit inverse G^-1 computed
 * once per subsystem and switch state, and lossless Bergeron lines cut the
 * network into subsystems that exchange history currents one or more steps
 * late.
 *
 * Node codes in every node argument:
 *   k >= 0       unknown node k (0 <= k < n_nodes)
 *   k == -1      ground
 *   k == -2 - s  known-voltage node of source s: v = A_s sin(2 pi f_s t + phi_s)
 *
 * Time: step n = 1, 2, ... is at t_n = n dt.  The loop starts de-energised
 * (all voltages, history currents and line histories zero; source voltages
 * count as zero at n = 0).
 */
#ifndef EMT_H
#define EMT_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EMT_OK = 0,
  EMT_EINVAL = 1,     /* invalid argument or network description */
  EMT_ESINGULAR = 2,  /* a subsystem conductance matrix is singular */
  EMT_ENOMEM = 3,     /* device or host allocation failed */
  EMT_ECUDA = 4,      /* a CUDA runtime call failed (message in emt_last_error) */
  EMT_ETIMEOUT = 5,   /* a device wait for another subsystem's line values ran out */
  EMT_ERESOURCE = 6,  /* the persistent launch cannot be co-resident / too large */
  EMT_ESTATE = 7      /* call out of order (e.g. step before prefactor) */
} emt_status;

typedef struct emt_ctx emt_ctx;  /* opaque; owns all device memory it allocates */

/* Network description.  All arrays are caller-owned and COPIED by
 * emt_build_network; they may be freed afterwards.
 *
 * Branches (R, L or C, one element each; trapezoidal companion model):
 *   br_k, br_m: end nodes (node codes; not both known, k != m)
 *   br_kind: 0 = R (ohm), 1 = L (henry), 2 = C (farad); br_value > 0
 * Sources: src_amp (peak volts), src_phase (rad), src_freq (Hz).
 * Lossless Bergeron lines: ln_k, ln_m unknown nodes, ln_zc > 0 (ohm),
 *   ln_delay >= 1 (travel time in whole steps).
 * Switches (ideal resistors while closed): sw_k, sw_m (unknown node or
 *   ground), sw_r > 0 (ohm); closed for sw_close_step <= n < sw_open_step,
 *   sw_open_step = -1 never opens, sw_close_step = -1 never closes.
 * Runtime switches (n_rswitches may be 0): two-state resistors, rs_ron
 *   while on and rs_roff while off (both > 0), between rs_k and rs_m
 *   (unknown node or ground), whose state in force at step n is decided
 *   from step n-1's solution (the state at step 1 is rs_on0):
 *     rs_kind 0, diode (anode rs_k, cathode rs_m): on iff v_k - v_m > 0;
 *     rs_kind 1, breaker: on until, at a step n >= rs_trip_step, its
 *       current (v_k - v_m) / rs_ron changes sign from step n-1 (product
 *       <= 0); off from step n+1 on, for good (rs_on0 is ignored: on).
 *   The paper's process 3 at run time (Sec. III-A): each subsystem with k
 *   runtime switches gets a prefactored G^-1 for every one of its 2^k
 *   states (k <= 8 per subsystem), and the time loop switches matrices
 *   when a state changes (with a scenario set: per scenario, every
 *   scenario matrix variant having its 2^k states); emt_adjoint
 *   differentiates with the decisions the forward run took held fixed.
 * Coupled three-phase lossless lines in modal form (n_clines may be 0):
 *   cl_k[3 l + p] / cl_m[3 l + p]: phase p's node (unknown) at each end;
 *   cl_tv[9 l + 3 p + j]: T_v, phase voltages = T_v modal voltages (modal
 *   currents use T_i = T_v^-T); cl_z[3 l + j], cl_tau[3 l + j]: mode j's
 *   Z_c (ohm) and travel time (s, >= dt, any real value).  Each end draws
 *   i_p = Y_p v_p + T_i I_mode with Y_p = T_i diag(1/Z) T_v^-1; mode j sends
 *   c_j(n) = -(2/Z_j) v_mode_j(n) - I_mode_j(n), and the far end's history
 *   is (1 - f) c(n - d) + f c(n - d - 1), tau = (d + f) dt, d = floor(tau/dt)
 *   (linear interpolation of the travel time).  An end's three phase nodes
 *   are one subsystem.  Scenario sets take them; emt_adjoint
 *   differentiates through them (their own Z, T_v and travel times are not
 *   parameters).
 * Control system (n_cblocks may be 0): the paper's control components as
 *   basic processes of its computation graph (Sec. III-A), layered into a
 *   directed acyclic graph whose layers run one after another (Sec. III-B).
 *   Block b: type cb_type[b], inputs cb_in0[b], cb_in1[b] (block indices;
 *   -1 where the type has no such input), parameters cb_p0[b], cb_p1[b]
 *   (finite), u0 / u1 its input values:
 *     0 CONST  y = p0                 5 LIMIT  y = min(max(u0, p0), p1), p0 <= p1
 *     1 MEAS   y = v(cb_node[b])      6 INTEG  y = y(n-1) + p0 (dt/2)(u0 + u0(n-1))
 *     2 GAIN   y = p0 u0              7 LAG    p0 / (1 + s p1), p1 > 0, trapezoidal:
 *     3 SUM    y = p0 u0 + p1 u1               y = a y(n-1) + b (u0 + u0(n-1)),
 *     4 MUL    y = p0 u0 u1                    a = (2 p1 - dt)/(2 p1 + dt),
 *     8 PI     y = p0 u0 + p1 I,               b = p0 dt / (2 p1 + dt)
 *              I = I(n-1) + (dt/2)(u0 + u0(n-1))
 *   (MEAS: cb_node an unknown node; states start at 0).  At step n, after
 *   v(n) is solved, the blocks act in index order: an input from a block of
 *   lower index sees its step-n output, one from a block of equal or higher
 *   index its step-(n-1) output (0 at step 1); that is how algebraic loops
 *   are broken.  Controlled current injections (n_cinj may be 0): the
 *   output of block ci_block[c] at step n enters unknown node ci_node[c]
 *   at step n + 1 (0 at step 1).  Every connected group of blocks, with the
 *   nodes it measures and drives, lies in one subsystem (a block group that
 *   touches no node runs in subsystem 0).  A scenario set may give blocks
 *   their own p0 per scenario (emt_scenario_desc).  Not supported by
 *   emt_adjoint.
 * Frequency-dependent lines (n_fdlines may be 0), one conductor each, ends
 *   fl_k / fl_m (unknown nodes, cut into different subsystems like any
 *   line): characteristic admittance and propagation function as
 *   pole-residue sums, up to 4 real poles each in slots [4 l + i] (unused
 *   slots ignored):
 *     Y_c(s) = fl_y0 + sum_{i < fl_ny} fl_yc_i / (s - fl_yq_i),
 *     A(s)   = e^{-s tau} (fl_a0 + sum_{i < fl_na} fl_ar_i / (s - fl_ap_i)),
 *   poles < 0, fl_y0 >= 0, tau = fl_tau >= dt (s, any real value).  Each
 *   pole term is discretised by the trapezoidal rule, x(n) = lam x(n-1) +
 *   mu (u(n) + u(n-1)), lam = (1 + p dt/2)/(1 - p dt/2), mu = r (dt/2)/
 *   (1 - p dt/2).  An end e (far end f) draws i_e(n) = yc_e(n) - b_e(n)
 *   with yc = Y_c applied to its voltage and b_e(n) = A applied to W_f,
 *   W_f(n) = (1 - phi) w_f(n - d) + phi w_f(n - d - 1), tau = (d + phi) dt,
 *   w_f(m) = 2 yc_f(m) - b_f(m): it stamps G_eq = fl_y0 + sum mu (> 0
 *   required) and draws a history current from the previous step.  With
 *   fl_y0 = 1/Z, fl_a0 = 1, no poles and tau = d dt this is the Bergeron
 *   line above.  Not supported by emt_adjoint.
 * Nonlinear resistors (n_nonlin may be 0), solved by the compensation
 *   method (the paper's process 3 at run time, Sec. III-A): element x between
 *   nl_k and nl_m (unknown node or ground, not both ground) carries
 *   i = f(v_k - v_m), f odd and piecewise linear through (0, 0) and
 *   (nl_v[8 x + j], nl_i[8 x + j]), j < nl_np[x] <= 8, 0 < v_1 < v_2 < ...,
 *   0 <= i_1 <= i_2 <= ..., continued past the last point with the last
 *   slope.  Each step solves the subsystem without the element (v0), takes
 *   the element's Thevenin source v_th = v0_k - v0_m behind R_th = z_k - z_m,
 *   z = G^-1 (e_k - e_m) (prefactored with G^-1 for every switch state), solves
 *   i = f(v_th - R_th i) exactly on the right segment and sets v = v0 - z i.
 *   At most one per subsystem (the element joins its two ends into one
 *   subsystem).  With a scenario set each scenario solves it against its
 *   own matrices.  Not supported by emt_adjoint. */
typedef struct {
  double dt;
  int64_t n_nodes;
  int64_t n_branches;
  const int32_t* br_k;
  const int32_t* br_m;
  const uint8_t* br_kind;
  const double* br_value;
  int64_t n_sources;
  const double* src_amp;
  const double* src_phase;
  const double* src_freq;
  int64_t n_lines;
  const int32_t* ln_k;
  const int32_t* ln_m;
  const double* ln_zc;
  const int32_t* ln_delay;
  int64_t n_switches;
  const int32_t* sw_k;
  const int32_t* sw_m;
  const double* sw_r;
  const int64_t* sw_close_step;
  const int64_t* sw_open_step;
  int64_t n_rswitches;
  const int32_t* rs_k;
  const int32_t* rs_m;
  const uint8_t* rs_kind;
  const double* rs_ron;
  const double* rs_roff;
  const uint8_t* rs_on0;
  const int64_t* rs_trip_step;
  int64_t n_clines;
  const int32_t* cl_k;
  const int32_t* cl_m;
  const double* cl_tv;
  const double* cl_z;
  const double* cl_tau;
  int64_t n_cblocks;
  const uint8_t* cb_type;
  const int32_t* cb_in0;
  const int32_t* cb_in1;
  const int32_t* cb_node;
  const double* cb_p0;
  const double* cb_p1;
  int64_t n_cinj;
  const int32_t* ci_block;
  const int32_t* ci_node;
  int64_t n_fdlines;
  const int32_t* fl_k;
  const int32_t* fl_m;
  const double* fl_tau;
  const double* fl_y0;
  const int32_t* fl_ny;
  const double* fl_yq;
  const double* fl_yc;
  const double* fl_a0;
  const int32_t* fl_na;
  const double* fl_ap;
  const double* fl_ar;
  int64_t n_nonlin;
  const int32_t* nl_k;
  const int32_t* nl_m;
  const int32_t* nl_np;
  const double* nl_v;
  const double* nl_i;
  /* Frequency-dependent line groups (n_fdgroups may be 0; appended here so
   * that descriptions without them keep their layout): three of the
   * frequency-dependent lines above carry the modes of one three-phase line.
   * fg_line[3 g + j] is the line of mode j, whose ends are phase j's nodes
   * (the three end-k nodes lie in one subsystem, as do the end-m ones);
   * fg_tv[9 g + 3 p + j]: T_v, phase voltages = T_v modal voltages (modal
   * currents: T_i = T_v^-T).  Mode j's Y_c acts on the modal voltage
   * (T_v^-1 v_phase)_j, its w and b as for one conductor; each end stamps
   * T_i diag(G_eq) T_v^-1 and draws T_i times the modal history currents.
   * A line belongs to at most one group.  Scenario sets take them; not
   * supported by emt_adjoint. */
  int64_t n_fdgroups;
  const int32_t* fg_line;
  const double* fg_tv;
} emt_network_desc;

/* Optional per-scenario overrides of one base network (the paper's
 * multi-scenario studies, Sec. III-B / IV-C).  NULL pointer fields mean
 * "same as the base network".  All arrays are caller-owned and copied.
 *   src_amp, src_phase: [n_scenarios][n_sources] row-major
 *   rm_branch_ptr[n_scenarios+1], rm_branch[]: branches removed per scenario
 *   rm_line_ptr[n_scenarios+1], rm_line[]:     lines removed per scenario
 *   sw_ptr[n_scenarios+1], sw_k[], sw_m[], sw_r[], sw_close_step[],
 *     sw_open_step[]: switches added per scenario (same rules as above).
 *   cbo_ptr[n_scenarios+1], cbo_block[], cbo_p0[]: control blocks whose
 *     parameter p0 a scenario sets (block index, finite value; a block at
 *     most once per scenario; for a LIMIT the new lower bound must not
 *     exceed p1), e.g. a set point per scenario.  NULL: none.
 * Scenario sets take every element kind (rm_line names lossless lines
 * only); each scenario keeps its own runtime-switch states. */
typedef struct {
  int64_t n_scenarios;
  const double* src_amp;
  const double* src_phase;
  const int64_t* rm_branch_ptr;
  const int32_t* rm_branch;
  const int64_t* rm_line_ptr;
  const int32_t* rm_line;
  const int64_t* sw_ptr;
  const int32_t* sw_k;
  const int32_t* sw_m;
  const double* sw_r;
  const int64_t* sw_close_step;
  const int64_t* sw_open_step;
  const int64_t* cbo_ptr;
  const int32_t* cbo_block;
  const double* cbo_p0;
} emt_scenario_desc;

/* Validate the description, split the network into subsystems (connected
 * components over branches and switches; lines are the cuts), number the
 * nodes subsystem by subsystem and upload the network to the current CUDA
 * device.  `scen` may be NULL (one scenario).  On success *out owns the
 * context; on failure *out is NULL (message via emt_last_error(NULL)). */
emt_status emt_build_network(const emt_network_desc* desc, const emt_scenario_desc* scen, emt_ctx** out);

/* Process 3 of Sec. III-A, done once: on the device, assemble each
 * subsystem's conductance matrix G (companion conductances g = 1/R,
 * dt/(2L), 2C/dt; 1/Z_c per line end; 1/R per closed switch) for every
 * switch state it meets and store G^-1 (Gauss-Jordan with partial pivoting
 * plus a Newton step whose residual is summed in twice the working
 * precision) as a double matrix plus its single-precision remainder, so
 * each solve applies G^-1 to well beyond double rounding.  Synchronous.
 * ESINGULAR names the subsystem. */
emt_status emt_prefactor(emt_ctx* ctx);

/* The same computation as emt_prefactor, without any device allocation: the
 * workspace emt_prefactor obtains from cudaMalloc (matrix lists, per-matrix
 * status, a copy of G and the Newton residual for every matrix) lives in a
 * fixed device array built into the library instead.  It is for callers
 * that must not allocate device memory when they refactorise, having built
 * the context beforehand: a service that reserves all device memory up
 * front and hands it out itself, or a loop that cannot take cudaMalloc's
 * implicit device synchronisation or risk its failure half-way through a
 * run.  The paper has no counterpart; it is a deployment convenience.
 *   Limit: at most 16383 matrices (subsystems x switch states) and 491,520
 *   solve-matrix entries (the "solve matrix" is n x (n + strong columns) per
 *   matrix); larger networks get EINVAL with a message (use emt_prefactor).
 *   The fixed array (about 7.7 MiB) is held on every device that loads the
 *   library until the process exits.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) and keeps it for the life of the process; make
 *   that first call before any stream capture.  A cudaDeviceReset frees the
 *   array with everything else on the device (every emt_ctx included), so
 *   the library is not usable on that device after a reset.
 *   The context's device must be current.  Single-scenario contexts only
 *   (EINVAL otherwise).  ESINGULAR names the subsystem, as emt_prefactor.
 *   Runs on `cuda_stream` and synchronises it.  It rewrites the context's
 *   solve matrices on that stream: order it after every earlier emt_step_n
 *   or emt_adjoint of the context issued on other streams (an event the
 *   stream waits on, or a synchronisation).  All calls share the one array:
 *   calls that overlap on the GPU (other threads, other streams, other
 *   contexts) race and must be serialised. */
emt_status emt_prefactor_noalloc(emt_ctx* ctx, void* cuda_stream);

/* Choose the recorded node voltages ("waveform channels", Sec. II-A):
 * channels = node ids (NULL = all nodes in order), every `decim`-th step
 * (steps decim, 2 decim, ...), room for `max_rows` recorded steps per
 * scenario.  Allocates the device record buffer; n_ch = 0 stops recording. */
emt_status emt_set_recording(emt_ctx* ctx, const int32_t* channels, int64_t n_ch, int32_t decim, int64_t max_rows);

/* Advance n_steps steps from the current step (resumable), asynchronously on
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream).  A source
 * kernel tabulates v_src(t_n) for the steps, then one persistent launch
 * runs them: each CTA owns a subsystem, keeps G^-1 and all element data in
 * shared memory, and meets other subsystems only through the line rings,
 * whose slots carry the step they belong to (no grid barrier, no flags).
 * A wait for line values exceeding its time budget latches an error that
 * emt_sync or the next call returns.
 * With a scenario set the whole study advances in one launch of the
 * multi-scenario kernel (one CTA per tile of scenarios, no waits between
 * CTAs), issued through a CUDA graph that is built once per launch shape
 * and whose kernel arguments are updated per call. */
emt_status emt_step_n(emt_ctx* ctx, int64_t n_steps, void* cuda_stream);

/* Copy recorded waveforms out.  channels: node ids that were recorded;
 * rows for steps step0, step0+decim, ... (n_rows of them; step0 a positive
 * multiple of decim); scenarios scen0 .. scen0+n_scen-1.
 * out: [n_rows][n_scen][n_ch] doubles, caller-owned, device memory if
 * out_on_device != 0 else host memory.  Every recorded channel in recording
 * order, over all scenarios (or one row), is one plain copy of the record
 * buffer; other requests gather on the device first.  Synchronous. */
emt_status emt_read_waveforms(emt_ctx* ctx, const int32_t* channels, int64_t n_ch, int64_t step0, int64_t n_rows,
                              int64_t scen0, int64_t n_scen, double* out, int32_t out_on_device);

/* emt_read_waveforms, stream-ordered: enqueues the gather (and, for a host
 * `out`, the device-to-host copy) on `cuda_stream` (NULL: the legacy
 * default stream) and returns without waiting, so that reading the rows of
 * one chunk of steps overlaps the run of the next.  The rows must be
 * recorded by steps enqueued before it on `cuda_stream`, or ordered before
 * it by the caller (an event the stream waits on); emt_step_n counts steps
 * as enqueued, so the bounds checks are those of emt_read_waveforms.  A
 * host `out` must be page-locked for the copy to run asynchronously, and
 * stays in use until the stream reaches this point; the temporary device
 * buffers are stream-ordered allocations.  Device errors of the steps
 * (wait timeouts) surface on emt_sync. */
emt_status emt_read_waveforms_async(emt_ctx* ctx, const int32_t* channels, int64_t n_ch, int64_t step0,
                                    int64_t n_rows, int64_t scen0, int64_t n_scen, double* out,
                                    int32_t out_on_device, void* cuda_stream);

/* Control block outputs of the last completed step (all 0 at step 0):
 * y[b] for b = 0 .. n_cblocks-1 in the caller's block order; n must equal
 * n_cblocks.  y is device memory if on_device != 0 else host memory.
 * Synchronous.  EINVAL for a context built with a scenario set. */
emt_status emt_read_controls(emt_ctx* ctx, double* y, int64_t n, int32_t on_device);

/* Pick the launch shape of the multi-scenario kernel by measurement: for
 * scenarios per CTA S_t (about k CTAs per SM for k = 1..6, and the powers
 * of two up to 32, where the subsystem groups fit in shared memory) and
 * 256, 512 or 1024 threads per CTA, run `trial_steps` steps from the
 * de-energised state on `cuda_stream` and keep the fastest; unless
 * "digit_solve" was set, both forms of the solve are timed (FP64, and the
 * tensor-core digit form when a solve matrix qualifies) and the faster
 * one is kept (emt_get_info "digit_solve" reports it).  Resets the
 * context to step 0 afterwards.  A context without a scenario set has no
 * tunable shape (EMT_OK, nothing changes).  The chosen shape is reported by
 * emt_get_info ("scenarios_per_cta", "batch_threads"); it can also be set
 * with emt_set_option.  Synchronous. */
emt_status emt_autotune(emt_ctx* ctx, int64_t trial_steps, void* cuda_stream);

/* Discrete adjoint: the loss J = sum_{n=1..N} sum_k (v_n[k] - v*_n[k])^2
 * over all node voltages of steps 1..N from the de-energised state, and
 * its exact gradient (reverse-mode of the discrete time loop, not of the
 * continuous equations) with respect to every branch value and source
 * amplitude.  Switch times, Z_c and line delays are fixed, not parameters.
 * The paper's fixed-step loop (Sec. III-A, processes 1-4) is run backwards:
 * w_n = G_n^-T vbar_n with G symmetric, so the same prefactored G^-1 serves
 * both directions.
 *   v_target:   [n_steps][n_nodes] doubles, caller's node order (v*_n in
 *               row n-1); treated as constant.
 *   ckpt_every: K >= 1: the forward state (history currents and line
 *               rings) is stored every K steps and each segment is run
 *               forward again before its reverse sweep (memory ~ N/K
 *               states + K x n_nodes tape); K = 0: the whole tape v_n is
 *               kept (N x n_nodes doubles), nothing is recomputed.  Both
 *               give bit-identical results.
 *   grad:       [n_branches + n_sources] doubles, or NULL: dJ/d(br_value[b])
 *               in the caller's branch order, then dJ/d(src_amp[s]).
 *   loss:       host double, or NULL (not both NULL).
 *   on_device:  non-zero: v_target and grad are device memory; else host.
 *   cuda_stream: stream for the launches (NULL: legacy default stream).
 * With runtime switches the reverse sweep uses the states the forward run
 * decided (the forward re-runs record them per step), i.e. the gradient of
 * the smooth piece of J the run lies on.  Coupled lines' own Z, T_v and
 * travel times are not parameters.  Requires emt_prefactor; a context built
 * with a scenario set, control blocks, frequency-dependent lines or nonlinear
 * resistors returns EINVAL.  Resets the context to step 0 before and after (the recording
 * buffer is not written).  Allocates its work buffers (about 8 N n_nodes
 * bytes for a host v_target, N/K checkpoints, the tape) and frees them
 * before returning.  Synchronous.  ETIMEOUT as for emt_step_n. */
emt_status emt_adjoint(emt_ctx* ctx, const double* v_target, int64_t n_steps, int32_t ckpt_every, double* grad,
                       double* loss, int32_t on_device, void* cuda_stream);

/* Return to the de-energised state at step 0 (keeps G^-1 and recording setup). */
emt_status emt_reset(emt_ctx* ctx);

/* Checkpoint / resume of a run (the paper runs each step from the previous
 * one, Sec. III-B; the run state is what one step hands to the next):
 * write the context's run state -- history currents, line rings and the
 * values consumed at the last step, runtime-switch words and breaker
 * currents, frequency-dependent line and control-block states, nonlinear
 * resistors' segments (per scenario in a scenario set) -- and its step
 * counter into buf (host memory, `cap` bytes), for emt_load_state into this
 * or another context built from the same description (and scenario set),
 * in this process or another.  *size receives the bytes needed; buf = NULL
 * only queries it; a smaller cap returns EINVAL.  Solve matrices and the
 * recording are not part of the state.  Synchronous. */
emt_status emt_save_state(emt_ctx* ctx, void* buf, int64_t cap, int64_t* size);

/* Restore a state written by emt_save_state: the context must be built from
 * the same network (EINVAL otherwise: the state carries the network's shape)
 * and prefactored (ESTATE otherwise); the next emt_step_n continues from the
 * saved step, bitwise as the saving context would have.  Clears a latched
 * device error.  Synchronous. */
emt_status emt_load_state(emt_ctx* ctx, const void* buf, int64_t size);

/* Wait for all work of this context; report a latched device error.
 * dev_err_info (may be NULL): [code, subsystem, line end, step]. */
emt_status emt_sync(emt_ctx* ctx, int32_t* dev_err_info);

/* Tuning and debug knobs (key = value): "wait_budget_ns" (per wait),
 * "batch_graph" (default 1: multi-scenario launches go through a CUDA
 * graph; 0: straight to the stream), "scenarios_per_cta" and
 * "batch_threads" (multi-scenario launch shape; see emt_autotune),
 * "adjoint_overlap" (default 1: emt_adjoint re-runs segment j-1 forward on
 * a second stream while the reverse sweep of segment j runs, when both
 * persistent grids fit on the device together; 0: one stream),
 * "debug_hold_lines" (that subsystem never sends line values; -1 none;
 * for failure-path tests), "warp_per_subsystem" (1: one warp per subsystem,
 * for networks of subsystems of at most 32 nodes with basic elements),
 * "state_space" (the step of each subsystem as one product y = M x with M
 * from G^-1, for networks whose subsystems hold basic elements only --
 * R/L/C branches, sources, fixed-time switches, lossless lines: 0 off,
 * 1 auto (default: while every subsystem's M has at most 2,048 entries),
 * 2 on), "digit_solve" (scenario sets: 1 runs process 4 of each subsystem
 * whose solve matrix a whole scenario tile shares, of at most 64 rows and
 * 128 columns, as exact base-256 digit products on the tensor cores
 * (tcgen05.mma, bf16 -> f32 accumulators in tensor memory), one rounding
 * per entry; 0 keeps the FP64 solve; unset (default) the FP64 solve runs
 * until emt_autotune picks the faster form; while on: at most 32 scenarios
 * and at least 128 threads per CTA, and one CTA per SM), "digit_min_rows"
 * (default 24: subsystems of fewer rows keep the FP64 solve in the digit
 * form, where a small product costs more on the tensor cores than in FP64).
 * EINVAL for an unknown key. */
emt_status emt_set_option(emt_ctx* ctx, const char* key, int64_t value);

/* Read-only facts: "n_subsystems", "n_ctas" (the CTAs of the persistent
 * kernel: one per subsystem, or several subsystems to a CTA when a single
 * network has more subsystems than the device holds CTAs at once),
 * "n_components" (the subsystems proper: components over branches and
 * switches), "sum_n2_components", "max_component_nodes", "step",
 * "max_subsystem_nodes" (nodes of the largest CTA),
 * "n_scenarios", "n_epochs_total", "sum_n2" (sum over subsystems of n_s^2),
 * "threads_per_cta", "kernel_launches", "n_nodes", "n_branches", "n_sources", "n_line_ends",
 * "smem_bytes" (dynamic shared memory per CTA of the persistent kernel),
 * "ctas_per_sm" (how many of its CTAs one SM holds; a single network needs
 * n_subsystems <= that x the SM count), "cta_max_line_ends",
 * "cta_max_lc_branches", "cta_max_control_blocks", "cta_max_lanes",
 * "cta_max_columns" (the per-CTA maxima that size its shared memory),
 * "n_strong_branches" (L/C branches applied through extra solve columns),
 * "n_runtime_switches", "n_coupled_lines", "n_fd_lines", "n_nonlinear", "n_control_blocks",
 * "n_control_injections", "max_control_layers" (largest layer count of one
 * subsystem's control graph),
 * "n_matrix_variants", "scenarios_per_cta", "batch_threads", "batch_groups"
 * (subsystem groups per step of the multi-scenario kernel),
 * "graph_launches", "autotuned", "digit_solve" (1 while on), "digit_matrices"
 * (solve matrices held in digit form), "state_space" (1 while the state-space
 * form runs emt_step_n), "warp_per_subsystem", "shard_rank" (-1 unless a shard),
 * "shard_window" (see emt_set_shard; 0 unless a shard), "shard_ctas" (CTAs
 * this context runs). */
emt_status emt_get_info(const emt_ctx* ctx, const char* key, int64_t* value);

/* Internal node order: perm[i] = original node id of internal slot i
 * (n_nodes entries). */
emt_status emt_get_node_order(const emt_ctx* ctx, int32_t* perm);

/* ---- Shards: one network over several devices (one context per rank) ----
 *
 * Subsystems meet only through line rings: the value a line end sends at
 * step n is consumed at the far end at step n + d, d its travel time in
 * whole steps (Sec. II-B: the line decouples its two ends).  Every rank
 * builds a context from the same description (so CTAs and line ends are
 * numbered alike) and runs only the CTAs it owns.  With D = the smallest d
 * of a line end whose two sides belong to different ranks, a window of
 * W <= D steps reads only values sent before it began, so the ranks run
 * each window independently and, between windows, swap the ring slots the
 * window wrote for the other side: point to point, 16 bytes per cut line
 * end and step, no collective.  The result is bitwise that of the whole
 * network in one context. */

/* CTA of every node: cta[i] for the caller's node i (n_nodes entries,
 * host memory).  EINVAL for a context built with a scenario set. */
emt_status emt_get_node_ctas(const emt_ctx* ctx, int32_t* cta);

/* The line ends ("n_line_ends" of them, library order; coupled lines
 * contribute one per mode and end): the CTA that owns each, the index of
 * the end at the other side of the line, and its travel time d in whole
 * steps.  Host arrays of n_line_ends entries, each may be NULL.  EINVAL for
 * a context built with a scenario set. */
emt_status emt_get_line_ends(const emt_ctx* ctx, int32_t* cta, int32_t* far_end, int32_t* d);

/* Make ctx a shard: it runs the CTAs c with owner[c] == rank (owner: host
 * array of "n_ctas" non-negative ranks, the same on every rank); owner =
 * NULL makes it the whole network again.  Sets "shard_window" (emt_get_info)
 * to D above (2^31 - 1 if no line is cut).  From then on each emt_step_n
 * is one window of at most D steps, and the next emt_step_n is refused
 * (ESTATE) until, for every peer, the window's values were packed
 * (emt_shard_pack) and the peer's window values unpacked (emt_shard_unpack).
 * Synchronises the device.  EINVAL: a scenario set, a rank owning no CTA, a
 * negative owner; the context then runs the whole network.  emt_adjoint is
 * refused while the context is a shard. */
emt_status emt_set_shard(emt_ctx* ctx, const int32_t* owner, int32_t rank);

/* The slots the last window wrote for rank `peer` (those its CTAs will
 * consume), as [cut line end][step of the window] 16-byte records (tag and
 * value words), cut line ends in ascending library order.  *bytes (may be
 * NULL) receives the size: 16 x (cut ends towards peer) x (window steps);
 * buf = NULL only queries it.  buf: device memory of `cap` bytes, 16-byte
 * aligned.  Enqueued on cuda_stream (NULL: legacy default stream), after the
 * window's launch when both are on one stream.  0 bytes for a peer that
 * shares no line with this rank. */
emt_status emt_shard_pack(emt_ctx* ctx, int32_t peer, void* buf, int64_t cap, int64_t* bytes, void* cuda_stream);

/* Write what rank `peer` packed for this rank after the same window into
 * this context's rings.  buf: device memory, 16-byte aligned, of exactly the
 * size the peer's emt_shard_pack reported (EINVAL otherwise).  Enqueued on
 * cuda_stream: the caller orders it after the buffer's arrival (and before
 * the next window). */
emt_status emt_shard_unpack(emt_ctx* ctx, int32_t peer, const void* buf, int64_t bytes, void* cuda_stream);

/* Per-phase cycle counts of the single-network kernel, from the phase-clock
 * build of the library (compiled with -DEMT_PHASE_CLOCKS; libemt_phases.so):
 * out[c * 8 + k] for every CTA c < n_ctas (host memory), summed over all
 * steps of all launches since the last reset, as clock64 cycles seen by the
 * CTA's thread 0:
 *   k = 0 process 2 (nodal injections), 1 process 4 (the solve's partial
 *   sums), 2 node voltages and the compensation method, 3 thread 0's own
 *   process-1 updates, 4 the wait of the thread that polls the CTA's first
 *   line end (its own count), 5 from thread 0's updates to the end-of-step
 *   barrier (the other updates and the line-value polls), 6 steps, 7 the
 *   cycles from the first step's start to the last step's end of the last
 *   launch.
 * While the state-space form runs (option "state_space"), its kernel's
 * counters instead: k = 0 thread 0's rows of the product, 1 the collection
 * of the next step's line values and source voltages (the poll warp's lane
 * 0), 2 thread 0 from its rows to the end-of-step barrier, 6 and 7 as above.
 * out may be NULL; reset != 0 zeroes the counters afterwards.  Synchronises
 * the device.  EINVAL in the normal build or with more than 2048 CTAs. */
emt_status emt_phase_clocks(emt_ctx* ctx, uint64_t* out, int32_t reset);

/* Last error message of ctx (or of the last failed build if ctx == NULL). */
const char* emt_last_error(const emt_ctx* ctx);

/* Free everything the context owns.  NULL is a no-op. */
void emt_destroy(emt_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
