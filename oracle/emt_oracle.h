/*
 * Plain FP64 CPU oracle for the EMTP-type time loop (test infrastructure).
 *
 * This library exists to check the CUDA path; only tests, the package's
 * smoke entry and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header or table with the CUDA library.
 *
 * Method (Sec. III-A of the CloudPSS paper lists the four basic processes of
 * the EMTP-type algorithm, ref. [2] gives the formulas):
 *   1. update Norton equivalent conductance / history current per element
 *      (trapezoidal companion models of R, L, C; Bergeron lossless lines),
 *   2. update nodal injected currents,
 *   3. factorise the conductance matrix (whenever it changes),
 *   4. forward / backward substitution for the node voltages.
 * Node codes: k >= 0 unknown node, -1 ground, -2-s known node of source s.
 */
#ifndef EMT_ORACLE_H
#define EMT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double dt;
  int64_t n_nodes;
  int64_t n_br;
  const int32_t* br_k;
  const int32_t* br_m;
  const uint8_t* br_kind;   /* 0 = R, 1 = L, 2 = C */
  const double* br_val;     /* ohm, henry, farad */
  int64_t n_src;
  const double* src_amp;
  const double* src_phase;
  const double* src_freq;
  int64_t n_ln;
  const int32_t* ln_k;
  const int32_t* ln_m;
  const double* ln_zc;
  const int32_t* ln_d;      /* travel time in steps, >= 1 */
  int64_t n_sw;
  const int32_t* sw_k;
  const int32_t* sw_m;
  const double* sw_r;
  const int64_t* sw_on;     /* closed for sw_on <= n < sw_off */
  const int64_t* sw_off;    /* -1 = never opens */
  /* Runtime switches: two-state resistors whose state in force at step n
   * is decided from step n-1's solution (state at step 1: rs_on0).
   *   kind 0, diode (anode k, cathode m): conducting iff v_k - v_m > 0;
   *   kind 1, breaker: closed until, at a step n >= rs_trip, its current
   *     g_on (v_k - v_m) changes sign from step n-1 (product <= 0); open
   *     from step n+1 on, for good.
   * Ends are unknown nodes or ground. */
  int64_t n_rs;
  const int32_t* rs_k;
  const int32_t* rs_m;
  const uint8_t* rs_kind;
  const double* rs_ron;
  const double* rs_roff;
  const uint8_t* rs_on0;
  const int64_t* rs_trip;
  /* Coupled three-phase lossless lines, modal form (Bergeron per mode):
   *   cl_k[3 l + p], cl_m[3 l + p]: phase p's node at end k / end m;
   *   cl_tv[9 l + 3 p + j]: T_v, phase voltages = T_v modal voltages
   *     (modal currents: T_i = T_v^-T);
   *   cl_z[3 l + j], cl_tau[3 l + j]: mode j's Z_c (ohm) and travel time
   *     (s, at least dt).
   * Each end draws i_p = Y_p v_p + T_i I_mode with Y_p = T_i diag(1/Z) T_v^-1;
   * mode j sends c_j(n) = -(2/Z_j) v_mode_j(n) - I_mode_j(n) to the far end,
   * whose history at step n is (1 - f_j) c_j(n - d_j) + f_j c_j(n - d_j - 1),
   * tau_j = (d_j + f_j) dt, d_j = floor(tau_j / dt). */
  int64_t n_cl;
  const int32_t* cl_k;
  const int32_t* cl_m;
  const double* cl_tv;
  const double* cl_z;
  const double* cl_tau;
  /* Control system (Sec. III-A: each control component is one basic process
   * of the computation graph).  Block b has one output y_b, inputs
   * cb_in0[b], cb_in1[b] (block indices, -1 = unused) and parameters p0, p1:
   *   0 CONST  y = p0                 5 LIMIT  y = min(max(u0, p0), p1)
   *   1 MEAS   y = v(cb_node[b])      6 INTEG  y = y(n-1) + p0 (dt/2)(u0 + u0(n-1))
   *   2 GAIN   y = p0 u0              7 LAG    p0 / (1 + s p1), trapezoidal:
   *   3 SUM    y = p0 u0 + p1 u1               y = a y(n-1) + b (u0 + u0(n-1)),
   *   4 MUL    y = p0 u0 u1                    a = (2 p1 - dt) / (2 p1 + dt),
   *   8 PI     y = p0 u0 + p1 I,               b = p0 dt / (2 p1 + dt)
   *            I = I(n-1) + (dt/2)(u0 + u0(n-1))
   * (states start at 0).  At step n, after the node voltages v(n) are
   * solved, the blocks are evaluated in index order: an input from a block
   * of lower index reads that block's step-n output, an input from a block
   * of equal or higher index its step-(n-1) output (0 at n = 1) -- this is
   * how algebraic loops are broken.  Controlled current injection c:
   * y_{ci_block[c]}(n) enters node ci_node[c] at step n + 1. */
  /* Frequency-dependent lines (one conductor each, ends fl_k / fl_m, both
   * unknown nodes): characteristic admittance and propagation function as
   * pole-residue sums,
   *   Y_c(s) = y0 + sum_i c_i / (s - q_i),  A(s) = e^{-s tau} (a0 + sum_i r_i / (s - p_i)),
   * up to 4 real poles each ([4 l + i] layout), poles < 0, tau >= dt.
   * Each first-order term is discretised by the trapezoidal rule,
   *   x(n) = lam x(n-1) + mu (u(n) + u(n-1)),  lam = (1 + p dt/2)/(1 - p dt/2),
   *   mu = r (dt/2)/(1 - p dt/2).
   * At an end e with far end f:
   *   yc_e(n) = y0 v_e(n) + sum_i s_ei(n)              (s_ei: Y_c's terms of v_e)
   *   i_e(n)  = yc_e(n) - b_e(n)                       (current into the line)
   *   b_e(n)  = a0 W_f(n) + sum_i z_ei(n)              (z_ei: A's terms of W_f)
   *   W_f(n)  = (1 - phi) w_f(n - d) + phi w_f(n - d - 1),  tau = (d + phi) dt
   *   w_f(m)  = yc_f(m) + i_f(m) = 2 yc_f(m) - b_f(m)  (0 for m <= 0).
   * So each end stamps G_eq = y0 + sum mu_i and draws the history current
   * sum_i (lam_i s_ei(n-1) + mu_i v_e(n-1)) - b_e(n).  With y0 = 1/Z, a0 = 1,
   * no poles and tau = d dt this is the lossless Bergeron line. */
  int64_t n_fl;
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
  /* Nonlinear resistors, solved by the compensation method: element e
   * between nl_k and nl_m (unknown node or ground, not both ground) carries
   * i = f(v_k - v_m), f odd and piecewise linear through (0, 0) and
   * (nl_v[8 e + j], nl_i[8 e + j]), j < nl_np[e] <= 8, with 0 < v_1 < v_2 <
   * ... and 0 <= i_1 <= i_2 <= ... (monotone), continued past the last
   * point with the last segment's slope.  At each step the subsystem is
   * solved without the element (v0), the element sees the Thevenin source
   * v_th = v0_k - v0_m behind R_th = z_k - z_m, z = G^-1 (e_k - e_m); its
   * current solves i = f(v_th - R_th i) (unique: f monotone, R_th > 0);
   * then v = v0 - z i.  A subsystem with several nonlinear resistors is
   * solved by the piecewise-linear Newton iteration on its nodal equations:
   * each element stamped as the line of the segment it was on at the last
   * step (i = c0 + slope u), the system solved, each element moved to the
   * segment its voltage lies on, until none moves (at most 64 rounds, else
   * the run fails).  The element joins k and m into one subsystem. */
  int64_t n_nl;
  const int32_t* nl_k;
  const int32_t* nl_m;
  const int32_t* nl_np;
  const double* nl_v;
  const double* nl_i;
  int64_t n_cb;
  const uint8_t* cb_type;
  const int32_t* cb_in0;
  const int32_t* cb_in1;
  const int32_t* cb_node;
  const double* cb_p0;
  const double* cb_p1;
  int64_t n_ci;
  const int32_t* ci_block;
  const int32_t* ci_node;
  /* Frequency-dependent line groups (n_fg may be 0): three of the
   * frequency-dependent lines above carry the modes of one three-phase line.
   * fg_line[3 g + j] is the line of mode j; its end nodes are phase j's
   * nodes at each end (the three end-k nodes lie in one subsystem, as do the
   * three end-m nodes); fg_tv[9 g + 3 p + j]: T_v, phase voltages = T_v modal
   * voltages (modal currents: T_i = T_v^-T).  Mode j's equations act on modal
   * quantities: its Y_c on the modal voltage (T_v^-1 v_phase)_j, its w and b
   * as for one conductor; each end draws the phase currents T_i i_mode, i.e.
   * it stamps T_i diag(G_eq) T_v^-1 and draws T_i times the modal history
   * currents.  A line belongs to at most one group. */
  int64_t n_fg;
  const int32_t* fg_line;
  const double* fg_tv;
} orc_net;

/* Run n_steps steps from the de-energised state.
 *   monolithic = 1: one conductance matrix over all unknown nodes;
 *   monolithic = 0: one matrix per subsystem (components joined by
 *                   branches and switches; lines cut them).
 *   rec / n_rec: recorded nodes (rec = NULL: all nodes in order);
 *   v_out: [n_steps][n_rec] node voltages of steps 1..n_steps (may be NULL);
 *   v_target / loss: if both non-NULL, loss = sum_n sum_k (v_n[k]-v*_n[k])^2
 *   over all nodes, v_target laid out [n_steps][n_nodes].
 * Returns 0, or a negative code: -1 invalid input, -2 singular matrix. */
int orc_run(const orc_net* net, int monolithic, int64_t n_steps, const int32_t* rec, int64_t n_rec,
            double* v_out, const double* v_target, double* loss);

/* Runtime-switch states in force at steps 1..n_steps: states[(n-1) n_rs + w]
 * (a run of orc_run's loop, partitioned mode). */
int orc_rs_states(const orc_net* net, int64_t n_steps, uint8_t* states);

/* Complex-step derivative of the loss with respect to parameter `param`
 * (0..n_br-1: branch value; n_br..n_br+n_src-1: source amplitude):
 * runs the same loop in complex arithmetic with p -> p + i*h.
 * loss = Re J, dloss = Im J / h. */
int orc_loss_cs(const orc_net* net, int64_t n_steps, const double* v_target, int64_t param, double h,
                double* loss, double* dloss);

/* Discrete adjoint of the loss over the full stored trajectory.
 * grad: [n_br + n_src] = dJ/d(branch value) then dJ/d(source amplitude).
 * With runtime switches the reverse sweep uses the states the forward run
 * decided (the gradient of the smooth piece the run lies on).  The
 * parameters of coupled lines themselves (Z, T_v, travel times) are not
 * differentiated.  Networks with control blocks, frequency-dependent
 * lines or nonlinear resistors are rejected (-1). */
int orc_adjoint(const orc_net* net, int64_t n_steps, const double* v_target, double* grad, double* loss);

/* Control block outputs of steps 1..n_steps: y_out[(n-1) n_cb + b]
 * (partitioned mode; node voltages as orc_run). */
int orc_controls(const orc_net* net, int64_t n_steps, double* y_out);

/* Subsystem of each unknown node (components over branches and switches). */
int orc_partition(const orc_net* net, int32_t* sub_of_node, int64_t* n_sub);

/* Sessions: the loop run window by window on a chosen part of the network
 * (partitioned mode), for checking a sharded run.  Subsystems meet only
 * through lines, and an end consumes at step n what the far end sent at
 * step n - d (Sec. II-B: the travel time decouples the two ends), so a part
 * can run up to d steps alone once the values its ends consume are put in.
 *   orc_open:      a session at step 0 (net must outlive it); NULL if invalid.
 *   orc_advance:   n_steps more steps; active[s] != 0 for the subsystems (of
 *                  orc_partition) whose processes 3 and 4 run, NULL = all;
 *                  v_out: [n_steps][n_nodes] or NULL.  Networks with control
 *                  blocks take active = NULL only (-1 otherwise).  An
 *                  inactive subsystem's voltages stay 0 and what its ends
 *                  send is wrong until orc_sent overwrites it.
 *   orc_line_ends: the 2 n_ln + 6 n_cl + 2 n_fl line ends, in the order
 *                  lines (k, m), coupled lines (end k modes 0-2, end m modes
 *                  0-2), frequency-dependent lines (k, m): a node of the end,
 *                  the far end's index, the travel time d in whole steps.
 *   orc_sent:      the values end `end` sent at steps n0 .. n0+w-1 (set = 0:
 *                  read into vals; 1: overwrite from vals); those steps must
 *                  be among the last d + 1 completed ones. */
typedef struct orc_session orc_session;
orc_session* orc_open(const orc_net* net);
int orc_advance(orc_session* s, int64_t n_steps, const uint8_t* active, double* v_out);
int orc_line_ends(const orc_net* net, int32_t* node, int32_t* far, int32_t* d);
int orc_sent(orc_session* s, int64_t end, int64_t n0, int64_t w, double* vals, int set);
void orc_close(orc_session* s);

/* Dense LU with partial pivoting: solve A x = b, A row-major n x n. */
int orc_lu_solve(int64_t n, const double* A, const double* b, double* x);

#ifdef __cplusplus
}
#endif
#endif
