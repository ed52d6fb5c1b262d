// Internal layout shared by the host driver (emt_api.cu) and the kernels.
// Everything here is an implementation detail behind include/emt.h.
#pragma once
#include <stdint.h>

#include <cuda_runtime.h>

namespace emt {

// Largest subsystem the persistent kernel keeps on chip (G^-1 in shared
// memory: 128 x 128 doubles = 128 KiB).
constexpr int kMaxSubsystemNodes = 128;

// Threads per CTA of the persistent forward kernel.
constexpr int kFwdThreads = 256;

// Injection entries (process 2).  Every node's injection is a signed sum of
// entries of one shared-memory input vector
//     inp = [ h (L/C slots) | g_b v_src (source-branch slots) |
//             I_e parity 0 (line ends) | I_e parity 1 | 0 |
//             controlled currents (one slot per control injection) |
//             Hy of the frequency-dependent line ends ]
// A parity block holds the line-end values, then the coupled ends' phase
// currents, then the frequency-dependent ends' b values.
// An entry is an int32: bit 31 = subtract, bits 0..30 = index into inp with
// line ends addressed in their parity-0 block.  A node's entries are split
// into "injection lanes" of 4 entries (padded with the trailing zero); the
// lanes of one node are consecutive and never straddle a warp, so the
// node's first lane can add the others' partial sums by warp shuffles.
constexpr uint32_t kEntryNeg = 0x80000000u;
constexpr int kMaxLanesPerNode = 32;

// One branch in device form.  Node fields are subsystem-local:
//   >= 0 local node, -1 ground, <= -2 local source -2-j.
struct BranchDev {
  int16_t k, m;
  uint8_t kind;      // 0 R, 1 L, 2 C
  uint8_t pad[3];
  double value;      // ohm / henry / farad (input)
  double g;          // companion conductance (written by the companion kernel)
  double e;          // history gain: +2g (L), -2g (C), 0 (R)
};

// One line end, owned by the subsystem of its node.  It consumes I_e(n)
// from its own ring and produces I_f(n+d) into the far end's ring.
// A ring slot is two 64-bit words, each = (step << 32) | one 32-bit half of
// the double I(step); each word is written and read as one single-copy
// atomic access, so a reader that finds the expected step in both words
// holds that step's value -- no fence or separate flag is needed.  A slot is
// rewritten (D = 2d steps later) only after its reader consumed it: the far
// end's write at step m carries a value computed from this end's output of
// step m - d, which this end produced after reading the slot.
struct LineEndDev {
  int32_t node;        // local node of this end (-1: a mode of a coupled line end)
  int32_t d;           // travel time in steps (whole part)
  int32_t depth;       // ring depth D = 2d
  int32_t ce;          // coupled line end (subsystem-local) this mode belongs to, or -1
  double y2;           // 2 / Z_c
  double y;            // 1 / Z_c (shunt stamped at node; 0 for modes, whose ends stamp Y_p)
  int64_t own_ring;    // first slot of this end's ring (values consumed here)
  int64_t far_ring;    // first slot of the far end's ring (values produced here)
  int32_t mode;        // mode index within its coupled end (0..2)
  int32_t fd;          // frequency-dependent end (subsystem-local FdEndDev) or -1
  double f;            // fractional travel time: history = (1 - f) c(n - d) + f c(n - d - 1)
};

// One end of a frequency-dependent line (one conductor): Y_c = y0 +
// sum c_i / (s - q_i) and A = e^{-s tau} (a0 + sum r_i / (s - p_i)), each
// pole term discretised by the trapezoidal rule, x(n) = lam x(n-1) +
// mu (u(n) + u(n-1)).  The end is a line end (node, rings, d, f) that
// stamps G_eq = y0 + sum mu_y and whose ring carries the far end's
//   w(m) = 2 yc(m) - b(m),  yc = y0 v + sum s_i  (s_i: Y_c's terms of v),
// while its own history is b(n) = a0 W(n) + sum z_i(n) (z_i: A's terms of
// W), W(n) = (1 - f) w(n - d) + f w(n - d - 1).  It draws the current
// G_eq v(n) + Hy(n) - b(n), Hy(n) = sum (lam_y s_i(n-1) + mu_y v(n-1)).
struct FdEndDev {
  int32_t le;          // subsystem-local line end
  int32_t ny, na;      // pole counts (<= 4)
  int32_t pad;
  double y0, a0;
  double mu_sum;       // sum of mu_y: G_eq - y0
  double omf;          // 1 - f of its line end (interpolation weight of w(n - d))
  double lam_y[4], mu_y[4], lam_a[4], mu_a[4];
};

// One end of a coupled three-phase lossless line in modal form.  Its three
// modes are consecutive line ends starting at le0; the phase-domain history
// currents T_i I_mode leave its three phase nodes, and the end stamps
// Y_p = T_i diag(1/Z) T_v^-1 into G (T_i = T_v^-T).  tinv, ti and yp are
// computed on the device from tv and z.
struct CoupledEndDev {
  int32_t node[3];     // phase nodes (subsystem-local)
  int32_t le0;         // subsystem-local index of the mode-0 line end
  double tv[9];        // T_v (phase voltages = T_v modal voltages), row-major
  double z[3];         // modal Z_c
  double tinv[9];      // T_v^-1
  double ti[9];        // T_i
  double yp[9];        // Y_p
};

// A switch in device form (subsystem-local ends, -1 = ground).
struct SwitchDev {
  int32_t k, m;
  double g;          // 1 / R while closed
};

// Per-subsystem descriptor.
struct SubDev {
  int32_t n;           // unknown nodes
  int32_t node_off;    // first internal node id
  int32_t br_off, n_br;        // all branches (stamping)
  int32_t lc_off, n_lc;        // L/C branch slots (history updates)
  int32_t sb_off, n_sb;        // source-branch slots (injection from known nodes)
  int32_t le_off, n_le;        // line ends owned here
  int32_t src_off, n_src;      // local sources (global ids in src_global)
  int32_t nb_off, n_nb;        // neighbour subsystems (reported by emt_get_info)
  int32_t ep_off, n_ep;        // switch epochs
  int32_t il_off, n_il;        // injection lanes (4 entries each; il_node / il_cnt per lane)
  int32_t str_off, n_str;      // strong L/C branches (L/C slots in str_slot)
  int32_t q;                   // column blocks per row in the matvec
  int32_t n_states;            // 2^(runtime switches): solve matrices per switch epoch
  int32_t rs_off, n_rs;        // runtime switches (RuntimeSwitchDev list)
  int32_t ce_off, n_ce;        // coupled line ends (CoupledEndDev list)
  int32_t cb_off, n_cb;        // control blocks (CtrlDev list, by layer)
  int32_t clay_off, n_clay;    // control layers: n_clay + 1 starts in clay (with the layer's type, see kLayerTypeShift)
  int32_t ci_off, n_ci;        // control injections: local block slot per injection in cinj
  int32_t fd_off, n_fd;        // frequency-dependent line ends (FdEndDev list)
  int32_t nl_off, n_nl;        // nonlinear resistors (NlDev list; at most kNlMaxPerSub)
  // More than kMaxRuntimeSwitches runtime switches: the solve matrix of a
  // (switch epoch, state word) is factorised by the CTA when the state is
  // first met (process 3 at run time) into one of n_cache slots, slot j at
  // ginv offset cache_goff + j n (n + n_str) (its nonlinear column at
  // cache_zoff + j n), tagged in cache_tag[cache_slot0 + j]; the
  // factorisation's two n x n workspaces at lazy_work + work_off.
  int32_t n_cache, cache_slot0;
  int64_t cache_goff, cache_zoff, work_off;
};

// A nonlinear resistor solved by the compensation method: odd, piecewise
// linear, segment j (0 <= j <= np) starting at (bv[j], bi[j]) with slope
// sl[j], (bv[0], bi[0]) = (0, 0), the last segment unbounded.  Each solve
// matrix entry of its subsystem carries the column z = G^-1 (e_k - e_m)
// (EpochDev::nlz_off); the step solves i = f(v_th - R_th i) against the
// linear solution, R_th = z_k - z_m, and corrects v by -z i.
constexpr int kNlMaxPoints = 8;
// Nonlinear resistors per subsystem (single networks; one in scenario
// sets).  With several, each solve matrix entry carries one column per
// element, z_j = G^-1 (e_kj - e_mj) at EpochDev::nlz_off + j n, and the step
// solves the elements together through the Thevenin matrix R = A^T Z.
constexpr int kNlMaxPerSub = 4;
// Device error code: the piecewise-linear iteration of a subsystem's
// nonlinear resistors found no consistent segments (reported as EMT_ESTATE).
constexpr int kErrNoSegments = 100;
// Device error code of the checks build: an index outside its array
// {kErrBounds, site, index, length} (emt_device.cuh; reported as EMT_ESTATE).
constexpr int kErrBounds = 101;
// Device error code of the multi-scenario kernel's tensor-core solve: a
// wait for the staged digit planes (what = 0) or for the products (1) ran
// past its budget {kErrTensorWait, subsystem, what, step} (EMT_ESTATE).
constexpr int kErrTensorWait = 102;
struct NlDev {
  int32_t k, m;        // subsystem-local ends, -1 = ground
  int32_t np;          // breakpoints after (0, 0)
  int32_t pad;
  double bv[kNlMaxPoints + 1], bi[kNlMaxPoints + 1], sl[kNlMaxPoints + 1];
};

// A control block in device form (subsystem-local, ordered by layer).  The
// CTA keeps block outputs as pairs y[2 slot + parity of the step]; an input
// is stored as i = 2 slot + late, where late = 1 marks a read of the
// previous step's output (the loop-breaking rule), so that the value read
// at a step of parity par is y[i ^ par].  An unused input points at the
// zero pair after the last block (i = 2 n_cb).  Coefficients: GAIN p0; SUM
// p0, p1; MUL p0; LIMIT lo p0, hi p1; INTEG p0 = k dt / 2; LAG p0 = a,
// p1 = b; PI kp p0, ki p1, p2 = dt / 2.
struct __align__(16) CtrlDev {
  int32_t type;        // 0 CONST .. 8 PI, as in the public header
  int32_t i0, i1;      // inputs, encoded as above
  int32_t node;        // MEAS: local node
  double p0, p1, p2;
  double ov;           // multi-scenario kernel: row of its per-scenario coefficients (BatchParams::cbo), or -1
};

// Control layer starts (local block slots) carry the layer's block type in
// bits 24..27 when all its blocks share one type, else kMixedLayer.
constexpr int kLayerTypeShift = 24;
constexpr int kMixedLayer = 15;

// Runtime switches per subsystem up to which every state word of every
// epoch is prefactored (2^k solve matrices per epoch); above it, and up to
// kMaxLazySwitches, states are factorised on the device when first met.
constexpr int kMaxRuntimeSwitches = 8;
constexpr int kMaxLazySwitches = 30;
// Cache slots per such subsystem beyond one per epoch.
constexpr int kLazyCacheExtra = 256;

// A runtime switch in device form: a two-state resistor whose state in
// force at step n is decided from step n-1's solution.  Bit `j` (its index
// within the subsystem) of the subsystem's state word is its state; the
// solve matrix of epoch e and state word w is entry e n_states + w.
struct RuntimeSwitchDev {
  int32_t k, m;        // subsystem-local ends, -1 = ground
  int32_t kind;        // 0 diode (anode k), 1 breaker
  int32_t pad;
  double r_on;         // breaker current = (v_k - v_m) / r_on while on
  int64_t trip;        // breaker: first step at which it may open
  double r_off;        // resistance while off (stamped by run-time factorisation)
};

// Strong L/C branches.  When a branch's conductance dwarfs the rest of
// what its two end nodes see, its history current h enters the injections
// of k and m with opposite signs and G^-1 i cancels two nearly equal large
// products.  Such a branch is kept out of the injections; its effect
// -(G^-1[:,k] - G^-1[:,m]) h is applied through an extra matvec column whose
// entries are formed without cancellation when G^-1 is built.  Criterion:
// g_b >= kStrongRatio * min(G_kk - g_b, G_mm - g_b).
constexpr double kStrongRatio = 3.0;

// Switch epoch of a subsystem: state holding from step `start` on.  Its
// solve matrix is n x nc, nc = n + n_str: [G^-1 | strong-branch columns].
// With runtime switches each epoch has n_states consecutive entries, one
// per state word (same start).
struct EpochDev {
  int64_t start;
  int64_t ginv_off;      // offset of this epoch's n x nc solve matrix
  int32_t sw_off, n_sw;  // closed switches (SwitchDev list)
  int64_t nlz_off;       // offset of its nonlinear resistor's column z (n doubles), or -1
  int32_t rs_word;       // >= 0: also stamp the subsystem's runtime switches in this state word
                         // (subsystems factorised at run time); -1: they are in the switch list
  int32_t pad;
};

// Lengths of the global arrays a launch indexes with device data, for the
// checks build (emt_device.cuh): ring slots, solve-matrix entries, record
// doubles, history slots, source-table doubles, nonlinear columns, tape and
// target doubles.
struct Bounds {
  int64_t ring, ginv, rec, h, src, nlz, tape, target, ssm;
};

// The step of one subsystem in state-space form (emt_ss.cu).  With
// x(n) = [h(n-1) | v_src(n) | J(n)] -- the history currents of its L/C
// slots, its sources' voltages, and per node with line ends the sum J of
// the values they consume -- both the node voltages v(n) and the new
// history currents h(n) are linear in x(n): y(n) = [h(n) | v(n)] = M x(n)
// (processes 2 and 4, v = G^-1 i, and process 1's h from v, in one
// matrix).  The values the line ends send follow from v directly, c_e =
// -(2/Z) v_node - I_e.  M per switch epoch, rows x cols, row-major at m_off
// + epoch rows cols in FwdParams::ss_m (ss_mlo: its single-precision
// remainder).  Used for networks of small subsystems with the basic
// elements only, where the step's chain of dependent FP64 operations, not
// its work, sets the time.
struct SsSubDev {
  int32_t rows, cols;   // rows = n_lc + n (compact: n); cols = n_lc + n_src + n_ln
  int32_t q;            // lanes per row of the matvec (a power of two <= 32)
  int32_t n_ln;         // nodes with line ends: ss_lnode[ln_off + j], their ends ss_lend[ss_lptr[ptr_off + j] ..]
  int32_t ln_off, ptr_off;
  // compact: M holds the node-voltage rows only, and one warp runs the whole
  // step (v, then h and the line outputs from v): fewer FP64 instructions,
  // for SMs that hold several CTAs
  int32_t compact, pad;
  int64_t m_off;
};

// Per-launch upper bounds that size the forward kernel's shared memory.
struct FwdLimits {
  int32_t n, nc, q, lc, sb, le, src, il, str;
  int32_t nbuf;                // solve-matrix buffers in shared memory: 1, or 2 (the last two states kept)
  int32_t ce;                  // coupled line ends per subsystem
  int32_t cb, clay, ci;        // control blocks, layers + 1 and injections per subsystem
  int32_t fd;                  // frequency-dependent line ends per subsystem
  int32_t nl;                  // most nonlinear resistors in one subsystem
};

struct FwdParams {
  int32_t n_sub;
  // a shard of the network (the other subsystems run elsewhere and meet it only
  // through line rings): CTA (or warp) i runs sub[i], subsystem active[i] of the
  // network, i < n_active; nullptr: all n_sub, active[i] = i
  const int32_t* active;
  int32_t n_active;
  FwdLimits lim;
  const SubDev* sub;
  const EpochDev* ep;
  const double* ginv;          // G^-1 rounded to double, per epoch
  const float* ginv_lo;        // G^-1 minus that rounding, in single precision
  const BranchDev* br;
  const int32_t* lc_idx;       // branch index per L/C slot
  const int32_t* sb_idx;       // branch index per source-branch slot
  double* h;                   // history current per L/C slot
  const int32_t* ent;          // injection entries, 4 per injection lane
  const int32_t* il_node;      // node of each injection lane (-1: padding)
  const int32_t* il_cnt;       // lanes of the node on its first lane, else 0
  const int32_t* str_slot;     // L/C slot of each strong branch
  const LineEndDev* le;
  unsigned long long* ring;    // [slots][2] tagged words
  const int32_t* src_global;   // global source id per local source slot
  const double* src_table;     // [n_steps][n_sources]: v_src(t_{n0+i})
  int32_t n_sources;
  int32_t* err;                // [4]: code, subsystem, line end, step
  double* rec;                 // [rows][n_rec], row r at rec + (r - rec_row0) * n_rec
  const int32_t* rec_pos;      // per internal node: column in rec, or -1
  int64_t rec_rows;            // rows below this are written
  int64_t rec_row0;            // first row held by rec (0 for a whole recording)
  int32_t rec_decim;
  int32_t n_rec;
  int64_t n0;                  // first step of this launch
  int64_t n_steps;
  unsigned long long wait_budget_ns;
  int32_t hold_sub;            // debug: this subsystem never writes its line outputs (-1: none)
  const CoupledEndDev* ce;     // coupled line ends (SubDev ce_off / n_ce)
  double* le_prev;             // per line end: value consumed at step n0 - 1 (modes' interpolation)
  const RuntimeSwitchDev* rs;  // runtime switches (SubDev rs_off / n_rs)
  int32_t* rs_word;            // per subsystem: state word in force at step n0 (carried across launches)
  double* rs_prev_i;           // per runtime switch: breaker current of the previous step
  int32_t* word_tape;          // optional [rows][n_sub]: state word in force at step n (row n - 1 - word_row0)
  int64_t word_row0;
  const CtrlDev* cb;           // control blocks (SubDev cb_off / n_cb)
  const int32_t* clay;         // control layer starts (SubDev clay_off)
  const int32_t* cinj;         // local block slot per control injection (SubDev ci_off / n_ci)
  double* cstate;              // per control block: two states (s0, s1)
  double* cy;                  // per control block: output of the last step (carried across launches)
  const FdEndDev* fd;          // frequency-dependent line ends (SubDev fd_off / n_fd)
  double* fd_state;            // per FD end: s[4], z[4], v(n-1), W(n-1), Hy(n) (11 doubles, carried)
  const NlDev* nl;             // nonlinear resistors (SubDev nl_off / n_nl)
  const double* nlz;           // their columns z per solve matrix entry (EpochDev::nlz_off, n per element)
  const float* nlz_lo;         // z minus that rounding, in single precision
  int32_t* nl_seg;             // per nonlinear resistor: its segment at the last step, sign * (j + 1) (carried)
  // run-time factorisation (SubDev::n_cache > 0): the same arrays, writable
  double* ginv_rw;
  float* ginv_lo_rw;
  double* nlz_rw;
  float* nlz_lo_rw;
  long long* cache_tag;        // per cache slot: (epoch << 32) | state word, or -1
  int32_t* cache_next;         // per subsystem: next slot to replace; then the count of run-time factorisations
  double* lazy_work;
  const SwitchDev* sw;         // closed switches of each epoch (EpochDev sw_off / n_sw)
  // state-space form (SsSubDev): per subsystem of the network, M and its remainder, the largest rows / cols
  const SsSubDev* ss;
  const double* ss_m;
  const float* ss_mlo;
  const int32_t* ss_lnode;     // local node of each line-end node slot
  const int32_t* ss_lptr;      // per slot: first position in ss_lend (n_ln + 1 per subsystem, from S.le_off)
  const int32_t* ss_lend;      // subsystem-local line ends grouped by node (n_le per subsystem, at S.le_off)
  int32_t ss_rows, ss_cols, ss_ln;   // maxima over subsystems (shared-memory layout)
  Bounds bnd;
};

constexpr int kFdState = 11;

struct PrefParams {
  int32_t n_mats;
  const int32_t* mat_sub;      // subsystem per matrix
  const int32_t* mat_ep;       // epoch index (into ep) per matrix
  const SubDev* sub;
  const EpochDev* ep;
  const BranchDev* br;
  const LineEndDev* le;
  const SwitchDev* sw;
  const CoupledEndDev* ce;     // coupled line ends: Y_p blocks
  const int32_t* lc_idx;       // branch index per L/C slot
  const int32_t* str_slot;     // L/C slot of each strong branch
  double* ginv;                // X_hi: G^-1 rounded to double
  float* ginv_lo;              // X_lo: G^-1 - X_hi in single precision
  const NlDev* nl;             // nonlinear resistors: their columns z are written to nlz / nlz_lo
  double* nlz;
  float* nlz_lo;
  const RuntimeSwitchDev* rs;  // runtime switches, stamped by EpochDev::rs_word where that is >= 0
  double* work_g;              // copy of G per matrix, at ep.ginv_off
  double* work_r;              // residual I - G X per matrix, at ep.ginv_off
  int32_t* status;             // per matrix: 0 ok, 1 singular
  // optional per-matrix removals (scenario variants): CSR over matrices of
  // branch indices / line-end indices left out of G (nullptr: none)
  const int32_t* rm_ptr_br;
  const int32_t* rm_br;
  const int32_t* rm_ptr_le;
  const int32_t* rm_le;
};

// Multi-scenario run (the paper's multi-scenario strategy, Sec. III-B):
// one CTA per tile of S_t scenarios runs the whole network for them; a
// warp's lanes are (item, scenario) with the scenario fastest, so every
// solve-matrix load is shared by the scenarios of a warp.  Subsystems meet
// only through lines of delay >= 1, so within a step the subsystems of a
// group are processed together: all injections, then all solves, then all
// updates (three barriers per group and step).  Groups are consecutive
// subsystems whose solve columns fit in shared memory.  Per-scenario state
// is scenario-contiguous in global memory: h[lc][S], ring[slot][S] (ring
// depth d+1: one CTA runs a scenario's subsystems in step order).
//
// Solve columns are numbered globally, subsystem by subsystem: column
// sub_col_off[s] + k is node k of s for k < n, else its strong branch
// k - n.  Batched injection entries name global slots: bits 28-30 the
// kind (0 L/C slot, 1 source-branch slot, 2 line end, 3 control injection:
// its block's output of the previous step, 4 / 5 a frequency-dependent
// end's b / Hy of the step, 6 a coupled end's phase history current of the
// step), bits 0-27 the index, bit 31 subtract.
constexpr uint32_t kBentKindShift = 28;
constexpr uint32_t kBentIndexMask = (1u << 28) - 1;
// Per-scenario state of a frequency-dependent end in the multi-scenario
// kernel: Y_c terms s 0..3, A terms z 4..7, v(n-1) 8, W(n-1) 9, Hy 10, b 11.
constexpr int kBatchFdState = 12;

struct BatchGroupDev {
  int32_t node0, node1;        // internal nodes [node0, node1)
  int32_t col0, col1;          // global solve columns
  int32_t lc0, lc1;            // L/C slots
  int32_t le0, le1;            // line ends
  int32_t lay0, n_lay;         // control layers: block lists cb_lay[lay0 .. lay0 + n_lay] into cb_list
  int32_t nl0, nl1;            // nonlinear resistors of its subsystems
  int32_t nlc0, nlc1;          // their (node, element) correction pairs in BatchParams::nlc
  int32_t fd0, fd1;            // frequency-dependent line ends of its subsystems
  int32_t ce0, ce1;            // coupled line ends of its subsystems
  int32_t sub0, sub1;          // its subsystems
};

struct BatchParams {
  int32_t n_sub, S, S_t;       // subsystems, scenarios, scenarios per CTA
  int32_t n_sources;
  int32_t n_groups, max_cols, max_nodes;
  const BatchGroupDev* grp;
  const double* ginv;
  const float* ginv_lo;
  const int32_t* col_code;     // per global column: internal node, or -1 - L/C slot of a strong branch
  const int32_t* col_sub;      // per global column: its subsystem
  const int32_t* node_sub;     // per internal node: subsystem
  const int32_t* node_r;       // per internal node: row within its subsystem
  const int32_t* sub_nc;       // per subsystem: solve columns n + n_str
  const int32_t* sub_col_off;  // per subsystem: first global column
  const int32_t* ent_ptr;      // [n_nodes + 1]: batched injection entries of each internal node
  const int32_t* bent;         // batched injection entries (no padding)
  const int32_t* lc_nk;        // per L/C slot: end k as internal node, -1 ground, -2-g source g
  const int32_t* lc_nm;
  const double* lc_e;          // history gain +2g (L) / -2g (C)
  const int8_t* lc_isl;        // 1 for L, 0 for C
  const double* sb_g;          // per source-branch slot: conductance
  const int32_t* sb_src;       // per source-branch slot: global source
  const int32_t* le_nd;        // per line end: internal node
  const int32_t* le_d1;        // per line end: d + 1
  const double* le_y2;         // per line end: 2 / Z_c
  const int64_t* le_bring;     // per line end: first slot of its own ring (depth d+1)
  const int64_t* le_bfar;      // per line end: first slot of the far end's ring
  const int64_t* ev_ptr;       // [S + 1]: solve-matrix selections per scenario, by step
  const int64_t* ev_step;      // first step of the selection (0 for the initial one)
  const int32_t* ev_sub;       // subsystem it applies to
  const int64_t* ev_off;       // offset of its solve matrix in ginv / ginv_lo
  const double* src_ac;        // [S][n_sources]: A cos(phase)
  const double* src_as;        // [S][n_sources]: A sin(phase)
  const double* src_omega;     // [n_sources]
  const uint8_t* keep_lc;      // [n_lc][S] 1 = present (nullptr: all present)
  const uint8_t* keep_sb;      // [n_sb][S]
  const uint8_t* keep_le;      // [n_le][S]
  double* h;                   // [n_lc][S]
  double* ring;                // [slots][S]
  // control blocks (global slots: subsystem by subsystem, by layer), their
  // inputs as 2 slot + late over all blocks (zero pair 2 n_cb); outputs
  // cy[(2 slot + parity) S + scenario], states cs[(2 slot + k) S + scenario]
  const CtrlDev* cb;
  const int32_t* cb_lay;       // per group and layer: first entry of cb_list (n_lay + 1 per group)
  const int32_t* cb_list;      // global block slots, layer by layer
  const int32_t* cinj;         // per control injection: global block slot
  const double* cbo;           // [rows][S][3]: per-scenario p0, p1, p2 of blocks with scenario parameters
  double* cy;
  double* cs;
  // nonlinear resistors (compensation method per scenario): records, per
  // element (subsystem, its nodes, its first internal node, 0), the
  // correction pairs (internal node, element), and the currents [n_nl][S];
  // a variant's column z (and its remainder) follows its matrix in ginv
  const NlDev* nl;
  const int32_t* nlinfo;
  const int32_t* nlc;
  double* nl_i;
  // frequency-dependent line ends: records, each one's line end, per line
  // end its FD end or -1, and the states [x][kBatchFdState][S]; an FD end's
  // ring (depth d + 2) holds w by the step it was sent
  const FdEndDev* fd;
  const int32_t* fd_le;
  const int32_t* le_fd;
  double* fds;
  // coupled line ends: records (T_v^-1, T_i, modal Z), each one's first
  // mode line end, per line end its coupled end or -1 and its interpolation
  // fraction f; modal histories [3 x + j][S] and phase currents [3 x + p][S]
  // of the step; a mode's ring (depth d + 2) holds c by the step it was sent
  // runtime switches (states per scenario): records, per subsystem (first
  // switch, count, matrix stride between state words, first internal node),
  // the state words [n_sub][S], breaker currents of the last step [n_rs][S]
  // and each scenario's current variant base [S][n_sub] (its matrix for
  // state word w is at base + w stride)
  const RuntimeSwitchDev* rs;
  const int32_t* sub_rs;
  int32_t* rs_word;
  double* rs_prev_i;
  long long* vbase;
  const CoupledEndDev* ce;
  const int32_t* ce_le0;
  const int32_t* ce_node;      // [3 x + p]: phase nodes as internal nodes
  const int32_t* le_ce;
  const double* le_f;
  double* cim;
  double* cph;
  double* rec;                 // [rows][S][n_rec]
  const int32_t* rec_pos;
  int64_t rec_rows;
  int32_t rec_decim, n_rec;
  int64_t n0, n_steps;
  double dt;
  int32_t* err;                // device error word (the checks build latches there)
  Bounds bnd;                  // ring: slots of the rings x S; h: L/C slots x S; ginv; rec
  // Digit form of the solve on the tensor cores (tcgen05, emt_digits.cuh)
  // for a subsystem whose matrix all scenarios of a tile share: per subsystem
  // s its matrices in digit form, dig_key[x] = ginv offset, dig_val[x] =
  // word offset in dig (x in dig_ptr[s] .. dig_ptr[s + 1]); per subsystem its
  // first internal node and rows; dig_grp: the most subsystems of a group
  // (nullptr dig: off).
  const uint32_t* dig;
  const int32_t* dig_ptr;
  const int64_t* dig_key;
  const int64_t* dig_val;
  const int32_t* sub_node0;
  const int32_t* sub_n;
  int32_t dig_grp;
  int32_t dig_min_rows;        // subsystems of fewer rows keep the FP64 solve (cheaper below ~24 rows)
};

// Digit matrices of the multi-scenario solve, in the shared-memory operand
// layout of tcgen05.mma (K-major, no swizzle: core matrices of 8 rows x 8
// bf16, 128 contiguous bytes, row i of a core matrix at byte 16 i), in
// chunks of 64 columns (kp = nc rounded up to 16; chunk c holds the kc =
// min(64, kp - 64 c) columns from 64 c, one bulk copy each): chunk c at byte
// 65536 c, in it digit plane a (8 planes) of 64 rows (rows past n are zero),
// element (a, r, k) at byte
//   2 a 64 kc + ((r / 8) (kc / 8) + (k - 64 c) / 8) 128 + (r % 8) 16 + (k % 8) 2,
// so that planes 2p and 2p + 1 form one 128-row operand; after the chunks
// the 64 row exponents (int32).  Subsystems of at most kDigRows rows and
// kDigCols columns.
constexpr int kDigRows = 64;
constexpr int kDigCols = 128;
constexpr int kDigChunk = 64;                         // columns of one staged chunk
constexpr int kDigChunkBytes = 16 * kDigRows * kDigChunk;   // 64 KiB: the shared-memory staging of a chunk
__host__ __device__ inline int dig_cols_pad(int nc) { return (nc + 15) & ~15; }
__host__ __device__ inline int dig_chunk_cols(int kp, int c) { return kp - kDigChunk * c < kDigChunk ? kp - kDigChunk * c : kDigChunk; }
// bytes of the digit planes of all chunks (the row exponents follow)
__host__ __device__ inline int64_t dig_planes_bytes(int nc) { return (int64_t)16 * kDigRows * dig_cols_pad(nc); }
__host__ __device__ inline int64_t dig_matrix_words(int nc) { return dig_planes_bytes(nc) / 4 + kDigRows; }
// Scenario rows of the injection digit table of a tile (the tcgen05 N
// blocks): 16 or 32, so that the digit groups of one MMA fit its at most
// 256 accumulator columns
__host__ __device__ inline int dig_tile_rows(int S_t) { return S_t <= 16 ? 16 : 32; }
constexpr int kDigMaxTile = 32;
// shared-memory bytes of the injection digit table of one chunk for a tile
// (8 planes x ts rows x 64 bf16), also the scratch of the accumulator
// read-back (64 rows x ts scenarios x 16 bytes)
__host__ __device__ inline int dig_table_bytes(int ts) { return 16 * ts * kDigChunk; }
cudaError_t launch_batch_digits(const double* ginv, const float* ginv_lo, const int64_t* mat_goff,
                                const int32_t* mat_n, const int32_t* mat_nc, const int64_t* mat_doff, int n_mats,
                                uint32_t* dig, cudaStream_t st);

// A CUDA graph holding the one multi-scenario launch; its kernel node's
// arguments are updated per call.
struct BatchGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t node = nullptr;
  int grid = 0, threads = 0;
  size_t smem = 0;
  const void* func = nullptr;   // the kernel instance of the node
  int64_t launches = 0;
};

// Per-launch upper bounds that size the adjoint kernel's shared memory.
struct AdjLimits {
  int32_t n, nc, q, br, lc, sb, le, src, il, ce;
};

// Reverse sweep of the discrete adjoint over steps n = n_hi, n_hi - 1, ...,
// n_hi - n_steps + 1 (one CTA per subsystem, like the forward kernel).
// Adjoint line values travel through tagged rings with the forward's slot
// layout; the tag of step n is n_total + 1 - n, so tags grow as the sweep
// runs backwards in time and the forward's de-energised ring start serves
// as the adjoint's zero final condition.
struct AdjParams {
  int32_t n_sub;
  AdjLimits lim;
  const SubDev* sub;
  const EpochDev* ep;
  const double* ginv;
  const float* ginv_lo;
  const BranchDev* br;
  const int32_t* br_lc;        // per branch: subsystem-local L/C slot, or -1
  const int32_t* lc_idx;
  const int32_t* ent;
  const int32_t* il_node;
  const int32_t* il_cnt;
  const int32_t* str_slot;
  const LineEndDev* le;
  unsigned long long* ring;    // adjoint rings
  const int32_t* src_global;
  const double* src_amp;       // per global source
  const double* sin_table;     // [n_total][n_sources]: sin(omega t_n + phase), row n - 1
  int32_t n_sources;
  const double* tape;          // [rows][n_nodes] internal order: v_n in row n - 1 - tape_row0
  int64_t tape_row0;
  const double* target;        // [n_total][n_nodes] caller's node order: v*_n in row n - 1
  const int32_t* word_tape;    // [rows][n_sub]: runtime-switch state word of step n (row n - 1 - tape_row0), or null
  const CoupledEndDev* ce;     // coupled line ends
  double* le_prev;             // per line end: adjoint value consumed at the previous reverse step (carried)
  const int32_t* orig_of;      // internal node -> caller's node
  int64_t n_nodes;
  double* hbar;                // per L/C slot: adjoint of h (carried across launches)
  double* dg;                  // per branch: dJ/dg accumulated
  double* dsrc;                // per branch: dJ/dA of its source accumulated
  double* loss_part;           // [n_sub][threads]: partial sums of (v - v*)^2
  int32_t* err;
  int64_t n_total;
  int64_t n_hi, n_steps;
  unsigned long long wait_budget_ns;
  Bounds bnd;
};

struct SourceParams {
  int32_t n_sources;
  const double* amp;           // per global source
  const double* phase;
  const double* omega;         // 2 pi f
  double dt;
  int64_t n0, n_steps;
  double* table;               // [n_steps][n_sources]
};

struct RingInitParams {
  const LineEndDev* le;        // all line ends
  int64_t n_le;
  unsigned long long* ring;
};

// kernels / launchers (emt_kernels.cu)
cudaError_t launch_ring_init(const RingInitParams& p, cudaStream_t st);

// Ring slots a shard exchanges: for each listed line end e and j < w, the
// slot its far ring holds for step n0 + d_e + j (the value e sent at step
// n0 + j), slot far_ring + (n0 + d + j) mod depth; 16 bytes (tag and value
// words) each.  pack = 1: ring -> buf[i w + j]; 0: buf -> ring.
struct RingCopyParams {
  const LineEndDev* le;
  const int32_t* ends;
  int32_t n_ends;
  int32_t w;
  int64_t n0;
  unsigned long long* ring;
  unsigned long long* buf;
  int32_t pack;
};
cudaError_t launch_ring_copy(const RingCopyParams& p, cudaStream_t st);

// Phase-clock build: per CTA, clock64 cycles summed over steps of
//   0 injection, 1 solve, 2 node voltages and compensation, 3 thread 0's
//   updates, 4 the wait of the thread polling line end 0, 5 thread 0 from
//   its updates to the end-of-step barrier (others' updates and polls),
//   6 steps, 7 cycles from the first step's start to the last step's end
//   (of the last launch);
// copied for CTAs 0 .. n-1 (n <= kPhaseCtas) into out, zeroed if reset.
// cudaErrorNotSupported in the normal build.
constexpr int kPhaseCtas = 2048;
constexpr int kPhaseCount = 8;
cudaError_t phase_clocks(unsigned long long* out, int n, bool reset);
// the same for the state-space kernel (emt_ss.cu): 0 thread 0's product rows,
// 1 the poll warp's collection, 2 thread 0 from its rows to the barrier, 6, 7 as above
cudaError_t ss_phase_clocks(unsigned long long* out, int n, bool reset);
cudaError_t launch_companion(BranchDev* br, int64_t n_br, double dt, cudaStream_t st);
cudaError_t launch_coupled_constants(CoupledEndDev* ce, int64_t n_ce, cudaStream_t st);
cudaError_t launch_prefactor(const PrefParams& p, int max_n, cudaStream_t st);
cudaError_t launch_sources(const SourceParams& p, cudaStream_t st);
// wide = false: the 64-register build only (while another persistent grid shares the device);
// ext: some subsystem factorises its switch states at run time (SubDev::n_cache > 0) or holds
// several nonlinear resistors; grp: the network has frequency-dependent line groups
cudaError_t launch_forward(const FwdParams& p, cudaStream_t st, bool wide = true, bool ext = false,
                           bool grp = false);
size_t forward_smem_bytes(const FwdLimits& lim);
// one warp per subsystem (emt_small.cu): subsystems of at most kSmallMaxNodes nodes with basic elements only
constexpr int kSmallMaxNodes = 32;
cudaError_t launch_forward_small(const FwdParams& p, cudaStream_t st);
size_t small_smem_bytes(const FwdLimits& lim);

// State-space form (emt_ss.cu): build M of every (subsystem, epoch) from the
// prefactored G^-1 (P's sub, ep, ginv, ginv_lo, br, lc_idx, sb_idx, le,
// str_slot, ss, ss_m, ss_mlo are used; one CTA per subsystem), and run steps
// with it (a cooperative launch of one CTA per subsystem, as launch_forward).
cudaError_t launch_ss_build(const FwdParams& p, cudaStream_t st);
cudaError_t launch_forward_ss(const FwdParams& p, bool compact, cudaStream_t st);
size_t ss_smem_bytes(int rows, int cols, int n, int le, int src, int ln, int lc);
constexpr int kSsThreads = 256;
int forward_blocks_per_sm(const FwdLimits& lim);   // resident CTAs per SM (0 on error)
cudaError_t launch_batch(const BatchParams& p, int threads, cudaStream_t st, BatchGraph* graph);
size_t batch_smem_bytes(int S_t, int n_sources, int n_sub, int max_cols, int max_nodes, bool digit = false,
                        int dig_grp = 0);
int batch_max_threads(bool digit);   // most threads of a multi-scenario CTA
int batch_min_threads(bool digit);   // fewest (the digit form: a warp per TMEM lane quarter)
// static shared memory the digit-form instance of the multi-scenario kernel
// keeps beside its dynamic shared memory (mbarriers, the TMEM address)
constexpr int kBatchDigitStaticSmem = 256;
void batch_graph_destroy(BatchGraph* graph);
cudaError_t launch_source_coefficients(const double* amp, const double* phase, int64_t count, double* ac, double* as,
                                       cudaStream_t st);
cudaError_t launch_slot_constants(const BranchDev* br, const int32_t* lc_idx, int64_t n_lc, const int32_t* sb_idx,
                                  int64_t n_sb, double* lc_e, double* sb_g, cudaStream_t st);
cudaError_t launch_adjoint(const AdjParams& p, cudaStream_t st);
size_t adjoint_smem_bytes(const AdjLimits& lim);
int adjoint_blocks_per_sm(const AdjLimits& lim);
int adjoint_threads();
cudaError_t launch_adj_finalize(const BranchDev* br, const int32_t* br_orig, int64_t n_br, const double* dg,
                                const double* dsrc, const int32_t* src_br_ptr, const int32_t* src_br, int64_t n_sources,
                                double dt, const double* loss_part, int64_t n_loss, double* grad, double* loss,
                                cudaStream_t st);
cudaError_t launch_gather(const double* rec, int32_t n_rec, int64_t n_scen_rec, const int32_t* col, int64_t n_ch,
                          int64_t row0, int64_t n_rows, int64_t scen0, int64_t n_scen, double* out, cudaStream_t st);

}  // namespace emt
