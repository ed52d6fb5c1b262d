// Host side of libemt: validation, partitioning into subsystems, device
// layout, launches and the C ABI of include/emt.h.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <queue>
#include <set>
#include <array>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/emt.h"
#include "emt_internal.h"

namespace {
// An NVTX range over one call of the C ABI, so that a timeline tool shows
// which entry point issued which launches (header-only NVTX: no cost
// without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

using namespace emt;

namespace {

thread_local std::string g_build_error;

const double kTwoPi = 2.0 * 3.14159265358979323846;

// Shared memory given to the solve matrix [G^-1 | strong columns] of one
// subsystem (double + single-precision parts).
const double kSolveSmemBytes = 150.0 * 1024;

// The state-space form runs by default while every subsystem's M has at
// most this many entries: beyond, its product's work outgrows what the
// shorter chain saves against the CTA kernel.
const int64_t kSsAutoEntries = 2048;

// Source-voltage table budget per chunk of a launch (doubles): 32 MiB.
const int64_t kSourceTableDoubles = 4 << 20;

}  // namespace

struct emt_ctx {
  std::string err;
  int device = 0;
  double dt = 0.0;
  int64_t n_nodes = 0, n_branches = 0, n_sources = 0, n_lines = 0;

  // partition and internal numbering
  int n_sub = 0;
  std::vector<int32_t> sub_of_node;     // original node -> subsystem
  std::vector<int32_t> internal_of;     // original node -> internal id
  std::vector<int32_t> original_of;     // internal id -> original node

  // host images of the device arrays
  std::vector<SubDev> subs;
  std::vector<EpochDev> epochs;
  std::vector<BranchDev> branches;
  std::vector<int32_t> lc_idx, sb_idx;
  std::vector<int32_t> ent, il_node, il_cnt, str_slot;
  std::vector<LineEndDev> line_ends;
  std::vector<int32_t> br_orig;                        // internal branch -> caller's branch index
  std::vector<int32_t> br_lc;                          // internal branch -> subsystem-local L/C slot or -1
  std::vector<int32_t> br_src;                         // internal branch -> global source at one end or -1
  std::vector<int32_t> src_br_ptr, src_br;             // per global source: its branches (CSR, internal order)
  std::vector<int32_t> src_global;                     // global source id per local source slot
  std::vector<double> src_amp, src_phase, src_omega;   // per global source
  std::vector<int32_t> nb_sub, nb_dmin;
  std::vector<SwitchDev> switches;
  std::vector<RuntimeSwitchDev> rswitches;             // runtime switches, grouped by subsystem
  std::vector<double> rs_roff;                         // their off resistances
  std::vector<CoupledEndDev> cends;                    // coupled line ends, grouped by subsystem
  std::vector<int32_t> rs_word0;                       // per subsystem: state word at step 1
  std::vector<FdEndDev> fdends;                        // frequency-dependent line ends, grouped by subsystem
  std::vector<NlDev> nls;                              // nonlinear resistors, grouped by subsystem
  int64_t nlz_len = 0;                                 // doubles of their columns over all matrix entries
  std::vector<CtrlDev> cblocks;                        // control blocks, grouped by subsystem, by layer
  std::vector<int32_t> clay, cinj;                     // layer starts; block slot per control injection
  std::vector<int32_t> cb_slot_of;                     // caller's block index -> subsystem-local slot
  std::vector<int32_t> cb_sub_of;                      // caller's block index -> subsystem
  int max_clayers = 0;
  int64_t ring_len = 0, ginv_len = 0, n_lc_total = 0;
  int64_t n_components = 0;
  // subsystems that factorise their switch states at run time (SubDev::n_cache)
  bool lazy = false;
  std::vector<long long> cache_tag0;   // initial tags of every cache slot
  std::vector<int32_t> cache_next0;    // per subsystem: initial slot to replace next; then 0 (factorisations)
  int64_t lazy_work_len = 0;
  long long* d_cache_tag = nullptr;
  long long* d_cache_tag0 = nullptr;
  int32_t* d_cache_next = nullptr;
  int32_t* d_cache_next0 = nullptr;
  double* d_lazy_work = nullptr;
  // one warp per subsystem (emt_small.cu), for networks whose subsystems are all small and hold basic
  // elements only; opt-in (option warp_per_subsystem): measured no faster than the CTA kernel, whose eight
  // warps spread a subsystem's FP64 work over all four FP64 pipes of its SM
  bool small_ok = false;
  bool use_small = false;
  // state-space form (emt_ss.cu): eligible networks (ss_ok) run it unless the option state_space is 0;
  // auto (1) only while every subsystem's M is at most kSsAutoEntries, 2 forces it
  bool ss_ok = false;
  bool ss_compact = false;   // every subsystem takes the compact step (several CTAs to an SM)
  int ss_mode = 1;
  int64_t ss_len = 0, ss_max_entries = 0;
  int ss_rows = 0, ss_cols = 0, ss_ln = 0;
  std::vector<SsSubDev> ss;
  std::vector<int32_t> ss_lnode, ss_lptr, ss_lend;
  SsSubDev* d_ss = nullptr;
  double* d_ss_m = nullptr;
  float* d_ss_mlo = nullptr;
  int32_t* d_ss_lnode = nullptr;
  int32_t* d_ss_lptr = nullptr;
  int32_t* d_ss_lend = nullptr;
  bool forward_narrow = false;   // emt_adjoint: its re-runs share the device with the reverse sweep
  bool fd_groups = false;        // frequency-dependent line groups (their code is in kernel builds of their own)
  int64_t comp_sum_n2 = 0, comp_max_n = 0;   // over the components
  FwdLimits lim{0, 0, 1, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0};

  // device arrays
  SubDev* d_sub = nullptr;
  EpochDev* d_ep = nullptr;
  BranchDev* d_br = nullptr;
  int32_t* d_lc_idx = nullptr;
  int32_t* d_sb_idx = nullptr;
  double* d_h = nullptr;
  int32_t* d_ent = nullptr;
  int32_t* d_il_node = nullptr;
  int32_t* d_il_cnt = nullptr;
  int32_t* d_str_slot = nullptr;
  LineEndDev* d_le = nullptr;
  unsigned long long* d_ring = nullptr;
  int32_t* d_src_global = nullptr;
  int32_t* d_br_orig = nullptr;
  int32_t* d_br_lc = nullptr;
  int32_t* d_br_src = nullptr;
  int32_t* d_src_br_ptr = nullptr;
  int32_t* d_src_br = nullptr;
  int32_t* d_original_of = nullptr;
  double* d_src_amp = nullptr;
  double* d_src_phase = nullptr;
  double* d_src_omega = nullptr;
  double* d_src_table = nullptr;
  int64_t src_table_steps = 0;
  SwitchDev* d_sw = nullptr;
  RuntimeSwitchDev* d_rs = nullptr;
  CoupledEndDev* d_ce = nullptr;
  double* d_le_prev = nullptr;
  int32_t* d_rs_word = nullptr;
  double* d_rs_prev_i = nullptr;
  FdEndDev* d_fd = nullptr;
  NlDev* d_nl = nullptr;
  int32_t* d_nl_seg = nullptr;                         // per nonlinear resistor: its segment at the last step
  double* d_nlz = nullptr;
  float* d_nlz_lo = nullptr;
  double* d_fd_state = nullptr;
  CtrlDev* d_cb = nullptr;
  int32_t* d_clay = nullptr;
  int32_t* d_cinj = nullptr;
  double* d_cstate = nullptr;
  double* d_cy = nullptr;
  double* d_ginv = nullptr;
  float* d_ginv_lo = nullptr;
  int32_t* d_err = nullptr;

  // recording
  std::vector<int32_t> rec_channels;     // original node ids, column order
  std::vector<int32_t> rec_col_of;       // original node -> column or -1
  int32_t rec_decim = 1;
  int64_t rec_rows = 0;
  double* d_rec = nullptr;
  int32_t* d_rec_pos = nullptr;          // internal node -> column or -1

  // run state and knobs
  int64_t step = 0;
  bool prefactored = false;
  bool overlap_adjoint = true;
  unsigned long long wait_budget_ns = 2000000000ull;
  int32_t hold_sub = -1;
  int64_t launches = 0;

  // multi-scenario mode (emt_build_network with a scenario set)
  bool batched = false;
  int64_t S = 1;
  int S_t = 1;
  int64_t n_base_epochs = 0;
  std::vector<int32_t> node_l0, node_nl;
  std::vector<int64_t> le_bring, le_bfar;
  int64_t bring_len = 0;
  std::vector<double> bsrc_amp, bsrc_phase;            // [S][n_sources]
  std::vector<uint8_t> keep_lc, keep_sb, keep_le;      // [slot][S], empty if nothing is removed
  std::vector<int64_t> msel_ptr, msel_start;
  std::vector<int32_t> msel_mat;
  std::vector<int32_t> var_sub;                        // subsystem of each variant matrix
  std::vector<int32_t> rm_ptr_br, rm_br, rm_ptr_le, rm_le;
  // flat per-slot arrays of the multi-scenario kernel (see BatchParams)
  std::vector<int32_t> b_col_code, b_col_sub, b_node_sub, b_node_r, b_sub_nc, b_sub_col_off, b_ent_ptr, b_bent;
  std::vector<int32_t> b_lc_nk, b_lc_nm, b_sb_src, b_le_nd, b_le_d1, b_ev_sub;
  std::vector<double> b_lc_e, b_sb_g, b_le_y2;
  std::vector<int8_t> b_lc_isl;
  std::vector<int64_t> b_ev_ptr, b_ev_step, b_ev_off;
  int32_t *d_col_code = nullptr, *d_col_sub = nullptr, *d_node_sub = nullptr, *d_node_r = nullptr, *d_sub_nc = nullptr,
          *d_sub_col_off = nullptr, *d_ent_ptr = nullptr, *d_bent = nullptr, *d_lc_nk = nullptr,
          *d_lc_nm = nullptr, *d_sb_src = nullptr, *d_le_nd = nullptr, *d_le_d1 = nullptr, *d_ev_sub = nullptr;
  double *d_lc_e = nullptr, *d_sb_g = nullptr, *d_le_y2 = nullptr, *d_src_ac = nullptr, *d_src_as = nullptr;
  int8_t* d_lc_isl = nullptr;
  int64_t *d_ev_ptr = nullptr, *d_ev_step = nullptr, *d_ev_off = nullptr;
  // launch configuration: scenarios per CTA, threads, subsystem groups
  int batch_threads = 512;
  std::vector<BatchGroupDev> groups;
  int max_cols = 0, max_nodes = 0;
  BatchGroupDev* d_grp = nullptr;
  BatchGraph graph;
  bool use_graph = true;
  // digit form of the multi-scenario solve (emt_batch.cu): matrices that
  // whole tiles share, in digit form; option digit_solve
  bool use_digit = false;
  bool digit_auto = true;   // digit_solve not set: emt_autotune times both forms and keeps the faster
  int dig_min_rows = 24;   // option digit_min_rows: smaller subsystems keep the FP64 solve
  bool dig_on = false;                                // the digit form runs (current configuration)
  int dig_grp = 0;                                    // most subsystems of a group (current S_t)
  int64_t dig_len = 0;
  std::vector<int32_t> dig_ptr, dig_sub_n, dig_node0, dig_mat_n, dig_mat_nc;
  std::vector<int64_t> dig_key, dig_val, dig_mat_goff;
  uint32_t* d_dig = nullptr;
  int32_t *d_dig_ptr = nullptr, *d_sub_node0 = nullptr, *d_sub_n = nullptr, *d_dig_mat_n = nullptr,
          *d_dig_mat_nc = nullptr;
  int64_t *d_dig_key = nullptr, *d_dig_val = nullptr, *d_dig_mat_goff = nullptr;
  bool tuned = false;
  int64_t* d_le_bring = nullptr;
  int64_t* d_le_bfar = nullptr;
  double* d_bsrc_amp = nullptr;
  double* d_bsrc_phase = nullptr;
  uint8_t* d_keep_lc = nullptr;
  uint8_t* d_keep_sb = nullptr;
  uint8_t* d_keep_le = nullptr;
  double* d_bh = nullptr;
  double* d_bring = nullptr;
  int32_t* d_rm_ptr_br = nullptr;
  int32_t* d_rm_br = nullptr;
  int32_t* d_rm_ptr_le = nullptr;
  int32_t* d_rm_le = nullptr;
  // control blocks of the multi-scenario kernel (see BatchParams)
  std::vector<CtrlDev> b_cb;
  std::vector<int32_t> b_cinj, b_cb_lay, b_cb_list;
  std::vector<double> b_cbo;
  CtrlDev* d_bcb = nullptr;
  int32_t *d_bcinj = nullptr, *d_bcb_lay = nullptr, *d_bcb_list = nullptr;
  double *d_bcbo = nullptr, *d_bcy = nullptr, *d_bcs = nullptr;
  // nonlinear resistors of the multi-scenario kernel (see BatchParams)
  std::vector<int32_t> b_nlinfo, b_nlc;
  int32_t *d_bnlinfo = nullptr, *d_bnlc = nullptr;
  double* d_bnli = nullptr;
  // frequency-dependent ends of the multi-scenario kernel (see BatchParams)
  std::vector<int32_t> b_fd_le, b_le_fd;
  int32_t *d_bfd_le = nullptr, *d_ble_fd = nullptr;
  double* d_bfds = nullptr;
  // runtime switches of the multi-scenario kernel (see BatchParams)
  std::vector<int32_t> b_sub_rs;
  int32_t *d_bsub_rs = nullptr, *d_bword = nullptr;
  double* d_brsi = nullptr;
  long long* d_bvbase = nullptr;
  // coupled ends of the multi-scenario kernel (see BatchParams)
  std::vector<int32_t> b_ce_le0, b_le_ce, b_ce_node;
  std::vector<double> b_le_f;
  int32_t *d_bce_le0 = nullptr, *d_ble_ce = nullptr, *d_bce_node = nullptr;
  double *d_ble_f = nullptr, *d_bcim = nullptr, *d_bcph = nullptr;

  // shard of the network this context runs (emt_set_shard): the CTAs it
  // owns, and per peer rank the line ends whose sent values cross over
  // (ascending library order, so that both sides list them alike)
  bool sharded = false;
  int32_t shard_rank = -1;
  int32_t shard_window = 0;                 // largest window: min d over the cut line ends
  std::vector<int32_t> shard_active;        // CTAs run here
  std::map<int32_t, std::vector<int32_t>> shard_send, shard_recv;
  std::map<int32_t, int64_t> shard_send_off, shard_recv_off;   // offsets into d_shard_ends
  std::set<int32_t> shard_to_pack, shard_to_unpack;         // peers the last window still owes
  int64_t win_n0 = 0, win_w = 0;            // steps of the last window
  int32_t* d_shard_active = nullptr;
  SubDev* d_shard_sub = nullptr;            // their descriptions, in that order
  int32_t* d_shard_ends = nullptr;

  std::vector<void*> allocations;

  emt_status fail(emt_status st, const std::string& msg) {
    err = msg;
    return st;
  }
  emt_status cuda_fail(cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? EMT_ENOMEM : EMT_ECUDA;
  }
  template <class T>
  cudaError_t upload(T** dst, const std::vector<T>& src) {
    const size_t n = std::max<size_t>(src.size(), 1);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) return e;
    allocations.push_back(p);
    if (!src.empty()) e = cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    *dst = static_cast<T*>(p);
    return e;
  }
  template <class T>
  cudaError_t alloc_zero(T** dst, size_t count) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return e;
    allocations.push_back(p);
    *dst = static_cast<T*>(p);
    return cudaMemset(p, 0, bytes);
  }
  void release(void* p) {
    if (!p) return;
    auto it = std::find(allocations.begin(), allocations.end(), p);
    if (it != allocations.end()) allocations.erase(it);
    cudaFree(p);
  }
};

namespace {

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Inverse of a 3 x 3 row-major matrix (cofactors); false if singular to working
// precision: |det| at most 1e-12 of Hadamard's bound, the product of the row norms.
bool invert3_host(const double* a, double* inv) {
  const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
  const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  double bound = 1.0;
  for (int r = 0; r < 3; ++r)
    bound *= std::sqrt(a[3 * r] * a[3 * r] + a[3 * r + 1] * a[3 * r + 1] + a[3 * r + 2] * a[3 * r + 2]);
  if (!std::isfinite(det) || !std::isfinite(bound) || !(std::fabs(det) > 1e-12 * bound)) return false;
  inv[0] = c00 / det;
  inv[3] = c01 / det;
  inv[6] = c02 / det;
  inv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  inv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  inv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
  return true;
}


std::string validate(const emt_network_desc* d) {
  if (!d) return "desc is NULL";
  if (!finite_pos(d->dt)) return "dt must be finite and > 0";
  if (d->n_nodes < 0 || d->n_branches < 0 || d->n_sources < 0 || d->n_lines < 0 || d->n_switches < 0)
    return "negative count";
  if (d->n_nodes > (1 << 28) || d->n_sources > (1 << 28)) return "too many nodes or sources";
  auto node_ok = [&](int32_t x) { return x >= -1 - d->n_sources && x < d->n_nodes; };
  if (d->n_branches && (!d->br_k || !d->br_m || !d->br_kind || !d->br_value)) return "branch array is NULL";
  for (int64_t b = 0; b < d->n_branches; ++b) {
    const int32_t k = d->br_k[b], m = d->br_m[b];
    if (!node_ok(k) || !node_ok(m)) return "branch " + std::to_string(b) + ": node out of range";
    if (k == m) return "branch " + std::to_string(b) + ": both ends on one node";
    if (k < 0 && m < 0) return "branch " + std::to_string(b) + ": no unknown end";
    if (d->br_kind[b] > 2) return "branch " + std::to_string(b) + ": kind must be 0 (R), 1 (L) or 2 (C)";
    if (!finite_pos(d->br_value[b])) return "branch " + std::to_string(b) + ": value must be finite and > 0";
  }
  if (d->n_sources && (!d->src_amp || !d->src_phase || !d->src_freq)) return "source array is NULL";
  for (int64_t s = 0; s < d->n_sources; ++s)
    if (!std::isfinite(d->src_amp[s]) || !std::isfinite(d->src_phase[s]) || !std::isfinite(d->src_freq[s]))
      return "source " + std::to_string(s) + ": non-finite parameter";
  if (d->n_lines && (!d->ln_k || !d->ln_m || !d->ln_zc || !d->ln_delay)) return "line array is NULL";
  for (int64_t l = 0; l < d->n_lines; ++l) {
    if (d->ln_k[l] < 0 || d->ln_k[l] >= d->n_nodes || d->ln_m[l] < 0 || d->ln_m[l] >= d->n_nodes)
      return "line " + std::to_string(l) + ": ends must be unknown nodes";
    if (d->ln_k[l] == d->ln_m[l]) return "line " + std::to_string(l) + ": both ends on one node";
    if (d->ln_delay[l] < 1) return "line " + std::to_string(l) + ": delay must be >= 1 step";
    if (d->ln_delay[l] > (1 << 20)) return "line " + std::to_string(l) + ": delay too large";
    if (!finite_pos(d->ln_zc[l])) return "line " + std::to_string(l) + ": Z_c must be finite and > 0";
  }
  if (d->n_clines < 0) return "negative count";
  if (d->n_clines && (!d->cl_k || !d->cl_m || !d->cl_tv || !d->cl_z || !d->cl_tau)) return "coupled line array is NULL";
  for (int64_t l = 0; l < d->n_clines; ++l) {
    const std::string nm = "coupled line " + std::to_string(l);
    for (int p = 0; p < 3; ++p)
      if (d->cl_k[3 * l + p] < 0 || d->cl_k[3 * l + p] >= d->n_nodes || d->cl_m[3 * l + p] < 0 ||
          d->cl_m[3 * l + p] >= d->n_nodes)
        return nm + ": ends must be unknown nodes";
    for (int j = 0; j < 3; ++j) {
      if (!finite_pos(d->cl_z[3 * l + j])) return nm + ": Z_c must be finite and > 0";
      if (!std::isfinite(d->cl_tau[3 * l + j]) || !(d->cl_tau[3 * l + j] >= d->dt))
        return nm + ": travel times must be finite and at least dt";
      if (d->cl_tau[3 * l + j] / d->dt > (double)(1 << 20)) return nm + ": travel time too large";
    }
    double inv[9];
    if (!invert3_host(d->cl_tv + 9 * l, inv)) return nm + ": T_v is singular";
  }
  if (d->n_rswitches < 0) return "negative count";
  if (d->n_rswitches && (!d->rs_k || !d->rs_m || !d->rs_kind || !d->rs_ron || !d->rs_roff || !d->rs_on0 ||
                         !d->rs_trip_step))
    return "runtime switch array is NULL";
  for (int64_t w = 0; w < d->n_rswitches; ++w) {
    const int32_t k = d->rs_k[w], m = d->rs_m[w];
    if (k < -1 || m < -1 || k >= d->n_nodes || m >= d->n_nodes || k == m || (k < 0 && m < 0))
      return "runtime switch " + std::to_string(w) + ": ends must be unknown nodes or ground";
    if (d->rs_kind[w] > 1) return "runtime switch " + std::to_string(w) + ": kind must be 0 (diode) or 1 (breaker)";
    if (!finite_pos(d->rs_ron[w]) || !finite_pos(d->rs_roff[w]))
      return "runtime switch " + std::to_string(w) + ": resistances must be finite and > 0";
  }
  if (d->n_nonlin < 0) return "negative count";
  if (d->n_nonlin && (!d->nl_k || !d->nl_m || !d->nl_np || !d->nl_v || !d->nl_i))
    return "nonlinear resistor array is NULL";
  for (int64_t x = 0; x < d->n_nonlin; ++x) {
    const std::string nm = "nonlinear resistor " + std::to_string(x);
    const int32_t k = d->nl_k[x], m = d->nl_m[x];
    if (k < -1 || m < -1 || k >= d->n_nodes || m >= d->n_nodes || k == m || (k < 0 && m < 0))
      return nm + ": ends must be unknown nodes or ground";
    if (d->nl_np[x] < 1 || d->nl_np[x] > kNlMaxPoints) return nm + ": 1 to 8 breakpoints";
    double pv = 0.0, pi = 0.0;
    for (int j = 0; j < d->nl_np[x]; ++j) {
      const double v = d->nl_v[kNlMaxPoints * x + j], i = d->nl_i[kNlMaxPoints * x + j];
      if (!std::isfinite(v) || !std::isfinite(i) || !(v > pv) || !(i >= pi))
        return nm + ": breakpoints need increasing v > 0 and nondecreasing i >= 0";
      pv = v;
      pi = i;
    }
  }
  if (d->n_fdlines < 0) return "negative count";
  if (d->n_fdlines && (!d->fl_k || !d->fl_m || !d->fl_tau || !d->fl_y0 || !d->fl_ny || !d->fl_yq || !d->fl_yc ||
                       !d->fl_a0 || !d->fl_na || !d->fl_ap || !d->fl_ar))
    return "frequency-dependent line array is NULL";
  for (int64_t l = 0; l < d->n_fdlines; ++l) {
    const std::string nm = "frequency-dependent line " + std::to_string(l);
    const int32_t k = d->fl_k[l], m = d->fl_m[l];
    if (k < 0 || m < 0 || k >= d->n_nodes || m >= d->n_nodes) return nm + ": ends must be unknown nodes";
    if (k == m) return nm + ": both ends on one node";
    if (!std::isfinite(d->fl_tau[l]) || !(d->fl_tau[l] >= d->dt)) return nm + ": travel time must be finite and at least dt";
    if (d->fl_tau[l] / d->dt > (double)(1 << 20)) return nm + ": travel time too large";
    if (!std::isfinite(d->fl_y0[l]) || !(d->fl_y0[l] >= 0.0) || !std::isfinite(d->fl_a0[l]))
      return nm + ": y0 must be finite and >= 0, a0 finite";
    if (d->fl_ny[l] < 0 || d->fl_ny[l] > 4 || d->fl_na[l] < 0 || d->fl_na[l] > 4)
      return nm + ": at most 4 poles each";
    double geq = d->fl_y0[l];
    for (int i = 0; i < d->fl_ny[l]; ++i) {
      const double q = d->fl_yq[4 * l + i], r = d->fl_yc[4 * l + i];
      if (!std::isfinite(q) || !(q < 0.0) || !std::isfinite(r)) return nm + ": poles must be finite and < 0";
      geq += r * (d->dt / 2.0) / (1.0 - q * d->dt / 2.0);
    }
    for (int i = 0; i < d->fl_na[l]; ++i)
      if (!std::isfinite(d->fl_ap[4 * l + i]) || !(d->fl_ap[4 * l + i] < 0.0) || !std::isfinite(d->fl_ar[4 * l + i]))
        return nm + ": poles must be finite and < 0";
    if (!(geq > 0.0)) return nm + ": its end conductance y0 + sum mu must be > 0";
  }
  if (d->n_fdgroups < 0) return "negative count";
  if (d->n_fdgroups && (!d->fg_line || !d->fg_tv)) return "frequency-dependent line group array is NULL";
  {
    std::vector<char> grouped((size_t)std::max<int64_t>(d->n_fdlines, 0), 0);
    for (int64_t gi = 0; gi < d->n_fdgroups; ++gi) {
      const std::string nm = "frequency-dependent line group " + std::to_string(gi);
      for (int j = 0; j < 3; ++j) {
        const int32_t l = d->fg_line[3 * gi + j];
        if (l < 0 || l >= d->n_fdlines) return nm + ": line index out of range";
        if (grouped[l]) return nm + ": line " + std::to_string(l) + " is in a group twice";
        grouped[l] = 1;
      }
      for (int k = 0; k < 9; ++k)
        if (!std::isfinite(d->fg_tv[9 * gi + k])) return nm + ": T_v must be finite";
      double inv[9];
      if (!invert3_host(d->fg_tv + 9 * gi, inv)) return nm + ": T_v must be invertible";
    }
  }
  if (d->n_cblocks < 0 || d->n_cinj < 0) return "negative count";
  if (d->n_cblocks && (!d->cb_type || !d->cb_in0 || !d->cb_in1 || !d->cb_node || !d->cb_p0 || !d->cb_p1))
    return "control block array is NULL";
  if (d->n_cinj && (!d->ci_block || !d->ci_node)) return "control injection array is NULL";
  if (d->n_cblocks >= (1 << 24)) return "too many control blocks";
  for (int64_t b = 0; b < d->n_cblocks; ++b) {
    const std::string nm = "control block " + std::to_string(b);
    const int t = d->cb_type[b];
    if (t > 8) return nm + ": type must be 0..8";
    if (!std::isfinite(d->cb_p0[b]) || !std::isfinite(d->cb_p1[b])) return nm + ": non-finite parameter";
    const int n_in = t <= 1 ? 0 : (t == 3 || t == 4) ? 2 : 1;
    const int32_t in[2] = {d->cb_in0[b], d->cb_in1[b]};
    for (int i = 0; i < n_in; ++i)
      if (in[i] < 0 || in[i] >= d->n_cblocks) return nm + ": input " + std::to_string(i) + " is not a block";
    if (t == 1 && (d->cb_node[b] < 0 || d->cb_node[b] >= d->n_nodes)) return nm + ": measured node must be unknown";
    if (t == 5 && !(d->cb_p0[b] <= d->cb_p1[b])) return nm + ": limits need p0 <= p1";
    if (t == 7 && !(d->cb_p1[b] > 0.0)) return nm + ": lag time constant must be > 0";
  }
  for (int64_t x = 0; x < d->n_cinj; ++x)
    if (d->ci_block[x] < 0 || d->ci_block[x] >= d->n_cblocks || d->ci_node[x] < 0 || d->ci_node[x] >= d->n_nodes)
      return "control injection " + std::to_string(x) + ": needs a block and an unknown node";
  if (d->n_switches && (!d->sw_k || !d->sw_m || !d->sw_r || !d->sw_close_step || !d->sw_open_step))
    return "switch array is NULL";
  for (int64_t w = 0; w < d->n_switches; ++w) {
    const int32_t k = d->sw_k[w], m = d->sw_m[w];
    if (k < -1 || m < -1 || k >= d->n_nodes || m >= d->n_nodes || k == m || (k < 0 && m < 0))
      return "switch " + std::to_string(w) + ": ends must be unknown nodes or ground";
    if (!finite_pos(d->sw_r[w])) return "switch " + std::to_string(w) + ": resistance must be finite and > 0";
  }
  return "";
}

int uf_find(std::vector<int>& p, int x) {
  while (p[x] != x) {
    p[x] = p[p[x]];
    x = p[x];
  }
  return x;
}

bool switch_closed(int64_t on, int64_t off, int64_t n) { return on >= 0 && n >= on && (off < 0 || n < off); }

// A control block's coefficients in device form (see CtrlDev) from its
// parameters p0, p1 and the step.
void ctrl_coefficients(CtrlDev& r, double p0, double p1, double dt) {
  r.p0 = p0;
  r.p1 = p1;
  r.p2 = 0.0;
  if (r.type == 6) r.p0 = p0 * (dt / 2.0);
  if (r.type == 7) {
    r.p0 = (2.0 * p1 - dt) / (2.0 * p1 + dt);
    r.p1 = p0 * dt / (2.0 * p1 + dt);
  }
  if (r.type == 8) r.p2 = dt / 2.0;
}

std::string validate_scenarios(const emt_network_desc* d, const emt_scenario_desc* sc) {
  if (sc->n_scenarios < 1 || sc->n_scenarios > (1 << 24)) return "n_scenarios must be in 1 .. 2^24";
  const int64_t S = sc->n_scenarios;
  for (int64_t i = 0; sc->src_amp && i < S * d->n_sources; ++i)
    if (!std::isfinite(sc->src_amp[i])) return "scenario source amplitude is not finite";
  for (int64_t i = 0; sc->src_phase && i < S * d->n_sources; ++i)
    if (!std::isfinite(sc->src_phase[i])) return "scenario source phase is not finite";
  auto csr = [&](const int64_t* ptr, const void* data, const char* what) -> std::string {
    if (!ptr) return "";
    if (!data && ptr[S] > 0) return std::string(what) + " list is NULL";
    if (ptr[0] != 0) return std::string(what) + " pointer must start at 0";
    for (int64_t s = 0; s < S; ++s)
      if (ptr[s + 1] < ptr[s]) return std::string(what) + " pointer must not decrease";
    return "";
  };
  std::string m = csr(sc->rm_branch_ptr, sc->rm_branch, "removed-branch");
  if (m.empty()) m = csr(sc->rm_line_ptr, sc->rm_line, "removed-line");
  if (m.empty()) m = csr(sc->sw_ptr, sc->sw_k, "scenario-switch");
  if (!m.empty()) return m;
  if (sc->rm_branch_ptr)
    for (int64_t i = 0; i < sc->rm_branch_ptr[S]; ++i)
      if (sc->rm_branch[i] < 0 || sc->rm_branch[i] >= d->n_branches) return "removed branch out of range";
  if (sc->rm_line_ptr)
    for (int64_t i = 0; i < sc->rm_line_ptr[S]; ++i)
      if (sc->rm_line[i] < 0 || sc->rm_line[i] >= d->n_lines) return "removed line out of range";
  if (sc->sw_ptr) {
    if (!sc->sw_m || !sc->sw_r || !sc->sw_close_step || !sc->sw_open_step) return "scenario-switch array is NULL";
    for (int64_t w = 0; w < sc->sw_ptr[S]; ++w) {
      const int32_t k = sc->sw_k[w], m2 = sc->sw_m[w];
      if (k < -1 || m2 < -1 || k >= d->n_nodes || m2 >= d->n_nodes || k == m2 || (k < 0 && m2 < 0))
        return "scenario switch " + std::to_string(w) + ": ends must be unknown nodes or ground";
      if (!finite_pos(sc->sw_r[w])) return "scenario switch " + std::to_string(w) + ": resistance must be > 0";
    }
  }
  if (sc->cbo_ptr) {
    m = csr(sc->cbo_ptr, sc->cbo_block, "control-parameter");
    if (!m.empty()) return m;
    if (sc->cbo_ptr[S] > 0 && !sc->cbo_p0) return "control-parameter value list is NULL";
    for (int64_t q = 0; q < S; ++q) {
      std::set<int32_t> seen;
      for (int64_t i = sc->cbo_ptr[q]; i < sc->cbo_ptr[q + 1]; ++i) {
        const int32_t b = sc->cbo_block[i];
        if (b < 0 || b >= d->n_cblocks) return "control-parameter block out of range";
        if (!seen.insert(b).second) return "a scenario sets the parameter of a control block twice";
        if (!std::isfinite(sc->cbo_p0[i])) return "control-parameter value is not finite";
        if (d->cb_type[b] == 5 && sc->cbo_p0[i] > d->cb_p1[b]) return "a LIMIT's lower bound exceeds its upper bound";
      }
    }
  }
  return "";
}

}  // namespace

// ------------------------------------------------------------------ scenarios

// Multi-scenario set: per (scenario, subsystem) the switch epochs and the
// solve-matrix variant of each (deduplicated by content: subsystem, removed
// branches and line ends, closed switches with their conductances), the
// removal masks, per-scenario sources and the batched line rings.
// Group consecutive subsystems so that one group's solve columns and nodes
// fit in the multi-scenario kernel's shared memory for S_t scenarios per
// CTA; upload the groups when `upload`.  False if one subsystem alone does
// not fit.
// Every scenario's runtime-switch state words back to the initial ones.
cudaError_t reset_batch_words(emt_ctx* c) {
  std::vector<int32_t> w((size_t)c->n_sub * c->S);
  for (int s = 0; s < c->n_sub; ++s)
    std::fill(w.begin() + (size_t)s * c->S, w.begin() + (size_t)(s + 1) * c->S, c->rs_word0[s]);
  return cudaMemcpy(c->d_bword, w.data(), w.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
}

// Shared memory a subsystem adds to its group in the digit form: its entry
// of the selections (0 with the digit form off).
size_t batch_dig_bytes(const emt_ctx* c, int s, int S_t) {
  (void)s;
  (void)S_t;
  return c->use_digit && !c->dig_key.empty() ? 8 + 16 + 4 * kDigMaxTile : 0;   // dsel, dmeta, exponents
}

bool batch_configure(emt_ctx* c, int S_t, bool upload) {
  const bool dig = c->use_digit && !c->dig_key.empty();
  if (dig && S_t > kDigMaxTile) return false;   // (the digit table holds at most 32 scenario rows)
  // the digit form's fixed part: the tile's exponents, alignment, one matrix's planes and the digit table
  const size_t fixed = batch_smem_bytes(S_t, (int)c->n_sources, c->n_sub, 0, 0, dig, 0) +
                       (dig ? kBatchDigitStaticSmem : 0);
  if (fixed >= 227 * 1024) return false;
  size_t budget = 227 * 1024 - fixed - 16;
  int dig_grp = 0;   // digit form: most subsystems of a group
  std::vector<BatchGroupDev> groups;
  std::vector<int32_t> lay, list;   // control layers per group (see BatchGroupDev)
  int max_cols = 0, max_nodes = 0;
  // (with the digit form the largest columns, nodes, members and tables may
  // come from different groups: the budget shrinks until their sum fits)
  for (int attempt = 0;; ++attempt) {
    groups.clear();
    lay.clear();
    list.clear();
    max_cols = max_nodes = dig_grp = 0;
    int s0 = 0;
    while (s0 < c->n_sub) {
      int s1 = s0, cols = 0, nodes = 0;
      size_t dbytes = 0;
      while (s1 < c->n_sub) {
        const SubDev& sd = c->subs[s1];
        const int nc2 = cols + sd.n + sd.n_str, n2 = nodes + sd.n;
        const size_t d2 = dbytes + batch_dig_bytes(c, s1, S_t);
        if (((size_t)nc2 * 12 + (size_t)n2 * 8) * S_t + d2 > budget) break;
        cols = nc2;
        nodes = n2;
        dbytes = d2;
        ++s1;
      }
      if (dig && s1 > s0) dig_grp = std::max(dig_grp, s1 - s0);
      if (s1 == s0) return false;
      const SubDev& a = c->subs[s0];
      const SubDev& b = c->subs[s1 - 1];
      BatchGroupDev G{};
      // control layers: layer l of the group = layer l of each of its subsystems
      G.lay0 = (int)lay.size();
      for (int s = s0; s < s1; ++s) G.n_lay = std::max(G.n_lay, c->subs[s].n_clay);
      for (int l = 0; l < G.n_lay; ++l) {
        lay.push_back((int32_t)list.size());
        for (int s = s0; s < s1; ++s) {
          const SubDev& sd = c->subs[s];
          if (l >= sd.n_clay) continue;
          constexpr int kSlotMask = (1 << kLayerTypeShift) - 1;
          const int j0 = c->clay[sd.clay_off + l] & kSlotMask, j1 = c->clay[sd.clay_off + l + 1] & kSlotMask;
          for (int j = j0; j < j1; ++j) list.push_back(sd.cb_off + j);
        }
      }
      lay.push_back((int32_t)list.size());
      // nonlinear resistors of the group's subsystems and their correction pairs
      G.nl0 = a.nl_off;
      G.nl1 = b.nl_off + b.n_nl;
      G.fd0 = a.fd_off;
      G.fd1 = b.fd_off + b.n_fd;
      G.ce0 = a.ce_off;
      G.ce1 = b.ce_off + b.n_ce;
      G.sub0 = s0;
      G.sub1 = s1;
      G.nlc0 = G.nlc1 = 0;
      for (int s = 0, pos = 0; s < s1; ++s) {
        const SubDev& sd = c->subs[s];
        if (s == s0) G.nlc0 = pos;
        pos += sd.n_nl * sd.n;
        G.nlc1 = pos;
      }
      G.node0 = a.node_off;
      G.node1 = b.node_off + b.n;
      G.col0 = c->b_sub_col_off[s0];
      G.col1 = c->b_sub_col_off[s1 - 1] + b.n + b.n_str;
      G.lc0 = a.lc_off;
      G.lc1 = b.lc_off + b.n_lc;
      G.le0 = a.le_off;
      G.le1 = b.le_off + b.n_le;
      groups.push_back(G);
      max_cols = std::max(max_cols, cols);
      max_nodes = std::max(max_nodes, nodes);
      s0 = s1;
    }
    const size_t total = batch_smem_bytes(S_t, (int)c->n_sources, c->n_sub, max_cols, max_nodes,
                                          dig, dig_grp);
    const size_t limit = 227 * 1024 - (dig ? kBatchDigitStaticSmem : 0);
    if (total <= limit) break;
    if (!dig || attempt >= 8 || total - limit >= budget) return false;
    budget -= total - limit;
  }
  if (!upload) return true;
  if (c->d_grp) {
    cudaDeviceSynchronize();
    c->release(c->d_grp);
    c->d_grp = nullptr;
  }
  if (c->upload(&c->d_grp, groups) != cudaSuccess) return false;
  if (!list.empty()) {
    c->release(c->d_bcb_lay);
    c->release(c->d_bcb_list);
    c->d_bcb_lay = nullptr;
    c->d_bcb_list = nullptr;
    if (c->upload(&c->d_bcb_lay, lay) != cudaSuccess || c->upload(&c->d_bcb_list, list) != cudaSuccess) return false;
  }
  c->b_cb_lay = lay;
  c->b_cb_list = list;
  c->groups = groups;
  c->max_cols = std::max(max_cols, 1);
  c->max_nodes = std::max(max_nodes, 1);
  c->S_t = S_t;
  c->dig_on = dig;
  c->dig_grp = dig_grp;
  return true;
}

std::string build_scenarios(emt_ctx* c, const emt_network_desc* d, const emt_scenario_desc* sc,
                            const std::vector<int>& local, const std::vector<int32_t>& new_of_orig,
                            const std::vector<int64_t>& le_of_end, const std::vector<int32_t>& lc_slot_of,
                            const std::vector<int32_t>& sb_slot_of) {
  c->batched = true;
  const int64_t S = sc->n_scenarios;
  c->S = S;
  const int nsub = c->n_sub;
  const int64_t nsrc = d->n_sources;
  c->bsrc_amp.resize(S * nsrc);
  c->bsrc_phase.resize(S * nsrc);
  for (int64_t q = 0; q < S; ++q)
    for (int64_t j = 0; j < nsrc; ++j) {
      c->bsrc_amp[q * nsrc + j] = sc->src_amp ? sc->src_amp[q * nsrc + j] : d->src_amp[j];
      c->bsrc_phase[q * nsrc + j] = sc->src_phase ? sc->src_phase[q * nsrc + j] : d->src_phase[j];
    }
  std::vector<int> sub_of_br(c->branches.size()), sub_of_le(c->line_ends.size());
  std::vector<int64_t> end_of_le(c->line_ends.size(), -1);
  for (int q = 0; q < nsub; ++q) {
    const SubDev& sd = c->subs[q];
    for (int b = sd.br_off; b < sd.br_off + sd.n_br; ++b) sub_of_br[b] = q;
    for (int e = sd.le_off; e < sd.le_off + sd.n_le; ++e) sub_of_le[e] = q;
  }
  for (int64_t e = 0; e < (int64_t)le_of_end.size(); ++e) end_of_le[le_of_end[e]] = e;
  const bool any_rm = (sc->rm_branch_ptr && sc->rm_branch_ptr[S] > 0) || (sc->rm_line_ptr && sc->rm_line_ptr[S] > 0);
  if (any_rm) {
    c->keep_lc.assign((size_t)c->lc_idx.size() * S, 1);
    c->keep_sb.assign((size_t)c->sb_idx.size() * S, 1);
    c->keep_le.assign((size_t)c->line_ends.size() * S, 1);
  }
  std::vector<std::vector<int64_t>> base_sw_of(nsub);
  for (int64_t w = 0; w < d->n_switches; ++w) {
    const int a = d->sw_k[w] >= 0 ? d->sw_k[w] : d->sw_m[w];
    base_sw_of[c->sub_of_node[a]].push_back(w);
  }
  struct Sw {
    int32_t k, m;
    double r;
    int64_t on, off;
  };
  std::map<std::vector<int64_t>, int> variants;
  c->n_base_epochs = (int64_t)c->epochs.size();
  int64_t goff = c->ginv_len;
  c->rm_ptr_br.assign(1, 0);
  c->rm_ptr_le.assign(1, 0);
  c->msel_ptr.assign(1, 0);
  std::vector<std::vector<int32_t>> rb(nsub), rl(nsub);
  std::vector<std::vector<Sw>> ssw(nsub);
  for (int64_t q = 0; q < S; ++q) {
    for (int k = 0; k < nsub; ++k) {
      rb[k].clear();
      rl[k].clear();
      ssw[k].clear();
    }
    if (sc->rm_branch_ptr)
      for (int64_t i = sc->rm_branch_ptr[q]; i < sc->rm_branch_ptr[q + 1]; ++i) {
        const int32_t nb = new_of_orig[sc->rm_branch[i]];
        const int k = sub_of_br[nb];
        rb[k].push_back(nb);
        if (lc_slot_of[nb] >= 0) c->keep_lc[(size_t)(c->subs[k].lc_off + lc_slot_of[nb]) * S + q] = 0;
        if (sb_slot_of[nb] >= 0) c->keep_sb[(size_t)(c->subs[k].sb_off + sb_slot_of[nb]) * S + q] = 0;
      }
    if (sc->rm_line_ptr)
      for (int64_t i = sc->rm_line_ptr[q]; i < sc->rm_line_ptr[q + 1]; ++i)
        for (int end = 0; end < 2; ++end) {
          const int64_t ge = le_of_end[2 * (int64_t)sc->rm_line[i] + end];
          rl[sub_of_le[ge]].push_back((int32_t)ge);
          c->keep_le[(size_t)ge * S + q] = 0;
        }
    for (int k = 0; k < nsub; ++k)
      for (int64_t w : base_sw_of[k])
        ssw[k].push_back({d->sw_k[w], d->sw_m[w], d->sw_r[w], d->sw_close_step[w], d->sw_open_step[w]});
    if (sc->sw_ptr)
      for (int64_t w = sc->sw_ptr[q]; w < sc->sw_ptr[q + 1]; ++w) {
        const int a = sc->sw_k[w] >= 0 ? sc->sw_k[w] : sc->sw_m[w];
        ssw[c->sub_of_node[a]].push_back({sc->sw_k[w], sc->sw_m[w], sc->sw_r[w], sc->sw_close_step[w], sc->sw_open_step[w]});
      }
    for (int k = 0; k < nsub; ++k) {
      const SubDev& sd = c->subs[k];
      std::sort(rb[k].begin(), rb[k].end());
      std::sort(rl[k].begin(), rl[k].end());
      std::vector<int64_t> events;
      for (const Sw& w : ssw[k]) {
        if (w.on >= 0) events.push_back(w.on);
        if (w.off >= 0) events.push_back(w.off);
      }
      std::sort(events.begin(), events.end());
      events.erase(std::unique(events.begin(), events.end()), events.end());
      std::vector<std::pair<int64_t, int64_t>> eps;
      eps.push_back({LLONG_MIN, events.empty() ? 1 : events[0] - 1});
      for (int64_t ev : events) eps.push_back({ev, ev});
      for (auto& ep : eps) {
        std::vector<std::array<int64_t, 3>> closed;
        for (const Sw& w : ssw[k]) {
          if (!switch_closed(w.on, w.off, ep.second)) continue;
          const double g = 1.0 / w.r;
          int64_t gb;
          std::memcpy(&gb, &g, sizeof(gb));
          closed.push_back({w.k >= 0 ? local[w.k] : -1, w.m >= 0 ? local[w.m] : -1, gb});
        }
        std::sort(closed.begin(), closed.end());
        std::vector<int64_t> key{k, (int64_t)rb[k].size()};
        key.insert(key.end(), rb[k].begin(), rb[k].end());
        key.push_back((int64_t)rl[k].size());
        key.insert(key.end(), rl[k].begin(), rl[k].end());
        for (auto& cl : closed) key.insert(key.end(), cl.begin(), cl.end());
        auto it = variants.find(key);
        int vid;
        if (it == variants.end()) {
          // one matrix per runtime-switch state word, consecutive (stride n (n + n_str) [+ n])
          vid = (int)((int64_t)c->epochs.size() - c->n_base_epochs);
          variants.emplace(key, vid);
          for (int word = 0; word < sd.n_states; ++word) {
            EpochDev E{};
            E.start = 0;
            E.rs_word = -1;   // the runtime switches are in its switch list
            E.ginv_off = goff;
            goff += (int64_t)sd.n * (sd.n + sd.n_str);
            E.nlz_off = -1;
            if (sd.n_nl > 0) {   // its nonlinear resistor's column z right after the matrix (and its remainder)
              E.nlz_off = goff;
              goff += sd.n;
            }
            E.sw_off = (int)c->switches.size();
            for (auto& cl : closed) {
              SwitchDev sw{};
              sw.k = (int32_t)cl[0];
              sw.m = (int32_t)cl[1];
              std::memcpy(&sw.g, &cl[2], sizeof(sw.g));
              c->switches.push_back(sw);
            }
            for (int j = 0; j < sd.n_rs; ++j) {   // runtime switches: r_on or r_off by the state word
              const RuntimeSwitchDev& r = c->rswitches[sd.rs_off + j];
              SwitchDev sw{};
              sw.k = r.k;
              sw.m = r.m;
              sw.g = 1.0 / (((word >> j) & 1) ? r.r_on : c->rs_roff[sd.rs_off + j]);
              c->switches.push_back(sw);
            }
            E.n_sw = (int)c->switches.size() - E.sw_off;
            c->epochs.push_back(E);
            c->var_sub.push_back(k);
            c->rm_br.insert(c->rm_br.end(), rb[k].begin(), rb[k].end());
            c->rm_ptr_br.push_back((int32_t)c->rm_br.size());
            c->rm_le.insert(c->rm_le.end(), rl[k].begin(), rl[k].end());
            c->rm_ptr_le.push_back((int32_t)c->rm_le.size());
          }
        } else {
          vid = it->second;
        }
        c->msel_start.push_back(ep.first);
        c->msel_mat.push_back((int32_t)(c->n_base_epochs + vid));
      }
      c->msel_ptr.push_back((int64_t)c->msel_start.size());
    }
  }
  if (c->epochs.size() > (size_t)INT32_MAX / 2) return "too many scenario matrix variants";
  c->ginv_len = goff;
  // batched rings: depth d + 1, scenario-contiguous
  c->le_bring.assign(c->line_ends.size(), 0);
  c->le_bfar.assign(c->line_ends.size(), 0);
  int64_t off = 0;
  for (size_t e = 0; e < c->line_ends.size(); ++e) {
    c->le_bring[e] = off;
    // FD ends and coupled modes interpolate: their values of steps n - d and n - d - 1 stay readable
    off += c->line_ends[e].d + (c->line_ends[e].fd >= 0 || c->line_ends[e].ce >= 0 ? 2 : 1);
  }
  // the far end of a lossless line by its line index, of a frequency-dependent one by its own ring
  std::map<int64_t, size_t> by_ring;   // FD ends and coupled modes by their own ring
  for (size_t e = 0; e < c->line_ends.size(); ++e)
    if (c->line_ends[e].fd >= 0 || c->line_ends[e].ce >= 0) by_ring[c->line_ends[e].own_ring] = e;
  for (size_t e = 0; e < c->line_ends.size(); ++e)
    c->le_bfar[e] = c->line_ends[e].fd >= 0 || c->line_ends[e].ce >= 0 ? c->le_bring[by_ring.at(c->line_ends[e].far_ring)]
                                                                        : c->le_bring[le_of_end[end_of_le[e] ^ 1]];
  c->bring_len = off;

  // flat per-slot arrays (global numbering of columns, lanes and slots)
  if (c->lc_idx.size() >= kBentIndexMask || c->sb_idx.size() >= kBentIndexMask ||
      c->line_ends.size() >= kBentIndexMask)
    return "too many element slots for the multi-scenario kernel";
  const int N = (int)c->original_of.size();
  c->b_node_sub.assign(N, 0);
  c->b_node_r.assign(N, 0);
  c->b_ent_ptr.assign(1, 0);
  int64_t col = 0;
  for (int q = 0; q < nsub; ++q) {
    const SubDev& sd = c->subs[q];
    const int nc = sd.n + sd.n_str;
    c->b_sub_nc.push_back(nc);
    if (col + nc > INT32_MAX / 2) return "too many solve columns";
    c->b_sub_col_off.push_back((int32_t)col);
    c->b_col_sub.insert(c->b_col_sub.end(), (size_t)nc, (int32_t)q);
    const int ie_base = sd.n_lc + sd.n_sb;
    for (int k = 0; k < sd.n; ++k) {
      c->b_col_code.push_back(sd.node_off + k);
      c->b_node_sub[sd.node_off + k] = q;
      c->b_node_r[sd.node_off + k] = k;
      // the node's entries in lane order, padding left out
      const int l0 = c->node_l0[sd.node_off + k], nl = c->node_nl[sd.node_off + k];
      for (int l = l0; l < l0 + nl; ++l)
        for (int u = 0; u < 4; ++u) {
          const uint32_t raw = (uint32_t)c->ent[4 * (size_t)(sd.il_off + l) + u];
          const int idx = (int)(raw & ~kEntryNeg);
          uint32_t code;
          const int blk = sd.n_le + 3 * sd.n_ce + sd.n_fd;
          const int zero = ie_base + 2 * blk, cph0 = ie_base + sd.n_le, fdb0 = cph0 + 3 * sd.n_ce;
          if (idx < sd.n_lc) code = (0u << kBentKindShift) | (uint32_t)(sd.lc_off + idx);
          else if (idx < ie_base) code = (1u << kBentKindShift) | (uint32_t)(sd.sb_off + idx - sd.n_lc);
          else if (idx < cph0) code = (2u << kBentKindShift) | (uint32_t)(sd.le_off + idx - ie_base);
          else if (idx < fdb0) code = (6u << kBentKindShift) | (uint32_t)(3 * sd.ce_off + idx - cph0);
          else if (idx < ie_base + blk) code = (4u << kBentKindShift) | (uint32_t)(sd.fd_off + idx - fdb0);
          else if (idx > zero && idx <= zero + sd.n_ci) code = (3u << kBentKindShift) | (uint32_t)(sd.ci_off + idx - zero - 1);
          else if (idx > zero + sd.n_ci && idx <= zero + sd.n_ci + sd.n_fd) {
            const int fx = sd.fd_off + idx - zero - 1 - sd.n_ci;
            // (a line group's modes: their Hy enters the phase history currents of the coupled fold)
            if (c->line_ends[sd.le_off + c->fdends[fx].le].ce >= 0) continue;
            code = (5u << kBentKindShift) | (uint32_t)fx;
          }
          else continue;
          c->b_bent.push_back((int32_t)(code | (raw & kEntryNeg)));
        }
      c->b_ent_ptr.push_back((int32_t)c->b_bent.size());
    }
    for (int t = 0; t < sd.n_str; ++t) c->b_col_code.push_back(-1 - (sd.lc_off + c->str_slot[sd.str_off + t]));
    col += nc;
    auto gnode = [&](int16_t x) -> int32_t {
      if (x >= 0) return sd.node_off + x;
      if (x == -1) return -1;
      return -2 - c->src_global[sd.src_off + (-2 - x)];
    };
    for (int x = 0; x < sd.n_lc; ++x) {
      const BranchDev& b = c->branches[c->lc_idx[sd.lc_off + x]];
      c->b_lc_nk.push_back(gnode(b.k));
      c->b_lc_nm.push_back(gnode(b.m));
      c->b_lc_isl.push_back(b.kind == 1 ? 1 : 0);
    }
    for (int x = 0; x < sd.n_sb; ++x) {
      const BranchDev& b = c->branches[c->sb_idx[sd.sb_off + x]];
      c->b_sb_src.push_back(c->src_global[sd.src_off + (b.k <= -2 ? -2 - b.k : -2 - b.m)]);
    }
    for (int e = 0; e < sd.n_le; ++e) {
      const LineEndDev& L = c->line_ends[sd.le_off + e];
      c->b_le_nd.push_back(sd.node_off + L.node);
      c->b_le_d1.push_back(L.d + 1);
      c->b_le_y2.push_back(L.y2);
    }
  }
  // solve-matrix selections as per-scenario events sorted by step
  c->b_ev_ptr.assign(1, 0);
  for (int64_t q = 0; q < S; ++q) {
    std::vector<std::array<int64_t, 3>> ev;   // (first step, subsystem, offset)
    for (int k = 0; k < nsub; ++k)
      for (int64_t x = c->msel_ptr[q * nsub + k]; x < c->msel_ptr[q * nsub + k + 1]; ++x)
        ev.push_back({std::max<int64_t>(c->msel_start[x], 0), k, c->epochs[c->msel_mat[x]].ginv_off});
    std::stable_sort(ev.begin(), ev.end(),
                     [](const std::array<int64_t, 3>& a, const std::array<int64_t, 3>& b) { return a[0] < b[0]; });
    for (auto& x : ev) {
      c->b_ev_step.push_back(x[0]);
      c->b_ev_sub.push_back((int32_t)x[1]);
      c->b_ev_off.push_back(x[2]);
    }
    c->b_ev_ptr.push_back((int64_t)c->b_ev_step.size());
  }
  // digit form: the matrices (of at most kDigRows rows and kDigCols columns)
  // that at least 16 scenarios (or all) select, so that whole tiles share them
  {
    const int64_t nvar = (int64_t)c->epochs.size() - c->n_base_epochs;
    std::vector<int64_t> users(nvar, 0), last(nvar, -1);
    for (int64_t q = 0; q < S; ++q)
      for (int k = 0; k < nsub; ++k)
        for (int64_t x = c->msel_ptr[q * nsub + k]; x < c->msel_ptr[q * nsub + k + 1]; ++x) {
          const int64_t v = c->msel_mat[x] - c->n_base_epochs;
          if (last[v] != q) {
            last[v] = q;
            ++users[v];
          }
        }
    std::vector<std::vector<int64_t>> mats(nsub);   // epoch entries per subsystem
    for (int64_t v = 0; v < nvar; ++v) {   // (selections name a variant's first state matrix; its others follow)
      const int k = c->var_sub[v];
      const SubDev& sd = c->subs[k];
      if (users[v] < std::min<int64_t>(16, S) || sd.n > kDigRows || sd.n + sd.n_str > kDigCols) continue;
      for (int w = 0; w < sd.n_states && v + w < nvar; ++w) mats[k].push_back(c->n_base_epochs + v + w);
    }
    c->dig_ptr.assign(1, 0);
    int64_t doff = 0;
    for (int k = 0; k < nsub; ++k) {
      const SubDev& sd = c->subs[k];
      for (int64_t e : mats[k]) {
        c->dig_key.push_back(c->epochs[e].ginv_off);
        c->dig_val.push_back(doff);
        c->dig_mat_goff.push_back(c->epochs[e].ginv_off);
        c->dig_mat_n.push_back(sd.n);
        c->dig_mat_nc.push_back(sd.n + sd.n_str);
        doff += (dig_matrix_words(sd.n + sd.n_str) + 3) & ~(int64_t)3;   // 16-byte aligned chunks
      }
      c->dig_ptr.push_back((int32_t)c->dig_key.size());
      c->dig_sub_n.push_back(sd.n);
      c->dig_node0.push_back(sd.node_off);
    }
    c->dig_len = doff;
  }
  // runtime switches: per subsystem (first switch, count, matrix stride,
  // first internal node); states are per scenario
  for (int q = 0; q < nsub; ++q) {
    const SubDev& sd = c->subs[q];
    const int64_t stride = (int64_t)sd.n * (sd.n + sd.n_str) + (sd.n_nl > 0 ? sd.n : 0);
    c->b_sub_rs.insert(c->b_sub_rs.end(), {sd.rs_off, sd.n_rs, (int32_t)stride, sd.node_off});
  }

  // coupled ends: each one's first mode line end; per line end its coupled
  // end (or -1) and interpolation fraction
  c->b_le_ce.assign(c->line_ends.size(), -1);
  c->b_le_f.assign(c->line_ends.size(), 0.0);
  for (size_t e = 0; e < c->line_ends.size(); ++e) c->b_le_f[e] = c->line_ends[e].f;
  for (int q = 0; q < nsub; ++q) {
    const SubDev& sd = c->subs[q];
    for (int x = 0; x < sd.n_ce; ++x) {
      const int ge0 = sd.le_off + c->cends[sd.ce_off + x].le0;
      c->b_ce_le0.push_back(ge0);
      for (int p = 0; p < 3; ++p) c->b_ce_node.push_back(sd.node_off + c->cends[sd.ce_off + x].node[p]);
      for (int j = 0; j < 3; ++j) c->b_le_ce[ge0 + j] = sd.ce_off + x;
    }
  }

  // frequency-dependent ends: each one's global line end, and per line end
  // its FD end (or -1)
  c->b_le_fd.assign(c->line_ends.size(), -1);
  for (int q = 0; q < nsub; ++q) {
    const SubDev& sd = c->subs[q];
    for (int x = 0; x < sd.n_fd; ++x) {
      const int ge = sd.le_off + c->fdends[sd.fd_off + x].le;
      c->b_fd_le.push_back(ge);
      c->b_le_fd[ge] = sd.fd_off + x;
    }
  }

  // nonlinear resistors: per element its subsystem, nodes and first
  // internal node; the (node, element) pairs its compensation corrects
  for (int q = 0; q < nsub; ++q) {
    const SubDev& sd = c->subs[q];
    for (int x = 0; x < sd.n_nl; ++x) {
      const int e = sd.nl_off + x;
      c->b_nlinfo.insert(c->b_nlinfo.end(), {q, sd.n, sd.node_off, 0});
      for (int r = 0; r < sd.n; ++r) c->b_nlc.insert(c->b_nlc.end(), {sd.node_off + r, e});
    }
  }

  // control blocks in global slots: inputs over all blocks (the zero pair
  // after the last one), MEAS nodes as internal nodes; the block of each
  // control injection; per-scenario coefficients of the blocks a scenario
  // sets a parameter of (the base ones in the other scenarios)
  const int NCB = (int)c->cblocks.size();
  c->b_cb = c->cblocks;
  for (int q = 0; q < nsub; ++q) {
    const SubDev& sd = c->subs[q];
    auto remap = [&](int32_t i) { return i >= 2 * sd.n_cb ? 2 * NCB : 2 * (sd.cb_off + (i >> 1)) + (i & 1); };
    for (int j = 0; j < sd.n_cb; ++j) {
      CtrlDev& r = c->b_cb[sd.cb_off + j];
      r.i0 = remap(r.i0);
      r.i1 = remap(r.i1);
      if (r.type == 1) r.node = sd.node_off + r.node;
    }
    for (int x = 0; x < sd.n_ci; ++x) c->b_cinj.push_back(sd.cb_off + c->cinj[sd.ci_off + x]);
  }
  if (sc->cbo_ptr && sc->cbo_ptr[S] > 0) {
    std::map<int32_t, int> row_of;
    for (int64_t i = 0; i < sc->cbo_ptr[S]; ++i) row_of.emplace(sc->cbo_block[i], (int)row_of.size());
    c->b_cbo.assign(row_of.size() * (size_t)S * 3, 0.0);
    auto slot = [&](int32_t b) { return c->subs[c->cb_sub_of[b]].cb_off + c->cb_slot_of[b]; };
    for (const auto& kv : row_of) {
      CtrlDev& r = c->b_cb[slot(kv.first)];
      r.ov = (double)kv.second;
      for (int64_t q = 0; q < S; ++q) {
        double* o = &c->b_cbo[((size_t)kv.second * S + q) * 3];
        o[0] = r.p0;
        o[1] = r.p1;
        o[2] = r.p2;
      }
    }
    for (int64_t q = 0; q < S; ++q)
      for (int64_t i = sc->cbo_ptr[q]; i < sc->cbo_ptr[q + 1]; ++i) {
        const int32_t b = sc->cbo_block[i];
        CtrlDev t{};
        t.type = d->cb_type[b];
        ctrl_coefficients(t, sc->cbo_p0[i], d->cb_p1[b], d->dt);
        double* o = &c->b_cbo[((size_t)row_of[b] * S + q) * 3];
        o[0] = t.p0;
        o[1] = t.p1;
        o[2] = t.p2;
      }
  }

  // default launch shape: about one CTA per SM
  c->S_t = (int)std::min<int64_t>(32, std::max<int64_t>(1, (S + 147) / 148));
  while (c->S_t > 1 && !batch_configure(c, c->S_t, false)) c->S_t = std::max(1, c->S_t / 2);
  if (!batch_configure(c, c->S_t, false)) return "network too large for the multi-scenario kernel's shared memory";
  return "";
}

// ------------------------------------------------------------------ build

// Components packed into at most `target` groups (one CTA each).  The
// smallest group merges with the smallest partner that keeps the merged
// group within `relax_n` times the largest component's nodes and `relax`
// times its line ends, L/C branches and control blocks (shared memory grows
// with the square of the nodes, linearly with the rest), while there are
// too many groups: the large components keep
// CTAs of their own, a merged group stays small (its solve runs the zero
// blocks too) and the per-CTA shared memory, sized by those maxima, hardly
// grows.  A component with runtime switches or a nonlinear resistor keeps a
// group of its own (switch states and compensation are per CTA).  A group's
// G is block-diagonal, so its inverse is the blocks' inverses.
std::vector<std::vector<int>> pack_components(const std::vector<std::vector<int>>& comps,
                                              const std::vector<char>& alone, const std::vector<int>& w_le,
                                              const std::vector<int>& w_lc, const std::vector<int>& w_cb,
                                              int target, double relax, double relax_n) {
  const size_t K = comps.size();
  size_t max_n = 0;
  int max_le = 0, max_lc = 0, max_cb = 0;
  for (size_t x = 0; x < K; ++x) {
    max_n = std::max(max_n, comps[x].size());
    max_le = std::max(max_le, w_le[x]);
    max_lc = std::max(max_lc, w_lc[x]);
    max_cb = std::max(max_cb, w_cb[x]);
  }
  const double cap_n = relax_n * (double)max_n, cap_le = relax * max_le, cap_lc = relax * max_lc;
  const double cap_cb = relax * max_cb;
  std::vector<std::vector<int>> groups(comps.begin(), comps.end());
  std::vector<int> le(w_le), lc(w_lc), cb(w_cb);
  std::vector<int> open;   // mergeable groups
  for (size_t x = 0; x < K; ++x)
    if (!alone[x]) open.push_back((int)x);
  int n_groups = (int)K;
  while (n_groups > target && open.size() >= 2) {
    std::sort(open.begin(), open.end(), [&](int a, int b) { return groups[a].size() < groups[b].size(); });
    const int a = open[0];
    int pick = -1;
    for (size_t j = 1; j < open.size() && pick < 0; ++j) {
      const int b = open[j];
      if ((double)(groups[a].size() + groups[b].size()) <= cap_n && le[a] + le[b] <= cap_le &&
          lc[a] + lc[b] <= cap_lc && cb[a] + cb[b] <= cap_cb)
        pick = (int)j;
    }
    if (pick < 0) {   // the smallest fits with nothing: it stays as it is
      open.erase(open.begin());
      continue;
    }
    const int b = open[pick];
    groups[a].insert(groups[a].end(), groups[b].begin(), groups[b].end());
    groups[b].clear();
    le[a] += le[b];
    lc[a] += lc[b];
    cb[a] += cb[b];
    open.erase(open.begin() + pick);
    --n_groups;
  }
  std::vector<std::vector<int>> out;
  for (auto& g : groups)
    if (!g.empty()) out.push_back(std::move(g));
  return out;
}

static emt_status build_network(const emt_network_desc* d, const emt_scenario_desc* scen, emt_ctx** out,
                                 int pack_to, double relax, double relax_n);

// Co-resident CTAs of the single-network kernel for this context's limits.
static int64_t forward_capacity(const emt_ctx* c) {
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  FwdLimits fl = c->lim;
  fl.n = std::max(fl.n, 1);
  fl.nc = std::max(fl.nc, 1);
  return (int64_t)n_sm * forward_blocks_per_sm(fl);
}

// A single network whose subsystems would not all be co-resident is built
// again with its subsystems packed several to a CTA (fewer CTAs, each with
// a block-diagonal solve), the merged groups allowed to grow past the
// largest component step by step until the packed network fits.  Scenario
// sets are not packed.
extern "C" emt_status emt_build_network(const emt_network_desc* d, const emt_scenario_desc* scen, emt_ctx** out) {
  NvtxRange nvtx_range("emt_build_network");
  emt_status st = build_network(d, scen, out, 0, 1.0, 1.0);
  if (st != EMT_OK || scen) return st;
  int64_t target = forward_capacity(*out);
  if (target <= 0 || (*out)->n_sub <= target) return st;
  // bounds on a merged group, loosest last: the linear counts first, the nodes last
  static const double kRelax[][2] = {{1.0, 1.0}, {1.5, 1.0}, {2.0, 1.0}, {3.0, 1.0}, {3.0, 1.25}, {3.0, 1.5}, {3.0, 2.0}};
  int step = 0;
  for (int attempt = 0; attempt < 16; ++attempt) {
    emt_destroy(*out);
    *out = nullptr;
    st = build_network(d, scen, out, (int)target, kRelax[step][0], kRelax[step][1]);
    if (st != EMT_OK) return st;
    const int64_t n = (*out)->n_sub, cap = forward_capacity(*out);
    if (n <= cap) return st;
    if (n <= target) {
      target = std::min(target - 1, cap);   // packed as asked, but its CTAs need more memory: aim lower
    } else if (step + 1 < (int)(sizeof(kRelax) / sizeof(kRelax[0]))) {
      ++step;                               // the bounds stop the merging short of the target
    } else {
      break;
    }
  }
  return st;   // still too many CTAs: emt_step_n reports EMT_ERESOURCE
}

static emt_status build_network(const emt_network_desc* d, const emt_scenario_desc* scen, emt_ctx** out,
                                 int pack_to, double relax, double relax_n) {
  if (!out) {
    g_build_error = "out is NULL";
    return EMT_EINVAL;
  }
  *out = nullptr;
  const std::string msg = validate(d);
  if (!msg.empty()) {
    g_build_error = msg;
    return EMT_EINVAL;
  }
  if (scen) {
    const std::string sm = validate_scenarios(d, scen);
    if (!sm.empty()) {
      g_build_error = sm;
      return EMT_EINVAL;
    }
  }
  emt_ctx* c = new emt_ctx();
  auto bail = [&](const std::string& m) {
    g_build_error = m;
    delete c;
    return EMT_EINVAL;
  };
  cudaGetDevice(&c->device);
  c->dt = d->dt;
  c->n_nodes = d->n_nodes;
  c->n_branches = d->n_branches;
  c->n_sources = d->n_sources;
  c->n_lines = d->n_lines;
  const int N = (int)d->n_nodes;

  // -------- subsystems: components over branches and switches
  std::vector<int> parent(N);
  std::iota(parent.begin(), parent.end(), 0);
  auto join = [&](int a, int b) {
    if (a < 0 || b < 0) return;
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a != b) parent[std::max(a, b)] = std::min(a, b);
  };
  for (int64_t b = 0; b < d->n_branches; ++b) join(d->br_k[b], d->br_m[b]);
  for (int64_t w = 0; w < d->n_switches; ++w) join(d->sw_k[w], d->sw_m[w]);
  for (int64_t w = 0; w < d->n_rswitches; ++w) join(d->rs_k[w], d->rs_m[w]);
  for (int64_t x = 0; x < d->n_nonlin; ++x) join(d->nl_k[x], d->nl_m[x]);
  for (int64_t l = 0; l < d->n_clines; ++l)   // an end's phases are coupled by Y_p
    for (int p = 1; p < 3; ++p) {
      join(d->cl_k[3 * l], d->cl_k[3 * l + p]);
      join(d->cl_m[3 * l], d->cl_m[3 * l + p]);
    }
  for (int64_t gi = 0; gi < d->n_fdgroups; ++gi)   // and those of a frequency-dependent line group
    for (int p = 1; p < 3; ++p) {
      join(d->fl_k[d->fg_line[3 * gi]], d->fl_k[d->fg_line[3 * gi + p]]);
      join(d->fl_m[d->fg_line[3 * gi]], d->fl_m[d->fg_line[3 * gi + p]]);
    }
  if (scen && scen->sw_ptr)   // scenario switches may join nodes too
    for (int64_t w = 0; w < scen->sw_ptr[scen->n_scenarios]; ++w) join(scen->sw_k[w], scen->sw_m[w]);
  c->sub_of_node.assign(N, -1);
  std::vector<int> label(N, -1);
  std::vector<std::vector<int>> nodes_of;
  for (int i = 0; i < N; ++i) {
    const int r = uf_find(parent, i);
    if (label[r] < 0) {
      label[r] = (int)nodes_of.size();
      nodes_of.emplace_back();
    }
    c->sub_of_node[i] = label[r];
    nodes_of[label[r]].push_back(i);
  }
  c->n_components = (int64_t)nodes_of.size();
  for (const auto& v : nodes_of) {
    c->comp_sum_n2 += (int64_t)v.size() * (int64_t)v.size();
    c->comp_max_n = std::max<int64_t>(c->comp_max_n, (int64_t)v.size());
  }
  if (pack_to > 0 && (int)nodes_of.size() > pack_to) {
    std::vector<char> alone(nodes_of.size(), 0);
    auto mark = [&](int32_t a) {
      if (a >= 0) alone[c->sub_of_node[a]] = 1;
    };
    for (int64_t w = 0; w < d->n_rswitches; ++w) mark(d->rs_k[w] >= 0 ? d->rs_k[w] : d->rs_m[w]);
    for (int64_t x = 0; x < d->n_nonlin; ++x) mark(d->nl_k[x] >= 0 ? d->nl_k[x] : d->nl_m[x]);
    std::vector<int> w_le(nodes_of.size(), 0), w_lc(nodes_of.size(), 0);
    for (int64_t l = 0; l < d->n_lines; ++l) {
      ++w_le[c->sub_of_node[d->ln_k[l]]];
      ++w_le[c->sub_of_node[d->ln_m[l]]];
    }
    for (int64_t l = 0; l < 3 * d->n_clines; ++l) {   // a mode per phase at each end
      ++w_le[c->sub_of_node[d->cl_k[l]]];
      ++w_le[c->sub_of_node[d->cl_m[l]]];
    }
    for (int64_t l = 0; l < d->n_fdlines; ++l) {
      ++w_le[c->sub_of_node[d->fl_k[l]]];
      ++w_le[c->sub_of_node[d->fl_m[l]]];
    }
    for (int64_t b = 0; b < d->n_branches; ++b)
      if (d->br_kind[b] != 0) ++w_lc[c->sub_of_node[d->br_k[b] >= 0 ? d->br_k[b] : d->br_m[b]]];
    // control blocks: a connected group of blocks sits with the nodes it measures or drives
    std::vector<int> w_cb(nodes_of.size(), 0);
    if (d->n_cblocks > 0) {
      const int64_t NB = d->n_cblocks;
      std::vector<int> bg(NB);
      std::iota(bg.begin(), bg.end(), 0);
      for (int64_t b = 0; b < NB; ++b)
        for (const int32_t in : {d->cb_in0[b], d->cb_in1[b]})
          if (in >= 0 && in < NB) {
            const int x = uf_find(bg, (int)b), y = uf_find(bg, in);
            if (x != y) bg[std::max(x, y)] = std::min(x, y);
          }
      std::vector<int> comp_of_group(NB, -1);
      for (int64_t b = 0; b < NB; ++b)
        if (d->cb_type[b] == 1) comp_of_group[uf_find(bg, (int)b)] = c->sub_of_node[d->cb_node[b]];
      for (int64_t x = 0; x < d->n_cinj; ++x) comp_of_group[uf_find(bg, d->ci_block[x])] = c->sub_of_node[d->ci_node[x]];
      for (int64_t b = 0; b < NB; ++b) {
        const int cp = comp_of_group[uf_find(bg, (int)b)];
        ++w_cb[cp >= 0 ? cp : 0];
      }
    }
    nodes_of = pack_components(nodes_of, alone, w_le, w_lc, w_cb, pack_to, relax, relax_n);
    for (size_t g = 0; g < nodes_of.size(); ++g)
      for (int v : nodes_of[g]) c->sub_of_node[v] = (int)g;
  }
  c->n_sub = (int)nodes_of.size();
  const int S = c->n_sub;
  c->internal_of.assign(N, -1);
  c->original_of.assign(N, -1);
  std::vector<int> local(N, -1);
  c->subs.assign(S, SubDev{});
  {
    int off = 0;
    for (int s = 0; s < S; ++s) {
      const int n = (int)nodes_of[s].size();
      if (n > kMaxSubsystemNodes)
        return bail("subsystem " + std::to_string(s) + " has " + std::to_string(n) + " nodes; at most " +
                    std::to_string(kMaxSubsystemNodes) + " are supported");
      c->subs[s].n = n;
      c->subs[s].node_off = off;
      for (int j = 0; j < n; ++j) {
        const int v = nodes_of[s][j];
        local[v] = j;
        c->internal_of[v] = off + j;
        c->original_of[off + j] = v;
      }
      off += n;
      c->lim.n = std::max(c->lim.n, n);
    }
  }

  // -------- branches and local sources, grouped by subsystem
  std::vector<std::vector<int64_t>> br_of(S);
  for (int64_t b = 0; b < d->n_branches; ++b) {
    const int a = d->br_k[b] >= 0 ? d->br_k[b] : d->br_m[b];
    br_of[c->sub_of_node[a]].push_back(b);
  }
  std::vector<int32_t> lc_slot_of, sb_slot_of;   // new branch index -> local slot
  std::vector<int32_t> new_of_orig(d->n_branches, -1);
  for (int s = 0; s < S; ++s) {
    SubDev& sd = c->subs[s];
    sd.br_off = (int)c->branches.size();
    sd.lc_off = (int)c->lc_idx.size();
    sd.sb_off = (int)c->sb_idx.size();
    sd.src_off = (int)c->src_global.size();
    std::map<int, int> src_local;
    auto code = [&](int32_t x) -> int16_t {
      if (x >= 0) return (int16_t)local[x];
      if (x == -1) return -1;
      const int g = -2 - x;
      auto it = src_local.find(g);
      if (it != src_local.end()) return (int16_t)(-2 - it->second);
      const int j = (int)src_local.size();
      src_local[g] = j;
      c->src_global.push_back(g);
      return (int16_t)(-2 - j);
    };
    for (int64_t b : br_of[s]) {
      BranchDev x{};
      x.k = code(d->br_k[b]);
      x.m = code(d->br_m[b]);
      x.kind = d->br_kind[b];
      x.value = d->br_value[b];
      const int32_t nb = (int32_t)c->branches.size();
      new_of_orig[b] = nb;
      lc_slot_of.push_back(-1);
      sb_slot_of.push_back(-1);
      if (x.kind != 0) {
        lc_slot_of[nb] = (int32_t)c->lc_idx.size() - sd.lc_off;
        c->lc_idx.push_back(nb);
      }
      c->br_orig.push_back((int32_t)b);
      c->br_lc.push_back(lc_slot_of[nb]);
      c->br_src.push_back(x.k <= -2 ? c->src_global[sd.src_off + (-2 - x.k)]
                                    : (x.m <= -2 ? c->src_global[sd.src_off + (-2 - x.m)] : -1));
      if (x.k <= -2 || x.m <= -2) {
        sb_slot_of[nb] = (int32_t)c->sb_idx.size() - sd.sb_off;
        c->sb_idx.push_back(nb);
      }
      c->branches.push_back(x);
    }
    sd.n_br = (int)c->branches.size() - sd.br_off;
    sd.n_lc = (int)c->lc_idx.size() - sd.lc_off;
    sd.n_sb = (int)c->sb_idx.size() - sd.sb_off;
    sd.n_src = (int)c->src_global.size() - sd.src_off;
    if (sd.n_src > kFwdThreads)
      return bail("subsystem " + std::to_string(s) + " uses more than " + std::to_string(kFwdThreads) + " sources");
    c->lim.lc = std::max(c->lim.lc, sd.n_lc);
    c->lim.sb = std::max(c->lim.sb, sd.n_sb);
    c->lim.src = std::max(c->lim.src, sd.n_src);
  }
  c->n_lc_total = (int64_t)c->lc_idx.size();
  c->src_br_ptr.assign(d->n_sources + 1, 0);
  for (int32_t s : c->br_src)
    if (s >= 0) ++c->src_br_ptr[s + 1];
  for (int64_t g = 0; g < d->n_sources; ++g) c->src_br_ptr[g + 1] += c->src_br_ptr[g];
  c->src_br.assign(c->src_br_ptr[d->n_sources], 0);
  {
    std::vector<int32_t> fill(c->src_br_ptr.begin(), c->src_br_ptr.end() - 1);
    for (size_t b = 0; b < c->br_src.size(); ++b)
      if (c->br_src[b] >= 0) c->src_br[fill[c->br_src[b]]++] = (int32_t)b;
  }
  if (c->branches.size() > (1u << 29)) return bail("too many branches");
  for (int64_t g = 0; g < d->n_sources; ++g) {
    c->src_amp.push_back(d->src_amp[g]);
    c->src_phase.push_back(d->src_phase[g]);
    c->src_omega.push_back(kTwoPi * d->src_freq[g]);
  }

  // -------- line ends: end 2l at ln_k, end 2l+1 at ln_m; ring depth 2d
  std::vector<int64_t> ring_off(2 * d->n_lines);
  std::vector<int64_t> cl_ring, cl_d, fl_ring;
  {
    int64_t off = 0;
    for (int64_t l = 0; l < d->n_lines; ++l) {
      const int64_t depth = 2 * (int64_t)d->ln_delay[l];
      ring_off[2 * l] = off;
      off += depth;
      ring_off[2 * l + 1] = off;
      off += depth;
    }
    // coupled lines: one ring per (end, mode), depth 2 floor(tau / dt)
    cl_ring.assign(6 * d->n_clines, 0);
    cl_d.assign(3 * d->n_clines, 0);
    for (int64_t l = 0; l < d->n_clines; ++l)
      for (int j = 0; j < 3; ++j) {
        const int64_t dd = (int64_t)std::floor(d->cl_tau[3 * l + j] / d->dt);
        cl_d[3 * l + j] = dd;
        for (int e = 0; e < 2; ++e) {
          cl_ring[6 * l + 3 * e + j] = off;
          off += 2 * dd;
        }
      }
    // frequency-dependent lines: one ring per end, depth 2 floor(tau / dt)
    fl_ring.assign(2 * d->n_fdlines, 0);
    for (int64_t l = 0; l < d->n_fdlines; ++l) {
      const int64_t dd = (int64_t)std::floor(d->fl_tau[l] / d->dt);
      for (int e = 0; e < 2; ++e) {
        fl_ring[2 * l + e] = off;
        off += 2 * dd;
      }
    }
    c->ring_len = off;
  }
  std::vector<std::vector<int64_t>> cends_of(S);   // coupled ends (2 l + e) per subsystem
  for (int64_t x = 0; x < 2 * d->n_clines; ++x)
    cends_of[c->sub_of_node[(x & 1) ? d->cl_m[3 * (x >> 1)] : d->cl_k[3 * (x >> 1)]]].push_back(x);
  // frequency-dependent line groups: per line its group (or -1); group ends (2 g + e) per subsystem
  std::vector<int64_t> fg_of_line((size_t)d->n_fdlines, -1);
  for (int64_t gi = 0; gi < d->n_fdgroups; ++gi)
    for (int j = 0; j < 3; ++j) fg_of_line[d->fg_line[3 * gi + j]] = gi;
  c->fd_groups = d->n_fdgroups > 0;
  std::vector<std::vector<int64_t>> gends_of(S);
  for (int64_t x = 0; x < 2 * d->n_fdgroups; ++x) {
    const int32_t l0 = d->fg_line[3 * (x >> 1)];
    gends_of[c->sub_of_node[(x & 1) ? d->fl_m[l0] : d->fl_k[l0]]].push_back(x);
  }
  std::vector<std::vector<int64_t>> fends_of(S);   // frequency-dependent ends (2 l + e) of lines in no group
  for (int64_t x = 0; x < 2 * d->n_fdlines; ++x)
    if (fg_of_line[x >> 1] < 0) fends_of[c->sub_of_node[(x & 1) ? d->fl_m[x >> 1] : d->fl_k[x >> 1]]].push_back(x);
  std::vector<std::vector<int64_t>> ends_of(S);
  std::vector<int64_t> le_of_end(2 * d->n_lines, -1);
  for (int64_t e = 0; e < 2 * d->n_lines; ++e) {
    const int node = (e & 1) ? d->ln_m[e >> 1] : d->ln_k[e >> 1];
    ends_of[c->sub_of_node[node]].push_back(e);
  }
  for (int s = 0; s < S; ++s) {
    SubDev& sd = c->subs[s];
    sd.le_off = (int)c->line_ends.size();
    std::map<int, int> dmin;
    for (int64_t e : ends_of[s]) {
      const int64_t l = e >> 1;
      const int node = (e & 1) ? d->ln_m[l] : d->ln_k[l];
      const int far_node = (e & 1) ? d->ln_k[l] : d->ln_m[l];
      LineEndDev le{};
      le.node = local[node];
      le.ce = -1;
      le.fd = -1;
      le.d = d->ln_delay[l];
      le.depth = 2 * d->ln_delay[l];
      le.y = 1.0 / d->ln_zc[l];
      le.y2 = 2.0 / d->ln_zc[l];
      le.own_ring = ring_off[e];
      le.far_ring = ring_off[e ^ 1];
      le_of_end[e] = (int64_t)c->line_ends.size();
      c->line_ends.push_back(le);
      const int fs = c->sub_of_node[far_node];
      if (fs != s) {
        auto it = dmin.find(fs);
        if (it == dmin.end() || it->second > le.d) dmin[fs] = le.d;
      }
    }
    // the discretised pole terms of frequency-dependent line l; its end conductance in geq
    auto fd_record = [&](int64_t l, double& geq) {
      const double dt = d->dt;
      FdEndDev r{};
      r.ny = d->fl_ny[l];
      r.na = d->fl_na[l];
      r.y0 = d->fl_y0[l];
      r.a0 = d->fl_a0[l];
      geq = r.y0;
      for (int i = 0; i < r.ny; ++i) {
        const double q = d->fl_yq[4 * l + i], den = 1.0 - q * dt / 2.0;
        r.lam_y[i] = (1.0 + q * dt / 2.0) / den;
        r.mu_y[i] = d->fl_yc[4 * l + i] * (dt / 2.0) / den;
        r.mu_sum += r.mu_y[i];
        geq += r.mu_y[i];
      }
      for (int i = 0; i < r.na; ++i) {
        const double p = d->fl_ap[4 * l + i], den = 1.0 - p * dt / 2.0;
        r.lam_a[i] = (1.0 + p * dt / 2.0) / den;
        r.mu_a[i] = d->fl_ar[4 * l + i] * (dt / 2.0) / den;
      }
      return r;
    };
    // frequency-dependent records of this subsystem: those of group modes (below), then of lone lines
    sd.fd_off = (int)c->fdends.size();
    // coupled line ends: a record each, then its three modes as line ends
    sd.ce_off = (int)c->cends.size();
    for (int64_t x : cends_of[s]) {
      const int64_t l = x >> 1;
      const int e = (int)(x & 1);
      const int32_t* nd = (e ? d->cl_m : d->cl_k) + 3 * l;
      CoupledEndDev ce{};
      for (int p = 0; p < 3; ++p) ce.node[p] = local[nd[p]];
      ce.le0 = (int)c->line_ends.size() - sd.le_off;
      for (int k = 0; k < 9; ++k) ce.tv[k] = d->cl_tv[9 * l + k];
      for (int j = 0; j < 3; ++j) ce.z[j] = d->cl_z[3 * l + j];
      const int ce_local = (int)c->cends.size() - sd.ce_off;
      c->cends.push_back(ce);
      const int fs = c->sub_of_node[(e ? d->cl_k : d->cl_m)[3 * l]];
      for (int j = 0; j < 3; ++j) {
        LineEndDev le{};
        le.node = -1;
        le.fd = -1;
        le.d = (int32_t)cl_d[3 * l + j];
        le.depth = 2 * le.d;
        le.ce = ce_local;
        le.mode = j;
        le.f = d->cl_tau[3 * l + j] / d->dt - (double)cl_d[3 * l + j];
        le.y2 = 2.0 / d->cl_z[3 * l + j];
        le.y = 0.0;
        le.own_ring = cl_ring[6 * l + 3 * e + j];
        le.far_ring = cl_ring[6 * l + 3 * (1 - e) + j];
        c->line_ends.push_back(le);
        if (fs != s) {
          auto it = dmin.find(fs);
          if (it == dmin.end() || it->second > le.d) dmin[fs] = le.d;
        }
      }
    }
    // frequency-dependent line group ends: a coupled end (T_v, modal 1 / G_eq, so that it stamps
    // T_i diag(G_eq) T_v^-1) whose three modes are frequency-dependent line ends on modal quantities
    for (int64_t x : gends_of[s]) {
      const int64_t gi = x >> 1;
      const int e = (int)(x & 1);
      CoupledEndDev ce{};
      ce.le0 = (int)c->line_ends.size() - sd.le_off;
      for (int k = 0; k < 9; ++k) ce.tv[k] = d->fg_tv[9 * gi + k];
      const int ce_local = (int)c->cends.size() - sd.ce_off;
      for (int j = 0; j < 3; ++j) {
        const int64_t l = d->fg_line[3 * gi + j];
        ce.node[j] = local[e ? d->fl_m[l] : d->fl_k[l]];
        double geq = 0.0;
        FdEndDev r = fd_record(l, geq);
        ce.z[j] = 1.0 / geq;
        const double steps = d->fl_tau[l] / d->dt;
        r.le = (int)c->line_ends.size() - sd.le_off;
        LineEndDev le{};
        le.node = -1;
        le.ce = ce_local;
        le.mode = j;
        le.fd = (int)c->fdends.size() - sd.fd_off;
        le.d = (int32_t)std::floor(steps);
        le.depth = 2 * le.d;
        le.f = steps - (double)le.d;
        r.omf = 1.0 - le.f;
        le.y = 0.0;
        le.y2 = 0.0;
        le.own_ring = fl_ring[2 * l + e];
        le.far_ring = fl_ring[2 * l + 1 - e];
        c->fdends.push_back(r);
        c->line_ends.push_back(le);
        const int fs = c->sub_of_node[e ? d->fl_k[l] : d->fl_m[l]];
        if (fs != s) {
          auto it = dmin.find(fs);
          if (it == dmin.end() || it->second > le.d) dmin[fs] = le.d;
        }
      }
      c->cends.push_back(ce);
    }
    sd.n_ce = (int)c->cends.size() - sd.ce_off;
    c->lim.ce = std::max(c->lim.ce, sd.n_ce);
    // frequency-dependent line ends: a line end each (the ring carries w)
    // and a record with the discretised pole terms
    for (int64_t x : fends_of[s]) {
      const int64_t l = x >> 1;
      const int e = (int)(x & 1);
      const double dt = d->dt, steps = d->fl_tau[l] / dt;
      double geq = 0.0;
      FdEndDev r = fd_record(l, geq);
      r.le = (int)c->line_ends.size() - sd.le_off;
      LineEndDev le{};
      le.node = local[e ? d->fl_m[l] : d->fl_k[l]];
      le.ce = -1;
      le.fd = (int)c->fdends.size() - sd.fd_off;
      le.d = (int32_t)std::floor(steps);
      le.depth = 2 * le.d;
      le.f = steps - (double)le.d;
      r.omf = 1.0 - le.f;
      le.y = geq;
      le.y2 = 0.0;
      le.own_ring = fl_ring[2 * l + e];
      le.far_ring = fl_ring[2 * l + 1 - e];
      c->fdends.push_back(r);
      c->line_ends.push_back(le);
      const int fs = c->sub_of_node[e ? d->fl_k[l] : d->fl_m[l]];
      if (fs != s) {
        auto it = dmin.find(fs);
        if (it == dmin.end() || it->second > le.d) dmin[fs] = le.d;
      }
    }
    sd.n_fd = (int)c->fdends.size() - sd.fd_off;
    c->lim.fd = std::max(c->lim.fd, sd.n_fd);
    sd.n_le = (int)c->line_ends.size() - sd.le_off;
    c->lim.le = std::max(c->lim.le, sd.n_le);
    sd.nb_off = (int)c->nb_sub.size();
    for (auto& kv : dmin) {
      c->nb_sub.push_back(kv.first);
      c->nb_dmin.push_back(kv.second);
    }
    sd.n_nb = (int)c->nb_sub.size() - sd.nb_off;
  }

  // -------- strong L/C branches (see kStrongRatio), from the companion
  // conductances and the line-end conductances at each node
  auto companion = [&](const BranchDev& x) {
    return x.kind == 0 ? 1.0 / x.value : (x.kind == 1 ? c->dt / (2.0 * x.value) : 2.0 * x.value / c->dt);
  };
  std::vector<char> strong(c->branches.size(), 0);
  for (int s = 0; s < S; ++s) {
    SubDev& sd = c->subs[s];
    std::vector<double> diag(sd.n, 0.0);
    for (int b = sd.br_off; b < sd.br_off + sd.n_br; ++b) {
      const BranchDev& x = c->branches[b];
      const double g = companion(x);
      if (x.k >= 0) diag[x.k] += g;
      if (x.m >= 0) diag[x.m] += g;
    }
    for (int e = sd.le_off; e < sd.le_off + sd.n_le; ++e)
      if (c->line_ends[e].node >= 0) diag[c->line_ends[e].node] += c->line_ends[e].y;
    for (int x = sd.ce_off; x < sd.ce_off + sd.n_ce; ++x) {   // Y_p diagonal of coupled ends
      const CoupledEndDev& ce = c->cends[x];
      double inv[9];
      invert3_host(ce.tv, inv);
      for (int p = 0; p < 3; ++p)
        for (int j = 0; j < 3; ++j) diag[ce.node[p]] += inv[3 * j + p] * inv[3 * j + p] / ce.z[j];
    }
    sd.str_off = (int)c->str_slot.size();
    std::vector<std::pair<double, int>> cand;   // (ratio, branch), strongest first
    for (int b = sd.br_off; b < sd.br_off + sd.n_br; ++b) {
      const BranchDev& x = c->branches[b];
      if (x.kind == 0 || x.k < 0 || x.m < 0) continue;
      const double g = companion(x);
      const double rest = std::min(diag[x.k] - g, diag[x.m] - g);
      if (g >= kStrongRatio * rest) cand.push_back({rest > 0.0 ? g / rest : 1e300, b});
    }
    std::sort(cand.begin(), cand.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
      return a.first > b.first || (a.first == b.first && a.second < b.second);
    });
    // the n x (n + n_str) solve matrix (double + float) must fit on chip
    const int max_nc = std::max(sd.n, (int)(kSolveSmemBytes / (12.0 * std::max(sd.n, 1))) - 1);
    const int keep = std::min((int)cand.size(), max_nc - sd.n);
    std::vector<int> chosen;
    for (int i = 0; i < keep; ++i) chosen.push_back(cand[i].second);
    std::sort(chosen.begin(), chosen.end());
    for (int b : chosen) {
      strong[b] = 1;
      c->str_slot.push_back(lc_slot_of[b]);
    }
    sd.n_str = (int)c->str_slot.size() - sd.str_off;
    c->lim.str = std::max(c->lim.str, sd.n_str);
    c->lim.nc = std::max(c->lim.nc, sd.n + sd.n_str);
  }

  // -------- nonlinear resistors (compensation method): at most one per
  // subsystem, the odd characteristic as segments from (0, 0)
  {
    std::vector<std::vector<int64_t>> nl_of(S);
    const int max_nl = scen ? 1 : kNlMaxPerSub;
    for (int64_t x = 0; x < d->n_nonlin; ++x) {
      const int a = d->nl_k[x] >= 0 ? d->nl_k[x] : d->nl_m[x];
      const int sb = c->sub_of_node[a];
      nl_of[sb].push_back(x);
      if ((int)nl_of[sb].size() > max_nl)
        return bail("subsystem " + std::to_string(sb) + " has more than " + std::to_string(max_nl) +
                    " nonlinear resistors" + (scen ? " (in a scenario set)" : ""));
    }
    for (int s = 0; s < S; ++s) {
      SubDev& sd = c->subs[s];
      sd.nl_off = (int)c->nls.size();
      sd.n_nl = (int)nl_of[s].size();
      for (int64_t x : nl_of[s]) {
        NlDev q{};
        q.k = d->nl_k[x] >= 0 ? local[d->nl_k[x]] : -1;
        q.m = d->nl_m[x] >= 0 ? local[d->nl_m[x]] : -1;
        q.np = d->nl_np[x];
        for (int j = 0; j < q.np; ++j) {
          q.bv[j + 1] = d->nl_v[kNlMaxPoints * x + j];
          q.bi[j + 1] = d->nl_i[kNlMaxPoints * x + j];
        }
        for (int j = 0; j < q.np; ++j) q.sl[j] = (q.bi[j + 1] - q.bi[j]) / (q.bv[j + 1] - q.bv[j]);
        q.sl[q.np] = q.sl[q.np - 1];   // past the last point, the last slope
        c->nls.push_back(q);
      }
      c->lim.nl = std::max(c->lim.nl, sd.n_nl);
    }
  }

  // -------- control blocks (Sec. III-A/B: control components as basic
  // processes, layered).  Each connected group of blocks runs in the
  // subsystem of the nodes it measures and drives; within a subsystem a
  // block's layer is one more than the deepest block it reads at the same
  // step (inputs of lower index), and the CTA evaluates layer after layer.
  std::vector<std::vector<int32_t>> ci_nodes_of(S);   // local node per control injection, by subsystem
  {
    const int64_t NB = d->n_cblocks;
    auto n_inputs = [&](int64_t b) { const int t = d->cb_type[b]; return t <= 1 ? 0 : (t == 3 || t == 4) ? 2 : 1; };
    auto input = [&](int64_t b, int i) { return i == 0 ? d->cb_in0[b] : d->cb_in1[b]; };
    std::vector<int> grp(NB);
    std::iota(grp.begin(), grp.end(), 0);
    for (int64_t b = 0; b < NB; ++b)
      for (int i = 0; i < n_inputs(b); ++i) {
        const int x = uf_find(grp, (int)b), y = uf_find(grp, input(b, i));
        if (x != y) grp[std::max(x, y)] = std::min(x, y);
      }
    std::vector<int> gsub(NB, -1);
    auto claim = [&](int64_t b, int32_t node) -> bool {
      const int r = uf_find(grp, (int)b), sn = c->sub_of_node[node];
      if (gsub[r] >= 0 && gsub[r] != sn) return false;
      gsub[r] = sn;
      return true;
    };
    for (int64_t b = 0; b < NB; ++b)
      if (d->cb_type[b] == 1 && !claim(b, d->cb_node[b]))
        return bail("control block " + std::to_string(b) + " belongs to a block group spanning two subsystems");
    for (int64_t x = 0; x < d->n_cinj; ++x)
      if (!claim(d->ci_block[x], d->ci_node[x]))
        return bail("control injection " + std::to_string(x) + " drives a node outside its block group's subsystem");
    c->cb_sub_of.assign(NB, 0);
    c->cb_slot_of.assign(NB, -1);
    std::vector<std::vector<int64_t>> cb_of(S);
    for (int64_t b = 0; b < NB; ++b) {
      const int r = uf_find(grp, (int)b);
      c->cb_sub_of[b] = gsub[r] >= 0 ? gsub[r] : 0;
      if (S > 0) cb_of[c->cb_sub_of[b]].push_back(b);   // increasing caller index
    }
    std::vector<int> layer(NB, 0);
    for (int s = 0; s < S; ++s) {
      SubDev& sd = c->subs[s];
      int n_layers = 0;
      for (int64_t b : cb_of[s]) {
        for (int i = 0; i < n_inputs(b); ++i)
          if (input(b, i) < b) layer[b] = std::max(layer[b], layer[input(b, i)] + 1);
        n_layers = std::max(n_layers, layer[b] + 1);
      }
      std::vector<int64_t> order = cb_of[s];
      std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return layer[a] < layer[b]; });
      for (size_t j = 0; j < order.size(); ++j) c->cb_slot_of[order[j]] = (int32_t)j;
      sd.cb_off = (int)c->cblocks.size();
      sd.n_cb = (int)order.size();
      sd.clay_off = (int)c->clay.size();
      sd.n_clay = sd.n_cb > 0 ? n_layers : 0;
      const double dt = d->dt;
      const int zero_pair = 2 * sd.n_cb;
      for (size_t j = 0; j < order.size(); ++j) {
        const int64_t b = order[j];
        if (j == 0 || layer[b] != layer[order[j - 1]]) {   // a layer starts: its type if uniform
          int lt = d->cb_type[b];
          for (size_t q = j; q < order.size() && layer[order[q]] == layer[b]; ++q)
            if (d->cb_type[order[q]] != lt) lt = kMixedLayer;
          c->clay.push_back((int32_t)j | (lt << kLayerTypeShift));
        }
        CtrlDev r{};
        r.type = d->cb_type[b];
        r.i0 = r.i1 = zero_pair;
        for (int i = 0; i < n_inputs(b); ++i)
          (i == 0 ? r.i0 : r.i1) = 2 * c->cb_slot_of[input(b, i)] + (input(b, i) >= b ? 1 : 0);
        r.node = r.type == 1 ? local[d->cb_node[b]] : -1;
        const double p0 = d->cb_p0[b], p1 = d->cb_p1[b];
        ctrl_coefficients(r, p0, p1, dt);
        r.ov = -1.0;
        c->cblocks.push_back(r);
      }
      if (sd.n_cb > 0) c->clay.push_back(sd.n_cb);
      c->lim.cb = std::max(c->lim.cb, sd.n_cb);
      c->lim.clay = std::max(c->lim.clay, sd.n_clay + 1);
      c->max_clayers = std::max(c->max_clayers, sd.n_clay);
    }
    std::vector<std::vector<int32_t>> ci_of(S);
    for (int64_t x = 0; x < d->n_cinj; ++x) ci_of[c->sub_of_node[d->ci_node[x]]].push_back((int32_t)x);
    for (int s = 0; s < S; ++s) {
      SubDev& sd = c->subs[s];
      sd.ci_off = (int)c->cinj.size();
      sd.n_ci = (int)ci_of[s].size();
      for (int32_t x : ci_of[s]) {
        c->cinj.push_back(c->cb_slot_of[d->ci_block[x]]);
        ci_nodes_of[s].push_back(local[d->ci_node[x]]);
      }
      c->lim.ci = std::max(c->lim.ci, sd.n_ci);
    }
  }

  // -------- injection lanes (see kEntryNeg): 4 entries each, a node's
  // lanes consecutive and inside one warp; strong branches stay out
  for (int s = 0; s < S; ++s) {
    SubDev& sd = c->subs[s];
    std::vector<std::vector<int32_t>> el(sd.n);
    const int ie_base = sd.n_lc + sd.n_sb, zero = ie_base + 2 * (sd.n_le + 3 * sd.n_ce + sd.n_fd);
    for (int x = 0; x < sd.n_ci; ++x)   // controlled currents enter their nodes
      el[ci_nodes_of[s][x]].push_back((int32_t)(zero + 1 + x));
    for (int x = 0; x < sd.n_fd; ++x) {   // FD ends draw Hy - b
      const LineEndDev& le = c->line_ends[sd.le_off + c->fdends[sd.fd_off + x].le];
      if (le.ce >= 0) {   // a group mode: its Hy slot carries phase `mode`'s T_i Hy; b enters the phase slots
        el[c->cends[sd.ce_off + le.ce].node[le.mode]].push_back((int32_t)(kEntryNeg | (uint32_t)(zero + 1 + sd.n_ci + x)));
        continue;
      }
      const int node = le.node;
      el[node].push_back((int32_t)(ie_base + sd.n_le + 3 * sd.n_ce + x));
      el[node].push_back((int32_t)(kEntryNeg | (uint32_t)(zero + 1 + sd.n_ci + x)));
    }
    for (int b = sd.br_off; b < sd.br_off + sd.n_br; ++b) {
      const BranchDev& x = c->branches[b];
      if (x.kind != 0 && !strong[b]) {
        const int32_t slot = lc_slot_of[b];
        if (x.k >= 0) el[x.k].push_back((int32_t)(kEntryNeg | (uint32_t)slot));   // current leaves k
        if (x.m >= 0) el[x.m].push_back(slot);                                     // and enters m
      }
      if (sb_slot_of[b] >= 0) el[x.k >= 0 ? x.k : x.m].push_back(sd.n_lc + sb_slot_of[b]);
    }
    for (int e = 0; e < sd.n_le; ++e)
      if (c->line_ends[sd.le_off + e].node >= 0 && c->line_ends[sd.le_off + e].fd < 0)
        el[c->line_ends[sd.le_off + e].node].push_back((int32_t)(kEntryNeg | (uint32_t)(ie_base + e)));
    for (int x = 0; x < sd.n_ce; ++x)   // coupled ends: phase-domain history currents leave the phase nodes
      for (int p = 0; p < 3; ++p)
        el[c->cends[sd.ce_off + x].node[p]].push_back(
            (int32_t)(kEntryNeg | (uint32_t)(ie_base + sd.n_le + 3 * x + p)));
    sd.il_off = (int)c->il_node.size();
    int lanes = 0;
    for (int k = 0; k < sd.n; ++k) {
      while (el[k].size() % 4 || el[k].empty()) el[k].push_back(zero);
      const int cnt = (int)el[k].size() / 4;
      if (cnt > kMaxLanesPerNode)
        return bail("node " + std::to_string(nodes_of[s][k]) + " has more than " +
                    std::to_string(4 * kMaxLanesPerNode) + " branch and line incidences");
      if (lanes % 32 + cnt > 32)
        while (lanes % 32) {   // pad to the next warp
          for (int u = 0; u < 4; ++u) c->ent.push_back(zero);
          c->il_node.push_back(-1);
          c->il_cnt.push_back(0);
          ++lanes;
        }
      for (int j = 0; j < cnt; ++j) {
        for (int u = 0; u < 4; ++u) c->ent.push_back(el[k][4 * j + u]);
        c->il_node.push_back(k);
        c->il_cnt.push_back(j == 0 ? cnt : 0);
        ++lanes;
      }
    }
    sd.n_il = lanes;
    c->lim.il = std::max(c->lim.il, lanes);
  }

  // -------- switch epochs per subsystem, sparse pattern of G per epoch
  {
    std::vector<std::vector<int64_t>> sw_of(S);
    for (int64_t w = 0; w < d->n_switches; ++w) {
      const int a = d->sw_k[w] >= 0 ? d->sw_k[w] : d->sw_m[w];
      sw_of[c->sub_of_node[a]].push_back(w);
    }
    std::vector<std::vector<int64_t>> rs_of(S);
    for (int64_t w = 0; w < d->n_rswitches; ++w) {
      const int a = d->rs_k[w] >= 0 ? d->rs_k[w] : d->rs_m[w];
      rs_of[c->sub_of_node[a]].push_back(w);
    }
    int64_t goff = 0;
    for (int s = 0; s < S; ++s) {
      SubDev& sd = c->subs[s];
      const int max_rs = scen ? kMaxRuntimeSwitches : kMaxLazySwitches;
      if ((int)rs_of[s].size() > max_rs)
        return bail("subsystem " + std::to_string(s) + " has more than " + std::to_string(max_rs) +
                    " runtime switches" + (scen ? " (in a scenario set)" : ""));
      sd.n_rs = (int)rs_of[s].size();
      // up to kMaxRuntimeSwitches every state word is prefactored; above it
      // the states are factorised on the device when first met
      const bool lazy = sd.n_rs > kMaxRuntimeSwitches;
      sd.n_states = lazy ? 1 : 1 << sd.n_rs;
      sd.rs_off = (int)c->rswitches.size();
      int32_t word0 = 0;
      for (int j = 0; j < sd.n_rs; ++j) {
        const int64_t w = rs_of[s][j];
        RuntimeSwitchDev r{};
        r.k = d->rs_k[w] >= 0 ? local[d->rs_k[w]] : -1;
        r.m = d->rs_m[w] >= 0 ? local[d->rs_m[w]] : -1;
        r.kind = d->rs_kind[w];
        r.r_on = d->rs_ron[w];
        r.trip = d->rs_trip_step[w];
        r.r_off = d->rs_roff[w];
        c->rswitches.push_back(r);
        c->rs_roff.push_back(d->rs_roff[w]);
        if (r.kind == 1 || d->rs_on0[w]) word0 |= 1 << j;
      }
      c->rs_word0.push_back(word0);
      std::vector<int64_t> events;
      for (int64_t w : sw_of[s]) {
        if (d->sw_close_step[w] >= 0) events.push_back(d->sw_close_step[w]);
        if (d->sw_open_step[w] >= 0) events.push_back(d->sw_open_step[w]);
      }
      std::sort(events.begin(), events.end());
      events.erase(std::unique(events.begin(), events.end()), events.end());
      std::vector<std::pair<int64_t, int64_t>> eps;   // (start, step at which the state is read)
      eps.push_back({LLONG_MIN, events.empty() ? 1 : events[0] - 1});
      for (int64_t e : events) eps.push_back({e, e});
      sd.ep_off = (int)c->epochs.size();
      const int64_t mat_len = (int64_t)sd.n * (sd.n + sd.n_str);
      if (lazy) {   // cache slots: epoch te's initial state in slot te, then spare slots
        const int n_te = (int)eps.size();
        sd.n_cache = n_te + kLazyCacheExtra;
        sd.cache_slot0 = (int)c->cache_tag0.size();
        sd.cache_goff = goff;
        goff += (int64_t)sd.n_cache * mat_len;
        sd.cache_zoff = c->nlz_len;
        c->nlz_len += (int64_t)sd.n_cache * sd.n_nl * sd.n;
        sd.work_off = c->lazy_work_len;
        c->lazy_work_len += 2 * (int64_t)sd.n * sd.n;
        for (int j = 0; j < sd.n_cache; ++j)
          c->cache_tag0.push_back(j < n_te ? (((long long)j << 32) | (unsigned)word0) : -1ll);
        c->cache_next0.push_back(n_te % sd.n_cache);
        c->lazy = true;
      } else {
        c->cache_next0.push_back(0);
      }
      for (int te = 0; te < (int)eps.size(); ++te) {
        const auto& ep = eps[te];
        for (int word = 0; word < sd.n_states; ++word) {
          EpochDev E{};
          E.start = ep.first;
          if (lazy) {
            E.ginv_off = sd.cache_goff + te * mat_len;
          } else {
            E.ginv_off = goff;
            goff += mat_len;
          }
          E.nlz_off = -1;
          if (sd.n_nl > 0) {   // one column per nonlinear resistor
            if (lazy) {
              E.nlz_off = sd.cache_zoff + (int64_t)te * sd.n_nl * sd.n;
            } else {
              E.nlz_off = c->nlz_len;
              c->nlz_len += (int64_t)sd.n_nl * sd.n;
            }
          }
          E.rs_word = lazy ? word0 : -1;
          E.sw_off = (int)c->switches.size();
          for (int64_t w : sw_of[s]) {
            if (!switch_closed(d->sw_close_step[w], d->sw_open_step[w], ep.second)) continue;
            SwitchDev sw{};
            sw.k = d->sw_k[w] >= 0 ? local[d->sw_k[w]] : -1;
            sw.m = d->sw_m[w] >= 0 ? local[d->sw_m[w]] : -1;
            sw.g = 1.0 / d->sw_r[w];
            c->switches.push_back(sw);
          }
          for (int j = 0; j < sd.n_rs && !lazy; ++j) {   // runtime switches: r_on or r_off by the state word
            const int64_t w = rs_of[s][j];
            SwitchDev sw{};
            sw.k = d->rs_k[w] >= 0 ? local[d->rs_k[w]] : -1;
            sw.m = d->rs_m[w] >= 0 ? local[d->rs_m[w]] : -1;
            sw.g = 1.0 / (((word >> j) & 1) ? d->rs_ron[w] : d->rs_roff[w]);
            c->switches.push_back(sw);
          }
          E.n_sw = (int)c->switches.size() - E.sw_off;
          c->epochs.push_back(E);
        }
      }
      sd.n_ep = (int)c->epochs.size() - sd.ep_off;
    }
    c->ginv_len = goff;
    c->cache_next0.push_back(0);   // the count of run-time factorisations
  }

  // -------- matvec blocking: n q tasks (at most one per thread) of
  // ceil(nc / q) dependent FMAs, then a node's q - 1 adds: q minimises that
  // chain of FP64 instructions (ties: nearest sqrt(nc))
  for (int s = 0; s < S; ++s) {
    SubDev& sd = c->subs[s];
    const int n = std::max(sd.n, 1), ncol = std::max(sd.n + sd.n_str, 1);
    int q = 1;
    long best = LONG_MAX;
    const double root = std::sqrt((double)ncol);
    for (int t = 1; t <= std::min(std::min(32, ncol), std::max(1, kFwdThreads / n)); ++t) {
      const long chain = (ncol + t - 1) / t + (t - 1);
      if (chain < best || (chain == best && std::fabs(t - root) < std::fabs(q - root))) {
        best = chain;
        q = t;
      }
    }
    sd.q = q;
    c->lim.q = std::max(c->lim.q, sd.q);
    // every task runs the same number of columns (zero columns pad the
    // last block), so that no warp diverges inside the FMA loop
    const int nc = sd.n + sd.n_str;
    c->lim.nc = std::max(c->lim.nc, sd.q * ((nc + sd.q - 1) / sd.q));
  }

  // -------- two solve-matrix buffers per CTA when runtime switches change
  // matrices at run time and both fit
  c->lim.nbuf = 1;
  if (!c->rswitches.empty()) {
    FwdLimits two = c->lim;
    two.nbuf = 2;
    two.n = std::max(two.n, 1);
    two.nc = std::max(two.nc, 1);
    if (forward_smem_bytes(two) <= 200 * 1024) c->lim.nbuf = 2;
  }

  // -------- the warp-per-subsystem kernel serves networks of small subsystems
  // with R/L/C branches, sources, fixed-time switches and lossless lines only
  c->small_ok = !scen && S > 0 && c->lim.n <= kSmallMaxNodes && c->lim.ce == 0 && c->lim.fd == 0 &&
                c->lim.cb == 0 && c->lim.ci == 0 && c->lim.nl == 0 && c->rswitches.empty() && !c->lazy;

  // -------- the state-space form (emt_ss.cu): the same element set; per
  // subsystem M's shape, its line-end nodes, and Q lanes per row of the
  // product chosen against a model of the step: its chain (ceil(cols/Q)
  // FMAs, log2 Q shuffle-adds, one add, the line outputs of a node) and the
  // FP64 instructions of the CTAs one SM holds, on its four pipes
  c->ss_ok = !scen && S > 0 && c->lim.ce == 0 && c->lim.fd == 0 && c->lim.cb == 0 && c->lim.ci == 0 &&
             c->lim.nl == 0 && c->rswitches.empty() && !c->lazy;
  if (c->ss_ok) {
    int n_sm = 148;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device);
    const int cps = (S + n_sm - 1) / std::max(n_sm, 1);
    c->ss.assign(S, SsSubDev{});
    c->ss_lend.assign(c->line_ends.size(), 0);
    c->ss_compact = cps > 1 && c->lim.n <= 32;
    int64_t off = 0;
    for (int s = 0; s < S && c->ss_ok; ++s) {
      const SubDev& sd = c->subs[s];
      std::map<int, std::vector<int>> by_node;   // ends grouped by their node, nodes ascending
      for (int x = 0; x < sd.n_le; ++x) by_node[c->line_ends[sd.le_off + x].node].push_back(x);
      SsSubDev& Q = c->ss[s];
      Q.n_ln = (int32_t)by_node.size();
      Q.ln_off = (int32_t)c->ss_lnode.size();
      Q.ptr_off = (int32_t)c->ss_lptr.size();
      int pos = 0, most = 0;
      for (const auto& kv : by_node) {
        c->ss_lnode.push_back(kv.first);
        c->ss_lptr.push_back(pos);
        for (int x : kv.second) c->ss_lend[sd.le_off + pos++] = x;
        most = std::max(most, (int)kv.second.size());
      }
      c->ss_lptr.push_back(pos);
      // several CTAs to an SM: the compact step (one warp, M's node rows only)
      Q.compact = c->ss_compact ? 1 : 0;
      Q.rows = Q.compact ? sd.n : sd.n_lc + sd.n;
      Q.cols = sd.n_lc + sd.n_src + Q.n_ln;
      if (Q.rows > kSsThreads - 32 || Q.cols < 1) {
        c->ss_ok = false;
        break;
      }
      if (Q.compact) {   // the most lanes per row that one warp holds
        Q.q = 1;
        while (Q.q < 32 && sd.n * Q.q * 2 <= 32 && Q.q < Q.cols) Q.q *= 2;
      } else {
        double best = 1e300;
        for (int qq = 1, lg = 0; qq <= 32 && Q.rows * qq <= kSsThreads - 32; qq *= 2, ++lg) {
          const double chain = (Q.cols + qq - 1) / qq + lg + 1 + (most + qq - 1) / qq;
          const double warps = (Q.rows * qq + 31) / 32;
          const double cost = std::max(chain, cps * warps * chain / 4.0);
          if (cost < best) {
            best = cost;
            Q.q = qq;
          }
        }
      }
      Q.m_off = off;
      off += (int64_t)sd.n_ep * Q.rows * Q.cols;
      c->ss_rows = std::max(c->ss_rows, Q.rows);
      c->ss_cols = std::max(c->ss_cols, Q.cols);
      c->ss_ln = std::max(c->ss_ln, Q.n_ln);
      c->ss_max_entries = std::max<int64_t>(c->ss_max_entries, (int64_t)Q.rows * Q.cols);
    }
    c->ss_len = off;
    if (c->ss_ok && ss_smem_bytes(c->ss_rows, c->ss_cols, std::max(c->lim.n, 1), c->lim.le, c->lim.src, c->ss_ln,
                                  c->lim.lc) *
                            (size_t)cps > 220 * 1024)
      c->ss_ok = false;
  }

  // -------- injection-lane range of every internal node
  c->node_l0.assign(N, 0);
  c->node_nl.assign(N, 0);
  for (int s = 0; s < S; ++s) {
    const SubDev& sd = c->subs[s];
    for (int l = 0; l < sd.n_il; ++l) {
      const int cnt = c->il_cnt[sd.il_off + l];
      if (cnt > 0) {
        c->node_l0[sd.node_off + c->il_node[sd.il_off + l]] = l;
        c->node_nl[sd.node_off + c->il_node[sd.il_off + l]] = cnt;
      }
    }
  }

  // -------- multi-scenario set
  if (scen) {
    const std::string bm = build_scenarios(c, d, scen, local, new_of_orig, le_of_end, lc_slot_of, sb_slot_of);
    if (!bm.empty()) return bail(bm);
  }

  // -------- upload
  cudaError_t e = cudaSuccess;
#define UP(dst, vec) \
  if (e == cudaSuccess) e = c->upload(&c->dst, c->vec);
  UP(d_sub, subs)
  UP(d_ep, epochs)
  UP(d_br, branches)
  UP(d_lc_idx, lc_idx)
  UP(d_sb_idx, sb_idx)
  UP(d_ent, ent)
  UP(d_il_node, il_node)
  UP(d_il_cnt, il_cnt)
  UP(d_str_slot, str_slot)
  UP(d_le, line_ends)
  UP(d_src_global, src_global)
  UP(d_src_amp, src_amp)
  UP(d_src_phase, src_phase)
  UP(d_src_omega, src_omega)
  UP(d_sw, switches)
  UP(d_rs, rswitches)
  UP(d_ce, cends)
  UP(d_rs_word, rs_word0)
  UP(d_fd, fdends)
  UP(d_nl, nls)
  if (e == cudaSuccess && !c->nls.empty()) {
    const std::vector<int32_t> one(c->nls.size(), 1);
    e = c->upload(&c->d_nl_seg, one);
  }
  UP(d_cb, cblocks)
  UP(d_clay, clay)
  UP(d_cinj, cinj)
  UP(d_br_orig, br_orig)
  UP(d_br_lc, br_lc)
  UP(d_br_src, br_src)
  UP(d_src_br_ptr, src_br_ptr)
  UP(d_src_br, src_br)
  UP(d_original_of, original_of)
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_h, (size_t)c->n_lc_total);
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_ring, 2 * (size_t)std::max<int64_t>(c->ring_len, 1));
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_ginv, (size_t)c->ginv_len);
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_ginv_lo, (size_t)c->ginv_len);
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_err, 4);
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_rs_prev_i, c->rswitches.size());
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_fd_state, kFdState * c->fdends.size());
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_nlz, (size_t)c->nlz_len);
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_nlz_lo, (size_t)c->nlz_len);
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_cstate, 2 * c->cblocks.size());
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_cy, c->cblocks.size());
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_le_prev, c->line_ends.size());
  if (c->ss_ok) {
    UP(d_ss, ss)
    UP(d_ss_lnode, ss_lnode)
    UP(d_ss_lptr, ss_lptr)
    UP(d_ss_lend, ss_lend)
    if (e == cudaSuccess) e = c->alloc_zero(&c->d_ss_m, (size_t)c->ss_len);
    if (e == cudaSuccess) e = c->alloc_zero(&c->d_ss_mlo, (size_t)c->ss_len);
  }
  if (c->lazy) {
    UP(d_cache_tag0, cache_tag0)
    UP(d_cache_tag, cache_tag0)
    UP(d_cache_next0, cache_next0)
    UP(d_cache_next, cache_next0)
    if (e == cudaSuccess) e = c->alloc_zero(&c->d_lazy_work, (size_t)c->lazy_work_len);
  }
  if (c->batched) {
    UP(d_col_code, b_col_code)
    UP(d_col_sub, b_col_sub)
    UP(d_node_sub, b_node_sub)
    UP(d_node_r, b_node_r)
    UP(d_sub_nc, b_sub_nc)
    UP(d_sub_col_off, b_sub_col_off)
    UP(d_ent_ptr, b_ent_ptr)
    UP(d_bent, b_bent)
    UP(d_lc_nk, b_lc_nk)
    UP(d_lc_nm, b_lc_nm)
    UP(d_lc_isl, b_lc_isl)
    UP(d_sb_src, b_sb_src)
    UP(d_le_nd, b_le_nd)
    UP(d_le_d1, b_le_d1)
    UP(d_le_y2, b_le_y2)
    UP(d_ev_ptr, b_ev_ptr)
    UP(d_ev_step, b_ev_step)
    UP(d_ev_sub, b_ev_sub)
    UP(d_ev_off, b_ev_off)
    UP(d_dig_ptr, dig_ptr)
    UP(d_dig_key, dig_key)
    UP(d_dig_val, dig_val)
    UP(d_sub_node0, dig_node0)
    UP(d_sub_n, dig_sub_n)
    UP(d_dig_mat_goff, dig_mat_goff)
    UP(d_dig_mat_n, dig_mat_n)
    UP(d_dig_mat_nc, dig_mat_nc)
    if (e == cudaSuccess) e = c->alloc_zero(&c->d_dig, (size_t)std::max<int64_t>(c->dig_len, 1));
    if (e == cudaSuccess) e = c->upload(&c->d_le_bring, c->le_bring);
    if (e == cudaSuccess) e = c->upload(&c->d_le_bfar, c->le_bfar);
    if (e == cudaSuccess) e = c->upload(&c->d_bsrc_amp, c->bsrc_amp);
    if (e == cudaSuccess) e = c->upload(&c->d_bsrc_phase, c->bsrc_phase);
    if (e == cudaSuccess) e = c->upload(&c->d_rm_ptr_br, c->rm_ptr_br);
    if (e == cudaSuccess) e = c->upload(&c->d_rm_br, c->rm_br);
    if (e == cudaSuccess) e = c->upload(&c->d_rm_ptr_le, c->rm_ptr_le);
    if (e == cudaSuccess) e = c->upload(&c->d_rm_le, c->rm_le);
    if (!c->keep_lc.empty()) {
      if (e == cudaSuccess) e = c->upload(&c->d_keep_lc, c->keep_lc);
      if (e == cudaSuccess) e = c->upload(&c->d_keep_sb, c->keep_sb);
      if (e == cudaSuccess) e = c->upload(&c->d_keep_le, c->keep_le);
    }
    if (!c->b_cb.empty()) {
      if (e == cudaSuccess) e = c->upload(&c->d_bcb, c->b_cb);
      if (e == cudaSuccess && !c->b_cinj.empty()) e = c->upload(&c->d_bcinj, c->b_cinj);
      if (e == cudaSuccess && !c->b_cbo.empty()) e = c->upload(&c->d_bcbo, c->b_cbo);
      if (e == cudaSuccess) e = c->alloc_zero(&c->d_bcy, (2 * c->b_cb.size() + 2) * (size_t)c->S);
      if (e == cudaSuccess) e = c->alloc_zero(&c->d_bcs, 2 * c->b_cb.size() * (size_t)c->S);
    }
    if (!c->rswitches.empty()) {
      if (e == cudaSuccess) e = c->upload(&c->d_bsub_rs, c->b_sub_rs);
      if (e == cudaSuccess) e = c->alloc_zero(&c->d_bword, (size_t)c->n_sub * c->S);
      if (e == cudaSuccess) e = c->alloc_zero(&c->d_brsi, c->rswitches.size() * (size_t)c->S);
      if (e == cudaSuccess) e = c->alloc_zero(&c->d_bvbase, (size_t)c->n_sub * c->S);
      if (e == cudaSuccess) e = reset_batch_words(c);
    }
    if (!c->b_ce_le0.empty()) {
      if (e == cudaSuccess) e = c->upload(&c->d_bce_le0, c->b_ce_le0);
      if (e == cudaSuccess) e = c->upload(&c->d_bce_node, c->b_ce_node);
      if (e == cudaSuccess) e = c->upload(&c->d_ble_ce, c->b_le_ce);
      if (e == cudaSuccess) e = c->upload(&c->d_ble_f, c->b_le_f);
      if (e == cudaSuccess) e = c->alloc_zero(&c->d_bcim, 3 * c->b_ce_le0.size() * (size_t)c->S);
      if (e == cudaSuccess) e = c->alloc_zero(&c->d_bcph, 3 * c->b_ce_le0.size() * (size_t)c->S);
    }
    if (!c->b_fd_le.empty()) {
      if (e == cudaSuccess) e = c->upload(&c->d_bfd_le, c->b_fd_le);
      if (e == cudaSuccess) e = c->upload(&c->d_ble_fd, c->b_le_fd);
      if (e == cudaSuccess) e = c->alloc_zero(&c->d_bfds, c->b_fd_le.size() * kBatchFdState * (size_t)c->S);
    }
    if (!c->b_nlinfo.empty()) {
      if (e == cudaSuccess) e = c->upload(&c->d_bnlinfo, c->b_nlinfo);
      if (e == cudaSuccess) e = c->upload(&c->d_bnlc, c->b_nlc);
      if (e == cudaSuccess) e = c->alloc_zero(&c->d_bnli, c->nls.size() * (size_t)c->S);
    }
    if (e == cudaSuccess) e = c->alloc_zero(&c->d_bh, (size_t)c->n_lc_total * c->S);
    if (e == cudaSuccess) e = c->alloc_zero(&c->d_bring, (size_t)std::max<int64_t>(c->bring_len, 1) * c->S);
    if (e == cudaSuccess) e = c->alloc_zero(&c->d_src_ac, (size_t)c->S * c->n_sources);
    if (e == cudaSuccess) e = c->alloc_zero(&c->d_src_as, (size_t)c->S * c->n_sources);
    if (e == cudaSuccess) e = c->alloc_zero(&c->d_lc_e, (size_t)c->lc_idx.size());
    if (e == cudaSuccess) e = c->alloc_zero(&c->d_sb_g, (size_t)c->sb_idx.size());
  }
#undef UP
  if (e == cudaSuccess && c->batched && !batch_configure(c, c->S_t, true)) e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = launch_companion(c->d_br, (int64_t)c->branches.size(), c->dt, nullptr);
  if (e == cudaSuccess) e = launch_coupled_constants(c->d_ce, (int64_t)c->cends.size(), nullptr);
  if (e == cudaSuccess && c->batched)
    e = launch_source_coefficients(c->d_bsrc_amp, c->d_bsrc_phase, c->S * c->n_sources, c->d_src_ac, c->d_src_as,
                                   nullptr);
  if (e == cudaSuccess && c->batched)
    e = launch_slot_constants(c->d_br, c->d_lc_idx, (int64_t)c->lc_idx.size(), c->d_sb_idx, (int64_t)c->sb_idx.size(),
                              c->d_lc_e, c->d_sb_g, nullptr);
  if (e == cudaSuccess) e = launch_ring_init(RingInitParams{c->d_le, (int64_t)c->line_ends.size(), c->d_ring}, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    g_build_error = std::string("device setup failed: ") + cudaGetErrorString(e);
    const emt_status st = (e == cudaErrorMemoryAllocation) ? EMT_ENOMEM : EMT_ECUDA;
    emt_destroy(c);
    return st;
  }
  *out = c;
  return EMT_OK;
}

// Subsystems that factorise their states at run time: after a prefactor,
// the cache holds each epoch's initial state (slot te) and nothing else.
// M of every (subsystem, epoch) of the state-space form, from the G^-1
// just prefactored (emt_ss.cu).
static cudaError_t build_state_space(emt_ctx* c, cudaStream_t st) {
  if (!c->ss_ok) return cudaSuccess;
  FwdParams p{};
  p.n_sub = c->n_sub;
  p.sub = c->d_sub;
  p.ep = c->d_ep;
  p.ginv = c->d_ginv;
  p.ginv_lo = c->d_ginv_lo;
  p.br = c->d_br;
  p.lc_idx = c->d_lc_idx;
  p.sb_idx = c->d_sb_idx;
  p.le = c->d_le;
  p.str_slot = c->d_str_slot;
  p.ss = c->d_ss;
  p.ss_m = c->d_ss_m;
  p.ss_mlo = c->d_ss_mlo;
  p.ss_lnode = c->d_ss_lnode;
  return launch_ss_build(p, st);
}

static cudaError_t reset_matrix_cache(emt_ctx* c, cudaStream_t st) {
  if (!c->lazy) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(c->d_cache_tag, c->d_cache_tag0, c->cache_tag0.size() * sizeof(long long),
                                  cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_cache_next, c->d_cache_next0, c->cache_next0.size() * sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, st);
  return e;
}

extern "C" emt_status emt_prefactor(emt_ctx* c) {
  NvtxRange nvtx_range("emt_prefactor");
  if (!c) return EMT_EINVAL;
  std::vector<int32_t> mat_sub, mat_ep;
  if (c->batched) {
    for (size_t v = 0; v < c->var_sub.size(); ++v) {
      mat_sub.push_back(c->var_sub[v]);
      mat_ep.push_back((int32_t)(c->n_base_epochs + v));
    }
  } else {
    for (int s = 0; s < c->n_sub; ++s)
      for (int k = 0; k < c->subs[s].n_ep; ++k) {
        mat_sub.push_back(s);
        mat_ep.push_back(c->subs[s].ep_off + k);
      }
  }
  int32_t *d_ms = nullptr, *d_me = nullptr, *d_status = nullptr;
  double *d_wg = nullptr, *d_wr = nullptr;
  cudaError_t e = c->upload(&d_ms, mat_sub);
  if (e == cudaSuccess) e = c->upload(&d_me, mat_ep);
  if (e == cudaSuccess) e = c->alloc_zero(&d_status, mat_sub.size());
  if (e == cudaSuccess) e = c->alloc_zero(&d_wg, (size_t)c->ginv_len);
  if (e == cudaSuccess) e = c->alloc_zero(&d_wr, (size_t)c->ginv_len);
  PrefParams p{};
  p.n_mats = (int32_t)mat_sub.size();
  p.mat_sub = d_ms;
  p.mat_ep = d_me;
  p.sub = c->d_sub;
  p.ep = c->d_ep;
  p.br = c->d_br;
  p.le = c->d_le;
  p.sw = c->d_sw;
  p.ce = c->d_ce;
  p.lc_idx = c->d_lc_idx;
  p.str_slot = c->d_str_slot;
  p.ginv = c->d_ginv;
  p.ginv_lo = c->d_ginv_lo;
  p.nl = c->d_nl;
  p.nlz = c->batched ? c->d_ginv : c->d_nlz;   // a scenario variant keeps z after its matrix
  p.nlz_lo = c->batched ? c->d_ginv_lo : c->d_nlz_lo;
  p.work_g = d_wg;
  p.work_r = d_wr;
  p.status = d_status;
  p.rs = c->d_rs;
  if (c->batched) {
    p.rm_ptr_br = c->d_rm_ptr_br;
    p.rm_br = c->d_rm_br;
    p.rm_ptr_le = c->d_rm_ptr_le;
    p.rm_le = c->d_rm_le;
  }
  if (e == cudaSuccess) e = launch_prefactor(p, std::max(c->lim.n, 1), nullptr);
  if (e == cudaSuccess) e = reset_matrix_cache(c, nullptr);
  if (e == cudaSuccess) e = build_state_space(c, nullptr);
  if (e == cudaSuccess && c->batched)   // the shared matrices in digit form
    e = launch_batch_digits(c->d_ginv, c->d_ginv_lo, c->d_dig_mat_goff, c->d_dig_mat_n, c->d_dig_mat_nc, c->d_dig_val,
                            (int)c->dig_key.size(), c->d_dig, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  std::vector<int32_t> status(mat_sub.size(), 0);
  if (e == cudaSuccess && !status.empty())
    e = cudaMemcpy(status.data(), d_status, status.size() * sizeof(int32_t), cudaMemcpyDeviceToHost);
  c->release(d_ms);
  c->release(d_me);
  c->release(d_status);
  c->release(d_wg);
  c->release(d_wr);
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_prefactor");
  for (size_t i = 0; i < status.size(); ++i)
    if (status[i] != 0) {
      const int s = mat_sub[i];
      return c->fail(EMT_ESINGULAR, "conductance matrix of subsystem " + std::to_string(s) + " (first node " +
                                        std::to_string(c->original_of[c->subs[s].node_off]) + ", switch state " +
                                        std::to_string(mat_ep[i] - c->subs[s].ep_off) + ") is singular");
    }
  c->prefactored = true;
  return EMT_OK;
}

extern "C" emt_status emt_set_recording(emt_ctx* c, const int32_t* channels, int64_t n_ch, int32_t decim,
                                        int64_t max_rows) {
  if (!c) return EMT_EINVAL;
  if (decim < 1 || max_rows < 0 || n_ch < 0) return c->fail(EMT_EINVAL, "decim must be >= 1, counts >= 0");
  cudaDeviceSynchronize();
  c->release(c->d_rec);
  c->release(c->d_rec_pos);
  c->d_rec = nullptr;
  c->d_rec_pos = nullptr;
  c->rec_channels.clear();
  c->rec_col_of.assign(c->n_nodes, -1);
  c->rec_rows = 0;
  if (n_ch == 0 || max_rows == 0) return EMT_OK;
  std::vector<int32_t> chans;
  if (channels) {
    for (int64_t i = 0; i < n_ch; ++i) {
      const int32_t x = channels[i];
      if (x < 0 || x >= c->n_nodes) return c->fail(EMT_EINVAL, "channel " + std::to_string(x) + " is not a node");
      if (c->rec_col_of[x] >= 0) return c->fail(EMT_EINVAL, "channel " + std::to_string(x) + " listed twice");
      c->rec_col_of[x] = (int32_t)chans.size();
      chans.push_back(x);
    }
  } else {
    for (int64_t i = 0; i < c->n_nodes; ++i) {
      c->rec_col_of[i] = (int32_t)i;
      chans.push_back((int32_t)i);
    }
  }
  std::vector<int32_t> pos(c->n_nodes, -1);
  for (int64_t i = 0; i < c->n_nodes; ++i) pos[c->internal_of[i]] = c->rec_col_of[i];
  cudaError_t e = c->upload(&c->d_rec_pos, pos);
  if (e == cudaSuccess) e = c->alloc_zero(&c->d_rec, (size_t)max_rows * c->S * chans.size());
  if (e != cudaSuccess) {
    c->rec_col_of.assign(c->n_nodes, -1);
    return c->cuda_fail(e, "emt_set_recording");
  }
  c->rec_channels = chans;
  c->rec_decim = decim;
  c->rec_rows = max_rows;
  return EMT_OK;
}

// Where a forward launch writes node voltages: rows of rec for steps
// decim, 2 decim, ..., row r (step (r + 1) decim) at rec + (r - row0) * n_rec.
struct RecSpec {
  double* rec = nullptr;
  const int32_t* pos = nullptr;
  int32_t n_rec = 0;
  int32_t decim = 1;
  int64_t rows = 0;
  int64_t row0 = 0;
  int32_t* word_tape = nullptr;   // optional per-step runtime-switch state words, rows from row0
};

// The one multi-scenario launch for steps n0 .. n0 + n_steps - 1.
static cudaError_t batch_launch(emt_ctx* c, int64_t n0, int64_t n_steps, cudaStream_t st, bool record) {
  BatchParams b{};
  b.n_sub = c->n_sub;
  b.S = (int32_t)c->S;
  b.S_t = c->S_t;
  b.n_sources = (int32_t)c->n_sources;
  b.n_groups = (int32_t)c->groups.size();
  b.max_cols = c->max_cols;
  b.max_nodes = c->max_nodes;
  b.grp = c->d_grp;
  b.ginv = c->d_ginv;
  b.ginv_lo = c->d_ginv_lo;
  b.col_code = c->d_col_code;
  b.col_sub = c->d_col_sub;
  b.node_sub = c->d_node_sub;
  b.node_r = c->d_node_r;
  b.sub_nc = c->d_sub_nc;
  b.sub_col_off = c->d_sub_col_off;
  b.ent_ptr = c->d_ent_ptr;
  b.bent = c->d_bent;
  b.lc_nk = c->d_lc_nk;
  b.lc_nm = c->d_lc_nm;
  b.lc_e = c->d_lc_e;
  b.lc_isl = c->d_lc_isl;
  b.sb_g = c->d_sb_g;
  b.sb_src = c->d_sb_src;
  b.le_nd = c->d_le_nd;
  b.le_d1 = c->d_le_d1;
  b.le_y2 = c->d_le_y2;
  b.le_bring = c->d_le_bring;
  b.le_bfar = c->d_le_bfar;
  b.ev_ptr = c->d_ev_ptr;
  b.ev_step = c->d_ev_step;
  b.ev_sub = c->d_ev_sub;
  b.ev_off = c->d_ev_off;
  b.src_ac = c->d_src_ac;
  b.src_as = c->d_src_as;
  b.src_omega = c->d_src_omega;
  b.keep_lc = c->d_keep_lc;
  b.keep_sb = c->d_keep_sb;
  b.keep_le = c->d_keep_le;
  b.h = c->d_bh;
  b.ring = c->d_bring;
  b.cb = c->d_bcb;
  b.cb_lay = c->d_bcb_lay;
  b.cb_list = c->d_bcb_list;
  b.cinj = c->d_bcinj;
  b.cbo = c->d_bcbo;
  b.cy = c->d_bcy;
  b.cs = c->d_bcs;
  b.nl = c->d_nl;
  b.nlinfo = c->d_bnlinfo;
  b.nlc = c->d_bnlc;
  b.nl_i = c->d_bnli;
  b.fd = c->d_fd;
  b.fd_le = c->d_bfd_le;
  b.le_fd = c->d_ble_fd;
  b.fds = c->d_bfds;
  b.rs = c->d_rs;
  b.sub_rs = c->d_bsub_rs;
  b.rs_word = c->d_bword;
  b.rs_prev_i = c->d_brsi;
  b.vbase = c->d_bvbase;
  b.ce = c->d_ce;
  b.ce_le0 = c->d_bce_le0;
  b.ce_node = c->d_bce_node;
  b.le_ce = c->d_ble_ce;
  b.le_f = c->d_ble_f;
  b.cim = c->d_bcim;
  b.cph = c->d_bcph;
  b.rec = record ? c->d_rec : nullptr;
  b.rec_pos = c->d_rec_pos;
  b.rec_rows = c->rec_rows;
  b.rec_decim = c->rec_decim;
  b.n_rec = (int32_t)c->rec_channels.size();
  b.n0 = n0;
  b.n_steps = n_steps;
  b.dt = c->dt;
  b.err = c->d_err;
  b.bnd.ring = std::max<int64_t>(c->bring_len, 1) * c->S;
  b.bnd.h = c->n_lc_total * c->S;
  b.bnd.ginv = c->ginv_len;
  b.bnd.rec = record ? c->rec_rows * c->S * (int64_t)c->rec_channels.size() : 0;
  if (c->use_digit && c->dig_on) {
    b.dig = c->d_dig;
    b.dig_ptr = c->d_dig_ptr;
    b.dig_key = c->d_dig_key;
    b.dig_val = c->d_dig_val;
    b.sub_node0 = c->d_sub_node0;
    b.sub_n = c->d_sub_n;
    b.dig_grp = std::max(c->dig_grp, 1);
    b.dig_min_rows = c->dig_min_rows;
  }
  return launch_batch(b, c->batch_threads, st, c->use_graph ? &c->graph : nullptr);
}

// Single-network forward run of n_steps steps from the context's step.
// A sharded context forgets its last window (after a reset or a loaded state).
static void shard_clear_window(emt_ctx* c) {
  c->shard_to_pack.clear();
  c->shard_to_unpack.clear();
  c->win_n0 = c->win_w = 0;
}

static bool state_space_runs(const emt_ctx* c) {
  return c->ss_ok && !(c->small_ok && c->use_small) &&
         (c->ss_mode == 2 || (c->ss_mode == 1 && c->ss_max_entries <= kSsAutoEntries));
}

static emt_status forward_steps(emt_ctx* c, int64_t n_steps, cudaStream_t st, const RecSpec& rs) {
  const bool small = c->small_ok && c->use_small;
  const bool ssf = state_space_runs(c);
  if (!ssf && (small ? small_smem_bytes(c->lim) : forward_smem_bytes(c->lim)) > 227 * 1024)
    return c->fail(EMT_ERESOURCE, "a subsystem needs more shared memory than one CTA has");
  // source table for one chunk of steps at a time (grow-only buffer)
  const int64_t chunk =
      std::min<int64_t>(n_steps, std::max<int64_t>(1, kSourceTableDoubles / std::max<int64_t>(c->n_sources, 1)));
  if (c->src_table_steps < chunk) {
    cudaStreamSynchronize(st);
    c->release(c->d_src_table);
    c->d_src_table = nullptr;
    c->src_table_steps = 0;
    cudaError_t e = c->alloc_zero(&c->d_src_table, (size_t)chunk * std::max<int64_t>(c->n_sources, 1));
    if (e != cudaSuccess) return c->cuda_fail(e, "emt_step_n source table");
    c->src_table_steps = chunk;
  }
  FwdParams p{};
  p.n_sub = c->n_sub;
  p.lim = c->lim;
  p.lim.n = std::max(p.lim.n, 1);
  p.lim.nc = std::max(p.lim.nc, 1);
  p.sub = c->d_sub;
  p.ep = c->d_ep;
  p.ginv = c->d_ginv;
  p.ginv_lo = c->d_ginv_lo;
  p.br = c->d_br;
  p.lc_idx = c->d_lc_idx;
  p.sb_idx = c->d_sb_idx;
  p.h = c->d_h;
  p.ent = c->d_ent;
  p.il_node = c->d_il_node;
  p.il_cnt = c->d_il_cnt;
  p.str_slot = c->d_str_slot;
  p.le = c->d_le;
  p.ring = c->d_ring;
  p.src_global = c->d_src_global;
  p.src_table = c->d_src_table;
  p.n_sources = (int32_t)c->n_sources;
  p.err = c->d_err;
  p.rec = rs.rec;
  p.rec_pos = rs.pos;
  p.rec_rows = rs.rows;
  p.rec_row0 = rs.row0;
  p.word_tape = rs.word_tape;
  p.word_row0 = rs.row0;
  p.rec_decim = rs.decim;
  p.n_rec = rs.n_rec;
  p.wait_budget_ns = c->wait_budget_ns;
  p.hold_sub = c->hold_sub;
  p.ce = c->d_ce;
  p.le_prev = c->d_le_prev;
  p.rs = c->d_rs;
  p.rs_word = c->d_rs_word;
  p.rs_prev_i = c->d_rs_prev_i;
  p.fd = c->d_fd;
  p.fd_state = c->d_fd_state;
  p.nl = c->d_nl;
  p.nlz = c->d_nlz;
  p.nlz_lo = c->d_nlz_lo;
  p.nl_seg = c->d_nl_seg;
  p.cb = c->d_cb;
  p.clay = c->d_clay;
  p.cinj = c->d_cinj;
  p.cstate = c->d_cstate;
  p.cy = c->d_cy;
  p.bnd.ring = std::max<int64_t>(c->ring_len, 1);
  p.bnd.ginv = c->ginv_len;
  p.bnd.rec = rs.rec ? (rs.rows - rs.row0) * rs.n_rec : 0;
  p.bnd.h = c->n_lc_total;
  p.bnd.src = c->src_table_steps * std::max<int64_t>(c->n_sources, 1);
  p.bnd.nlz = c->nlz_len;
  p.ginv_rw = c->d_ginv;
  p.ginv_lo_rw = c->d_ginv_lo;
  p.nlz_rw = c->d_nlz;
  p.nlz_lo_rw = c->d_nlz_lo;
  p.cache_tag = c->d_cache_tag;
  p.cache_next = c->d_cache_next;
  p.lazy_work = c->d_lazy_work;
  p.sw = c->d_sw;
  p.ss = c->d_ss;
  p.ss_m = c->d_ss_m;
  p.ss_mlo = c->d_ss_mlo;
  p.ss_lnode = c->d_ss_lnode;
  p.ss_lptr = c->d_ss_lptr;
  p.ss_lend = c->d_ss_lend;
  p.ss_rows = c->ss_rows;
  p.ss_cols = c->ss_cols;
  p.ss_ln = c->ss_ln;
  p.bnd.ssm = std::max<int64_t>(c->ss_len, 1);
  if (c->sharded) {
    p.sub = c->d_shard_sub;
    p.active = c->d_shard_active;
    p.n_active = (int32_t)c->shard_active.size();
  }
  for (int64_t done = 0; done < n_steps; done += chunk) {
    const int64_t len = std::min(chunk, n_steps - done);
    SourceParams sp{};
    sp.n_sources = (int32_t)c->n_sources;
    sp.amp = c->d_src_amp;
    sp.phase = c->d_src_phase;
    sp.omega = c->d_src_omega;
    sp.dt = c->dt;
    sp.n0 = c->step + 1;
    sp.n_steps = len;
    sp.table = c->d_src_table;
    cudaError_t e = launch_sources(sp, st);
    if (e != cudaSuccess) return c->cuda_fail(e, "emt_step_n source table");
    p.n0 = c->step + 1;
    p.n_steps = len;
    e = ssf     ? launch_forward_ss(p, c->ss_compact, st)
        : small ? launch_forward_small(p, st)
                : launch_forward(p, st, !c->forward_narrow, c->lazy || c->lim.nl > 1, c->fd_groups);
    if (e == cudaErrorCooperativeLaunchTooLarge)
      return c->fail(EMT_ERESOURCE, "persistent launch of " + std::to_string(c->n_sub) +
                                        " CTAs cannot be co-resident on this device");
    if (e != cudaSuccess) return c->cuda_fail(e, "emt_step_n launch");
    c->step += len;
    c->launches += (c->n_sources > 0 ? 2 : 1);
  }
  return EMT_OK;
}


extern "C" emt_status emt_step_n(emt_ctx* c, int64_t n_steps, void* stream) {
  NvtxRange nvtx_range("emt_step_n");
  if (!c) return EMT_EINVAL;
  if (!c->prefactored) return c->fail(EMT_ESTATE, "emt_prefactor has not run");
  if (n_steps < 0) return c->fail(EMT_EINVAL, "n_steps < 0");
  if (n_steps == 0 || c->n_sub == 0) return EMT_OK;
  if (c->step + n_steps > (int64_t)INT32_MAX - (int64_t)(1 << 21))
    return c->fail(EMT_EINVAL, "step counter would exceed 2^31 - 2^21");
  if (!c->rec_channels.empty() && (c->step + n_steps) / c->rec_decim > c->rec_rows)
    return c->fail(EMT_EINVAL, "recording capacity exceeded: raise max_rows in emt_set_recording");
  if (c->sharded) {
    if (n_steps > c->shard_window)
      return c->fail(EMT_EINVAL, "a shard advances at most " + std::to_string(c->shard_window) +
                                     " steps (its shortest cut line) between exchanges, not " + std::to_string(n_steps));
    if (!c->shard_to_pack.empty())
      return c->fail(EMT_ESTATE, "the last window's line values for rank " + std::to_string(*c->shard_to_pack.begin()) +
                                     " are not packed (emt_shard_pack)");
    if (!c->shard_to_unpack.empty())
      return c->fail(EMT_ESTATE, "the last window's line values from rank " +
                                     std::to_string(*c->shard_to_unpack.begin()) + " are not unpacked (emt_shard_unpack)");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (c->batched) {
    cudaError_t e = batch_launch(c, c->step + 1, n_steps, st, !c->rec_channels.empty());
    if (e != cudaSuccess) return c->cuda_fail(e, "emt_step_n multi-scenario launch");
    c->step += n_steps;
    c->launches += 1;
    return EMT_OK;
  }
  RecSpec rs;
  if (!c->rec_channels.empty()) {
    rs.rec = c->d_rec;
    rs.pos = c->d_rec_pos;
    rs.n_rec = (int32_t)c->rec_channels.size();
    rs.decim = c->rec_decim;
    rs.rows = c->rec_rows;
  }
  const int64_t n0 = c->step + 1;
  const emt_status r = forward_steps(c, n_steps, st, rs);
  if (r == EMT_OK && c->sharded) {   // the window just enqueued: its sent values go out, the peers' come in
    c->win_n0 = n0;
    c->win_w = n_steps;
    for (auto& kv : c->shard_send) c->shard_to_pack.insert(kv.first);
    for (auto& kv : c->shard_recv) c->shard_to_unpack.insert(kv.first);
  }
  return r;
}

extern "C" emt_status emt_sync(emt_ctx* c, int32_t* info) {
  if (!c) return EMT_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_sync");
  int32_t h[4] = {0, 0, 0, 0};
  e = cudaMemcpy(h, c->d_err, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_sync");
  if (info) std::memcpy(info, h, sizeof(h));
  if (h[0] == EMT_ETIMEOUT)
    return c->fail(EMT_ETIMEOUT, "subsystem " + std::to_string(h[1]) + " timed out at step " + std::to_string(h[3]) +
                                     " waiting for the value of its line end " + std::to_string(h[2]));
  if (h[0] == kErrBounds) {
    static const char* kSite[] = {"?", "ring read", "ring write", "solve matrix", "record", "history current",
                                  "source table", "nonlinear column", "adjoint tape", "adjoint target",
                                  "injection entry"};
    const int site = (h[1] >= 1 && h[1] <= 10) ? h[1] : 0;
    return c->fail(EMT_ESTATE, std::string("checks build: ") + kSite[site] + " index " + std::to_string(h[2]) +
                                   " outside its array of " + std::to_string(h[3]));
  }
  if (h[0] == kErrNoSegments)
    return c->fail(EMT_ESTATE, "the nonlinear resistors of subsystem " + std::to_string(h[1]) +
                                   " found no consistent segments at step " + std::to_string(h[3]));
  if (h[0] == kErrTensorWait)
    return c->fail(EMT_ESTATE, std::string("tensor-core solve of subsystem ") + std::to_string(h[1]) + " at step " +
                                   std::to_string(h[3]) + ": the wait for its " +
                                   (h[2] == 0 ? "staged digit planes" : "products") + " ran out of time");
  if (h[0] == EMT_ESINGULAR)
    return c->fail(EMT_ESINGULAR, "conductance matrix of subsystem " + std::to_string(h[1]) + " in switch epoch " +
                                      std::to_string(h[3]) + ", runtime-switch state word " + std::to_string(h[2]) +
                                      " (factorised at run time) is singular");
  if (h[0] != 0) return c->fail((emt_status)h[0], "device error");
  return EMT_OK;
}

// The recorded block itself when the request is every recorded channel in
// recording order over rows whose scenarios lie contiguously in the record
// buffer ([row][scenario][column]); else NULL (a gather is needed).
static const double* contiguous_rows(const emt_ctx* c, const std::vector<int32_t>& col, int64_t row0, int64_t n_rows,
                                     int64_t scen0, int64_t n_scen) {
  const int64_t n_rec = (int64_t)c->rec_channels.size();
  if ((int64_t)col.size() != n_rec) return nullptr;
  for (int64_t i = 0; i < n_rec; ++i)
    if (col[i] != i) return nullptr;
  if (!(scen0 == 0 && n_scen == c->S) && n_rows != 1) return nullptr;
  return c->d_rec + (row0 * c->S + scen0) * n_rec;
}

extern "C" emt_status emt_read_waveforms(emt_ctx* c, const int32_t* channels, int64_t n_ch, int64_t step0,
                                         int64_t n_rows, int64_t scen0, int64_t n_scen, double* out,
                                         int32_t out_on_device) {
  NvtxRange nvtx_range("emt_read_waveforms");
  if (!c) return EMT_EINVAL;
  if (n_ch < 0 || n_rows < 0 || n_scen < 0) return c->fail(EMT_EINVAL, "negative count");
  if (n_ch == 0 || n_rows == 0 || n_scen == 0) return EMT_OK;
  if (!out || !channels) return c->fail(EMT_EINVAL, "NULL buffer");
  if (c->rec_channels.empty()) return c->fail(EMT_ESTATE, "nothing is being recorded");
  if (scen0 < 0 || scen0 + n_scen > c->S) return c->fail(EMT_EINVAL, "scenario range out of bounds");
  if (step0 < c->rec_decim || step0 % c->rec_decim != 0)
    return c->fail(EMT_EINVAL, "step0 must be a positive multiple of the recording decimation");
  const int64_t row0 = step0 / c->rec_decim - 1;
  if (row0 + n_rows > c->rec_rows || (row0 + n_rows) * c->rec_decim > c->step)
    return c->fail(EMT_EINVAL, "requested steps have not been recorded");
  std::vector<int32_t> col(n_ch);
  for (int64_t i = 0; i < n_ch; ++i) {
    const int32_t x = channels[i];
    if (x < 0 || x >= c->n_nodes || c->rec_col_of[x] < 0)
      return c->fail(EMT_EINVAL, "channel " + std::to_string(x) + " is not recorded");
    col[i] = c->rec_col_of[x];
  }
  const emt_status st = emt_sync(c, nullptr);
  if (st != EMT_OK) return st;
  const size_t bytes = (size_t)n_rows * n_scen * n_ch * sizeof(double);
  if (const double* src = contiguous_rows(c, col, row0, n_rows, scen0, n_scen)) {   // one plain copy
    const cudaError_t e = cudaMemcpy(out, src, bytes, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return c->cuda_fail(e, "emt_read_waveforms");
    return EMT_OK;
  }
  int32_t* d_col = nullptr;
  double* d_out = out;
  cudaError_t e = c->upload(&d_col, col);
  if (e == cudaSuccess && !out_on_device) {
    void* p = nullptr;
    e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) c->allocations.push_back(p);
    d_out = static_cast<double*>(p);
  }
  if (e == cudaSuccess)
    e = launch_gather(c->d_rec, (int32_t)c->rec_channels.size(), c->S, d_col, n_ch, row0, n_rows, scen0, n_scen, d_out,
                      nullptr);
  if (e == cudaSuccess && !out_on_device) e = cudaMemcpy(out, d_out, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  c->release(d_col);
  if (!out_on_device) c->release(d_out);
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_read_waveforms");
  return EMT_OK;
}

extern "C" emt_status emt_read_waveforms_async(emt_ctx* c, const int32_t* channels, int64_t n_ch, int64_t step0,
                                               int64_t n_rows, int64_t scen0, int64_t n_scen, double* out,
                                               int32_t out_on_device, void* cuda_stream) {
  NvtxRange nvtx_range("emt_read_waveforms_async");
  if (!c) return EMT_EINVAL;
  if (n_ch < 0 || n_rows < 0 || n_scen < 0) return c->fail(EMT_EINVAL, "negative count");
  if (n_ch == 0 || n_rows == 0 || n_scen == 0) return EMT_OK;
  if (!out || !channels) return c->fail(EMT_EINVAL, "NULL buffer");
  if (c->rec_channels.empty()) return c->fail(EMT_ESTATE, "nothing is being recorded");
  if (scen0 < 0 || scen0 + n_scen > c->S) return c->fail(EMT_EINVAL, "scenario range out of bounds");
  if (step0 < c->rec_decim || step0 % c->rec_decim != 0)
    return c->fail(EMT_EINVAL, "step0 must be a positive multiple of the recording decimation");
  const int64_t row0 = step0 / c->rec_decim - 1;
  if (row0 + n_rows > c->rec_rows || (row0 + n_rows) * c->rec_decim > c->step)
    return c->fail(EMT_EINVAL, "requested steps have not been recorded");
  std::vector<int32_t> col(n_ch);
  for (int64_t i = 0; i < n_ch; ++i) {
    const int32_t x = channels[i];
    if (x < 0 || x >= c->n_nodes || c->rec_col_of[x] < 0)
      return c->fail(EMT_EINVAL, "channel " + std::to_string(x) + " is not recorded");
    col[i] = c->rec_col_of[x];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t bytes = (size_t)n_rows * n_scen * n_ch * sizeof(double);
  if (const double* src = contiguous_rows(c, col, row0, n_rows, scen0, n_scen)) {   // the copy engine alone
    const cudaError_t e =
        cudaMemcpyAsync(out, src, bytes, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return c->cuda_fail(e, "emt_read_waveforms_async");
    return EMT_OK;
  }
  void* d_col = nullptr;
  void* d_tmp = nullptr;
  cudaError_t e = cudaMallocAsync(&d_col, col.size() * sizeof(int32_t), st);
  // from pageable memory the copy is staged before the call returns, so `col` may go
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_col, col.data(), col.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  double* d_out = out;
  if (e == cudaSuccess && !out_on_device) {
    e = cudaMallocAsync(&d_tmp, bytes, st);
    d_out = static_cast<double*>(d_tmp);
  }
  if (e == cudaSuccess)
    e = launch_gather(c->d_rec, (int32_t)c->rec_channels.size(), c->S, static_cast<const int32_t*>(d_col), n_ch,
                      row0, n_rows, scen0, n_scen, d_out, st);
  if (e == cudaSuccess && !out_on_device) e = cudaMemcpyAsync(out, d_out, bytes, cudaMemcpyDeviceToHost, st);
  if (d_tmp) cudaFreeAsync(d_tmp, st);
  if (d_col) cudaFreeAsync(d_col, st);
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_read_waveforms_async");
  return EMT_OK;
}

extern "C" emt_status emt_read_controls(emt_ctx* c, double* y, int64_t n, int32_t on_device) {
  if (!c) return EMT_EINVAL;
  if (c->batched) return c->fail(EMT_EINVAL, "emt_read_controls: a scenario set's block outputs are per scenario");
  if (n != (int64_t)c->cb_slot_of.size())
    return c->fail(EMT_EINVAL, "emt_read_controls: n must equal the number of control blocks");
  if (n == 0) return EMT_OK;
  if (!y) return c->fail(EMT_EINVAL, "NULL buffer");
  const emt_status st = emt_sync(c, nullptr);
  if (st != EMT_OK) return st;
  std::vector<double> dev(c->cblocks.size()), out(n);
  cudaError_t e = cudaMemcpy(dev.data(), c->d_cy, dev.size() * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_read_controls");
  for (int64_t b = 0; b < n; ++b) out[b] = dev[c->subs[c->cb_sub_of[b]].cb_off + c->cb_slot_of[b]];
  if (on_device) {
    e = cudaMemcpy(y, out.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return c->cuda_fail(e, "emt_read_controls");
  } else {
    std::copy(out.begin(), out.end(), y);
  }
  return EMT_OK;
}

extern "C" emt_status emt_reset(emt_ctx* c) {
  if (!c) return EMT_EINVAL;
  shard_clear_window(c);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemset(c->d_h, 0, std::max<int64_t>(c->n_lc_total, 1) * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemset(c->d_ring, 0, 2 * std::max<int64_t>(c->ring_len, 1) * sizeof(unsigned long long));
  if (e == cudaSuccess) e = launch_ring_init(RingInitParams{c->d_le, (int64_t)c->line_ends.size(), c->d_ring}, nullptr);
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, 4 * sizeof(int32_t));
  if (e == cudaSuccess && !c->rs_word0.empty())
    e = cudaMemcpy(c->d_rs_word, c->rs_word0.data(), c->rs_word0.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !c->rswitches.empty())
    e = cudaMemset(c->d_rs_prev_i, 0, c->rswitches.size() * sizeof(double));
  if (e == cudaSuccess && !c->line_ends.empty())
    e = cudaMemset(c->d_le_prev, 0, c->line_ends.size() * sizeof(double));
  if (e == cudaSuccess && !c->fdends.empty())
    e = cudaMemset(c->d_fd_state, 0, kFdState * c->fdends.size() * sizeof(double));
  if (e == cudaSuccess && !c->cblocks.empty()) e = cudaMemset(c->d_cstate, 0, 2 * c->cblocks.size() * sizeof(double));
  if (e == cudaSuccess && !c->cblocks.empty()) e = cudaMemset(c->d_cy, 0, c->cblocks.size() * sizeof(double));
  if (e == cudaSuccess && !c->nls.empty()) {   // every nonlinear resistor on its first positive segment
    const std::vector<int32_t> one(c->nls.size(), 1);
    e = cudaMemcpy(c->d_nl_seg, one.data(), one.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  }
  if (c->batched) {
    if (e == cudaSuccess) e = cudaMemset(c->d_bh, 0, std::max<size_t>((size_t)c->n_lc_total * c->S, 1) * sizeof(double));
    if (e == cudaSuccess)
      e = cudaMemset(c->d_bring, 0, std::max<size_t>((size_t)std::max<int64_t>(c->bring_len, 1) * c->S, 1) * sizeof(double));
    if (e == cudaSuccess && c->d_bcy) e = cudaMemset(c->d_bcy, 0, (2 * c->b_cb.size() + 2) * (size_t)c->S * sizeof(double));
    if (e == cudaSuccess && c->d_bcs) e = cudaMemset(c->d_bcs, 0, 2 * c->b_cb.size() * (size_t)c->S * sizeof(double));
    if (e == cudaSuccess && c->d_bfds)
      e = cudaMemset(c->d_bfds, 0, c->b_fd_le.size() * kBatchFdState * (size_t)c->S * sizeof(double));
    if (e == cudaSuccess && c->d_bcim) e = cudaMemset(c->d_bcim, 0, 3 * c->b_ce_le0.size() * (size_t)c->S * sizeof(double));
    if (e == cudaSuccess && c->d_bword) e = reset_batch_words(c);
    if (e == cudaSuccess && c->d_brsi) e = cudaMemset(c->d_brsi, 0, c->rswitches.size() * (size_t)c->S * sizeof(double));
    if (e == cudaSuccess && c->d_bcph) e = cudaMemset(c->d_bcph, 0, 3 * c->b_ce_le0.size() * (size_t)c->S * sizeof(double));
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_reset");
  c->step = 0;
  return EMT_OK;
}

extern "C" emt_status emt_autotune(emt_ctx* c, int64_t trial_steps, void* stream) {
  NvtxRange nvtx_range("emt_autotune");
  if (!c) return EMT_EINVAL;
  if (trial_steps < 1) return c->fail(EMT_EINVAL, "emt_autotune: trial_steps must be >= 1");
  if (!c->prefactored) return c->fail(EMT_ESTATE, "emt_prefactor has not run");
  if (!c->batched) {   // the single-network kernel's shape is fixed by the partition
    c->tuned = true;
    return EMT_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  // scenarios per CTA: about k CTAs per SM for k = 1..6, and powers of two
  std::set<int> cand;
  for (int k = 1; k <= 6; ++k)
    cand.insert((int)std::min<int64_t>(32, std::max<int64_t>(1, (c->S + (int64_t)n_sm * k - 1) / ((int64_t)n_sm * k))));
  for (int p2 = 1; p2 <= 32; p2 *= 2)
    if (p2 <= c->S) cand.insert(p2);
  const int threads[3] = {256, 512, 1024};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  int best_st = c->S_t, best_th = c->batch_threads;
  bool best_digit = c->use_digit;
  // the solve form: the one set by digit_solve, else both (FP64, and the digit form when a matrix qualifies)
  std::vector<bool> forms{c->use_digit};
  if (c->digit_auto && !c->dig_key.empty()) forms = {false, true};
  for (bool form : forms)
  for (int St : cand) {
    c->use_digit = form;
    if (!batch_configure(c, St, true)) continue;
    for (int th : threads) {
      const bool dg = c->use_digit && c->dig_on;
      if (th > batch_max_threads(dg) || th < batch_min_threads(dg)) continue;
      c->batch_threads = th;
      emt_status rs = emt_reset(c);
      if (rs != EMT_OK) return rs;
      cudaEventRecord(e0, st);
      cudaError_t e = batch_launch(c, 1, trial_steps, st, false);
      cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      c->launches += 1;
      if (ms < best_ms) {
        best_ms = ms;
        best_st = St;
        best_th = th;
        best_digit = form;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->use_digit = best_digit;
  if (!batch_configure(c, best_st, true)) return c->fail(EMT_ERESOURCE, "emt_autotune: no launch shape fits");
  c->batch_threads = best_th;
  c->tuned = true;
  return emt_reset(c);
}

extern "C" emt_status emt_set_option(emt_ctx* c, const char* key, int64_t value) {
  if (!c || !key) return EMT_EINVAL;
  const std::string k(key);
  if (k == "wait_budget_ns") {
    if (value < 0) return c->fail(EMT_EINVAL, "wait_budget_ns must be >= 0");
    c->wait_budget_ns = (unsigned long long)value;
    return EMT_OK;
  }
  if (k == "batch_graph") {   // 0: multi-scenario launches go straight to the stream, not through a graph
    c->use_graph = value != 0;
    return EMT_OK;
  }
  if (k == "scenarios_per_cta" || k == "batch_threads") {
    if (!c->batched) return c->fail(EMT_EINVAL, k + " applies to a context built with a scenario set");
    if (k == "batch_threads") {
      const bool dg = c->use_digit && c->dig_on;
      const int most = batch_max_threads(dg), fewest = batch_min_threads(dg);
      if (value < fewest || value > most || value % 32)
        return c->fail(EMT_EINVAL, "batch_threads must be a multiple of 32 in [" + std::to_string(fewest) + ", " +
                                       std::to_string(most) + "]");
      c->batch_threads = (int)value;
      return EMT_OK;
    }
    if (value < 1 || value > 1024 || !batch_configure(c, (int)value, true))
      return c->fail(EMT_EINVAL, "scenarios_per_cta " + std::to_string(value) + " does not fit in shared memory");
    return EMT_OK;
  }
  if (k == "warp_per_subsystem") {   // 1: networks of small subsystems run one warp per subsystem (emt_small.cu)
    if (value != 0 && !c->small_ok)
      return c->fail(EMT_EINVAL, "this network does not fit the warp-per-subsystem kernel (subsystems of at most " +
                                     std::to_string(kSmallMaxNodes) + " nodes with basic elements only)");
    cudaDeviceSynchronize();
    c->use_small = value != 0;
    return EMT_OK;
  }
  if (k == "digit_solve") {   // 1: the multi-scenario solve of shared matrices on the tensor cores (digit form)
    if (!c->batched) return c->fail(EMT_EINVAL, "digit_solve applies to a context built with a scenario set");
    cudaDeviceSynchronize();
    c->use_digit = value != 0;
    c->digit_auto = false;   // (the autotuner keeps the form set here)
    if (c->use_digit)
      c->batch_threads = std::max(std::min(c->batch_threads, batch_max_threads(true)), batch_min_threads(true));
    if (!batch_configure(c, c->S_t, true)) {
      c->use_digit = false;
      batch_configure(c, c->S_t, true);
      return c->fail(EMT_EINVAL, "digit_solve: scenarios_per_cta " + std::to_string(c->S_t) +
                                     " is above 32, or the digit planes and table do not fit in shared memory "
                                     "beside it");
    }
    c->tuned = false;
    return EMT_OK;
  }
  if (k == "digit_min_rows") {   // the digit form takes subsystems of at least this many rows (default 24)
    if (value < 1 || value > kDigRows)
      return c->fail(EMT_EINVAL, "digit_min_rows must be in [1, " + std::to_string(kDigRows) + "]");
    c->dig_min_rows = (int)value;
    c->tuned = false;
    return EMT_OK;
  }
  if (k == "state_space") {   // 0 off, 1 auto (default), 2 on: the state-space form (emt_ss.cu)
    if (value < 0 || value > 2) return c->fail(EMT_EINVAL, "state_space is 0, 1 or 2");
    if (value == 2 && !c->ss_ok)
      return c->fail(EMT_EINVAL, "this network does not fit the state-space form (subsystems of basic elements "
                                 "whose M has at most " + std::to_string(kSsThreads - 32) + " rows)");
    cudaDeviceSynchronize();
    c->ss_mode = (int)value;
    return EMT_OK;
  }
  if (k == "adjoint_overlap") {   // 0: the adjoint re-runs segments on the caller's stream only
    c->overlap_adjoint = value != 0;
    return EMT_OK;
  }
  if (k == "debug_hold_lines") {   // failure-path tests: one subsystem never sends line values
    if (value < -1 || value >= c->n_sub) return c->fail(EMT_EINVAL, "debug_hold_lines out of range");
    c->hold_sub = (int32_t)value;
    return EMT_OK;
  }
  return c->fail(EMT_EINVAL, "unknown option '" + k + "'");
}

extern "C" emt_status emt_get_info(const emt_ctx* c, const char* key, int64_t* value) {
  if (!c || !key || !value) return EMT_EINVAL;
  const std::string k(key);
  if (k == "n_subsystems" || k == "n_ctas") *value = c->n_sub;
  else if (k == "step") *value = c->step;
  else if (k == "max_subsystem_nodes") *value = c->lim.n;
  else if (k == "n_scenarios") *value = c->S;
  else if (k == "n_matrix_variants") *value = c->batched ? (int64_t)c->var_sub.size() : (int64_t)c->epochs.size();
  else if (k == "scenarios_per_cta") *value = c->batched ? c->S_t : 1;
  else if (k == "batch_threads") *value = c->batched ? c->batch_threads : 0;
  else if (k == "batch_groups") *value = c->batched ? (int64_t)c->groups.size() : 0;
  else if (k == "graph_launches") *value = c->graph.launches;
  else if (k == "autotuned") *value = c->tuned ? 1 : 0;
  else if (k == "n_epochs_total") *value = (int64_t)c->epochs.size();
  else if (k == "n_components") *value = c->n_components;
  else if (k == "cta_max_line_ends") *value = c->lim.le;
  else if (k == "cta_max_lc_branches") *value = c->lim.lc;
  else if (k == "cta_max_control_blocks") *value = c->lim.cb;
  else if (k == "cta_max_lanes") *value = c->lim.il;
  else if (k == "cta_max_columns") *value = c->lim.nc;
  else if (k == "sum_n2_components") *value = c->comp_sum_n2;
  else if (k == "max_component_nodes") *value = c->comp_max_n;
  else if (k == "sum_n2") {
    int64_t s2 = 0;
    for (const SubDev& s : c->subs) s2 += (int64_t)s.n * s.n;
    *value = s2;
  } else if (k == "threads_per_cta") *value = kFwdThreads;
  else if (k == "kernel_launches") *value = c->launches;
  else if (k == "n_branches") *value = (int64_t)c->branches.size();
  else if (k == "n_sources") *value = c->n_sources;
  else if (k == "n_nodes") *value = c->n_nodes;
  else if (k == "n_line_ends") *value = (int64_t)c->line_ends.size();
  else if (k == "n_strong_branches") *value = (int64_t)c->str_slot.size();
  else if (k == "n_runtime_switches") *value = (int64_t)c->rswitches.size();
  else if (k == "n_coupled_lines") *value = (int64_t)c->cends.size() / 2;
  else if (k == "n_fd_lines") *value = (int64_t)c->fdends.size() / 2;
  else if (k == "n_nonlinear") *value = (int64_t)c->nls.size();
  else if (k == "n_control_blocks") *value = (int64_t)c->cblocks.size();
  else if (k == "n_control_injections") *value = (int64_t)c->cinj.size();
  else if (k == "max_control_layers") *value = c->max_clayers;
  else if (k == "smem_bytes") *value = (int64_t)forward_smem_bytes(c->lim);
  else if (k == "shard_rank") *value = c->sharded ? c->shard_rank : -1;
  else if (k == "shard_window") *value = c->sharded ? c->shard_window : 0;
  else if (k == "shard_ctas") *value = c->sharded ? (int64_t)c->shard_active.size() : c->n_sub;
  else if (k == "state_space") *value = state_space_runs(c) ? 1 : 0;
  else if (k == "digit_solve") *value = c->batched && c->use_digit && c->dig_on ? 1 : 0;
  else if (k == "digit_matrices") *value = (int64_t)c->dig_key.size();
  else if (k == "digit_min_rows") *value = c->dig_min_rows;
  else if (k == "warp_per_subsystem") *value = c->small_ok && c->use_small ? 1 : 0;
  else if (k == "lazy_subsystems") {   // subsystems whose switch states are factorised at run time
    int64_t m = 0;
    for (const SubDev& sd : c->subs) m += sd.n_cache > 0 ? 1 : 0;
    *value = m;
  } else if (k == "runtime_factorisations") {   // switch states factorised by the kernel since the prefactor
    int32_t v = 0;
    cudaDeviceSynchronize();
    if (c->lazy && cudaMemcpy(&v, c->d_cache_next + c->n_sub, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return EMT_ECUDA;
    *value = v;
  } else if (k == "factorised_states") {   // solve matrices held by their caches (synchronises the device)
    std::vector<long long> tag(c->cache_tag0.size());
    cudaDeviceSynchronize();
    if (!tag.empty() &&
        cudaMemcpy(tag.data(), c->d_cache_tag, tag.size() * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess)
      return EMT_ECUDA;
    int64_t m = 0;
    for (long long t : tag) m += t >= 0 ? 1 : 0;
    *value = m;
  }
  else if (k == "ctas_per_sm") {   // co-resident persistent CTAs per SM (occupancy of the single-network kernel)
    FwdLimits fl = c->lim;
    fl.n = std::max(fl.n, 1);
    fl.nc = std::max(fl.nc, 1);
    *value = forward_blocks_per_sm(fl);
  }
  else return EMT_EINVAL;
  return EMT_OK;
}

extern "C" emt_status emt_get_node_order(const emt_ctx* c, int32_t* perm) {
  if (!c || !perm) return EMT_EINVAL;
  for (int64_t i = 0; i < c->n_nodes; ++i) perm[i] = c->original_of[i];
  return EMT_OK;
}

// ---------------------------------------------------------------- shards
//
// Subsystems meet only through line rings, and a value sent at step n is
// consumed at step n + d (Sec. II-B: the line's travel time decouples its
// two ends).  A shard runs the CTAs one rank owns; with every cut line end
// at least D steps long, a window of W <= D steps reads only values sent
// before the window began, so each rank runs its window alone and the
// ranks swap, between windows, the slots the window wrote for the other
// side.

static std::vector<int32_t> far_ends(const emt_ctx* c) {
  std::map<int64_t, int32_t> by_own;
  for (size_t e = 0; e < c->line_ends.size(); ++e) by_own[c->line_ends[e].own_ring] = (int32_t)e;
  std::vector<int32_t> far(c->line_ends.size(), -1);
  for (size_t e = 0; e < c->line_ends.size(); ++e) {
    auto it = by_own.find(c->line_ends[e].far_ring);
    if (it != by_own.end()) far[e] = it->second;
  }
  return far;
}

static std::vector<int32_t> cta_of_line_end(const emt_ctx* c) {
  std::vector<int32_t> cta(c->line_ends.size(), -1);
  for (int s = 0; s < c->n_sub; ++s)
    for (int x = 0; x < c->subs[s].n_le; ++x) cta[c->subs[s].le_off + x] = s;
  return cta;
}

extern "C" emt_status emt_get_node_ctas(const emt_ctx* c, int32_t* cta) {
  if (!c || !cta) return EMT_EINVAL;
  if (c->batched) return const_cast<emt_ctx*>(c)->fail(EMT_EINVAL, "emt_get_node_ctas: a scenario set's CTAs hold scenarios, not subsystems");
  for (int64_t i = 0; i < c->n_nodes; ++i) cta[i] = c->sub_of_node[i];
  return EMT_OK;
}

extern "C" emt_status emt_get_line_ends(const emt_ctx* c, int32_t* cta, int32_t* far_end, int32_t* d) {
  if (!c) return EMT_EINVAL;
  if (c->batched) return const_cast<emt_ctx*>(c)->fail(EMT_EINVAL, "emt_get_line_ends: not for a context built with a scenario set");
  const std::vector<int32_t> own = cta_of_line_end(c), far = far_ends(c);
  for (size_t e = 0; e < c->line_ends.size(); ++e) {
    if (cta) cta[e] = own[e];
    if (far_end) far_end[e] = far[e];
    if (d) d[e] = c->line_ends[e].d;
  }
  return EMT_OK;
}

extern "C" emt_status emt_set_shard(emt_ctx* c, const int32_t* owner, int32_t rank) {
  if (!c) return EMT_EINVAL;
  if (c->batched) return c->fail(EMT_EINVAL, "emt_set_shard: a context built with a scenario set is not sharded");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_set_shard");
  c->release(c->d_shard_active);
  c->release(c->d_shard_ends);
  c->release(c->d_shard_sub);
  c->d_shard_active = c->d_shard_ends = nullptr;
  c->d_shard_sub = nullptr;
  c->sharded = false;
  c->shard_rank = -1;
  c->shard_window = 0;
  c->shard_active.clear();
  c->shard_send.clear();
  c->shard_recv.clear();
  c->shard_send_off.clear();
  c->shard_recv_off.clear();
  shard_clear_window(c);
  if (owner == nullptr) return EMT_OK;   // the whole network again
  if (rank < 0) return c->fail(EMT_EINVAL, "emt_set_shard: rank < 0");
  for (int s = 0; s < c->n_sub; ++s) {
    if (owner[s] < 0) return c->fail(EMT_EINVAL, "emt_set_shard: CTA " + std::to_string(s) + " has a negative owner");
    if (owner[s] == rank) c->shard_active.push_back(s);
  }
  if (c->shard_active.empty()) return c->fail(EMT_EINVAL, "emt_set_shard: rank " + std::to_string(rank) + " owns no CTA");
  const std::vector<int32_t> own = cta_of_line_end(c), far = far_ends(c);
  int64_t window = INT32_MAX;
  for (size_t x = 0; x < c->line_ends.size(); ++x) {
    if (far[x] < 0) return c->fail(EMT_ESTATE, "emt_set_shard: line end without a far end");
    const int32_t a = owner[own[x]], b = owner[own[far[x]]];
    if (a == b) continue;
    window = std::min<int64_t>(window, c->line_ends[x].d);
    if (a == rank) c->shard_send[b].push_back((int32_t)x);   // sent here, consumed at rank b
    if (b == rank) c->shard_recv[a].push_back((int32_t)x);   // sent at rank a, consumed here
  }
  std::vector<int32_t> all;
  for (auto& kv : c->shard_send) {
    c->shard_send_off[kv.first] = (int64_t)all.size();
    all.insert(all.end(), kv.second.begin(), kv.second.end());
  }
  for (auto& kv : c->shard_recv) {
    c->shard_recv_off[kv.first] = (int64_t)all.size();
    all.insert(all.end(), kv.second.begin(), kv.second.end());
  }
  std::vector<SubDev> ssub;
  for (int32_t s : c->shard_active) ssub.push_back(c->subs[s]);
  e = c->upload(&c->d_shard_active, c->shard_active);
  if (e == cudaSuccess) e = c->upload(&c->d_shard_sub, ssub);
  if (e == cudaSuccess) e = c->upload(&c->d_shard_ends, all);
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_set_shard");
  c->sharded = true;
  c->shard_rank = rank;
  c->shard_window = (int32_t)window;
  return EMT_OK;
}

static emt_status shard_copy(emt_ctx* c, int32_t peer, void* buf, int64_t bytes, void* stream, bool pack) {
  const char* fn = pack ? "emt_shard_pack" : "emt_shard_unpack";
  if (!c->sharded) return c->fail(EMT_ESTATE, std::string(fn) + ": the context is not a shard (emt_set_shard)");
  const auto& lists = pack ? c->shard_send : c->shard_recv;
  auto it = lists.find(peer);
  const int64_t n_ends = it == lists.end() ? 0 : (int64_t)it->second.size();
  const int64_t need = n_ends * c->win_w * 16;
  if (buf == nullptr && pack) return EMT_OK;   // size query only (the caller read *bytes)
  if (bytes != need)
    return c->fail(EMT_EINVAL, std::string(fn) + ": the window's buffer for rank " + std::to_string(peer) + " holds " +
                                   std::to_string(need) + " bytes, not " + std::to_string(bytes));
  if (need > 0) {
    if ((reinterpret_cast<uintptr_t>(buf) & 15u) != 0)
      return c->fail(EMT_EINVAL, std::string(fn) + ": buffer not 16-byte aligned");
    RingCopyParams p{};
    p.le = c->d_le;
    p.ends = c->d_shard_ends + (pack ? c->shard_send_off[peer] : c->shard_recv_off[peer]);
    p.n_ends = (int32_t)n_ends;
    p.w = (int32_t)c->win_w;
    p.n0 = c->win_n0;
    p.ring = c->d_ring;
    p.buf = static_cast<unsigned long long*>(buf);
    p.pack = pack ? 1 : 0;
    cudaError_t e = launch_ring_copy(p, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return c->cuda_fail(e, fn);
    c->launches += 1;
  }
  (pack ? c->shard_to_pack : c->shard_to_unpack).erase(peer);
  return EMT_OK;
}

extern "C" emt_status emt_shard_pack(emt_ctx* c, int32_t peer, void* buf, int64_t cap, int64_t* bytes, void* stream) {
  if (!c) return EMT_EINVAL;
  if (!c->sharded) return c->fail(EMT_ESTATE, "emt_shard_pack: the context is not a shard (emt_set_shard)");
  auto it = c->shard_send.find(peer);
  const int64_t need = (it == c->shard_send.end() ? 0 : (int64_t)it->second.size()) * c->win_w * 16;
  if (bytes) *bytes = need;
  if (buf == nullptr) return EMT_OK;
  if (cap < need) return c->fail(EMT_EINVAL, "emt_shard_pack: buffer of " + std::to_string(cap) + " bytes, " +
                                                 std::to_string(need) + " needed");
  return shard_copy(c, peer, buf, need, stream, true);
}

extern "C" emt_status emt_shard_unpack(emt_ctx* c, int32_t peer, const void* buf, int64_t bytes, void* stream) {
  if (!c) return EMT_EINVAL;
  return shard_copy(c, peer, const_cast<void*>(buf), bytes, stream, false);
}

extern "C" emt_status emt_phase_clocks(emt_ctx* c, uint64_t* out, int32_t reset) {
  if (!c) return EMT_EINVAL;
  if (c->n_sub > kPhaseCtas)
    return c->fail(EMT_EINVAL, "emt_phase_clocks: more than " + std::to_string(kPhaseCtas) + " CTAs");
  cudaError_t e = state_space_runs(c) ? ss_phase_clocks(reinterpret_cast<unsigned long long*>(out), c->n_sub, reset != 0)
                                      : phase_clocks(reinterpret_cast<unsigned long long*>(out), c->n_sub, reset != 0);
  if (e == cudaErrorNotSupported) return c->fail(EMT_EINVAL, "emt_phase_clocks: not the phase-clock build");
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_phase_clocks");
  return EMT_OK;
}

extern "C" const char* emt_last_error(const emt_ctx* c) { return c ? c->err.c_str() : g_build_error.c_str(); }

extern "C" void emt_destroy(emt_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  batch_graph_destroy(&c->graph);
  for (void* p : c->allocations) cudaFree(p);
  c->allocations.clear();
  delete c;
}

// ---------------------------------------------------------------- save / load state
//
// The run state of a context -- everything a launch carries to the next:
// history currents, line rings, the values consumed at the last step,
// runtime-switch words and breaker currents, frequency-dependent line and
// control-block states, nonlinear segments (per scenario in a scenario set)
// -- and the step counter, as a header followed by the arrays in a fixed
// order.  Solve matrices are not part of it: a context built from the same
// description and prefactored has the same ones.

namespace {

constexpr uint32_t kStateMagic = 0x53544d45u;   // "EMTS"
constexpr uint32_t kStateVersion = 1;

struct StateHeader {
  uint32_t magic, version;
  int64_t n_nodes, n_sub, S, step, n_arrays, shape;
};

// (device pointer, bytes) of every state array, in the serialised order
std::vector<std::pair<void*, size_t>> state_arrays(emt_ctx* c) {
  std::vector<std::pair<void*, size_t>> a;
  auto add = [&](void* p, size_t bytes) { a.push_back({bytes ? p : nullptr, p ? bytes : 0}); };
  if (!c->batched) {
    add(c->d_h, (size_t)c->n_lc_total * sizeof(double));
    add(c->d_ring, 2 * (size_t)std::max<int64_t>(c->ring_len, 1) * sizeof(unsigned long long));
    add(c->d_le_prev, c->line_ends.size() * sizeof(double));
    add(c->d_rs_word, c->rs_word0.size() * sizeof(int32_t));
    add(c->d_rs_prev_i, c->rswitches.size() * sizeof(double));
    add(c->d_fd_state, kFdState * c->fdends.size() * sizeof(double));
    add(c->d_cstate, 2 * c->cblocks.size() * sizeof(double));
    add(c->d_cy, c->cblocks.size() * sizeof(double));
    add(c->d_nl_seg, c->nls.size() * sizeof(int32_t));
  } else {
    const size_t S = (size_t)c->S;
    add(c->d_bh, (size_t)c->n_lc_total * S * sizeof(double));
    add(c->d_bring, (size_t)std::max<int64_t>(c->bring_len, 1) * S * sizeof(double));
    add(c->d_bcy, c->d_bcy ? (2 * c->b_cb.size() + 2) * S * sizeof(double) : 0);
    add(c->d_bcs, c->d_bcs ? 2 * c->b_cb.size() * S * sizeof(double) : 0);
    add(c->d_bfds, c->d_bfds ? c->b_fd_le.size() * kBatchFdState * S * sizeof(double) : 0);
    add(c->d_bcim, c->d_bcim ? 3 * c->b_ce_le0.size() * S * sizeof(double) : 0);
    add(c->d_bcph, c->d_bcph ? 3 * c->b_ce_le0.size() * S * sizeof(double) : 0);
    add(c->d_bword, c->d_bword ? (size_t)c->n_sub * S * sizeof(int32_t) : 0);
    add(c->d_brsi, c->d_brsi ? c->rswitches.size() * S * sizeof(double) : 0);
    add(c->d_bvbase, c->d_bvbase ? (size_t)c->n_sub * S * sizeof(long long) : 0);
    add(c->d_bnli, c->d_bnli ? c->nls.size() * S * sizeof(double) : 0);
  }
  return a;
}

// FNV-1a over the context's shape (counts and array sizes), so that a state
// only loads into a context of the same network
int64_t state_shape(emt_ctx* c, const std::vector<std::pair<void*, size_t>>& a) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t x) {
    for (int i = 0; i < 8; ++i) {
      h ^= (x >> (8 * i)) & 0xffu;
      h *= 1099511628211ull;
    }
  };
  mix((uint64_t)c->n_nodes);
  mix((uint64_t)c->n_branches);
  mix((uint64_t)c->n_lines);
  mix((uint64_t)c->n_sources);
  mix((uint64_t)c->n_sub);
  mix((uint64_t)c->S);
  mix(c->batched ? 1u : 0u);
  for (const auto& x : a) mix((uint64_t)x.second);
  return (int64_t)(h >> 1);
}

}  // namespace

extern "C" emt_status emt_save_state(emt_ctx* c, void* buf, int64_t cap, int64_t* size) {
  if (!c || !size) return c ? c->fail(EMT_EINVAL, "emt_save_state: size is NULL") : EMT_EINVAL;
  const auto arrays = state_arrays(c);
  int64_t need = (int64_t)sizeof(StateHeader);
  for (const auto& x : arrays) need += (int64_t)(sizeof(uint64_t) + x.second);
  *size = need;
  if (!buf) return EMT_OK;   // a size query
  if (cap < need) return c->fail(EMT_EINVAL, "emt_save_state: buffer of " + std::to_string(cap) + " bytes, " +
                                                 std::to_string(need) + " needed");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_save_state");
  unsigned char* out = static_cast<unsigned char*>(buf);
  StateHeader hd{kStateMagic, kStateVersion, c->n_nodes, c->n_sub, c->S, c->step, (int64_t)arrays.size(),
                 state_shape(c, arrays)};
  std::memcpy(out, &hd, sizeof(hd));
  size_t off = sizeof(hd);
  for (const auto& x : arrays) {
    const uint64_t bytes = x.second;
    std::memcpy(out + off, &bytes, sizeof(bytes));
    off += sizeof(bytes);
    if (bytes) {
      e = cudaMemcpy(out + off, x.first, bytes, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return c->cuda_fail(e, "emt_save_state");
    }
    off += bytes;
  }
  return EMT_OK;
}

extern "C" emt_status emt_load_state(emt_ctx* c, const void* buf, int64_t size) {
  if (!c) return EMT_EINVAL;
  if (!buf || size < (int64_t)sizeof(StateHeader)) return c->fail(EMT_EINVAL, "emt_load_state: no state in the buffer");
  const auto arrays = state_arrays(c);
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != kStateMagic || hd.version != kStateVersion)
    return c->fail(EMT_EINVAL, "emt_load_state: not a state written by emt_save_state (or another version)");
  if (hd.n_nodes != c->n_nodes || hd.n_sub != c->n_sub || hd.S != c->S || hd.n_arrays != (int64_t)arrays.size() ||
      hd.shape != state_shape(c, arrays))
    return c->fail(EMT_EINVAL, "emt_load_state: the state belongs to a context of another network");
  if (!c->prefactored) return c->fail(EMT_ESTATE, "emt_prefactor has not run");
  if (hd.step < 0 || hd.step > (int64_t)INT32_MAX - (int64_t)(1 << 21))
    return c->fail(EMT_EINVAL, "emt_load_state: step counter out of range");
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  size_t off = sizeof(hd);
  cudaError_t e = cudaDeviceSynchronize();
  for (const auto& x : arrays) {
    uint64_t bytes = 0;
    if (off + sizeof(bytes) > (size_t)size) return c->fail(EMT_EINVAL, "emt_load_state: truncated state");
    std::memcpy(&bytes, in + off, sizeof(bytes));
    off += sizeof(bytes);
    if (bytes != x.second || off + bytes > (size_t)size) return c->fail(EMT_EINVAL, "emt_load_state: truncated state");
    if (e == cudaSuccess && bytes) e = cudaMemcpy(x.first, in + off, bytes, cudaMemcpyHostToDevice);
    off += bytes;
  }
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, 4 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_load_state");
  c->step = hd.step;
  shard_clear_window(c);
  return EMT_OK;
}

// ---------------------------------------------------------------- adjoint
//
// Forward pass from the de-energised state, saving (h, line rings) before
// every segment of K steps but the last; the last segment records its tape
// v_n directly.  Reverse pass, segments last to first: restore the
// segment's checkpoint, run it forward again recording the tape, then run
// the reverse kernel over it.  K = 0 keeps the whole tape (one segment).
static emt_status adjoint_run(emt_ctx* c, const double* v_target, int64_t n_steps, int32_t ckpt_every,
                              double* grad, double* loss, int32_t on_device, void* stream);

extern "C" emt_status emt_adjoint(emt_ctx* c, const double* v_target, int64_t n_steps, int32_t ckpt_every,
                                  double* grad, double* loss, int32_t on_device, void* stream) {
  NvtxRange nvtx_range("emt_adjoint");
  if (!c) return EMT_EINVAL;
  c->forward_narrow = true;   // the re-runs may share the device with the reverse sweep
  const emt_status st = adjoint_run(c, v_target, n_steps, ckpt_every, grad, loss, on_device, stream);
  c->forward_narrow = false;
  return st;
}

static emt_status adjoint_run(emt_ctx* c, const double* v_target, int64_t n_steps, int32_t ckpt_every,
                              double* grad, double* loss, int32_t on_device, void* stream) {
  if (c->batched) return c->fail(EMT_EINVAL, "emt_adjoint: a context built with a scenario set has no adjoint");
  if (c->sharded) return c->fail(EMT_EINVAL, "emt_adjoint: runs the whole network; clear the shard (emt_set_shard NULL)");
  if (!c->cblocks.empty()) return c->fail(EMT_EINVAL, "emt_adjoint: control blocks have no adjoint");
  if (!c->fdends.empty()) return c->fail(EMT_EINVAL, "emt_adjoint: frequency-dependent lines have no adjoint");
  if (!c->nls.empty()) return c->fail(EMT_EINVAL, "emt_adjoint: nonlinear resistors have no adjoint");
  if (c->lazy)
    return c->fail(EMT_EINVAL, "emt_adjoint: a subsystem with more than " + std::to_string(kMaxRuntimeSwitches) +
                                   " runtime switches (states factorised at run time) has no adjoint");
  if (!c->prefactored) return c->fail(EMT_ESTATE, "emt_prefactor has not run");
  if (n_steps < 1) return c->fail(EMT_EINVAL, "emt_adjoint: n_steps must be >= 1");
  if (n_steps > (int64_t)INT32_MAX - (int64_t)(1 << 21))
    return c->fail(EMT_EINVAL, "emt_adjoint: n_steps exceeds 2^31 - 2^21");
  if (ckpt_every < 0) return c->fail(EMT_EINVAL, "emt_adjoint: ckpt_every must be >= 0");
  if (!v_target) return c->fail(EMT_EINVAL, "emt_adjoint: v_target is NULL");
  if (!grad && !loss) return c->fail(EMT_EINVAL, "emt_adjoint: grad and loss are both NULL");
  AdjLimits al{};
  al.n = std::max(c->lim.n, 1);
  al.nc = std::max(c->lim.nc, 1);
  al.q = c->lim.q;
  for (const SubDev& sd : c->subs) al.br = std::max(al.br, sd.n_br);
  al.lc = c->lim.lc;
  al.sb = c->lim.sb;
  al.le = c->lim.le;
  al.src = c->lim.src;
  al.il = c->lim.il;
  al.ce = c->lim.ce;
  if (adjoint_smem_bytes(al) > 227 * 1024)
    return c->fail(EMT_ERESOURCE, "emt_adjoint: a subsystem needs more shared memory than one CTA has");
  emt_status rs0 = emt_reset(c);
  if (rs0 != EMT_OK) return rs0;
  if (c->n_sub == 0) {
    if (grad) {
      if (on_device) cudaMemset(grad, 0, (size_t)(c->n_branches + c->n_sources) * sizeof(double));
      else std::fill(grad, grad + c->n_branches + c->n_sources, 0.0);
    }
    if (loss) *loss = 0.0;
    return EMT_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t N = n_steps, nn = c->n_nodes, ns = c->n_sources, nbr = (int64_t)c->branches.size();
  const int64_t K = ckpt_every > 0 ? std::min<int64_t>(ckpt_every, N) : N;
  const int64_t n_seg = (N + K - 1) / K;
  const int64_t n_lc = std::max<int64_t>(c->n_lc_total, 1);
  const int64_t ring_words = 2 * std::max<int64_t>(c->ring_len, 1);
  const int T = adjoint_threads();

  // The forward re-run of segment j-1 overlaps the reverse sweep of
  // segment j (second stream, two tapes) when both persistent grids fit on
  // the device together: every SM holds at least min(per-SM residency) CTAs
  // of either kernel, so 2 n_sub <= n_SM * that is enough.
  bool overlap = false;
  if (K < N) {
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    FwdLimits fl = c->lim;
    fl.n = std::max(fl.n, 1);
    fl.nc = std::max(fl.nc, 1);
    const int m = std::min(forward_blocks_per_sm(fl), adjoint_blocks_per_sm(al));
    overlap = m > 0 && 2 * (int64_t)c->n_sub <= (int64_t)n_sm * m && c->overlap_adjoint;
  }
  std::vector<void*> mine;   // this call's buffers, released before returning
  const double* d_tgt = v_target;
  double *d_tgt_copy = nullptr, *d_sin = nullptr, *d_ones = nullptr, *d_ck_h = nullptr, *d_tape = nullptr;
  double *d_hbar = nullptr, *d_dg = nullptr, *d_dsrc = nullptr, *d_lp = nullptr, *d_grad = grad, *d_loss = nullptr;
  unsigned long long *d_ck_ring = nullptr, *d_aring = nullptr;
  int32_t* d_pos = nullptr;
  int32_t *d_wtape = nullptr, *d_ck_word = nullptr;   // runtime switches: per-step state words, checkpoints
  double* d_ck_rsi = nullptr;
  double *d_adj_lep = nullptr, *d_ck_lep = nullptr;    // line ends: adjoint carry; forward carry checkpoints
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    e = c->alloc_zero(&d_tgt_copy, (size_t)(N * nn));
    if (e == cudaSuccess) {
      mine.push_back(d_tgt_copy);
      e = cudaMemcpyAsync(d_tgt_copy, v_target, (size_t)(N * nn) * sizeof(double), cudaMemcpyHostToDevice, st);
    }
    d_tgt = d_tgt_copy;
  }
#define ADJ_ALLOC(ptr, count) \
  if (e == cudaSuccess) {     \
    e = c->alloc_zero(&ptr, (size_t)(count)); \
    if (e == cudaSuccess) mine.push_back(ptr); \
  }
  ADJ_ALLOC(d_sin, std::max<int64_t>(N * ns, 1))
  ADJ_ALLOC(d_ones, std::max<int64_t>(ns, 1))
  ADJ_ALLOC(d_ck_h, std::max<int64_t>((n_seg - 1) * n_lc, 1))
  ADJ_ALLOC(d_ck_ring, std::max<int64_t>((n_seg - 1) * ring_words, 1))
  ADJ_ALLOC(d_tape, (overlap ? 2 : 1) * K * nn)
  const bool rsw = !c->rswitches.empty();
  const int64_t n_rsw = (int64_t)c->rswitches.size();
  const bool cpl = !c->cends.empty();
  const int64_t n_lend = std::max<int64_t>((int64_t)c->line_ends.size(), 1);
  ADJ_ALLOC(d_adj_lep, n_lend)
  if (cpl) ADJ_ALLOC(d_ck_lep, std::max<int64_t>((n_seg - 1) * n_lend, 1))
  if (rsw) {
    ADJ_ALLOC(d_wtape, (overlap ? 2 : 1) * K * c->n_sub)
    ADJ_ALLOC(d_ck_word, std::max<int64_t>((n_seg - 1) * c->n_sub, 1))
    ADJ_ALLOC(d_ck_rsi, std::max<int64_t>((n_seg - 1) * n_rsw, 1))
  }
  ADJ_ALLOC(d_aring, ring_words)
  ADJ_ALLOC(d_hbar, n_lc)
  ADJ_ALLOC(d_dg, std::max<int64_t>(nbr, 1))
  ADJ_ALLOC(d_dsrc, std::max<int64_t>(nbr, 1))
  ADJ_ALLOC(d_lp, (int64_t)c->n_sub * T)
  ADJ_ALLOC(d_loss, 1)
  if (!on_device || !grad) ADJ_ALLOC(d_grad, nbr + ns)
#undef ADJ_ALLOC
  if (e == cudaSuccess) {
    std::vector<int32_t> pos(nn);
    std::iota(pos.begin(), pos.end(), 0);
    e = c->upload(&d_pos, pos);
    if (e == cudaSuccess) mine.push_back(d_pos);
  }
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    for (void* p : mine) c->release(p);
  };
  if (e != cudaSuccess) {
    cleanup();
    return c->cuda_fail(e, "emt_adjoint allocation");
  }
  // sin(omega t_n + phase) for n = 1..N: the source table with unit amplitudes
  if (ns > 0) {
    std::vector<double> ones(ns, 1.0);
    e = cudaMemcpyAsync(d_ones, ones.data(), ns * sizeof(double), cudaMemcpyHostToDevice, st);
    SourceParams sp{};
    sp.n_sources = (int32_t)ns;
    sp.amp = d_ones;
    sp.phase = c->d_src_phase;
    sp.omega = c->d_src_omega;
    sp.dt = c->dt;
    sp.n0 = 1;
    sp.n_steps = N;
    sp.table = d_sin;
    if (e == cudaSuccess) e = launch_sources(sp, st);
    if (e == cudaSuccess) cudaStreamSynchronize(st);   // ones[] leaves scope
    c->launches += 1;
  }
  if (e != cudaSuccess) {
    cleanup();
    return c->cuda_fail(e, "emt_adjoint sin table");
  }
  auto tape_of = [&](int64_t j) { return d_tape + (overlap ? (j & 1) : 0) * K * nn; };
  auto wtape_of = [&](int64_t j) { return rsw ? d_wtape + (overlap ? (j & 1) : 0) * K * c->n_sub : nullptr; };
  auto tape_spec = [&](int64_t j, int64_t seg0, int64_t len) {
    RecSpec r;
    r.word_tape = wtape_of(j);
    r.rec = tape_of(j);
    r.pos = d_pos;
    r.n_rec = (int32_t)nn;
    r.decim = 1;
    r.rows = seg0 + len;
    r.row0 = seg0;
    return r;
  };
  // forward pass with checkpoints
  emt_status stt = EMT_OK;
  for (int64_t j = 0; j < n_seg && stt == EMT_OK; ++j) {
    const int64_t s0 = j * K, len = std::min(K, N - s0);
    if (j < n_seg - 1) {
      e = cudaMemcpyAsync(d_ck_h + j * n_lc, c->d_h, n_lc * sizeof(double), cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ck_ring + j * ring_words, c->d_ring, ring_words * sizeof(unsigned long long),
                            cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess && rsw)
        e = cudaMemcpyAsync(d_ck_word + j * c->n_sub, c->d_rs_word, c->n_sub * sizeof(int32_t),
                            cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess && rsw)
        e = cudaMemcpyAsync(d_ck_rsi + j * n_rsw, c->d_rs_prev_i, n_rsw * sizeof(double), cudaMemcpyDeviceToDevice,
                            st);
      if (e == cudaSuccess && cpl)
        e = cudaMemcpyAsync(d_ck_lep + j * n_lend, c->d_le_prev, c->line_ends.size() * sizeof(double),
                            cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) break;
    }
    stt = forward_steps(c, len, st, j == n_seg - 1 ? tape_spec(j, s0, len) : RecSpec());
  }
  // reverse pass
  if (e == cudaSuccess && stt == EMT_OK)
    e = launch_ring_init(RingInitParams{c->d_le, (int64_t)c->line_ends.size(), d_aring}, st);
  AdjParams a{};
  a.n_sub = c->n_sub;
  a.lim = al;
  a.sub = c->d_sub;
  a.ep = c->d_ep;
  a.ginv = c->d_ginv;
  a.ginv_lo = c->d_ginv_lo;
  a.br = c->d_br;
  a.br_lc = c->d_br_lc;
  a.lc_idx = c->d_lc_idx;
  a.ent = c->d_ent;
  a.il_node = c->d_il_node;
  a.il_cnt = c->d_il_cnt;
  a.str_slot = c->d_str_slot;
  a.le = c->d_le;
  a.ring = d_aring;
  a.src_global = c->d_src_global;
  a.src_amp = c->d_src_amp;
  a.sin_table = d_sin;
  a.n_sources = (int32_t)ns;
  a.target = d_tgt;
  a.ce = c->d_ce;
  a.le_prev = d_adj_lep;
  a.orig_of = c->d_original_of;
  a.n_nodes = nn;
  a.hbar = d_hbar;
  a.dg = d_dg;
  a.dsrc = d_dsrc;
  a.loss_part = d_lp;
  a.err = c->d_err;
  a.n_total = N;
  a.wait_budget_ns = c->wait_budget_ns;
  a.bnd.ring = std::max<int64_t>(c->ring_len, 1);
  a.bnd.ginv = c->ginv_len;
  a.bnd.tape = K * nn;
  a.bnd.target = N * nn;
  // Re-run of segment j from its checkpoint, recording its tape, on `rs`.
  auto rerun = [&](int64_t j, cudaStream_t rs) -> emt_status {
    const int64_t s0 = j * K, len = std::min(K, N - s0);
    e = cudaMemcpyAsync(c->d_h, d_ck_h + j * n_lc, n_lc * sizeof(double), cudaMemcpyDeviceToDevice, rs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->d_ring, d_ck_ring + j * ring_words, ring_words * sizeof(unsigned long long),
                          cudaMemcpyDeviceToDevice, rs);
    if (e == cudaSuccess && rsw)
      e = cudaMemcpyAsync(c->d_rs_word, d_ck_word + j * c->n_sub, c->n_sub * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                          rs);
    if (e == cudaSuccess && rsw)
      e = cudaMemcpyAsync(c->d_rs_prev_i, d_ck_rsi + j * n_rsw, n_rsw * sizeof(double), cudaMemcpyDeviceToDevice, rs);
    if (e == cudaSuccess && cpl)
      e = cudaMemcpyAsync(c->d_le_prev, d_ck_lep + j * n_lend, c->line_ends.size() * sizeof(double),
                          cudaMemcpyDeviceToDevice, rs);
    if (e != cudaSuccess) return c->cuda_fail(e, "emt_adjoint checkpoint restore");
    c->step = s0;
    return forward_steps(c, len, rs, tape_spec(j, s0, len));
  };
  // Host order of the overlapped schedule (each event is recorded before
  // any wait on it is enqueued):
  //   st:  ... reverse(j) [waits rerun_done(j)], records rev_done(j)
  //   st2: rerun(j-1) [waits rev_done(j+1), the last user of its tape], records rerun_done(j-1)
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fwd = nullptr, ev_rerun[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr};
  if (overlap && e == cudaSuccess && stt == EMT_OK) {
    e = cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_fwd, cudaEventDisableTiming);
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
      e = cudaEventCreateWithFlags(&ev_rerun[q], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_rev[q], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev_fwd, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st2, ev_fwd, 0);
  }
  for (int64_t j = n_seg - 1; j >= 0 && e == cudaSuccess && stt == EMT_OK; --j) {
    const int64_t s0 = j * K, len = std::min(K, N - s0);
    if (j < n_seg - 1) {
      if (overlap) {
        e = cudaStreamWaitEvent(st, ev_rerun[j & 1], 0);
      } else {
        stt = rerun(j, st);
      }
      if (e != cudaSuccess || stt != EMT_OK) break;
    }
    a.tape = tape_of(j);
    a.word_tape = wtape_of(j);
    a.tape_row0 = s0;
    a.n_hi = s0 + len;
    a.n_steps = len;
    e = launch_adjoint(a, st);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
      stt = c->fail(EMT_ERESOURCE, "adjoint launch of " + std::to_string(c->n_sub) +
                                       " CTAs cannot be co-resident on this device");
      break;
    }
    c->launches += 1;
    if (overlap && e == cudaSuccess) e = cudaEventRecord(ev_rev[j & 1], st);
    if (overlap && e == cudaSuccess && j >= 1) {
      if (j + 1 <= n_seg - 1) e = cudaStreamWaitEvent(st2, ev_rev[(j + 1) & 1], 0);
      if (e == cudaSuccess) stt = rerun(j - 1, st2);
      if (e == cudaSuccess && stt == EMT_OK) e = cudaEventRecord(ev_rerun[(j - 1) & 1], st2);
    }
  }
  if (st2) {
    cudaStreamSynchronize(st2);
    cudaStreamDestroy(st2);
  }
  if (ev_fwd) cudaEventDestroy(ev_fwd);
  for (int q = 0; q < 2; ++q) {
    if (ev_rerun[q]) cudaEventDestroy(ev_rerun[q]);
    if (ev_rev[q]) cudaEventDestroy(ev_rev[q]);
  }
  if (e == cudaSuccess && stt == EMT_OK) {
    e = launch_adj_finalize(c->d_br, c->d_br_orig, nbr, d_dg, d_dsrc, c->d_src_br_ptr, c->d_src_br, ns, c->dt, d_lp,
                            (int64_t)c->n_sub * T, d_grad, d_loss, st);
    c->launches += 2;
  }
  double h_loss = 0.0;
  if (e == cudaSuccess && stt == EMT_OK) {
    if (grad && !on_device)
      e = cudaMemcpyAsync(grad, d_grad, (size_t)(nbr + ns) * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_loss, d_loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cleanup();
  if (stt != EMT_OK) return stt;
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_adjoint");
  int32_t info[4] = {0, 0, 0, 0};
  e = cudaMemcpy(info, c->d_err, sizeof(info), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_adjoint");
  if (info[0] == EMT_ETIMEOUT)
    return c->fail(EMT_ETIMEOUT, "emt_adjoint: subsystem " + std::to_string(info[1]) + " timed out at tag " +
                                     std::to_string(info[3]) + " waiting for the value of its line end " +
                                     std::to_string(info[2]));
  if (info[0] != 0) return c->fail((emt_status)info[0], "emt_adjoint: device error");
  if (loss) *loss = h_loss;
  return emt_reset(c);
}

// ------------------------------------------------------------------ no-alloc prefactor
//
// emt_prefactor allocates temporary device buffers (the matrix lists, a
// status word per matrix, and two n x nc workspaces per matrix: a copy of G
// and the Newton residual).  Callers that must not allocate device memory
// when they refactorise -- services that reserve all device memory up front
// and hand it out themselves, loops that cannot take cudaMalloc's implicit
// device synchronisation or risk its failure half-way through a run -- use
// emt_prefactor_noalloc instead, which keeps that workspace in the fixed
// array below.

namespace {

constexpr size_t kNoAllocMaxMats = 16384;                    // matrices (subsystem x switch state)
constexpr size_t kNoAllocMaxWorkDoubles = 480 * 1024;        // per workspace (G copy / residual)
constexpr size_t kNoAllocScratchBytes =
    3 * kNoAllocMaxMats * sizeof(int32_t) + 2 * kNoAllocMaxWorkDoubles * sizeof(double) + 256;

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up on the first
// call on that device.  Every thread that looks it up stores the same
// value; the atomics make concurrent first calls well defined.
constexpr int kNoAllocMaxDevices = 64;
std::atomic<void*> g_noalloc_ptr[kNoAllocMaxDevices];

// Matrix m is epoch m: epochs are stored subsystem by subsystem.
__global__ void noalloc_mat_lists(const SubDev* sub, int n_sub, int32_t* mat_sub, int32_t* mat_ep) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_sub) return;
  for (int k = 0; k < sub[s].n_ep; ++k) {
    mat_sub[sub[s].ep_off + k] = s;
    mat_ep[sub[s].ep_off + k] = sub[s].ep_off + k;
  }
}

// first[0] = 1 + index of the first singular matrix, or 0 if none
__global__ void noalloc_first_singular(const int32_t* status, int n_mats, int32_t* first) {
  for (int m = threadIdx.x; m < n_mats; m += blockDim.x)
    if (status[m] != 0) atomicMin(first, m + 1);
}

}  // namespace

extern "C" emt_status emt_prefactor_noalloc(emt_ctx* c, void* stream) {
  if (!c) return EMT_EINVAL;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_prefactor_noalloc");
  if (dev != c->device) return c->fail(EMT_EINVAL, "make the context's device current first");
  if (c->batched) return c->fail(EMT_EINVAL, "emt_prefactor_noalloc serves single-scenario contexts; use emt_prefactor");
  if (dev < 0 || dev >= kNoAllocMaxDevices) return c->fail(EMT_EINVAL, "device index beyond the supported range");
  const size_t n_mats = c->epochs.size();
  if (n_mats + 1 > kNoAllocMaxMats || (size_t)c->ginv_len > kNoAllocMaxWorkDoubles)
    return c->fail(EMT_EINVAL, "network too large for emt_prefactor_noalloc's fixed workspace "
                               "(at most 16383 matrices and 491520 solve-matrix entries); use emt_prefactor");
  void* sym = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!sym) {   // one-time set-up on this device (the device is current)
    e = cudaGetSymbolAddress(&sym, g_noalloc_scratch);
    if (e != cudaSuccess) return c->cuda_fail(e, "emt_prefactor_noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[dev].store(sym, std::memory_order_release);
  }
  unsigned char* base = static_cast<unsigned char*>(sym);
  int32_t* mat_sub = reinterpret_cast<int32_t*>(base);
  int32_t* mat_ep = mat_sub + kNoAllocMaxMats;
  int32_t* status = mat_ep + kNoAllocMaxMats;      // status[0 .. n_mats), then the "first" word
  double* work_g = reinterpret_cast<double*>(base + 3 * kNoAllocMaxMats * sizeof(int32_t));
  double* work_r = work_g + kNoAllocMaxWorkDoubles;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n_mats == 0) {
    c->prefactored = true;
    return EMT_OK;
  }
  e = cudaMemsetAsync(status, 0, (n_mats + 1) * sizeof(int32_t), st);
  if (e == cudaSuccess) {
    noalloc_mat_lists<<<(c->n_sub + 127) / 128, 128, 0, st>>>(c->d_sub, c->n_sub, mat_sub, mat_ep);
    e = cudaGetLastError();
  }
  PrefParams p{};
  p.n_mats = (int32_t)n_mats;
  p.mat_sub = mat_sub;
  p.mat_ep = mat_ep;
  p.sub = c->d_sub;
  p.ep = c->d_ep;
  p.br = c->d_br;
  p.le = c->d_le;
  p.sw = c->d_sw;
  p.ce = c->d_ce;
  p.lc_idx = c->d_lc_idx;
  p.str_slot = c->d_str_slot;
  p.ginv = c->d_ginv;
  p.ginv_lo = c->d_ginv_lo;
  p.nl = c->d_nl;
  p.nlz = c->d_nlz;
  p.nlz_lo = c->d_nlz_lo;
  p.work_g = work_g;
  p.work_r = work_r;
  p.status = status;
  p.rs = c->d_rs;
  if (e == cudaSuccess) e = launch_prefactor(p, std::max(c->lim.n, 1), st);
  if (e == cudaSuccess) e = reset_matrix_cache(c, st);
  if (e == cudaSuccess) e = build_state_space(c, st);
  int32_t* first = status + n_mats;
  if (e == cudaSuccess) e = cudaMemsetAsync(first, 0x7f, sizeof(int32_t), st);
  if (e == cudaSuccess) {
    noalloc_first_singular<<<1, 256, 0, st>>>(status, (int)n_mats, first);
    e = cudaGetLastError();
  }
  int32_t h_first = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_first, first, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return c->cuda_fail(e, "emt_prefactor_noalloc");
  if (h_first != 0x7f7f7f7f) {   // matrix h_first - 1 is epoch h_first - 1 (epochs subsystem by subsystem)
    const int m = h_first - 1;
    for (int s = 0; s < c->n_sub; ++s)
      if (m >= c->subs[s].ep_off && m < c->subs[s].ep_off + c->subs[s].n_ep)
        return c->fail(EMT_ESINGULAR, "conductance matrix of subsystem " + std::to_string(s) + " (first node " +
                                          std::to_string(c->original_of[c->subs[s].node_off]) + ", switch state " +
                                          std::to_string(m - c->subs[s].ep_off) + ") is singular");
    return c->fail(EMT_ESINGULAR, "a subsystem conductance matrix is singular");
  }
  c->prefactored = true;
  return EMT_OK;
}
