// CUDA kernels of the EMTP-type time loop for sm_103a (B300).
//
// companion_kernel   process 1 constants: g = 1/R, dt/(2L), 2C/dt and the
//                    history gain e = +2g (L) / -2g (C)
// prefactor_kernel   process 3, once per subsystem and switch state: stamp G,
//                    invert it in place (Gauss-Jordan, partial pivoting),
//                    then a Newton step with the residual summed in twice
//                    the working precision, giving G^-1 = X_hi + X_lo
//                    (double + single-precision remainder)
// source_kernel      process 1 for sources: the table v_src(t_n) of a launch
// ring_init_kernel   de-energised line histories in the tagged rings
// fwd_kernel         the persistent time loop (processes 1, 2, 4 and the
//                    Bergeron line update), one CTA per subsystem, G^-1 and
//                    all per-element data in shared memory for the whole
//                    launch; subsystems meet only through the line rings,
//                    whose slots carry the step they belong to (no flags,
//                    no fences, no grid barrier)
// gather_kernel      copies recorded channels into the caller's layout
//
// Formulas (CloudPSS paper Sec. III-A processes; textbook trapezoidal
// companions of its ref. [2]; lossless Bergeron line):
//   i_n[k] = sum_src g_b v_src(t_n) - sum_b a_bk h_b(n-1) - sum_e I_e(n)
//   v_n    = G^-1 i_n
//   h_b(n) = +h_b(n-1) + 2 g v_b(n)   (L)      -h_b(n-1) - 2 g v_b(n)   (C)
//   I_far(n+d) = -(2/Z_c) v_near(n) - I_near(n)
#include <stdint.h>

#include <algorithm>
#include <climits>

#include <cuda_runtime.h>

#include "emt_internal.h"
#include "emt_device.cuh"

namespace emt {

namespace {

// error-free transformations (Knuth TwoSum; TwoProd by FMA)
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// hi + lo += a * b, products exact, sum carried in two doubles (Dot2)
__device__ __forceinline__ void dot2_acc(double& hi, double& lo, double a, double b) {
  const double p = __dmul_rn(a, b);
  const double pe = fma(a, b, -p);
  double s, e;
  two_sum(hi, p, s, e);
  hi = s;
  lo = __dadd_rn(lo, __dadd_rn(e, pe));
}

// ------------------------------------------------------------ companion

__global__ void companion_kernel(BranchDev* br, int64_t n_br, double dt) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_br) return;
  const BranchDev x = br[b];
  double g;
  if (x.kind == 0) g = 1.0 / x.value;
  else if (x.kind == 1) g = dt / (2.0 * x.value);
  else g = 2.0 * x.value / dt;
  br[b].g = g;
  br[b].e = x.kind == 1 ? 2.0 * g : (x.kind == 2 ? -2.0 * g : 0.0);
}

// ------------------------------------------------------------ coupled lines

// Per coupled line end: T_v^-1 (cofactors), T_i = T_v^-T and
// Y_p = T_i diag(1/Z) T_v^-1.
__global__ void coupled_constants_kernel(CoupledEndDev* ce, int64_t n_ce) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_ce) return;
  CoupledEndDev& c = ce[i];
  const double* a = c.tv;
  const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
  const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  double inv[9];
  inv[0] = c00 / det;
  inv[3] = c01 / det;
  inv[6] = c02 / det;
  inv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  inv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  inv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
  for (int k = 0; k < 9; ++k) c.tinv[k] = inv[k];
  for (int p = 0; p < 3; ++p)
    for (int j = 0; j < 3; ++j) c.ti[3 * p + j] = inv[3 * j + p];
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) {
      double acc = 0.0;
      for (int j = 0; j < 3; ++j) acc += c.ti[3 * p + j] * (1.0 / c.z[j]) * inv[3 * j + q];
      c.yp[3 * p + q] = acc;
    }
}

// ------------------------------------------------------------ prefactor

__device__ __forceinline__ void stamp(double* A, int n, int k, int m, double g) {
  if (k >= 0) A[k * n + k] += g;
  if (m >= 0) A[m * n + m] += g;
  if (k >= 0 && m >= 0) {
    A[k * n + m] -= g;
    A[m * n + k] -= g;
  }
}

// One solve matrix (process 3), by all threads of a CTA: stamp G, invert it
// in place (Gauss-Jordan, partial pivoting), then a Newton step with the
// residual summed in twice the working precision, giving G^-1 = X_hi +
// X_lo; then the strong-branch columns and the nonlinear resistor's column.
// Used by the prefactor (one CTA per matrix) and by the forward kernel when
// a subsystem meets a switch state for the first time.
struct FactorJob {
  SubDev S;
  const SwitchDev* sw;                   // closed switches
  int n_sw;
  const RuntimeSwitchDev* rs;            // the subsystem's runtime switches, stamped by rs_word if >= 0
  int rs_word;
  const BranchDev* br;
  const LineEndDev* le;
  const CoupledEndDev* ce;
  const int32_t* lc_idx;
  const int32_t* str_slot;
  const NlDev* nl;
  int rb0, rb1, rl0, rl1;                // removed branches / line ends (scenario variants)
  const int32_t* rm_br;
  const int32_t* rm_le;
  double* out;                           // X_hi, n x nc (nc = n + strong columns)
  float* out_lo;                         // X_lo
  double* nlz;                           // the nonlinear resistor's column (n), or nullptr
  float* nlz_lo;
  double* Gw;                            // two n x n workspaces
  double* Rw;
};

// A: n x n doubles, fcol: n doubles, perm: n ints, all in shared memory, and
// two shared ints; returns true on every thread if G is singular.
__device__ __noinline__ bool factor_cta(const FactorJob& J, double* A, double* fcol, int* perm, int* s_p, int* s_sing) {
  const SubDev& S = J.S;
  const int n = S.n, T = blockDim.x, tid = threadIdx.x;
  for (int i = tid; i < n * n; i += T) A[i] = 0.0;
  __syncthreads();
  if (tid == 0) {
    // a source end acts as ground in G (its voltage goes to the injection);
    // elements a scenario variant removes are left out
    for (int b = 0; b < S.n_br; ++b) {
      bool removed = false;
      for (int x = J.rb0; x < J.rb1; ++x) removed |= (J.rm_br[x] == S.br_off + b);
      if (removed) continue;
      const BranchDev x = J.br[S.br_off + b];
      stamp(A, n, x.k >= 0 ? x.k : -1, x.m >= 0 ? x.m : -1, x.g);
    }
    for (int e = 0; e < S.n_le; ++e) {
      bool removed = false;
      for (int x = J.rl0; x < J.rl1; ++x) removed |= (J.rm_le[x] == S.le_off + e);
      if (removed) continue;
      const LineEndDev le = J.le[S.le_off + e];
      if (le.node >= 0) A[le.node * n + le.node] += le.y;
    }
    for (int x = 0; x < S.n_ce; ++x) {   // coupled line ends: the 3 x 3 block Y_p
      const CoupledEndDev& c = J.ce[S.ce_off + x];
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) A[c.node[p] * n + c.node[q]] += c.yp[3 * p + q];
    }
    for (int w = 0; w < J.n_sw; ++w) {
      const SwitchDev sw = J.sw[w];
      stamp(A, n, sw.k, sw.m, sw.g);
    }
    if (J.rs_word >= 0)   // runtime switches by the state word: r_on or r_off
      for (int j = 0; j < S.n_rs; ++j) {
        const RuntimeSwitchDev r = J.rs[S.rs_off + j];
        stamp(A, n, r.k, r.m, 1.0 / (((J.rs_word >> j) & 1) ? r.r_on : r.r_off));
      }
    *s_sing = 0;
  }
  __syncthreads();
  double* Gw = J.Gw;
  double* Rw = J.Rw;
  for (int i = tid; i < n * n; i += T) Gw[i] = A[i];
  // in-place Gauss-Jordan inversion with row pivoting
  for (int k = 0; k < n; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int arg = k;
      for (int i = k + tid; i < n; i += 32) {
        const double m = fabs(A[i * n + k]);
        if (m > best) { best = m; arg = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oa = __shfl_down_sync(0xffffffffu, arg, off);
        if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
      }
      if (tid == 0) {
        *s_p = arg;
        perm[k] = arg;
        if (!(best > 1e-300) || !isfinite(best)) *s_sing = 1;
      }
    }
    __syncthreads();
    if (*s_sing) break;
    const int p = *s_p;
    if (p != k)
      for (int j = tid; j < n; j += T) {
        const double t = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / A[k * n + k];
    __syncthreads();
    for (int j = tid; j < n; j += T) A[k * n + j] = (j == k) ? inv : A[k * n + j] * inv;
    for (int i = tid; i < n; i += T) fcol[i] = (i == k) ? 0.0 : A[i * n + k];
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += T) {
      const int i = idx / n, j = idx - i * n;
      if (i == k) continue;
      if (j == k) A[i * n + k] = -fcol[i] * A[k * n + k];
      else A[i * n + j] -= fcol[i] * A[k * n + j];
    }
    __syncthreads();
  }
  const bool singular = *s_sing != 0;
  __syncthreads();
  if (singular) return true;
  // undo the row interchanges as column interchanges, last pivot first
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int i = tid; i < n; i += T) {
        const double t = A[i * n + k];
        A[i * n + k] = A[i * n + p];
        A[i * n + p] = t;
      }
    __syncthreads();
  }
  // Newton step: R0 = I - G X0 with Dot2 (exact products, sum carried in
  // two doubles), X_hi = X0 + X0 R0, which is G^-1 to about an ulp.  Then
  // the remainder X_lo = X_hi (I - G X_hi) in single precision: a rounded
  // inverse is the exact inverse of a matrix off from G by ~cond(G) eps,
  // a systematic error the long recursion would integrate; X_hi + X_lo
  // removes it at the cost of single-precision work per solve.
  for (int idx = tid; idx < n * n; idx += T) {
    const int i = idx / n, j = idx - i * n;
    double hi = (i == j) ? 1.0 : 0.0, lo = 0.0;
    for (int k = 0; k < n; ++k) dot2_acc(hi, lo, -Gw[i * n + k], A[k * n + j]);
    Rw[idx] = __dadd_rn(hi, lo);
  }
  __syncthreads();
  const int nc = n + S.n_str;
  double* out = J.out;
  for (int idx = tid; idx < n * n; idx += T) {
    const int i = idx / n, j = idx - i * n;
    double c = 0.0;
    for (int k = 0; k < n; ++k) c = fma(A[i * n + k], Rw[k * n + j], c);
    out[i * nc + j] = A[idx] + c;
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += T) A[idx] = out[(idx / n) * nc + idx % n];
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += T) {
    const int i = idx / n, j = idx - i * n;
    double hi = (i == j) ? 1.0 : 0.0, lo = 0.0;
    for (int k = 0; k < n; ++k) dot2_acc(hi, lo, -Gw[i * n + k], A[k * n + j]);
    Rw[idx] = __dadd_rn(hi, lo);
  }
  __syncthreads();
  float* out_lo = J.out_lo;
  for (int idx = tid; idx < n * n; idx += T) {
    const int i = idx / n, j = idx - i * n;
    double c = 0.0;
    for (int k = 0; k < n; ++k) c = fma(A[i * n + k], Rw[k * n + j], c);
    out_lo[i * nc + j] = (float)c;
  }
  __syncthreads();
  // strong-branch columns (G^-1[:,k] - G^-1[:,m]) from X_hi + X_lo with
  // error-free differences, split again into double + single remainder
  for (int idx = tid; idx < n * S.n_str; idx += T) {
    const int i = idx / S.n_str, t = idx - i * S.n_str;
    const BranchDev b = J.br[J.lc_idx[S.lc_off + J.str_slot[S.str_off + t]]];
    double d1, e1;
    two_sum(out[i * nc + b.k], -out[i * nc + b.m], d1, e1);
    const double rest = e1 + ((double)out_lo[i * nc + b.k] - (double)out_lo[i * nc + b.m]);
    double s, e;
    two_sum(d1, rest, s, e);
    out[i * nc + n + t] = s;
    out_lo[i * nc + n + t] = (float)e;
  }
  // each nonlinear resistor's column G^-1 (e_k - e_m), formed the same way
  if (S.n_nl > 0 && J.nlz != nullptr) {
    for (int idx = tid; idx < n * S.n_nl; idx += T) {
      const int x = idx / n, i = idx - x * n;
      const NlDev& q = J.nl[S.nl_off + x];
      const double a = q.k >= 0 ? out[i * nc + q.k] : 0.0, b = q.m >= 0 ? out[i * nc + q.m] : 0.0;
      const double al = q.k >= 0 ? (double)out_lo[i * nc + q.k] : 0.0;
      const double bl = q.m >= 0 ? (double)out_lo[i * nc + q.m] : 0.0;
      double d1, e1;
      two_sum(a, -b, d1, e1);
      double s, e;
      two_sum(d1, e1 + (al - bl), s, e);
      J.nlz[idx] = s;
      J.nlz_lo[idx] = (float)e;
    }
  }
  __syncthreads();
  return false;
}

__global__ void __launch_bounds__(256) prefactor_kernel(PrefParams P) {
  extern __shared__ double A[];
  __shared__ double fcol[kMaxSubsystemNodes];
  __shared__ int perm[kMaxSubsystemNodes];
  __shared__ int s_p, s_sing;
  const int mi = blockIdx.x;
  FactorJob J;
  J.S = P.sub[P.mat_sub[mi]];
  const EpochDev E = P.ep[P.mat_ep[mi]];
  J.sw = P.sw + E.sw_off;
  J.n_sw = E.n_sw;
  J.rs = P.rs;
  J.rs_word = E.rs_word;
  J.br = P.br;
  J.le = P.le;
  J.ce = P.ce;
  J.lc_idx = P.lc_idx;
  J.str_slot = P.str_slot;
  J.nl = P.nl;
  J.rb0 = P.rm_ptr_br ? P.rm_ptr_br[mi] : 0;
  J.rb1 = P.rm_ptr_br ? P.rm_ptr_br[mi + 1] : 0;
  J.rl0 = P.rm_ptr_le ? P.rm_ptr_le[mi] : 0;
  J.rl1 = P.rm_ptr_le ? P.rm_ptr_le[mi + 1] : 0;
  J.rm_br = P.rm_br;
  J.rm_le = P.rm_le;
  J.out = P.ginv + E.ginv_off;
  J.out_lo = P.ginv_lo + E.ginv_off;
  J.nlz = E.nlz_off >= 0 ? P.nlz + E.nlz_off : nullptr;
  J.nlz_lo = E.nlz_off >= 0 ? P.nlz_lo + E.nlz_off : nullptr;
  J.Gw = P.work_g + E.ginv_off;
  J.Rw = P.work_r + E.ginv_off;
  const bool singular = factor_cta(J, A, fcol, perm, &s_p, &s_sing);
  if (threadIdx.x == 0) P.status[mi] = singular ? 1 : 0;
}

// ------------------------------------------------------------ sources

__global__ void source_kernel(SourceParams P) {
  const int64_t total = P.n_steps * P.n_sources;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / P.n_sources;
    const int s = (int)(i - r * P.n_sources);
    const double t = (double)(P.n0 + r) * P.dt;
    // argument rounded as (omega * t) + phase, each operation once
    P.table[i] = P.amp[s] * sin(__dadd_rn(__dmul_rn(P.omega[s], t), P.phase[s]));
  }
}

// ------------------------------------------------------------ line rings

// De-energised start: the slot consumed at step s (1 <= s <= d) holds 0
// tagged s; every other slot holds tag 0, which no step matches.
__global__ void ring_init_kernel(RingInitParams P) {
  const int64_t e = blockIdx.x;
  if (e >= P.n_le) return;
  const LineEndDev L = P.le[e];
  for (int j = threadIdx.x; j < L.depth; j += blockDim.x) {
    const unsigned s = (j == 0) ? (unsigned)L.depth : (unsigned)j;
    const unsigned long long w = (s <= (unsigned)L.d) ? ((unsigned long long)s << 32) : 0ull;
    P.ring[2 * (L.own_ring + j)] = w;
    P.ring[2 * (L.own_ring + j) + 1] = w;
  }
}

// Between the windows of a sharded run: copy the slots a window wrote for
// remote readers (pack) or write them into this context's copy of the
// rings (unpack).  No kernel of the run is in flight at either point, so
// plain 16-byte accesses suffice.
__global__ void ring_copy_kernel(RingCopyParams P) {
  const int64_t total = (int64_t)P.n_ends * P.w;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i / P.w, j = i - x * P.w;
    const LineEndDev L = P.le[P.ends[x]];
    const int64_t slot = L.far_ring + (P.n0 + L.d + j) % L.depth;
    ulonglong2* r = reinterpret_cast<ulonglong2*>(P.ring) + slot;
    ulonglong2* b = reinterpret_cast<ulonglong2*>(P.buf) + i;
    if (P.pack) *b = *r;
    else *r = *b;
  }
}

// ------------------------------------------------------------ phase clocks
//
// The phase-clock build (compiled with -DEMT_PHASE_CLOCKS, the library
// libemt_phases.so): thread 0 of every CTA of fwd_kernel adds the clock64
// cycles of each phase of each step to per-CTA counters, and the thread
// that polls the CTA's first line end adds the cycles of its wait; read by
// emt_phase_clocks.  In the normal build the marks compile to nothing.
#ifdef EMT_PHASE_CLOCKS
__device__ unsigned long long g_phase[kPhaseCtas][kPhaseCount];
// (32-bit clocks and shared-memory sums: the instrumented kernel keeps the
// register budget of the normal one)
#define PH_DECL                                                   \
  __shared__ unsigned long long s_ph[kPhaseCount];                \
  __shared__ unsigned s_ph_first;                                 \
  unsigned ph_t0 = 0, ph_t1 = 0;                                  \
  if (threadIdx.x < kPhaseCount) s_ph[threadIdx.x] = 0;
#define PH_MARK(t) const unsigned t = (unsigned)clock();
#define PH_ADD(k, a, b) \
  if (threadIdx.x == 0) s_ph[k] += (unsigned)((b) - (a));
#else
#define PH_DECL
#define PH_MARK(t)
#define PH_ADD(k, a, b)
#endif

// ------------------------------------------------------------ forward
//
// On B300 a warp issues at most one FP64 instruction per ~64 cycles however
// many of its lanes are active, and two warps on one SM sub-partition share
// that rate.  The step is therefore laid out to keep the FP64 instruction
// count of the busiest warp small: four-entry injection lanes joined by
// shuffles, one FMA chain per matvec task over a contiguous block of
// columns (plus a single-precision chain for X_lo), node sums in their own
// phase, and update items of one kind per warp.  The next step's line
// values are collected by the update threads once their items are done, one
// thread per line end (per coupled end), so that all waits run at once.

// the last warp: collects the first step's line values of a launch, and
// serves the source-value prefetch; the warp before it evaluates control
// blocks when the subsystem has some
constexpr int kPollWarp = kFwdThreads / 32 - 1;
constexpr int kItemThreads = kFwdThreads - 32;

// A CTA's nonlinear resistor in shared memory: its record, the constants
// of the current matrix (see nl_setup), the current of the step, the record
// row of the step being compensated (or -1) and whether the constants need
// recomputing after a matrix load; then the current matrix's column z
// (n doubles, then n floats of remainder).  Its address is recomputed where
// it is used (only CTAs with a nonlinear resistor), so that the step loop of
// the others keeps no extra pointer live.
struct NlState {
  NlDev q[kNlMaxPerSub];
  double c[1 + 3 * (kNlMaxPoints + 1)];
  double inl;
  long long row;
  int dirty;
  int m;                                 // elements (several: the fields below)
  double R[kNlMaxPerSub * kNlMaxPerSub];   // Thevenin matrix R_jl = z_l[k_j] - z_l[m_j]
  double minv[kNlMaxPerSub * kNlMaxPerSub];  // (I + D R)^-1 for the slopes of minv_key
  double work[kNlMaxPerSub * kNlMaxPerSub];  // its elimination
  double cur[kNlMaxPerSub];              // element currents of the step
  double c0[kNlMaxPerSub], slope[kNlMaxPerSub];   // the current segments' lines
  double a[kNlMaxPerSub], f[kNlMaxPerSub];        // c = a + B y, u = E y - f for the current segments
  double B[kNlMaxPerSub * kNlMaxPerSub], E[kNlMaxPerSub * kNlMaxPerSub];
  int seg[kNlMaxPerSub];                 // segments, sign * (j + 1)
  int minv_key;                          // segment indices (4 bits each) minv belongs to, -1: none
  int coef_key;                          // segments with signs (5 bits each) a, B, E, f belong to, -1: none
  // the columns z_j (m n doubles), then their single-precision remainders
  __device__ double* z() { return reinterpret_cast<double*>(this + 1); }
  __device__ float* zl(int n, int m = 1) { return reinterpret_cast<float*>(z() + (size_t)m * n); }
};

// Shared-memory layout of fwd_kernel, from the per-launch limits.  G^-1
// rows are stored with an odd stride (n | 1) so that the rows a warp reads
// together fall in different banks.
struct FwdSmem {
  size_t gi, part, iv, vv, inp, vs, lce, sbg, ley2, leown, lefar, lef, imode, ceti, cetinv, cbr, cy, cs, fdr,
      fdst, nls;                                                                           // 8-byte
  size_t gilo, ivf, partf;                                                                 // float
  size_t lck, lcm, lckind, lcstr, sbsrc, lenode, ledepth, led, rslot, wslot, ent, ilnode, ilcnt, srcg, recp,
      lece, lemode, cele0, cenode, clay, cinj, lefd, cecnt, cecnt2;                        // int
  size_t bytes;
};

// doubles of the shared input vector inp (see kEntryNeg)
__host__ __device__ inline size_t fwd_inp_len(const FwdLimits& L) {
  return (size_t)L.lc + L.sb + 2 * ((size_t)L.le + 3 * (size_t)L.ce + L.fd) + 1 + (size_t)L.ci + L.fd;
}

__host__ __device__ inline FwdSmem fwd_smem(const FwdLimits& L) {
  FwdSmem s{};
  size_t o = 0;
  auto d = [&](size_t count) { size_t r = o; o += count * 8; return r; };
  auto w = [&](size_t count) { size_t r = o; o += count * 4; return r; };
  auto d16 = [&](size_t count) { o = (o + 15) & ~(size_t)15; return d(count); };
  const size_t ldg = (size_t)(L.nc | 1);
  const size_t nbuf = L.nbuf > 1 ? 2 : 1;
  s.gi = d(nbuf * (size_t)L.n * ldg);
  const size_t nq = (size_t)L.n * L.q;
  const size_t n_tasks = nq < (size_t)kFwdThreads ? nq : (size_t)kFwdThreads;   // a CTA's n q <= its threads
  s.part = d(n_tasks);
  s.iv = d(L.nc);
  s.vv = d(L.n);
  s.inp = d(fwd_inp_len(L));
  s.vs = d(2 * (size_t)L.src);
  s.lce = d(L.lc);
  s.sbg = d(L.sb);
  s.ley2 = d(L.le);
  s.leown = d(L.le);
  s.lefar = d(L.le);
  s.lef = d(L.le);
  s.imode = d(2 * (size_t)L.le);
  s.ceti = d(9 * (size_t)L.ce);
  s.cetinv = d(9 * (size_t)L.ce);
  s.cbr = d16(sizeof(CtrlDev) / 8 * (size_t)L.cb);
  s.cy = d16(2 * (size_t)L.cb + 2);
  s.cs = d16(2 * (size_t)L.cb);
  s.nls = d(L.nl ? sizeof(NlState) / 8 + (size_t)L.nl * L.n + ((size_t)L.nl * L.n + 1) / 2 : 0);
  s.fdr = d(sizeof(FdEndDev) / 8 * (size_t)L.fd);
  s.fdst = d(kFdState * (size_t)L.fd);
  s.gilo = w(nbuf * (size_t)L.n * ldg);
  s.ivf = w(L.nc);
  s.partf = w(n_tasks);
  s.lcstr = w(L.lc);
  s.lck = w(L.lc);
  s.lcm = w(L.lc);
  s.lckind = w(L.lc);
  s.sbsrc = w(L.sb);
  s.lenode = w(L.le);
  s.ledepth = w(L.le);
  s.led = w(L.le);
  s.rslot = w(L.le);
  s.wslot = w(L.le);
  s.ent = w(4 * (size_t)L.il);
  s.ilnode = w(L.il);
  s.ilcnt = w(L.il);
  s.srcg = w(L.src);
  s.recp = w(L.n);
  s.lece = w(L.le);
  s.lemode = w(L.le);
  s.cele0 = w(L.ce);
  s.cenode = w(3 * (size_t)L.ce);
  s.clay = w(L.clay);
  s.cinj = w(L.ci);
  s.lefd = w(L.le);
  s.cecnt = w(L.ce);
  s.cecnt2 = w(L.ce);
  s.bytes = (o + 15) & ~(size_t)15;
  return s;
}

// Coupled line modes at the first step of a launch (the last warp, after
// collecting step m's values into blk_new; later steps fold them as they
// arrive): each mode's interpolated history I_mode(m) = (1 - f) c(m - d)
// + f c(m - d - 1) from the values consumed at steps m (blk_new) and m - 1
// (blk_old), then the phase-domain history currents T_i I_mode of each
// coupled end into the phase slots that follow the n_le line-end slots.
__device__ void fold_modes(int lane, int n_le, int n_ce, const int* lece, const double* lef, const double* blk_old,
                           double* blk_new, double* imode_new, const int* cele0, const double* ceti, const int* lefd,
                           int fd_base) {
  for (int e = lane; e < n_le; e += 32)
    if (lece[e] >= 0)   // (a mode of a frequency-dependent line group: -b, already folded on arrival)
      imode_new[e] = lefd != nullptr && lefd[e] >= 0 ? -blk_new[fd_base + lefd[e]]
                                                     : fma(lef[e], blk_old[e], (1.0 - lef[e]) * blk_new[e]);
  __syncwarp();
  for (int x = lane; x < 3 * n_ce; x += 32) {
    const int c = x / 3, p = x - 3 * c;
    const double* ti = ceti + 9 * c + 3 * p;
    const double* im = imode_new + cele0[c];
    blk_new[n_le + x] = fma(ti[0], im[0], fma(ti[1], im[1], ti[2] * im[2]));
  }
  __syncwarp();
}

// Total order of finite doubles as signed 64-bit integers (the magnitude
// bits of negative values flipped), so that a limiter compares on the
// integer pipe instead of spending FP64 latency.
__device__ __forceinline__ long long ordered_bits(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}

// One control block of type `type` at a step of parity par (its layer's
// current inputs are final): inputs are y[i ^ par] (see CtrlDev), st = the
// block's two states, updated into *ns (and *has_state set) for the types
// that keep state; the caller stores only for its own block.  FP64
// instructions cost ~64 cycles of the warp each, so each type uses as few
// as it can; a limiter compares on the integer pipe.
__device__ __forceinline__ double control_block(int type, const CtrlDev& r, const double* y, int par,
                                                const double* vv, const double* st, double2* ns, bool* has_state) {
  const double u0 = y[r.i0 ^ par];
  const double u1 = y[r.i1 ^ par];
  double out;
  switch (type) {
    case 0: out = r.p0; break;
    case 1: out = vv[r.node]; break;
    case 2: out = r.p0 * u0; break;
    case 3: out = fma(r.p0, u0, r.p1 * u1); break;
    case 4: out = r.p0 * u0 * u1; break;
    case 5: {   // lo if u0 < lo, hi if u0 > hi, else u0 (finite values)
      const long long k = ordered_bits(u0);
      out = k < ordered_bits(r.p0) ? r.p0 : (k > ordered_bits(r.p1) ? r.p1 : u0);
      break;
    }
    case 6: {   // trapezoidal integral
      const double2 s = *reinterpret_cast<const double2*>(st);
      out = fma(r.p0, u0 + s.y, s.x);
      *ns = make_double2(out, u0);
      *has_state = true;
      break;
    }
    case 7: {   // first-order lag, Tustin: a y(n-1) + b (u0 + u0(n-1))
      const double2 s = *reinterpret_cast<const double2*>(st);
      out = fma(r.p1, u0 + s.y, r.p0 * s.x);
      *ns = make_double2(out, u0);
      *has_state = true;
      break;
    }
    default: {   // PI: proportional + trapezoidal integral
      const double2 s = *reinterpret_cast<const double2*>(st);
      const double integral = fma(r.p2, u0 + s.y, s.x);
      out = fma(r.p1, integral, r.p0 * u0);
      *ns = make_double2(integral, u0);
      *has_state = true;
      break;
    }
  }
  return out;
}

// Block b of a layer (type lt, or each block's own for a mixed layer);
// lanes past the layer's end evaluate the layer's first block and store
// nothing (a straight path without a per-lane loop is much shorter here).
__device__ __forceinline__ void control_slot(int b, int first, bool act, int lt, const CtrlDev* cbr, double* cy,
                                             double* cs, int par, const double* vv) {
  const int bb = act ? b : first;
  const CtrlDev& r = cbr[bb];
  double2 ns = make_double2(0.0, 0.0);
  bool has_state = false;
  const double y = control_block(lt == kMixedLayer ? r.type : lt, r, cy, par, vv, cs + 2 * bb, &ns, &has_state);
  if (act) {
    cy[2 * b + par] = y;
    if (has_state) *reinterpret_cast<double2*>(cs + 2 * b) = ns;
  }
}

// Nonlinear resistor (compensation method), per solve-matrix entry: the
// Thevenin resistance R = z_k - z_m of its column and, per segment j, the
// image H_j = v_j + R i_j of the segment's start, 1 / (1 + R s_j) and
// R (i_j - s_j v_j).  c = [R, H[9], a[9], b[9]].
__device__ void nl_setup(const NlDev& q, const double* zh, const float* zl, double* c) {
  const double zk = q.k >= 0 ? zh[q.k] + (double)zl[q.k] : 0.0;
  const double zm = q.m >= 0 ? zh[q.m] + (double)zl[q.m] : 0.0;
  const double R = zk - zm;
  c[0] = R;
  for (int j = 0; j <= q.np; ++j) {
    c[1 + j] = fma(R, q.bi[j], q.bv[j]);
    c[1 + (kNlMaxPoints + 1) + j] = 1.0 / fma(R, q.sl[j], 1.0);
    c[1 + 2 * (kNlMaxPoints + 1) + j] = R * fma(-q.sl[j], q.bv[j], q.bi[j]);
  }
}

// Its current from the Thevenin voltage: the segment whose image holds
// |v_th| (integer compares of finite doubles), then u on that segment and
// i = f(u) with the sign of v_th.
__device__ double nl_current(const NlDev& q, const double* c, double vth) {
  const double x = fabs(vth);
  const long long kx = ordered_bits(x);
  int j = 0;
  while (j < q.np && kx >= ordered_bits(c[1 + j + 1])) ++j;
  const double u = (x - c[1 + 2 * (kNlMaxPoints + 1) + j]) * c[1 + (kNlMaxPoints + 1) + j];
  const double i = fma(q.sl[j], u - q.bv[j], q.bi[j]);
  return vth < 0.0 ? -i : i;
}

// The compensation step of a CTA with a nonlinear resistor (after the node
// sums, two barriers inside; every thread of the CTA calls it): the current
// from the Thevenin source on thread 0, then v -= z i and the record.
__device__ __forceinline__ void compensate(const FwdParams& P, int n, NlState* s, double* vv, const int* recp) {
  const int tid = threadIdx.x, T = blockDim.x;
  const double* z = s->z();
  const float* zl = s->zl(n);
  if (tid == 0) {
    if (s->dirty) {
      nl_setup(s->q[0], z, zl, s->c);
      s->dirty = 0;
    }
    const double vth = (s->q[0].k >= 0 ? vv[s->q[0].k] : 0.0) - (s->q[0].m >= 0 ? vv[s->q[0].m] : 0.0);
    s->inl = nl_current(s->q[0], s->c, vth);
  }
  __syncthreads();
  const double inl = s->inl;
  const long long row = s->row;
  for (int r = tid; r < n; r += T) {
    const double v = fma(-(double)zl[r], inl, fma(-z[r], inl, vv[r]));
    vv[r] = v;
    if (row >= 0 && recp[r] >= 0) P.rec[EMT_CHK(P.err, (row - P.rec_row0) * P.n_rec + recp[r], P.bnd.rec, kChkRecord)] = v;
  }
  __syncthreads();
}

// Segment of nonlinear resistor q that holds the voltage u: sign * (j + 1),
// j the number of breakpoints at or below |u| (independent integer compares
// of the bit patterns, which order non-negative doubles).
__device__ __forceinline__ int nl_segment_of(const NlDev& q, double u) {
  const long long bu = __double_as_longlong(u);
  const long long kx = bu & 0x7fffffffffffffffll;   // |u|
  int j = 0;
#pragma unroll
  for (int p = 1; p <= kNlMaxPoints; ++p)
    j += (p <= q.np && kx >= __double_as_longlong(q.bv[p])) ? 1 : 0;
  return bu < 0 ? -(j + 1) : j + 1;
}

// (I + D R)^-1 of the current segments' slopes D into s->minv (Gauss-Jordan
// with partial pivoting, on one thread, in the state's shared memory; it
// runs only when a segment's slope changes).
__device__ __forceinline__ void nl_invert(NlState* s, int m) {
  constexpr int W = kNlMaxPerSub;
  double* M = s->work;
  double* X = s->minv;
  for (int j = 0; j < m; ++j)
    for (int l = 0; l < m; ++l) {
      M[j * W + l] = fma(s->q[j].sl[abs(s->seg[j]) - 1], s->R[j * W + l], j == l ? 1.0 : 0.0);
      X[j * W + l] = j == l ? 1.0 : 0.0;
    }
  for (int k = 0; k < m; ++k) {
    int p = k;
    for (int i = k + 1; i < m; ++i)
      if (fabs(M[i * W + k]) > fabs(M[p * W + k])) p = i;
    for (int l = 0; l < m; ++l) {
      double t = M[k * W + l];
      M[k * W + l] = M[p * W + l];
      M[p * W + l] = t;
      t = X[k * W + l];
      X[k * W + l] = X[p * W + l];
      X[p * W + l] = t;
    }
    const double inv = 1.0 / M[k * W + k];
    for (int l = 0; l < m; ++l) {
      M[k * W + l] *= inv;
      X[k * W + l] *= inv;
    }
    for (int i = 0; i < m; ++i) {
      if (i == k) continue;
      const double f = M[i * W + k];
      for (int l = 0; l < m; ++l) {
        M[i * W + l] = fma(-f, M[k * W + l], M[i * W + l]);
        X[i * W + l] = fma(-f, X[k * W + l], X[i * W + l]);
      }
    }
  }
}

// Several nonlinear resistors in the CTA (m >= 2), the compensation method
// with the Thevenin matrix R = A^T Z: with each element on a segment's line
// i = c0 + slope u, the currents solve (I + D R) c = c0 + D y, D =
// diag(slope), y = A^T v0 (v0 the linear solution), i.e. c = a + B y and
// the element voltages u = y - R c = E y - f, with M = (I + D R)^-1,
// a = M c0, B = M D, E = I - R B, f = R a, all fixed while the segments are;
// each element is moved to the segment its voltage lies on until none
// moves, starting from the last step's segments; then v -= Z c.  Warp 0,
// lane j = element j; M is kept while the slopes stay (a sign change keeps
// them), a, B, E, f while the segments stay.  Every thread of the CTA calls
// it (two barriers inside).
__device__ void compensate_multi(const FwdParams& P, int n, int m, NlState* s, double* vv, const int* recp,
                                 int* seg_g, int sidx, long long step, int* abort_flag) {
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31;
  const double* z = s->z();
  const float* zl = s->zl(n, m);
  constexpr int W = kNlMaxPerSub;
  if (tid < 32) {
    if (s->dirty) {   // a newly loaded matrix: its Thevenin matrix
      if (lane < m * m) {
        const int j = lane / m, l = lane - j * m;
        const NlDev& q = s->q[j];
        const double* zc = z + (size_t)l * n;
        const float* zlc = zl + (size_t)l * n;
        const double a = q.k >= 0 ? zc[q.k] + (double)zlc[q.k] : 0.0;
        const double b = q.m >= 0 ? zc[q.m] + (double)zlc[q.m] : 0.0;
        s->R[j * W + l] = a - b;
      }
      __syncwarp();
      if (lane == 0) {
        s->dirty = 0;
        s->minv_key = -1;
        s->coef_key = -1;
      }
      __syncwarp();
    }
    double y = 0.0;
    if (lane < m) {
      const NlDev& q = s->q[lane];
      y = (q.k >= 0 ? vv[q.k] : 0.0) - (q.m >= 0 ? vv[q.m] : 0.0);
    }
    double yl[W];   // every element's y on every lane (0 past the m elements)
#pragma unroll
    for (int l = 0; l < W; ++l) yl[l] = __shfl_sync(0xffffffffu, y, l);
    bool settled = false;
    double cc = 0.0;
    for (int it = 0; it < 32 && !settled; ++it) {
      int key = 0, full = 0;
      for (int j = 0; j < m; ++j) {
        key |= (abs(s->seg[j]) - 1) << (4 * j);
        full |= (s->seg[j] + 9) << (5 * j);   // with the signs
      }
      if (full != s->coef_key) {   // new segments: M (if the slopes changed), then a, B, E, f
        if (key != s->minv_key) {
          if (lane == 0) {
            nl_invert(s, m);
            s->minv_key = key;
          }
          __syncwarp();
        }
        if (lane < m) {
          const NlDev& q = s->q[lane];
          const int sg = s->seg[lane], jj = abs(sg) - 1;
          const double c0 = fma(-q.sl[jj], q.bv[jj], q.bi[jj]);
          s->c0[lane] = sg < 0 ? -c0 : c0;
          s->slope[lane] = q.sl[jj];
        }
        __syncwarp();
        if (lane < m) {
          double a = 0.0;
          for (int l = 0; l < W; ++l) {
            if (l < m) a = fma(s->minv[lane * W + l], s->c0[l], a);
            s->B[lane * W + l] = l < m ? s->minv[lane * W + l] * s->slope[l] : 0.0;
          }
          s->a[lane] = a;
        }
        __syncwarp();
        if (lane < m) {
          double f = 0.0;
          for (int l = 0; l < W; ++l) {
            if (l < m) f = fma(s->R[lane * W + l], s->a[l], f);
            double rb = 0.0;
            for (int p = 0; p < m; ++p) rb = fma(s->R[lane * W + p], s->B[p * W + l], rb);
            s->E[lane * W + l] = l < m ? (lane == l ? 1.0 : 0.0) - rb : 0.0;
          }
          s->f[lane] = f;
        }
        __syncwarp();
        if (lane == 0) s->coef_key = full;
        __syncwarp();
      }
      // c = a + B y and u = E y - f: two independent dot products per lane
      double c = 0.0, u = 0.0;
      if (lane < m) {   // (B and E are zero past the m elements)
        c = s->a[lane];
        u = -s->f[lane];
#pragma unroll
        for (int l = 0; l < W; ++l) {
          c = fma(s->B[lane * W + l], yl[l], c);
          u = fma(s->E[lane * W + l], yl[l], u);
        }
      }
      int sg = 0;
      bool moved = false;
      if (lane < m) {
        sg = nl_segment_of(s->q[lane], u);
        moved = sg != s->seg[lane];
      }
      if (__any_sync(0xffffffffu, moved)) {
        __syncwarp();
        if (lane < m) s->seg[lane] = sg;
        __syncwarp();
      } else {
        settled = true;
        cc = c;
      }
    }
    if (lane < m) {
      s->cur[lane] = cc;
      seg_g[lane] = s->seg[lane];
    }
    if (!settled && lane == 0) {
      if (atomicCAS(P.err, 0, kErrNoSegments) == 0) {
        P.err[1] = sidx;
        P.err[2] = -1;
        P.err[3] = (int)step;
      }
      *abort_flag = 1;
    }
  }
  __syncthreads();
  const long long row = s->row;
  double cur[W];
#pragma unroll
  for (int j = 0; j < W; ++j) cur[j] = j < m ? s->cur[j] : 0.0;
  for (int r = tid; r < n; r += T) {   // the remainders' products first (each column's conversion on the integer pipe)
    double lo = 0.0, hi = vv[r];
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (j < m) {
        lo = fma(f64_of(zl[(size_t)j * n + r]), cur[j], lo);
        hi = fma(-z[(size_t)j * n + r], cur[j], hi);
      }
    const double v = hi - lo;
    vv[r] = v;
    if (row >= 0 && recp[r] >= 0) P.rec[EMT_CHK(P.err, (row - P.rec_row0) * P.n_rec + recp[r], P.bnd.rec, kChkRecord)] = v;
  }
  __syncthreads();
}

// A frequency-dependent line end's history at step m, folded by the poll
// lane that just collected its ring value w_far(m - d) (so the fold of an
// early value hides behind the wait for a late one): W(m) interpolated like
// a mode, A's pole terms z_i(m) = lam z_i(m-1) + mu (W(m) + W(m-1)), and
// b(m) = a0 W(m) + sum z_i into its b slot.  sx = the end's states (z at
// 4..7, W(m-1) at 9).
struct FdFold {
  const int* lefd;          // per line end: FD end or -1 (nullptr: none in this subsystem)
  const FdEndDev* fdr;
  double* fdst;
  const double* lef;
  const double* blk_old;    // the previous step's collected values
  int b_base;               // first b slot in the parity block
};

__device__ __forceinline__ void fold_fd_end(const FdFold& F, int e, double w_new, double* blk_new) {
  const int x = F.lefd[e];
  if (x < 0) return;
  const FdEndDev& r = F.fdr[x];
  double* sx = F.fdst + kFdState * x;
  const double W = fma(F.lef[e], F.blk_old[e], r.omf * w_new);
  const double ws = W + sx[9];
  double zsum = 0.0;
  for (int i = 0; i < r.na; ++i) {
    const double z = fma(r.lam_a[i], sx[4 + i], r.mu_a[i] * ws);
    sx[4 + i] = z;
    zsum = i == 0 ? z : zsum + z;
  }
  sx[9] = W;
  blk_new[F.b_base + x] = fma(r.a0, W, zsum);
}

// One warp collects one step's line-end histories I_e(n) from the tagged
// rings.  Bounded: on exceeding the time budget (or seeing another CTA's
// error) it latches an error and returns false.
// One warp collects the values of step `tag` of every line end (the first
// step of a launch; frequency-dependent ends folded on arrival).
__device__ bool collect_lines(const FwdParams& P, int n_le, unsigned tag, int lane, int sidx, const long long* leown,
                              const int* ledepth, int* rslot, double* ie, const FdFold& F) {
  bool ok = true;
  for (int e = lane; e < n_le && ok; e += 32) {
    const bool fd = F.lefd != nullptr && F.lefd[e] >= 0;
    double v = 0.0;
    ok = poll_slot(P, P.ring + 2 * EMT_CHK(P.err, leown[e] + rslot[e], P.bnd.ring, kChkRingRead), tag, sidx, e, v);
    ie[e] = v;
    if (ok && fd) fold_fd_end(F, e, v, ie);
    const int nx = rslot[e] + 1;
    rslot[e] = nx == ledepth[e] ? 0 : nx;
  }
  return __all_sync(0xffffffffu, ok);
}

// Two builds: at most 64 registers per thread (four CTAs per SM, for
// networks of many subsystems) and at most 128 (two per SM): the second
// keeps more of the step loop's state in registers and is used whenever its
// residency holds every CTA.
// kExt: the network has subsystems that factorise their switch states at
// run time or hold several nonlinear resistors; kGrp: it has
// frequency-dependent line groups (the code for each is compiled only into
// the instances that need it, so that the step loop of every other network
// keeps its registers and its schedule).
template <int kMinBlocks, bool kExt, bool kGrp>
__global__ void __launch_bounds__(kFwdThreads, kMinBlocks) fwd_kernel(FwdParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_abort;
  constexpr int kRs = kExt ? kMaxLazySwitches : kMaxRuntimeSwitches;
  __shared__ RuntimeSwitchDev s_rs[kRs];
  __shared__ double s_rsi[kRs];   // breaker currents of the previous step
  __shared__ int s_rsbit[kRs];    // states decided for the next step
  __shared__ int s_slot, s_fp, s_fsing;        // run-time factorisation: cache slot, pivot, singular flag
  const FwdSmem L = fwd_smem(P.lim);
  const int inp_len = (int)fwd_inp_len(P.lim);
  (void)inp_len;
  double* gi_buf = reinterpret_cast<double*>(smem_raw + L.gi);
  double* part = reinterpret_cast<double*>(smem_raw + L.part);
  double* iv = reinterpret_cast<double*>(smem_raw + L.iv);
  double* vv = reinterpret_cast<double*>(smem_raw + L.vv);
  double* inp = reinterpret_cast<double*>(smem_raw + L.inp);
  double* vs = reinterpret_cast<double*>(smem_raw + L.vs);     // [2][src]
  double* lce = reinterpret_cast<double*>(smem_raw + L.lce);
  double* sbg = reinterpret_cast<double*>(smem_raw + L.sbg);
  double* ley2 = reinterpret_cast<double*>(smem_raw + L.ley2);
  long long* leown = reinterpret_cast<long long*>(smem_raw + L.leown);
  long long* lefar = reinterpret_cast<long long*>(smem_raw + L.lefar);
  float* gilo_buf = reinterpret_cast<float*>(smem_raw + L.gilo);
  float* ivf = reinterpret_cast<float*>(smem_raw + L.ivf);
  float* partf = reinterpret_cast<float*>(smem_raw + L.partf);   // X_lo partial sums per task
  int* lck = reinterpret_cast<int*>(smem_raw + L.lck);
  int* lcm = reinterpret_cast<int*>(smem_raw + L.lcm);
  int* lckind = reinterpret_cast<int*>(smem_raw + L.lckind);
  int* lcstr = reinterpret_cast<int*>(smem_raw + L.lcstr);
  int* sbsrc = reinterpret_cast<int*>(smem_raw + L.sbsrc);
  int* lenode = reinterpret_cast<int*>(smem_raw + L.lenode);
  int* ledepth = reinterpret_cast<int*>(smem_raw + L.ledepth);
  int* led = reinterpret_cast<int*>(smem_raw + L.led);
  int* rslot = reinterpret_cast<int*>(smem_raw + L.rslot);
  int* wslot = reinterpret_cast<int*>(smem_raw + L.wslot);
  int* ent = reinterpret_cast<int*>(smem_raw + L.ent);
  int* ilnode = reinterpret_cast<int*>(smem_raw + L.ilnode);
  int* ilcnt = reinterpret_cast<int*>(smem_raw + L.ilcnt);
  int* srcg = reinterpret_cast<int*>(smem_raw + L.srcg);
  int* recp = reinterpret_cast<int*>(smem_raw + L.recp);    // per node: record column or -1
  double* lef = reinterpret_cast<double*>(smem_raw + L.lef);        // per line end: fractional delay
  double* imode = reinterpret_cast<double*>(smem_raw + L.imode);    // [2][le]: modal histories by parity
  double* ceti = reinterpret_cast<double*>(smem_raw + L.ceti);      // per coupled end: T_i
  double* cetinv = reinterpret_cast<double*>(smem_raw + L.cetinv);  // per coupled end: T_v^-1
  int* lece = reinterpret_cast<int*>(smem_raw + L.lece);            // per line end: coupled end or -1
  int* lemode = reinterpret_cast<int*>(smem_raw + L.lemode);
  int* cele0 = reinterpret_cast<int*>(smem_raw + L.cele0);
  int* cenode = reinterpret_cast<int*>(smem_raw + L.cenode);
  CtrlDev* cbr = reinterpret_cast<CtrlDev*>(smem_raw + L.cbr);      // control blocks, by layer
  double* cy = reinterpret_cast<double*>(smem_raw + L.cy);          // [cb + 1][2]: outputs by step parity, zero pair
  double* cs = reinterpret_cast<double*>(smem_raw + L.cs);          // [cb][2]: block states
  int* clay = reinterpret_cast<int*>(smem_raw + L.clay);            // layer starts and types
  int* cinj = reinterpret_cast<int*>(smem_raw + L.cinj);            // block slot per control injection
  FdEndDev* fdr = reinterpret_cast<FdEndDev*>(smem_raw + L.fdr);   // frequency-dependent line ends
  double* fdst = reinterpret_cast<double*>(smem_raw + L.fdst);      // their states (kFdState each)
  int* lefd = reinterpret_cast<int*>(smem_raw + L.lefd);            // per line end: FD end or -1
  int* cecnt = reinterpret_cast<int*>(smem_raw + L.cecnt);          // per coupled end: modes collected this step

  // the subsystem this CTA runs: its description P.sub[blockIdx.x], its index in
  // the network sidx0 (kept in shared memory: a register held through the step
  // loop would cost the narrow instance a spill)
  __shared__ int s_sidx;
  const int sidx0 = P.active != nullptr ? P.active[blockIdx.x] : (int)blockIdx.x;
  s_sidx = sidx0;   // every thread stores the same value and reads back its own store
  const SubDev S = P.sub[blockIdx.x];
#define SIDX (*(volatile int*)&s_sidx)
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = S.n, Q = S.q, n_str = S.n_str, nc = n + n_str, ldg = nc | 1;
  const int blk = (nc + Q - 1) / Q;   // columns per matvec task
  const int n_lc = S.n_lc, n_sb = S.n_sb, n_le = S.n_le, n_il = S.n_il, n_ce = S.n_ce;
  const int ie_base = n_lc + n_sb;
  const int n_fd = S.n_fd;
  const int fd_base = n_le + 3 * n_ce;   // b values of the FD ends within a parity block
  const int blk_len = n_le + 3 * n_ce + n_fd;   // per parity: line-end values, coupled phase currents, FD b
  const int zero_slot = ie_base + 2 * blk_len;
  const int ci_base = zero_slot + 1;   // controlled currents
  const int n_cb = S.n_cb, n_clay = S.n_clay, n_ci = S.n_ci;
  const int hy_base = ci_base + n_ci;   // Hy of the FD ends
  // with control blocks the warp before the poll warp evaluates them in the
  // update phase, layer by layer; the update items take the other warps
  const int item_threads = n_cb > 0 ? kItemThreads - 32 : kItemThreads;
  const int lv = P.lim.le;
  const int src_vs = P.lim.src;
  const bool writes_lines = sidx0 != P.hold_sub;
  PH_DECL
  const int src_thread = T - 1 - tid;
  // update items: L/C branches, then line ends, then source branches, each
  // block starting on a warp boundary so that a warp runs one kind
  const int it_le = (n_lc + 31) & ~31;
  const int it_sb = it_le + ((n_le + 31) & ~31);
  const int it_end = it_sb + n_sb;

  // ---- prologue: this subsystem's data into shared memory
  for (int x = tid; x < n_lc; x += T) {
    const BranchDev b = P.br[P.lc_idx[S.lc_off + x]];
    inp[x] = P.h[EMT_CHK(P.err, S.lc_off + x, P.bnd.h, kChkHistory)];
    lce[x] = b.e;
    lck[x] = b.k;
    lcm[x] = b.m;
    lckind[x] = b.kind;
    lcstr[x] = -1;
  }
  for (int x = tid; x < n_sb; x += T) {
    const BranchDev b = P.br[P.sb_idx[S.sb_off + x]];
    sbg[x] = b.g;
    sbsrc[x] = b.k <= -2 ? -2 - b.k : -2 - b.m;
  }
  for (int x = tid; x < n_le; x += T) {
    const LineEndDev e = P.le[S.le_off + x];
    ley2[x] = e.y2;
    leown[x] = e.own_ring;
    lefar[x] = e.far_ring;
    lenode[x] = e.node;
    ledepth[x] = e.depth;
    led[x] = e.d;
    rslot[x] = (int)(P.n0 % e.depth);
    wslot[x] = (int)((P.n0 + e.d) % e.depth);
    lef[x] = e.f;
    lece[x] = e.ce;
    lemode[x] = e.mode;
    lefd[x] = e.fd;
    // the value consumed at step n0 - 1 (for interpolated modal histories)
    inp[ie_base + (int)((P.n0 - 1) & 1) * blk_len + x] = P.le_prev[S.le_off + x];
  }
  for (int c = tid; c < n_ce; c += T) {
    const CoupledEndDev& ce = P.ce[S.ce_off + c];
    cecnt[c] = 0;
    reinterpret_cast<int*>(smem_raw + L.cecnt2)[c] = 0;
    cele0[c] = ce.le0;
    for (int k = 0; k < 3; ++k) cenode[3 * c + k] = ce.node[k];
    for (int k = 0; k < 9; ++k) {
      ceti[9 * c + k] = ce.ti[k];
      cetinv[9 * c + k] = ce.tinv[k];
    }
  }
  for (int x = tid; x < n_cb; x += T) {
    cbr[x] = P.cb[S.cb_off + x];
    cs[2 * x] = P.cstate[2 * (size_t)(S.cb_off + x)];
    cs[2 * x + 1] = P.cstate[2 * (size_t)(S.cb_off + x) + 1];
    cy[2 * x + (int)((P.n0 - 1) & 1)] = P.cy[S.cb_off + x];
  }
  if (tid < 2 && n_cb > 0) cy[2 * n_cb + tid] = 0.0;   // the zero pair read by unused inputs
  for (int x = tid; x < (n_cb > 0 ? n_clay + 1 : 0); x += T) clay[x] = P.clay[S.clay_off + x];
  for (int x = tid; x < n_ci; x += T) {
    const int b = P.cinj[S.ci_off + x];
    cinj[x] = b;
    inp[ci_base + x] = P.cy[S.cb_off + b];   // the last step's output drives this step
  }
  for (int x = tid; x < n_fd; x += T) {
    fdr[x] = P.fd[S.fd_off + x];
    for (int k = 0; k < kFdState; ++k) fdst[kFdState * x + k] = P.fd_state[kFdState * (size_t)(S.fd_off + x) + k];
    inp[hy_base + x] = P.fd_state[kFdState * (size_t)(S.fd_off + x) + 10];
  }
  for (int r = tid; r < n; r += T) recp[r] = P.rec != nullptr ? P.rec_pos[S.node_off + r] : -1;
  for (int x = tid; x < 4 * n_il; x += T) ent[x] = P.ent[4 * (size_t)S.il_off + x];
  for (int x = tid; x < n_il; x += T) {
    ilnode[x] = P.il_node[S.il_off + x];
    ilcnt[x] = P.il_cnt[S.il_off + x];
  }
  for (int x = tid; x < S.n_src; x += T) {
    srcg[x] = P.src_global[S.src_off + x];
    vs[(P.n0 & 1) * src_vs + x] = P.src_table[EMT_CHK(P.err, P.src_global[S.src_off + x], P.bnd.src, kChkSource)];
  }
  if (tid == 0) {
    inp[zero_slot] = 0.0;
    s_abort = 0;
  }
  // solve matrix: switch epoch te (by step) and runtime-switch state word
  const int n_rs = S.n_rs, n_states = S.n_states, n_te = S.n_ep / n_states;
  int word = n_rs > 0 ? P.rs_word[SIDX] : 0;
  for (int x = tid; x < n_rs; x += T) {
    s_rs[x] = P.rs[S.rs_off + x];
    s_rsi[x] = P.rs_prev_i[S.rs_off + x];
    s_rsbit[x] = (word >> x) & 1;
  }
  int te = 0;
  while (te + 1 < n_te && P.ep[S.ep_off + (te + 1) * n_states].start <= P.n0) ++te;
  long long next_ep_start = (te + 1 < n_te) ? P.ep[S.ep_off + (te + 1) * n_states].start : LLONG_MAX;
  // Solve-matrix buffers: with two, the previous state's matrix stays
  // resident, so a switch that goes back and forth reloads nothing.
  const size_t buf_len = (size_t)P.lim.n * (size_t)(P.lim.nc | 1);
  int cur_buf = 0;
  int tag_cur = -1, tag_other = -1;   // solve-matrix entries (or cache slots) held by the two buffers
  double* gi = gi_buf;
  float* gilo = gilo_buf;
  // A subsystem with more runtime switches than are prefactored keeps its
  // solve matrices in a cache of slots: the slot of (epoch te, state word),
  // factorised by the CTA into the slot (shared-memory buffer wbuf as the
  // workspace) when the state is met for the first time; -1 if singular.
  auto lazy_slot = [&](int te_, int word_, int wbuf, bool& factored) -> int {
    factored = false;
    const long long key = ((long long)te_ << 32) | (unsigned)word_;
    if (tid == 0) {
      int f = -1;
      for (int j = 0; j < S.n_cache && f < 0; ++j)
        if (P.cache_tag[S.cache_slot0 + j] == key) f = j;
      if (f < 0) {   // replace the next slot in turn
        f = P.cache_next[SIDX];
        P.cache_next[SIDX] = f + 1 == S.n_cache ? 0 : f + 1;
        P.cache_tag[S.cache_slot0 + f] = -1;
        s_slot = -1 - f;
      } else {
        s_slot = f;
      }
    }
    __syncthreads();
    int slot = s_slot;
    if (slot >= 0) return slot;
    slot = -1 - slot;
    factored = true;
    const EpochDev E = P.ep[S.ep_off + te_];
    FactorJob J;
    J.S = S;
    J.sw = P.sw + E.sw_off;
    J.n_sw = E.n_sw;
    J.rs = P.rs;
    J.rs_word = word_;
    J.br = P.br;
    J.le = P.le;
    J.ce = P.ce;
    J.lc_idx = P.lc_idx;
    J.str_slot = P.str_slot;
    J.nl = P.nl;
    J.rb0 = J.rb1 = J.rl0 = J.rl1 = 0;
    J.rm_br = J.rm_le = nullptr;
    J.out = P.ginv_rw + S.cache_goff + (int64_t)slot * n * nc;
    J.out_lo = P.ginv_lo_rw + S.cache_goff + (int64_t)slot * n * nc;
    J.nlz = S.n_nl > 0 ? P.nlz_rw + S.cache_zoff + (int64_t)slot * S.n_nl * n : nullptr;
    J.nlz_lo = S.n_nl > 0 ? P.nlz_lo_rw + S.cache_zoff + (int64_t)slot * S.n_nl * n : nullptr;
    J.Gw = P.lazy_work + S.work_off;
    J.Rw = J.Gw + (size_t)n * n;
    // workspaces: the buffer the matrix is loaded into next, and the solve's partial sums
    if (factor_cta(J, gi_buf + wbuf * buf_len, part, reinterpret_cast<int*>(partf), &s_fp, &s_fsing)) {
      if (tid == 0 && atomicCAS(P.err, 0, 2) == 0) {   // EMT_ESINGULAR, subsystem, -, epoch
        P.err[1] = SIDX;
        P.err[2] = word_;
        P.err[3] = te_;
      }
      return -1;
    }
    if (tid == 0) {
      P.cache_tag[S.cache_slot0 + slot] = key;
      atomicAdd(P.cache_next + P.n_sub, 1);   // run-time factorisations so far (the counter after the slots)
    }
    return slot;
  };
  const bool lazy = kExt && S.n_cache > 0;
  {
    bool factored;
    const int entry = lazy ? lazy_slot(te, word, 0, factored) : te * n_states + word;
    if (entry < 0) {
      if (tid == 0) s_abort = 1;
    } else {
      tag_cur = entry;
      const int64_t off =
          EMT_CHK_BLOCK(P.err, lazy ? S.cache_goff + (int64_t)entry * n * nc : P.ep[S.ep_off + entry].ginv_off,
                        n * nc, P.bnd.ginv, kChkMatrix);
      for (int i = tid; i < n * nc; i += T) {
        const int r = i / nc, c = i - r * nc;
        gi[r * ldg + c] = P.ginv[off + i];
        gilo[r * ldg + c] = P.ginv_lo[off + i];
      }
    }
  }
  // nonlinear resistor: its record and the column of the current matrix;
  // its constants are (re)computed before the first compensation after a load
  const int n_nl = S.n_nl;
  if (n_nl > 0 && tag_cur >= 0) {
    NlState* nls = reinterpret_cast<NlState*>(smem_raw + fwd_smem(P.lim).nls);
    for (int x = tid; x < n_nl; x += T) nls->q[x] = P.nl[S.nl_off + x];
    if (kExt)   // several elements: their segments of the last step
      for (int x = tid; x < n_nl; x += T) nls->seg[x] = P.nl_seg[S.nl_off + x];
    if (tid == 0) {
      nls->dirty = 1;
      nls->m = n_nl;
      nls->minv_key = -1;
    }
    const int64_t zoff =
        EMT_CHK_BLOCK(P.err, lazy ? S.cache_zoff + (int64_t)tag_cur * n_nl * n : P.ep[S.ep_off + tag_cur].nlz_off,
                      n_nl * n, P.bnd.nlz, kChkNlColumn);
    for (int i = tid; i < n_nl * n; i += T) {   // one column per element
      nls->z()[i] = P.nlz[zoff + i];
      nls->zl(n, n_nl)[i] = P.nlz_lo[zoff + i];
    }
  }
  __syncthreads();
  for (int x = tid; x < n_sb; x += T) inp[n_lc + x] = sbg[x] * vs[(P.n0 & 1) * src_vs + sbsrc[x]];
  // frequency-dependent line groups: the modes' Hy (kept modal in the state) into the phase slots, T_i Hy
  for (int c = tid; c < (kGrp && n_fd > 0 ? n_ce : 0); c += T) {
    const int e0 = cele0[c];
    if (lefd[e0] < 0) continue;   // (a coupled Bergeron end)
    const double h0 = fdst[kFdState * lefd[e0] + 10], h1 = fdst[kFdState * lefd[e0 + 1] + 10],
                 h2 = fdst[kFdState * lefd[e0 + 2] + 10];
    for (int p = 0; p < 3; ++p) {
      const double* ti = ceti + 9 * c + 3 * p;
      inp[hy_base + lefd[e0 + p]] = fma(ti[0], h0, fma(ti[1], h1, ti[2] * h2));
    }
  }
  for (int t = tid; t < n_str; t += T) {
    const int x = P.str_slot[S.str_off + t];
    lcstr[x] = t;
    iv[n + t] = -inp[x];
    ivf[n + t] = (float)(-inp[x]);
  }
  if (warp == kPollWarp && n_le > 0) {
    const int p0 = (int)(P.n0 & 1);
    const FdFold F{n_fd > 0 ? lefd : nullptr, fdr, fdst, lef, inp + ie_base + (p0 ^ 1) * blk_len, fd_base};
    const bool ok = collect_lines(P, n_le, (unsigned)P.n0, lane, SIDX, leown, ledepth, rslot,
                                  inp + ie_base + p0 * blk_len, F);
    if (!ok && lane == 0) s_abort = 1;
    if (n_ce > 0)
      fold_modes(lane, n_le, n_ce, lece, lef, inp + ie_base + (p0 ^ 1) * blk_len, inp + ie_base + p0 * blk_len,
                 imode + p0 * lv, cele0, ceti, kGrp && n_fd > 0 ? lefd : nullptr, fd_base);
  }
  // control layer starts 0..31 in the control warp's registers (lane l)
  int lay_reg = 0;
  if (n_cb > 0 && lane <= n_clay) lay_reg = clay[lane];
  // recording counters: steps decim, 2 decim, ... go to rows 0, 1, ...
  const int decim = P.rec_decim > 0 ? P.rec_decim : 1;
  int dec = (int)(P.n0 % decim);
  long long rec_row = P.n0 / decim - (dec == 0 ? 1 : 0);
  __syncthreads();

  const long long n_end = P.n0 + P.n_steps;
  for (long long step = P.n0; step < n_end && !s_abort; ++step) {
    const int par = (int)(step & 1);
    const double* vsc = vs + par * src_vs;
    const int parshift = par * blk_len;
    // runtime-switch states decided from the previous step's solution
    int new_word = 0;
    for (int j = 0; j < n_rs; ++j) new_word |= s_rsbit[j] << j;
    if (P.word_tape != nullptr && tid == 0) P.word_tape[(step - 1 - P.word_row0) * P.n_sub + SIDX] = new_word;
    if (step >= next_ep_start || new_word != word) {
      while (te + 1 < n_te && P.ep[S.ep_off + (te + 1) * n_states].start <= step) ++te;
      next_ep_start = (te + 1 < n_te) ? P.ep[S.ep_off + (te + 1) * n_states].start : LLONG_MAX;
      word = new_word;
      int entry = te * n_states + word;
      if (lazy) {
        // a miss factorises into the buffer loaded next (whose copy is then
        // stale) and replaces a slot (whose copies are then stale)
        const int wbuf = P.lim.nbuf > 1 ? (cur_buf ^ 1) : cur_buf;
        bool factored;
        entry = lazy_slot(te, word, wbuf, factored);
        if (entry < 0) {
          if (tid == 0) s_abort = 1;
          __syncthreads();
          break;
        }
        if (factored) {
          if (P.lim.nbuf > 1) tag_other = -1;
          else tag_cur = -1;
          if (entry == tag_cur) tag_cur = -1;
          if (entry == tag_other) tag_other = -1;
        }
      }
      if (entry != tag_cur) {
        if (n_nl > 0) {   // the nonlinear resistors' columns follow the matrix
          NlState* nls = reinterpret_cast<NlState*>(smem_raw + fwd_smem(P.lim).nls);
          const int64_t zoff =
              EMT_CHK_BLOCK(P.err, lazy ? S.cache_zoff + (int64_t)entry * n_nl * n : P.ep[S.ep_off + entry].nlz_off,
                            n_nl * n, P.bnd.nlz, kChkNlColumn);
          for (int i = tid; i < n_nl * n; i += T) {
            nls->z()[i] = P.nlz[zoff + i];
            nls->zl(n, n_nl)[i] = P.nlz_lo[zoff + i];
          }
          if (tid == 0) nls->dirty = 1;
        }
        if (P.lim.nbuf > 1) {   // the other buffer: a hit, or overwritten below
          cur_buf ^= 1;
          const int t = tag_cur;
          tag_cur = tag_other;
          tag_other = t;
        }
        gi = gi_buf + cur_buf * buf_len;
        gilo = gilo_buf + cur_buf * buf_len;
        if (entry != tag_cur) {
          tag_cur = entry;
          const int64_t off =
              EMT_CHK_BLOCK(P.err, lazy ? S.cache_goff + (int64_t)entry * n * nc : P.ep[S.ep_off + entry].ginv_off,
                            n * nc, P.bnd.ginv, kChkMatrix);
          for (int i = tid; i < n * nc; i += T) {
            const int r = i / nc, c = i - r * nc;
            gi[r * ldg + c] = P.ginv[off + i];
            gilo[r * ldg + c] = P.ginv_lo[off + i];
          }
        }
      }
    }
    // next step's source voltages: load issued now, stored after process 4
    double vnext = 0.0;
    if (src_thread < S.n_src && step + 1 < n_end)
      vnext = __ldg(P.src_table + EMT_CHK(P.err, (step + 1 - P.n0) * P.n_sources + srcg[src_thread], P.bnd.src,
                                          kChkSource));

    PH_MARK(c0)
#ifdef EMT_PHASE_CLOCKS
    if (step == P.n0 && tid == 0) s_ph_first = c0;
#endif
    // process 2: nodal injections; each lane sums four entries, the node's
    // first lane adds its other lanes' sums
    for (int base = 0; base < n_il; base += T) {
      const int l = base + tid;
      double s = 0.0;
      int node = -1, cnt = 0;
      if (l < n_il) {
        node = ilnode[l];
        cnt = ilcnt[l];
        const int* e4 = ent + 4 * l;
        s = (signed_entry(inp, (unsigned)e4[0], ie_base, blk_len, parshift, P.err, inp_len) +
             signed_entry(inp, (unsigned)e4[1], ie_base, blk_len, parshift, P.err, inp_len)) +
            (signed_entry(inp, (unsigned)e4[2], ie_base, blk_len, parshift, P.err, inp_len) +
             signed_entry(inp, (unsigned)e4[3], ie_base, blk_len, parshift, P.err, inp_len));
      }
      const int wmax = __reduce_max_sync(0xffffffffu, cnt);
      double acc = s;
      for (int j = 1; j < wmax; ++j) {
        const double o = __shfl_down_sync(0xffffffffu, s, j);
        if (j < cnt) acc += o;
      }
      if (cnt > 0) {
        iv[node] = acc;
        ivf[node] = f32_trunc(acc);   // (the X_lo chain's operand: truncation on the integer pipe)
      }
    }
    __syncthreads();
    PH_MARK(c1)

    // process 4: v = (X_hi + X_lo) i; task (r, q) runs one FMA chain over
    // the contiguous column block q (the warp issue rate, not the FMA
    // latency, is the limit; contiguous blocks keep the rounding of the
    // partial sums small, measured over long runs)
    for (int task = tid; task < n * Q; task += T) {
      const int r = task / Q, q = task - r * Q;
      const double* row = gi + r * ldg;
      const float* rowl = gilo + r * ldg;
      const int j1 = min(nc, (q + 1) * blk);
      double a = 0.0;
      float b = 0.f;
#pragma unroll 2   // measured: 2 beats 1, 3 and 4 (the loop is not unrolled by default)
      for (int j = q * blk; j < j1; ++j) {
        a = fma(row[j], iv[j], a);
        b = fmaf(rowl[j], ivf[j], b);
      }
      part[task] = a;
      partf[task] = b;
    }
    if (src_thread < S.n_src) vs[(par ^ 1) * src_vs + src_thread] = vnext;
    __syncthreads();
    PH_MARK(c2)

    // node voltages
    const bool rec_now = P.rec != nullptr && dec == 0 && rec_row < P.rec_rows;
    for (int r = tid; r < n; r += T) {
      // the X_hi partial sums in double, the X_lo ones in single precision
      double v = part[r * Q];
      float vl = partf[r * Q];
      for (int q = 1; q < Q; ++q) {
        v += part[r * Q + q];
        vl += partf[r * Q + q];
      }
      v += f64_of(vl);
      vv[r] = v;
      if (rec_now && recp[r] >= 0)
        P.rec[EMT_CHK(P.err, (rec_row - P.rec_row0) * P.n_rec + recp[r], P.bnd.rec, kChkRecord)] = v;
    }
    if (n_nl > 0 && tid == 0)   // rewritten after the compensation
      reinterpret_cast<NlState*>(smem_raw + fwd_smem(P.lim).nls)->row = rec_now ? rec_row : -1;
    if (dec == 0) ++rec_row;
    if (++dec == decim) dec = 0;
    __syncthreads();

    // compensation method: the nonlinear resistor against the linear
    // solution, its current from the Thevenin source, then v -= z i
    if (n_nl == 1) {
      compensate(P, n, reinterpret_cast<NlState*>(smem_raw + fwd_smem(P.lim).nls), vv, recp);
    } else if (kExt && n_nl > 1) {
      compensate_multi(P, n, n_nl, reinterpret_cast<NlState*>(smem_raw + fwd_smem(P.lim).nls), vv, recp,
                       P.nl_seg + S.nl_off, SIDX, step, &s_abort);
      if (s_abort) break;
    }
    PH_MARK(c3)

    // process 1: history currents, line outputs, next step's source
    // injections; then the update threads collect next step's line values
    if (warp == kPollWarp) {
      // (the update threads collect the next step's line values below)
    } else if (n_cb > 0 && warp == kPollWarp - 1) {
      // control blocks at this step, one layer after another; then the
      // controlled currents of the next step
      constexpr int kSlotMask = (1 << kLayerTypeShift) - 1;
      int cur = __shfl_sync(0xffffffffu, lay_reg, 0);
      for (int l = 0; l < n_clay; ++l) {
        const int nxt = l + 1 < 32 ? __shfl_sync(0xffffffffu, lay_reg, l + 1) : clay[l + 1];
        const int lt = cur >> kLayerTypeShift, first = cur & kSlotMask, b1 = nxt & kSlotMask;
        control_slot(first + lane, first, first + lane < b1, lt, cbr, cy, cs, par, vv);
        for (int b = first + 32 + lane; b - lane < b1; b += 32)   // layers wider than a warp
          control_slot(b, first, b < b1, lt, cbr, cy, cs, par, vv);
        cur = nxt;
        __syncwarp();
      }
      for (int c = lane; c < n_ci; c += 32) inp[ci_base + c] = cy[2 * cinj[c] + par];
    } else {
      // runtime switches: the states in force at the next step (oracle rules)
      if (tid < n_rs) {
        const RuntimeSwitchDev r = s_rs[tid];
        const double vb = (r.k >= 0 ? vv[r.k] : 0.0) - (r.m >= 0 ? vv[r.m] : 0.0);
        int bit = (word >> tid) & 1;
        if (r.kind == 0) {
          bit = vb > 0.0 ? 1 : 0;
        } else if (bit) {
          const double i = vb / r.r_on;
          if (step >= r.trip && s_rsi[tid] * i <= 0.0) bit = 0;
          s_rsi[tid] = i;
        }
        s_rsbit[tid] = bit;
      }
      const double* ie_cur = inp + ie_base + parshift;
      const double* vs_next = vs + (par ^ 1) * src_vs;
      // the next step's slot of this thread's first line end, loaded now so
      // that its L2 round trip overlaps the update items (checked after them;
      // a slot written later, by a one-step line, is polled as before).  Not
      // in the line-group builds, whose longer collection it slowed (5.72
      // against 5.54 us per step).
      const int e_pre = kGrp ? -1 : item_threads - 1 - tid;
      unsigned long long pw0 = 0, pw1 = 0;
      if (e_pre >= 0 && e_pre < n_le && step + 1 < n_end)
        ld_tagged_raw(P.ring + 2 * EMT_CHK(P.err, leown[e_pre] + rslot[e_pre], P.bnd.ring, kChkRingRead), pw0, pw1);
      for (int it = tid; it < it_end; it += item_threads) {
        if (it < n_lc) {
          const int k = lck[it], m = lcm[it];
          const double vk = k >= 0 ? vv[k] : (k == -1 ? 0.0 : vsc[-2 - k]);
          const double vm = m >= 0 ? vv[m] : (m == -1 ? 0.0 : vsc[-2 - m]);
          const double vb = vk - vm;
          const double hn = lckind[it] == 1 ? fma(lce[it], vb, inp[it]) : fma(lce[it], vb, -inp[it]);
          inp[it] = hn;
          const int t = lcstr[it];
          if (t >= 0) {   // strong branch: its current drives the extra matvec column
            iv[n + t] = -hn;
            ivf[n + t] = f32_trunc(-hn);
          }
        } else if (it >= it_le && it < it_le + n_le) {
          const int e = it - it_le;
          double out;
          const int c = lece[e], fx = lefd[e];
          if (fx >= 0) {   // frequency-dependent end: Y_c's terms of v, then w = 2 yc - b
            const FdEndDev& r = fdr[fx];
            double* sx = fdst + kFdState * fx;
            double v;
            if (kGrp && c >= 0) {   // a mode of a line group: the modal voltage (T_v^-1 v_phase)_mode
              const double* tr = cetinv + 9 * c + 3 * lemode[e];
              const int* nd = cenode + 3 * c;
              v = fma(tr[0], vv[nd[0]], fma(tr[1], vv[nd[1]], tr[2] * vv[nd[2]]));
            } else {
              v = vv[lenode[e]];
            }
            const double vsum = v + sx[8];
            double ssum = 0.0, lam_s = 0.0;
            for (int i = 0; i < r.ny; ++i) {
              const double si = fma(r.lam_y[i], sx[i], r.mu_y[i] * vsum);
              sx[i] = si;
              ssum = i == 0 ? si : ssum + si;
              lam_s = i == 0 ? r.lam_y[i] * si : fma(r.lam_y[i], si, lam_s);
            }
            const double yc = fma(r.y0, v, ssum);
            out = fma(2.0, yc, -ie_cur[fd_base + fx]);
            sx[8] = v;
            const double hy = fma(r.mu_sum, v, lam_s);   // Hy(n+1)
            sx[10] = hy;
            if (!kGrp || c < 0) {
              inp[hy_base + fx] = hy;
            } else {   // the last of its end's three modes puts T_i Hy_mode into the phase slots
              __threadfence_block();
              int* cnt2 = reinterpret_cast<int*>(smem_raw + fwd_smem(P.lim).cecnt2);
              if (atomicAdd(&cnt2[c], 1) == 2) {
                __threadfence_block();
                cnt2[c] = 0;
                const int e0 = cele0[c];
                const volatile double* st = fdst;
                const double h0 = st[kFdState * lefd[e0] + 10], h1 = st[kFdState * lefd[e0 + 1] + 10],
                             h2 = st[kFdState * lefd[e0 + 2] + 10];
                for (int p = 0; p < 3; ++p) {
                  const double* ti = ceti + 9 * c + 3 * p;
                  inp[hy_base + lefd[e0 + p]] = fma(ti[0], h0, fma(ti[1], h1, ti[2] * h2));
                }
              }
            }
          } else if (c < 0) {
            out = fma(-ley2[e], vv[lenode[e]], -ie_cur[e]);
          } else {   // a mode: c_j = -(2/Z_j) (T_v^-1 v_p)_j - I_mode_j(n)
            const double* tr = cetinv + 9 * c + 3 * lemode[e];
            const int* nd = cenode + 3 * c;
            const double vm = fma(tr[0], vv[nd[0]], fma(tr[1], vv[nd[1]], tr[2] * vv[nd[2]]));
            out = fma(-ley2[e], vm, -imode[par * lv + e]);
          }
          if (writes_lines)
            st_tagged(P.ring + 2 * EMT_CHK(P.err, lefar[e] + wslot[e], P.bnd.ring, kChkRingWrite),
                      (unsigned)(step + led[e]), out);
          const int nx = wslot[e] + 1;
          wslot[e] = nx == ledepth[e] ? 0 : nx;
        } else if (it >= it_sb) {
          const int x = it - it_sb;
          inp[n_lc + x] = sbg[x] * vs_next[sbsrc[x]];
        }
      }
#ifdef EMT_PHASE_CLOCKS
      ph_t0 = (unsigned)clock();
#endif
      // next step's ring values: one update thread per line end, counted
      // from the last thread (the first threads hold the update items), so
      // that all waits run at once and the folds spread over several warps.
      // A coupled end's phase currents are formed by whichever thread
      // collects the last of its three modes.
      if (n_le > 0 && step + 1 < n_end) {
        const unsigned tag = (unsigned)(step + 1);
        double* ie_old = inp + ie_base + par * blk_len;
        double* ie_next = inp + ie_base + (par ^ 1) * blk_len;
        double* imode_next = imode + (par ^ 1) * lv;
        const FdFold F{n_fd > 0 ? lefd : nullptr, fdr, fdst, lef, ie_old, fd_base};
        bool ok = true;
        for (int e = item_threads - 1 - tid; e < n_le && ok; e += item_threads) {
          double v = 0.0;
          if (e != e_pre || !tagged_value(pw0, pw1, tag, v))
            ok = poll_slot(P, P.ring + 2 * EMT_CHK(P.err, leown[e] + rslot[e], P.bnd.ring, kChkRingRead), tag, SIDX,
                           e, v);
          ie_next[e] = v;
          const int nx = rslot[e] + 1;
          rslot[e] = nx == ledepth[e] ? 0 : nx;
          if (!ok) break;
          const int c = lece[e];
          if (c >= 0) {   // a mode: its interpolated history; the third of its end's modes forms T_i I_mode
            if (kGrp && F.lefd != nullptr && F.lefd[e] >= 0) {   // a line group's mode: b folded now, -b its history
              fold_fd_end(F, e, v, ie_next);
              imode_next[e] = -ie_next[F.b_base + F.lefd[e]];
            } else {
              imode_next[e] = fma(lef[e], ie_old[e], (1.0 - lef[e]) * v);
            }
            __threadfence_block();
            if (atomicAdd(&cecnt[c], 1) == 2) {
              __threadfence_block();
              cecnt[c] = 0;
              const volatile double* im = imode_next + cele0[c];
              const double m0 = im[0], m1 = im[1], m2 = im[2];
              for (int p = 0; p < 3; ++p) {
                const double* ti = ceti + 9 * c + 3 * p;
                ie_next[n_le + 3 * c + p] = fma(ti[0], m0, fma(ti[1], m1, ti[2] * m2));
              }
            }
          } else if (F.lefd != nullptr) {
            fold_fd_end(F, e, v, ie_next);
          }
        }
        if (!ok) s_abort = 1;
      }
#ifdef EMT_PHASE_CLOCKS
      ph_t1 = (unsigned)clock();
      if (tid == item_threads - 1) s_ph[4] += ph_t1 - ph_t0;   // the wait of line end 0's poll thread
#endif
    }
    __syncthreads();
    PH_MARK(c5)
    PH_ADD(0, c0, c1)
    PH_ADD(1, c1, c2)
    PH_ADD(2, c2, c3)
    PH_ADD(3, c3, ph_t0)
    PH_ADD(5, ph_t1, c5)
#ifdef EMT_PHASE_CLOCKS
    if (tid == 0) {
      s_ph[6] += 1;
      s_ph[7] = (unsigned)(c5 - s_ph_first);
    }
#endif
  }
#ifdef EMT_PHASE_CLOCKS
  __syncthreads();
  if (SIDX < kPhaseCtas && tid < kPhaseCount) {
    if (tid == 7) g_phase[SIDX][7] = s_ph[7];   // the last launch's span
    else atomicAdd(&g_phase[SIDX][tid], s_ph[tid]);
  }
#endif
  if (!s_abort) {
    for (int b = tid; b < n_lc; b += T) P.h[EMT_CHK(P.err, S.lc_off + b, P.bnd.h, kChkHistory)] = inp[b];
    if (P.n_steps > 0)   // the values consumed at the last step, for the next launch's interpolation
      for (int x = tid; x < n_le; x += T)
        P.le_prev[S.le_off + x] = inp[ie_base + (int)((n_end - 1) & 1) * blk_len + x];
    for (int x = tid; x < n_rs; x += T) P.rs_prev_i[S.rs_off + x] = s_rsi[x];
    if (P.n_steps > 0)   // (the prologue advanced A's terms to step n0, which a launch of 0 steps never ran)
      for (int x = tid; x < n_fd; x += T)
        for (int k = 0; k < kFdState; ++k) P.fd_state[kFdState * (size_t)(S.fd_off + x) + k] = fdst[kFdState * x + k];
    for (int x = tid; x < n_cb; x += T) {
      P.cstate[2 * (size_t)(S.cb_off + x)] = cs[2 * x];
      P.cstate[2 * (size_t)(S.cb_off + x) + 1] = cs[2 * x + 1];
      P.cy[S.cb_off + x] = cy[2 * x + (int)((n_end - 1) & 1)];
    }
    if (n_rs > 0 && tid == 0) {
      int w = 0;
      for (int j = 0; j < n_rs; ++j) w |= s_rsbit[j] << j;
      P.rs_word[SIDX] = w;
    }
  }
}

// ------------------------------------------------------------ gather

__global__ void gather_kernel(const double* rec, int32_t n_rec, int64_t n_scen_rec, const int32_t* col, int64_t n_ch,
                              int64_t row0, int64_t n_rows, int64_t scen0, int64_t n_scen, double* out) {
  const int64_t total = n_rows * n_scen * n_ch;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i % n_ch, rs = i / n_ch;
    const int64_t s = rs % n_scen, r = rs / n_scen;
    out[i] = rec[((row0 + r) * n_scen_rec + scen0 + s) * n_rec + col[c]];
  }
}

}  // namespace

#undef SIDX

cudaError_t launch_ring_init(const RingInitParams& p, cudaStream_t st) {
  if (p.n_le <= 0) return cudaSuccess;
  ring_init_kernel<<<(unsigned)p.n_le, 64, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t phase_clocks(unsigned long long* out, int n, bool reset) {
#ifdef EMT_PHASE_CLOCKS
  const size_t bytes = (size_t)std::min(n, kPhaseCtas) * kPhaseCount * sizeof(unsigned long long);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && out != nullptr && bytes > 0) e = cudaMemcpyFromSymbol(out, g_phase, bytes);
  if (e == cudaSuccess && reset) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_phase);
    if (e == cudaSuccess) e = cudaMemset(p, 0, sizeof(g_phase));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  return e;
#else
  (void)out;
  (void)n;
  (void)reset;
  return cudaErrorNotSupported;
#endif
}

cudaError_t launch_ring_copy(const RingCopyParams& p, cudaStream_t st) {
  const int64_t total = (int64_t)p.n_ends * p.w;
  if (total <= 0) return cudaSuccess;
  const int th = 256;
  const int64_t blocks = std::min<int64_t>((total + th - 1) / th, 148 * 8);
  ring_copy_kernel<<<(unsigned)blocks, th, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_companion(BranchDev* br, int64_t n_br, double dt, cudaStream_t st) {
  if (n_br <= 0) return cudaSuccess;
  const int th = 256;
  companion_kernel<<<(unsigned)((n_br + th - 1) / th), th, 0, st>>>(br, n_br, dt);
  return cudaGetLastError();
}

cudaError_t launch_coupled_constants(CoupledEndDev* ce, int64_t n_ce, cudaStream_t st) {
  if (n_ce <= 0) return cudaSuccess;
  coupled_constants_kernel<<<(unsigned)((n_ce + 127) / 128), 128, 0, st>>>(ce, n_ce);
  return cudaGetLastError();
}

cudaError_t launch_prefactor(const PrefParams& p, int max_n, cudaStream_t st) {
  if (p.n_mats <= 0) return cudaSuccess;
  const size_t smem = (size_t)max_n * max_n * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(prefactor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  prefactor_kernel<<<p.n_mats, 256, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_sources(const SourceParams& p, cudaStream_t st) {
  const int64_t total = p.n_steps * p.n_sources;
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 8);
  source_kernel<<<blocks, 256, 0, st>>>(p);
  return cudaGetLastError();
}

size_t forward_smem_bytes(const FwdLimits& lim) { return fwd_smem(lim).bytes; }

int forward_blocks_per_sm(const FwdLimits& lim) {
  const size_t smem = forward_smem_bytes(lim);
  if (smem > 227 * 1024) return 0;
  if (cudaFuncSetAttribute(fwd_kernel<4, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fwd_kernel<4, false, false>, kFwdThreads, smem) != cudaSuccess)
    return 0;
  return per_sm;
}

cudaError_t launch_forward(const FwdParams& p, cudaStream_t st, bool wide, bool ext, bool grp) {
  const size_t smem = forward_smem_bytes(p.lim);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  // the 128-register build when allowed and its residency holds every CTA, else the 64-register one
  const void* fns[2] = {
      ext ? (grp ? (const void*)fwd_kernel<2, true, true> : (const void*)fwd_kernel<2, true, false>)
          : (grp ? (const void*)fwd_kernel<2, false, true> : (const void*)fwd_kernel<2, false, false>),
      ext ? (grp ? (const void*)fwd_kernel<4, true, true> : (const void*)fwd_kernel<4, true, false>)
          : (grp ? (const void*)fwd_kernel<4, false, true> : (const void*)fwd_kernel<4, false, false>)};
  for (int v = wide ? 0 : 1; v < 2; ++v) {
    cudaError_t e = cudaFuncSetAttribute(fns[v], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[v], kFwdThreads, smem);
    if (e != cudaSuccess) return e;
    const int grid = p.active != nullptr ? p.n_active : p.n_sub;
    if ((long long)per_sm * n_sm < grid) continue;
    FwdParams arg = p;
    void* args[] = {&arg};
    // cooperative launch: all CTAs co-resident, so every ring wait can end
    return cudaLaunchCooperativeKernel(fns[v], dim3(grid), dim3(kFwdThreads), args, smem, st);
  }
  return cudaErrorCooperativeLaunchTooLarge;
}

cudaError_t launch_gather(const double* rec, int32_t n_rec, int64_t n_scen_rec, const int32_t* col, int64_t n_ch,
                          int64_t row0, int64_t n_rows, int64_t scen0, int64_t n_scen, double* out, cudaStream_t st) {
  const int64_t total = n_rows * n_scen * n_ch;
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 16);
  gather_kernel<<<blocks, 256, 0, st>>>(rec, n_rec, n_scen_rec, col, n_ch, row0, n_rows, scen0, n_scen, out);
  return cudaGetLastError();
}

}  // namespace emt
