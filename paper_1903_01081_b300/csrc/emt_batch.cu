// Multi-scenario time loop for sm_103a (B300).
//
// The paper's multi-scenario strategy (Sec. III-B): the scenarios of a
// study share the network structure, so every basic process becomes one
// SIMT operation over all scenarios.  Here one CTA runs the whole network
// for a tile of S_t scenarios; a warp's lanes are (item, scenario) with the
// scenario fastest, so each solve-matrix entry a warp loads serves all its
// scenarios (for a shared G^-1 the solve over the tile is a dense product
// G^-1 [i^(1) ... i^(S_t)], done with DFMA: on B300 the FP64 MMA path shares
// the DFMA pipe and adds no throughput).  A scenario that changes a
// subsystem's G (an element removed, a switch closed) selects its own
// prefactored matrix for that subsystem from the step the change applies.
// Scenarios are independent, so CTAs never wait on each other.
//
// Subsystems exchange values only through lines of delay >= 1, so within
// one step all subsystems of a group run each process together: all
// injections, then all solves, then all updates -- three barriers per
// group and step, and thousands of independent items per phase to hide
// the FP64 and memory latencies.
//
// Formulas as in emt_kernels.cu (trapezoidal companions, Bergeron lines;
// the paper's Sec. III-A processes with the textbook forms of its ref. [2]).
#include <stdint.h>

#include <algorithm>

#include <cuda_runtime.h>

#include "emt_internal.h"
#include "emt_device.cuh"
#include "emt_digits.cuh"

namespace emt {

namespace {

constexpr int kBatchMaxThreads = 1024;
// the digit-form instance takes at most 512 threads (128 registers each: its
// tensor-core loop keeps two accumulator chains and the 64-bit sums live)
constexpr int kBatchDigitThreads = 512;

// ---------------------------------------------------------------- digit form
//
// For a subsystem whose solve matrix X every scenario of the tile shares,
// process 4 over the tile, V = X [i^(1) .. i^(S_t)], is a dense product; it
// runs exactly on the bf16 tensor cores in the digit form of emt_digits.cuh
// (62-bit fixed point, balanced base-256 digits, exact fp32 sums of digit
// products, one rounding to double).  mma.m16n8k16 with M = 16 scenarios
// (the injection digits b, from a shared-memory table), N = 8 rows of X
// (its digits a, prepared once per matrix), K = 16 solve columns; the
// pairs with a + b = u go to one fp32 accumulator (at most 8 pairs of 64
// columns: below 2^23, exact), turned into integers per u.

__device__ __forceinline__ void dg_mma(float* d, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                       unsigned b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ long long dg_shl64(int x, int sh) {
  return (long long)((unsigned long long)(long long)x << sh);
}

// One CTA per matrix: each row as 62-bit fixed point against its own scale
// (X_hi + X_lo), split into digits, written in the B-fragment order
// (dig_matrix_words), then the row exponents.  Padding stays zero.
__global__ void __launch_bounds__(256) batch_digits_kernel(const double* ginv, const float* ginv_lo,
                                                           const int64_t* mat_goff, const int32_t* mat_n,
                                                           const int32_t* mat_nc, const int64_t* mat_doff,
                                                           uint32_t* dig) {
  __shared__ unsigned s_em[kDigRows];
  const int mi = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int n = mat_n[mi], nc = mat_nc[mi], r8n = (n + 7) / 8, ks = (nc + 15) / 16;
  const double* xh = ginv + mat_goff[mi];
  const float* xl = ginv_lo + mat_goff[mi];
  uint32_t* out = dig + mat_doff[mi];
  int* ex = reinterpret_cast<int*>(out + (int64_t)8 * r8n * ks * 64);
  for (int r = tid; r < 8 * r8n; r += T) {
    unsigned em = 1;
    for (int k = 0; r < n && k < nc; ++k)
      em = max(em, max(dg_expo(xh[r * nc + k]), dg_expo((double)xl[r * nc + k])));
    if (r < n) s_em[r] = em;
    ex[r] = (int)em;
  }
  __syncthreads();
  unsigned short* o16 = reinterpret_cast<unsigned short*>(out);
  for (int idx = tid; idx < n * nc; idx += T) {
    const int r = idx / nc, k = idx - r * nc;
    const long long np = dg_fixed(xh[idx], s_em[r]) + dg_fixed((double)xl[idx], s_em[r]) + kDigitBias;
    const int R8 = r >> 3, g = r & 7, st = k >> 4, kk = k & 15, t = (kk & 7) >> 1, half = kk >> 3, el = kk & 1;
    for (int a = 0; a < kDigits; ++a) {
      const int64_t word = ((int64_t)(a * r8n + R8) * ks + st) * 64 + 2 * (4 * g + t) + half;
      o16[2 * word + el] = (unsigned short)dg_digit_bf16(np, a);
    }
  }
}

// Ring slot of step `step` in a ring of depth d1 (steps stay below 2^31).
__device__ __forceinline__ int64_t ring_slot(long long step, int d1) { return (int64_t)((unsigned)step % (unsigned)d1); }

// Signed value of one batched injection entry for scenario sg (tile lane sl).
__device__ __forceinline__ double entry_value(const BatchParams& P, uint32_t raw, int sg, int sl, long long step,
                                              const double* vs) {
  const uint32_t kind = (raw >> kBentKindShift) & 7u;
  const int idx = (int)(raw & kBentIndexMask);
  double val;
  if (kind > 2u) {   // the rarer kinds
    if (kind == 3u)   // a controlled current: its block's output of the previous step
      val = P.cy[(int64_t)(2 * __ldg(P.cinj + idx) + (int)((step - 1) & 1)) * P.S + sg];
    else if (kind == 6u)   // a coupled end's phase history current of this step
      val = P.cph[(int64_t)idx * P.S + sg];
    else   // a frequency-dependent end's b (4) or Hy (5) of this step
      val = P.fds[((int64_t)idx * kBatchFdState + (kind == 4u ? 11 : 10)) * P.S + sg];
  } else if (kind == 0u) {
    val = P.h[EMT_CHK(P.err, (int64_t)idx * P.S + sg, P.bnd.h, kChkHistory)];
  } else if (kind == 1u) {
    val = __ldg(P.sb_g + idx) * vs[__ldg(P.sb_src + idx) * P.S_t + sl];
    if (P.keep_sb && !P.keep_sb[(int64_t)idx * P.S + sg]) val = 0.0;
  } else {
    val = P.ring[EMT_CHK(P.err, (__ldg(P.le_bring + idx) + ring_slot(step, __ldg(P.le_d1 + idx))) * P.S + sg,
                         P.bnd.ring, kChkRingRead)];
  }
  // the sign by flipping the sign bit (integer pipe)
  return __longlong_as_double(__double_as_longlong(val) ^ ((long long)(raw & kEntryNeg) << 32));
}

// Control block g (global slot) for scenario sg at a step of parity par:
// the same formulas as the single-network kernel, with inputs, outputs and
// states per scenario in global memory and, for a block with scenario
// parameters, this scenario's coefficients; MEAS reads the group's node
// voltages (vv, tile lane sl, nodes from node0).
__device__ __forceinline__ void batch_control(const BatchParams& P, int g, int sg, int sl, int par, const double* vv,
                                              int node0, int St) {
  const CtrlDev& r = P.cb[g];
  const int64_t S = P.S;
  double p0 = r.p0, p1 = r.p1, p2 = r.p2;
  if (r.ov >= 0.0) {
    const double* o = P.cbo + ((int64_t)r.ov * S + sg) * 3;
    p0 = o[0];
    p1 = o[1];
    p2 = o[2];
  }
  const double u0 = P.cy[(int64_t)(r.i0 ^ par) * S + sg];
  const double u1 = P.cy[(int64_t)(r.i1 ^ par) * S + sg];
  double* sx = P.cs + (int64_t)(2 * g) * S + sg;   // (y or integral of the last step, u0 of the last step)
  double out;
  switch (r.type) {
    case 0: out = p0; break;
    case 1: out = vv[(size_t)(r.node - node0) * St + sl]; break;
    case 2: out = p0 * u0; break;
    case 3: out = fma(p0, u0, p1 * u1); break;
    case 4: out = p0 * u0 * u1; break;
    case 5: out = u0 < p0 ? p0 : (u0 > p1 ? p1 : u0); break;
    case 6:
      out = fma(p0, u0 + sx[S], sx[0]);
      sx[0] = out;
      sx[S] = u0;
      break;
    case 7:
      out = fma(p1, u0 + sx[S], p0 * sx[0]);
      sx[0] = out;
      sx[S] = u0;
      break;
    default: {
      const double integral = fma(p2, u0 + sx[S], sx[0]);
      out = fma(p1, integral, p0 * u0);
      sx[0] = integral;
      sx[S] = u0;
      break;
    }
  }
  P.cy[(int64_t)(2 * g + par) * S + sg] = out;
}

// Nonlinear resistor e for tile lane sl: the Thevenin voltage from the
// linear solution vv, R_th from the column z of the scenario's current
// matrix (after the matrix in ginv), then the segment j of the odd
// piecewise-linear f whose image u + R_th f(u) holds |v_th| (images of the
// breakpoints compared, no division), u on it and i = f(u) with v_th's sign.
__device__ __forceinline__ double batch_nl_current(const BatchParams& P, int e, int sl, const long long* cur,
                                                   const double* vv, int node0, int St) {
  const NlDev& q = P.nl[e];
  const int s = __ldg(P.nlinfo + 4 * e), n = __ldg(P.nlinfo + 4 * e + 1), node_off = __ldg(P.nlinfo + 4 * e + 2);
  const int64_t zoff =
      EMT_CHK_BLOCK(P.err, cur[(size_t)sl * P.n_sub + s] + (int64_t)n * __ldg(P.sub_nc + s), n, P.bnd.ginv, kChkNlColumn);
  const double* z = P.ginv + zoff;
  const float* zl = P.ginv_lo + zoff;
  const double vk = q.k >= 0 ? vv[(size_t)(node_off + q.k - node0) * St + sl] : 0.0;
  const double vm = q.m >= 0 ? vv[(size_t)(node_off + q.m - node0) * St + sl] : 0.0;
  const double zk = q.k >= 0 ? z[q.k] + (double)zl[q.k] : 0.0;
  const double zm = q.m >= 0 ? z[q.m] + (double)zl[q.m] : 0.0;
  const double R = zk - zm, vth = vk - vm, x = fabs(vth);
  int j = 0;
  while (j < q.np && x >= fma(R, q.bi[j + 1], q.bv[j + 1])) ++j;
  const double u = (x - R * fma(-q.sl[j], q.bv[j], q.bi[j])) / fma(R, q.sl[j], 1.0);
  const double i = fma(q.sl[j], u - q.bv[j], q.bi[j]);
  return vth < 0.0 ? -i : i;
}

// The far end's w of step m from this FD end's ring (depth d + 2); 0 before step 1.
__device__ __forceinline__ double fd_ring_w(const BatchParams& P, int ge, long long m, int sg) {
  if (m < 1) return 0.0;
  const int depth = __ldg(P.le_d1 + ge) + 1;
  return P.ring[EMT_CHK(P.err, (__ldg(P.le_bring + ge) + (int64_t)((unsigned long long)m % (unsigned)depth)) * P.S + sg,
                        P.bnd.ring, kChkRingRead)];
}

// FD end x at the start of step n (scenario sg): b(n) and the A terms.
__device__ __forceinline__ void batch_fd_fold(const BatchParams& P, int x, int sg, long long step) {
  const FdEndDev& r = P.fd[x];
  const int ge = __ldg(P.fd_le + x);
  const int d = __ldg(P.le_d1 + ge) - 1;
  const int64_t S = P.S;
  double* st = P.fds + (int64_t)x * kBatchFdState * S + sg;
  const double w_new = fd_ring_w(P, ge, step - d, sg), w_old = fd_ring_w(P, ge, step - d - 1, sg);
  const double W = fma(1.0 - r.omf, w_old, r.omf * w_new);
  const double ws = W + st[9 * S];
  double zsum = 0.0;
  for (int i = 0; i < r.na; ++i) {
    const double z = fma(r.lam_a[i], st[(4 + i) * S], r.mu_a[i] * ws);
    st[(4 + i) * S] = z;
    zsum = i == 0 ? z : zsum + z;
  }
  st[9 * S] = W;
  st[11 * S] = fma(r.a0, W, zsum);
}

// FD end x (line end ge) after the solve of step n: Y_c's terms of v, the
// line output w = 2 yc - b into the far end's ring, and Hy(n+1).
__device__ __forceinline__ void batch_fd_update(const BatchParams& P, int ge, int x, int sg, long long step, double v) {
  const FdEndDev& r = P.fd[x];
  const int64_t S = P.S;
  double* st = P.fds + (int64_t)x * kBatchFdState * S + sg;
  const double vsum = v + st[8 * S];
  double ssum = 0.0, lam_s = 0.0;
  for (int i = 0; i < r.ny; ++i) {
    const double si = fma(r.lam_y[i], st[i * S], r.mu_y[i] * vsum);
    st[i * S] = si;
    ssum = i == 0 ? si : ssum + si;
    lam_s = i == 0 ? r.lam_y[i] * si : fma(r.lam_y[i], si, lam_s);
  }
  const double yc = fma(r.y0, v, ssum);
  const double w = fma(2.0, yc, -st[11 * S]);
  const int depth = __ldg(P.le_d1 + ge) + 1;
  P.ring[EMT_CHK(P.err, (__ldg(P.le_bfar + ge) + (int64_t)((unsigned long long)step % (unsigned)depth)) * S + sg,
                 P.bnd.ring, kChkRingWrite)] = w;
  st[8 * S] = v;
  st[10 * S] = fma(r.mu_sum, v, lam_s);
}

// Coupled end x at the start of step n (scenario sg): mode j's history
// I_j(n) = (1 - f_j) c_j(n - d_j) + f_j c_j(n - d_j - 1) from the far end's
// values in its ring, then the phase history currents T_i I.
__device__ __forceinline__ void batch_ce_fold(const BatchParams& P, int x, int sg, long long step) {
  const CoupledEndDev& r = P.ce[x];
  const int64_t S = P.S;
  const int ge0 = __ldg(P.ce_le0 + x);
  double im[3];
  for (int j = 0; j < 3; ++j) {
    const int ge = ge0 + j, d = __ldg(P.le_d1 + ge) - 1;
    const double f = __ldg(P.le_f + ge);
    const double c_new = fd_ring_w(P, ge, step - d, sg), c_old = fd_ring_w(P, ge, step - d - 1, sg);
    im[j] = fma(f, c_old, (1.0 - f) * c_new);
    P.cim[(int64_t)(3 * x + j) * S + sg] = im[j];
  }
  for (int p = 0; p < 3; ++p)
    P.cph[(int64_t)(3 * x + p) * S + sg] = fma(r.ti[3 * p], im[0], fma(r.ti[3 * p + 1], im[1], r.ti[3 * p + 2] * im[2]));
}

// A coupled line's mode (line end ge, end x) after the solve of step n:
// c_j(n) = -(2/Z_j) (T_v^-1 v_p)_j - I_j(n) into the far end's ring.
__device__ __forceinline__ void batch_ce_update(const BatchParams& P, int ge, int x, int sg, int sl, long long step,
                                                const double* vv, int node0, int St) {
  const CoupledEndDev& r = P.ce[x];
  const int64_t S = P.S;
  const int j = ge - __ldg(P.ce_le0 + x);
  double v[3];
  for (int p = 0; p < 3; ++p) v[p] = vv[(size_t)(__ldg(P.ce_node + 3 * x + p) - node0) * St + sl];
  const double vm = fma(r.tinv[3 * j], v[0], fma(r.tinv[3 * j + 1], v[1], r.tinv[3 * j + 2] * v[2]));
  const double out = fma(-__ldg(P.le_y2 + ge), vm, -P.cim[(int64_t)(3 * x + j) * S + sg]);
  const int depth = __ldg(P.le_d1 + ge) + 1;
  P.ring[EMT_CHK(P.err, (__ldg(P.le_bfar + ge) + (int64_t)((unsigned long long)step % (unsigned)depth)) * S + sg,
                 P.bnd.ring, kChkRingWrite)] = out;
}

// Scenario sg selects variant base `base` for subsystem s: its matrix is
// the one of the scenario's current runtime-switch state word.
__device__ __forceinline__ void select_matrix(const BatchParams& P, long long* cur, int sl, int sg, int s,
                                              long long base) {
  long long off = base;
  if (P.vbase != nullptr) {
    P.vbase[(int64_t)sg * P.n_sub + s] = base;
    off += (long long)P.rs_word[(int64_t)s * P.S + sg] * __ldg(P.sub_rs + 4 * s + 2);
  }
  cur[(size_t)sl * P.n_sub + s] = off;
}

// Subsystem s, scenario sg, after the solve of step n: the state in force
// at step n+1 of each runtime switch (a diode conducts iff v_k - v_m > 0; a
// breaker, once past its trip step, opens for good at a sign change of its
// current), and the matrix of the new state word.
__device__ __forceinline__ void batch_rs_decide(const BatchParams& P, long long* cur, int s, int sl, int sg,
                                                long long step, const double* vv, int node0, int St) {
  const int n_rs = __ldg(P.sub_rs + 4 * s + 1);
  if (n_rs == 0) return;
  const int rs0 = __ldg(P.sub_rs + 4 * s), node_off = __ldg(P.sub_rs + 4 * s + 3);
  const int64_t S = P.S;
  int* wp = P.rs_word + (int64_t)s * S + sg;
  const int word = *wp;
  int nw = 0;
  for (int j = 0; j < n_rs; ++j) {
    const RuntimeSwitchDev& r = P.rs[rs0 + j];
    const double vk = r.k >= 0 ? vv[(size_t)(node_off + r.k - node0) * St + sl] : 0.0;
    const double vm = r.m >= 0 ? vv[(size_t)(node_off + r.m - node0) * St + sl] : 0.0;
    const double vb = vk - vm;
    int bit = (word >> j) & 1;
    if (r.kind == 0) {
      bit = vb > 0.0 ? 1 : 0;
    } else if (bit) {
      double* ip = P.rs_prev_i + (int64_t)(rs0 + j) * S + sg;
      const double i = vb / r.r_on;
      if (step >= r.trip && *ip * i <= 0.0) bit = 0;
      *ip = i;
    }
    nw |= bit << j;
  }
  if (nw != word) {
    *wp = nw;
    cur[(size_t)sl * P.n_sub + s] = P.vbase[(int64_t)sg * P.n_sub + s] + (long long)nw * __ldg(P.sub_rs + 4 * s + 2);
  }
}

// kDigit: the instance with the digit-form solve (P.dig set); the other keeps
// the FP64 kernel's registers free of it
template <bool kDigit>
__global__ void __launch_bounds__(kDigit ? kBatchDigitThreads : kBatchMaxThreads, 1) batch_kernel(BatchParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int St = P.S_t;
  const int sigma0 = blockIdx.x * St;
  const int n_here = min(St, P.S - sigma0);   // scenarios of this tile
  const int T = blockDim.x, tid = threadIdx.x;
  const int S = P.S, n_sub = P.n_sub;
  // item x = tid + i T of a phase is (x / St, x % St); both advance by
  // (T / St, T % St) per iteration, so no phase loop divides
  const int q0 = tid / St, r0 = tid - q0 * St, dq = T / St, dr = T - dq * St;
  double* vs = reinterpret_cast<double*>(smem_raw);                      // [n_sources][St]
  long long* cur = reinterpret_cast<long long*>(vs + (size_t)P.n_sources * St);   // [St][n_sub] matrix offsets
  long long* evn = cur + (size_t)St * n_sub;                             // [St] next selection event
  double* iv = reinterpret_cast<double*>(evn + St);                      // [max_cols][St]
  double* vv = iv + (size_t)P.max_cols * St;                             // [max_nodes][St]
  float* ivf = reinterpret_cast<float*>(vv + (size_t)P.max_nodes * St);  // [max_cols][St]
  double* wsc = reinterpret_cast<double*>(ivf + (((size_t)P.max_cols * St + 1) & ~(size_t)1));   // [n_sources][2]
  // digit form: per subsystem of the group its digit matrix (or -1), the
  // injection exponents of a batch [dig_grp][TS], the digit table
  const int TS = 16 * ((St + 15) / 16);
  long long* dsel = reinterpret_cast<long long*>(wsc + 2 * (size_t)P.n_sources);   // [dig_grp]
  int* dem = reinterpret_cast<int*>(dsel + P.dig_grp);
  uint32_t* dtab = reinterpret_cast<uint32_t*>(
      (reinterpret_cast<uintptr_t>(dem + (P.dig != nullptr ? P.dig_grp * TS : 0)) + 15) & ~(uintptr_t)15);

  // solve matrices in force at the first step
  for (int sl = tid; sl < n_here; sl += T) {
    const int sg = sigma0 + sl;
    int64_t x = P.ev_ptr[sg];
    const int64_t x1 = P.ev_ptr[sg + 1];
    for (; x < x1 && P.ev_step[x] <= P.n0; ++x) select_matrix(P, cur, sl, sg, P.ev_sub[x], P.ev_off[x]);
    evn[sl] = x;
  }

  const int decim = P.rec_decim > 0 ? P.rec_decim : 1;
  const long long n_end = P.n0 + P.n_steps;
  for (long long step = P.n0; step < n_end; ++step) {
    const double t = (double)step * P.dt;
    // switch events of this step
    for (int sl = tid; sl < n_here; sl += T) {
      const int sg = sigma0 + sl;
      int64_t x = evn[sl];
      const int64_t x1 = P.ev_ptr[sg + 1];
      if (x < x1 && P.ev_step[x] <= step) {
        for (; x < x1 && P.ev_step[x] <= step; ++x) select_matrix(P, cur, sl, sg, P.ev_sub[x], P.ev_off[x]);
        evn[sl] = x;
      }
    }
    // process 1 for sources: v_src(t_n) = A sin(omega t + phase)
    //   = (A cos phase) sin(omega t) + (A sin phase) cos(omega t),
    // one sin/cos pair per source and step, two FP64 operations per scenario
    for (int x = tid; x < P.n_sources; x += T) {
      double sn, cs;
      sincos(__dmul_rn(P.src_omega[x], t), &sn, &cs);
      wsc[2 * x] = sn;
      wsc[2 * x + 1] = cs;
    }
    __syncthreads();
    for (int x = tid, src = q0, sl = r0; x < P.n_sources * St; x += T, src += dq, sl += dr) {
      if (sl >= St) {
        sl -= St;
        ++src;
      }
      if (sl < n_here) {
        const int64_t q = (int64_t)(sigma0 + sl) * P.n_sources + src;
        vs[x] = fma(__ldg(P.src_ac + q), wsc[2 * src], __ldg(P.src_as + q) * wsc[2 * src + 1]);
      }
    }
    __syncthreads();
    const bool rec_now = P.rec != nullptr && step % decim == 0 && step / decim - 1 < P.rec_rows;
    const long long rec_row = step / decim - 1;

    for (int g = 0; g < P.n_groups; ++g) {
      const BatchGroupDev G = P.grp[g];

      // frequency-dependent ends: W(n) interpolated from the far end's w of
      // steps n - d and n - d - 1 (its ring, depth d + 2), A's pole terms
      // z_i(n) = lam z_i(n-1) + mu (W(n) + W(n-1)) and b(n) = a0 W + sum z_i
      // (and coupled ends: each mode's interpolated history, then T_i I_mode)
      if (G.fd1 > G.fd0 || G.ce1 > G.ce0) {
        const int n_fdg = G.fd1 - G.fd0, n_fold = n_fdg + (G.ce1 - G.ce0);
        for (int x = tid, j = q0, sl = r0; x < n_fold * St; x += T, j += dq, sl += dr) {
          if (sl >= St) {
            sl -= St;
            ++j;
          }
          if (sl >= n_here) continue;
          if (j < n_fdg) batch_fd_fold(P, G.fd0 + j, sigma0 + sl, step);
          else batch_ce_fold(P, G.ce0 + j - n_fdg, sigma0 + sl, step);
        }
        __syncthreads();
      }

      // process 2: nodal injections (and the strong-branch inputs -h)
      const int n_cols = G.col1 - G.col0;
      for (int x = tid, c = q0, sl = r0; x < n_cols * St; x += T, c += dq, sl += dr) {
        if (sl >= St) {
          sl -= St;
          ++c;
        }
        if (sl >= n_here) continue;
        const int sg = sigma0 + sl;
        const int code = __ldg(P.col_code + G.col0 + c);
        double acc = 0.0;
        if (code >= 0) {
          const int e0 = __ldg(P.ent_ptr + code), e1 = __ldg(P.ent_ptr + code + 1);
          if (e0 < e1) acc = entry_value(P, (uint32_t)__ldg(P.bent + e0), sg, sl, step, vs);
          for (int e = e0 + 1; e < e1; ++e) acc += entry_value(P, (uint32_t)__ldg(P.bent + e), sg, sl, step, vs);
        } else {
          acc = -P.h[EMT_CHK(P.err, (int64_t)(-1 - code) * S + sg, P.bnd.h, kChkHistory)];
        }
        iv[x] = acc;
        ivf[x] = f32_trunc(acc);
      }
      // digit form: a subsystem whose matrix the whole tile shares, and that
      // matrix in digit form
      if (kDigit)
        for (int j = tid; j < G.sub1 - G.sub0; j += T) {
          const int s = G.sub0 + j;
          const long long c0 = cur[s];
          bool same = true;
          for (int sl = 1; sl < n_here && same; ++sl) same = cur[(size_t)sl * n_sub + s] == c0;
          long long d = -1;
          if (same)
            for (int x = __ldg(P.dig_ptr + s); x < __ldg(P.dig_ptr + s + 1); ++x)
              if (__ldg(P.dig_key + x) == c0) d = __ldg(P.dig_val + x);
          dsel[j] = d;
        }
      __syncthreads();

      // process 4: v = (X_hi + X_lo) [i; -h_strong], each scenario with its
      // own solve matrix for the row's subsystem
      const int n_nodes = G.node1 - G.node0;
      for (int x = tid, k = q0, sl = r0; x < n_nodes * St; x += T, k += dq, sl += dr) {
        if (sl >= St) {
          sl -= St;
          ++k;
        }
        if (sl >= n_here) continue;
        const int node = G.node0 + k;
        const int s = __ldg(P.node_sub + node), r = __ldg(P.node_r + node);
        if (kDigit && dsel[s - G.sub0] >= 0) continue;   // (the digit form below)
        const int nc = __ldg(P.sub_nc + s);
        const int cb = __ldg(P.sub_col_off + s) - G.col0;
        const int64_t off =
            EMT_CHK_BLOCK(P.err, cur[(size_t)sl * n_sub + s] + (int64_t)r * nc, nc, P.bnd.ginv, kChkMatrix);
        const double* row = P.ginv + off;
        const float* rowl = P.ginv_lo + off;
        const double* ivc = iv + (size_t)cb * St + sl;
        const float* ivfc = ivf + (size_t)cb * St + sl;
        double a = 0.0;
        float b = 0.f;
        int j = 0;
        // four row entries loaded ahead of their FMAs (same summation order)
        for (; j + 4 <= nc; j += 4) {
          const double x0 = __ldg(row + j), x1 = __ldg(row + j + 1), x2 = __ldg(row + j + 2), x3 = __ldg(row + j + 3);
          const float y0 = __ldg(rowl + j), y1 = __ldg(rowl + j + 1), y2 = __ldg(rowl + j + 2), y3 = __ldg(rowl + j + 3);
          a = fma(x0, ivc[(size_t)j * St], a);
          b = fmaf(y0, ivfc[(size_t)j * St], b);
          a = fma(x1, ivc[(size_t)(j + 1) * St], a);
          b = fmaf(y1, ivfc[(size_t)(j + 1) * St], b);
          a = fma(x2, ivc[(size_t)(j + 2) * St], a);
          b = fmaf(y2, ivfc[(size_t)(j + 2) * St], b);
          a = fma(x3, ivc[(size_t)(j + 3) * St], a);
          b = fmaf(y3, ivfc[(size_t)(j + 3) * St], b);
        }
        for (; j < nc; ++j) {
          a = fma(__ldg(row + j), ivc[(size_t)j * St], a);
          b = fmaf(__ldg(rowl + j), ivfc[(size_t)j * St], b);
        }
        const double v = a + f64_of(b);
        vv[x] = v;
        if (rec_now) {
          const int pos = P.rec_pos[node];
          if (pos >= 0) P.rec[EMT_CHK(P.err, (rec_row * S + sigma0 + sl) * P.n_rec + pos, P.bnd.rec, kChkRecord)] = v;
        }
      }
      // the digit-form subsystems, in batches whose injection digits fit the table
      if (kDigit) {
        const int warp = tid >> 5, lane = tid & 31, n_warps = T >> 5, g = lane >> 2, t = lane & 3;
        for (int jb0 = 0; jb0 < G.sub1 - G.sub0;) {
          // the batch [jb0, jb1): the digit subsystems whose tables fit dig_words (all of the group's, as sized)
          int jb1 = jb0, used = 0, cnt = 0;
          for (; jb1 < G.sub1 - G.sub0; ++jb1) {
            if (dsel[jb1] < 0) continue;
            const int w = dig_table_words(__ldg(P.sub_nc + G.sub0 + jb1), TS);
            if (used + w > P.dig_words) break;
            used += w;
            ++cnt;
          }
          if (cnt == 0) {   // (every digit subsystem's table fits by construction; a step past one never loops)
            jb0 = jb1 + (jb1 < G.sub1 - G.sub0 ? 1 : 0);
            continue;
          }
          // injection digits: a warp per (subsystem, scenario): its scale (largest exponent), then the table
          for (int it = warp; it < cnt * n_here; it += n_warps) {
            int jj = it / n_here, sl = it - jj * n_here, j = jb0, off = 0;
            for (;; ++j) {   // the jj-th digit subsystem of the batch, and its table offset
              if (dsel[j] < 0) continue;
              if (jj == 0) break;
              off += dig_table_words(__ldg(P.sub_nc + G.sub0 + j), TS);
              --jj;
            }
            const int s = G.sub0 + j, nc = __ldg(P.sub_nc + s), ks = (nc + 15) >> 4, sw = 8 * ks + 4;
            const double* ivc = iv + (size_t)(__ldg(P.sub_col_off + s) - G.col0) * St + sl;
            unsigned em = 1;
            for (int k = lane; k < nc; k += 32) em = max(em, dg_expo(ivc[(size_t)k * St]));
            em = max(__reduce_max_sync(0xffffffffu, em), 1u);
            uint32_t* tab = dtab + off;
            for (int kw = lane; kw < 8 * ks; kw += 32) {
              const int k = 2 * kw;
              const double x0 = k < nc ? ivc[(size_t)k * St] : 0.0, x1 = k + 1 < nc ? ivc[(size_t)(k + 1) * St] : 0.0;
              const long long n0 = dg_fixed(x0, em) + kDigitBias, n1 = dg_fixed(x1, em) + kDigitBias;
#pragma unroll
              for (int b = 0; b < kDigits; ++b)
                tab[(b * TS + sl) * sw + kw] = dg_digit_bf16(n0, b) | (dg_digit_bf16(n1, b) << 16);
            }
            if (lane == 0) dem[it - (it / n_here) * n_here + (it / n_here) * TS] = (int)em;
          }
          __syncthreads();
          // products: a warp per (subsystem, 16 scenarios, 8 rows)
          int n_task = 0;
          for (int j = jb0; j < jb1; ++j)
            if (dsel[j] >= 0) n_task += (TS / 16) * ((__ldg(P.sub_n + G.sub0 + j) + 7) >> 3);
          for (int it = warp; it < n_task; it += n_warps) {
            int rem = it, j = jb0, jj = 0, off = 0, ntile = 0;
            for (;; ++j) {
              if (dsel[j] < 0) continue;
              ntile = (TS / 16) * ((__ldg(P.sub_n + G.sub0 + j) + 7) >> 3);
              if (rem < ntile) break;
              rem -= ntile;
              off += dig_table_words(__ldg(P.sub_nc + G.sub0 + j), TS);
              ++jj;
            }
            const int s = G.sub0 + j, n = __ldg(P.sub_n + s), nc = __ldg(P.sub_nc + s);
            const int ks = (nc + 15) >> 4, sw = 8 * ks + 4, r8n = (n + 7) >> 3;
            const int stile = rem / r8n, R8 = rem - stile * r8n;
            const uint32_t* dm = P.dig + dsel[j];
            const uint32_t* tab = dtab + off + (16 * stile + g) * sw + t;
            long long ta[4] = {0, 0, 0, 0}, tb[4] = {0, 0, 0, 0};
            for (int u = kDigitGroupLo; u <= 2 * kDigits - 2; ++u) {
              // pairs (a, u - a) two at a time on two accumulators, so that two MMA chains are in flight
              float e0[4] = {0.f, 0.f, 0.f, 0.f}, e1[4] = {0.f, 0.f, 0.f, 0.f};
              const int a_hi = min(kDigits - 1, u);
              for (int a = max(0, u - (kDigits - 1)); a <= a_hi; a += 2) {
                const bool two = a + 1 <= a_hi;
                const uint32_t* tA = tab + (u - a) * TS * sw;
                const uint32_t* tB = tab + (u - a - (two ? 1 : 0)) * TS * sw;
                const uint2* fA = reinterpret_cast<const uint2*>(dm) + ((size_t)(a * r8n + R8) * ks) * 32 + lane;
                const uint2* fB = fA + (size_t)r8n * ks * 32;
                for (int st = 0; st < ks; ++st) {
                  const uint2 bA = __ldg(fA + st * 32);
                  dg_mma(e0, tA[8 * st], tA[8 * sw + 8 * st], tA[8 * st + 4], tA[8 * sw + 8 * st + 4], bA.x, bA.y);
                  if (two) {
                    const uint2 bB = __ldg(fB + st * 32);
                    dg_mma(e1, tB[8 * st], tB[8 * sw + 8 * st], tB[8 * st + 4], tB[8 * sw + 8 * st + 4], bB.x, bB.y);
                  }
                }
                if (ks > 4) {   // more than 64 columns: each pair's sums leave the accumulators at once
#pragma unroll
                  for (int c = 0; c < 4; ++c) {
                    const int q = dg_acc_int(e0[c]) + dg_acc_int(e1[c]);
                    if (u >= 11) ta[c] += dg_shl64(q, 8 * (u - 11));
                    else tb[c] += dg_shl64(q, 8 * (u - kDigitGroupLo));
                    e0[c] = e1[c] = 0.f;
                  }
                }
              }
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const int q = dg_acc_int(e0[c]) + dg_acc_int(e1[c]);
                if (u >= 11) ta[c] += dg_shl64(q, 8 * (u - 11));
                else tb[c] += dg_shl64(q, 8 * (u - kDigitGroupLo));
              }
            }
            const int* ex = reinterpret_cast<const int*>(dm + (size_t)8 * r8n * ks * 64);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int sl = 16 * stile + g + (c >= 2 ? 8 : 0), r = 8 * R8 + 2 * t + (c & 1);
              if (sl < n_here && r < n) {
                const double v = dg_to_double(ta[c], tb[c], __ldg(ex + r) + dem[jj * TS + sl] - 2120);
                const int node = __ldg(P.sub_node0 + s) + r;
                vv[(size_t)(node - G.node0) * St + sl] = v;
                if (rec_now) {
                  const int pos = P.rec_pos[node];
                  if (pos >= 0)
                    P.rec[EMT_CHK(P.err, (rec_row * S + sigma0 + sl) * P.n_rec + pos, P.bnd.rec, kChkRecord)] = v;
                }
              }
            }
          }
          jb0 = jb1;
          if (jb0 < G.sub1 - G.sub0) __syncthreads();   // (the table is refilled by the next batch)
        }
      }
      __syncthreads();

      // compensation method: each nonlinear resistor against its
      // subsystem's linear solution, per scenario (its current from the
      // Thevenin source v_th behind R_th = z_k - z_m), then v -= z i
      if (G.nl1 > G.nl0) {
        const int n_nlg = G.nl1 - G.nl0;
        for (int x = tid, j = q0, sl = r0; x < n_nlg * St; x += T, j += dq, sl += dr) {
          if (sl >= St) {
            sl -= St;
            ++j;
          }
          if (sl >= n_here) continue;
          const int e = G.nl0 + j, sg = sigma0 + sl;
          P.nl_i[(int64_t)e * S + sg] = batch_nl_current(P, e, sl, cur, vv, G.node0, St);
        }
        __syncthreads();
        const int n_c = G.nlc1 - G.nlc0;
        for (int x = tid, j = q0, sl = r0; x < n_c * St; x += T, j += dq, sl += dr) {
          if (sl >= St) {
            sl -= St;
            ++j;
          }
          if (sl >= n_here) continue;
          const int node = __ldg(P.nlc + 2 * (G.nlc0 + j)), e = __ldg(P.nlc + 2 * (G.nlc0 + j) + 1);
          const int s = __ldg(P.nlinfo + 4 * e), n = __ldg(P.nlinfo + 4 * e + 1), node_off = __ldg(P.nlinfo + 4 * e + 2);
          const int64_t zoff = cur[(size_t)sl * n_sub + s] + (int64_t)n * __ldg(P.sub_nc + s);
          const int r = node - node_off;
          const double i = P.nl_i[(int64_t)e * S + sigma0 + sl];
          double* vp = vv + (size_t)(node - G.node0) * St + sl;
          const int64_t zr = EMT_CHK(P.err, zoff + r, P.bnd.ginv, kChkNlColumn);
          const double v = fma(-(double)__ldg(P.ginv_lo + zr), i, fma(-__ldg(P.ginv + zr), i, *vp));
          *vp = v;
          if (rec_now) {
            const int pos = P.rec_pos[node];
            if (pos >= 0)
              P.rec[EMT_CHK(P.err, (rec_row * S + sigma0 + sl) * P.n_rec + pos, P.bnd.rec, kChkRecord)] = v;
          }
        }
        __syncthreads();
      }

      // runtime switches: each subsystem's state word for the next step from
      // this step's solution (its matrix for that word from then on)
      if (P.vbase != nullptr) {
        const int n_sg = G.sub1 - G.sub0;
        for (int x = tid, j = q0, sl = r0; x < n_sg * St; x += T, j += dq, sl += dr) {
          if (sl >= St) {
            sl -= St;
            ++j;
          }
          if (sl >= n_here) continue;
          batch_rs_decide(P, cur, G.sub0 + j, sl, sigma0 + sl, step, vv, G.node0, St);
        }
      }

      // control blocks of the group's subsystems at this step, layer by
      // layer (their controlled currents enter the next step's injections)
      for (int l = 0; l < G.n_lay; ++l) {
        const int b0 = __ldg(P.cb_lay + G.lay0 + l), nb = __ldg(P.cb_lay + G.lay0 + l + 1) - b0;
        for (int x = tid, k = q0, sl = r0; x < nb * St; x += T, k += dq, sl += dr) {
          if (sl >= St) {
            sl -= St;
            ++k;
          }
          if (sl >= n_here) continue;
          batch_control(P, __ldg(P.cb_list + b0 + k), sigma0 + sl, sl, (int)(step & 1), vv, G.node0, St);
        }
        __syncthreads();
      }

      // process 1: history currents and line outputs of the group
      const int n_lc = G.lc1 - G.lc0, n_items = n_lc + (G.le1 - G.le0);
      for (int x = tid, it = q0, sl = r0; x < n_items * St; x += T, it += dq, sl += dr) {
        if (sl >= St) {
          sl -= St;
          ++it;
        }
        if (sl >= n_here) continue;
        const int sg = sigma0 + sl;
        if (it < n_lc) {
          const int gl = G.lc0 + it;
          if (P.keep_lc && !P.keep_lc[(int64_t)gl * S + sg]) continue;   // removed: h stays 0
          const int nk = __ldg(P.lc_nk + gl), nm = __ldg(P.lc_nm + gl);
          const double vk = nk >= 0 ? vv[(size_t)(nk - G.node0) * St + sl] : (nk == -1 ? 0.0 : vs[(-2 - nk) * St + sl]);
          const double vm = nm >= 0 ? vv[(size_t)(nm - G.node0) * St + sl] : (nm == -1 ? 0.0 : vs[(-2 - nm) * St + sl]);
          const double e = __ldg(P.lc_e + gl);
          double* hp = P.h + EMT_CHK(P.err, (int64_t)gl * S + sg, P.bnd.h, kChkHistory);
          const double hv = *hp;
          *hp = __ldg(P.lc_isl + gl) ? fma(e, vk - vm, hv) : fma(e, vk - vm, -hv);
        } else if (P.le_fd != nullptr && __ldg(P.le_fd + G.le0 + (it - n_lc)) >= 0) {
          const int ge = G.le0 + (it - n_lc);
          batch_fd_update(P, ge, __ldg(P.le_fd + ge), sg, step, vv[(size_t)(__ldg(P.le_nd + ge) - G.node0) * St + sl]);
        } else if (P.le_ce != nullptr && __ldg(P.le_ce + G.le0 + (it - n_lc)) >= 0) {
          const int ge = G.le0 + (it - n_lc);
          batch_ce_update(P, ge, __ldg(P.le_ce + ge), sg, sl, step, vv, G.node0, St);
        } else {
          const int ge = G.le0 + (it - n_lc);
          const int d1 = __ldg(P.le_d1 + ge);
          const double ie =
              P.ring[EMT_CHK(P.err, (__ldg(P.le_bring + ge) + ring_slot(step, d1)) * S + sg, P.bnd.ring, kChkRingRead)];
          double out = fma(-__ldg(P.le_y2 + ge), vv[(size_t)(__ldg(P.le_nd + ge) - G.node0) * St + sl], -ie);
          if (P.keep_le && !P.keep_le[(int64_t)ge * S + sg]) out = 0.0;   // removed line
          P.ring[EMT_CHK(P.err, (__ldg(P.le_bfar + ge) + ring_slot(step + d1 - 1, d1)) * S + sg, P.bnd.ring,
                         kChkRingWrite)] = out;
        }
      }
      __syncthreads();
    }
  }
}

// Per-slot constants of the multi-scenario kernel, gathered from the
// companion conductances: e of each L/C slot, g of each source-branch slot.
__global__ void slot_constants_kernel(const BranchDev* br, const int32_t* lc_idx, int64_t n_lc, const int32_t* sb_idx,
                                      int64_t n_sb, double* lc_e, double* sb_g) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_lc + n_sb;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n_lc) lc_e[i] = br[lc_idx[i]].e;
    else sb_g[i - n_lc] = br[sb_idx[i - n_lc]].g;
  }
}

// A cos(phase), A sin(phase) per scenario and source (set-up, once).
__global__ void source_coefficients_kernel(const double* amp, const double* phase, int64_t count, double* ac,
                                           double* as) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    double sn, cs;
    sincos(phase[i], &sn, &cs);
    ac[i] = amp[i] * cs;
    as[i] = amp[i] * sn;
  }
}

}  // namespace

cudaError_t launch_source_coefficients(const double* amp, const double* phase, int64_t count, double* ac, double* as,
                                       cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, 148 * 8);
  source_coefficients_kernel<<<blocks, 256, 0, st>>>(amp, phase, count, ac, as);
  return cudaGetLastError();
}

cudaError_t launch_slot_constants(const BranchDev* br, const int32_t* lc_idx, int64_t n_lc, const int32_t* sb_idx,
                                  int64_t n_sb, double* lc_e, double* sb_g, cudaStream_t st) {
  const int64_t total = n_lc + n_sb;
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 4);
  slot_constants_kernel<<<blocks, 256, 0, st>>>(br, lc_idx, n_lc, sb_idx, n_sb, lc_e, sb_g);
  return cudaGetLastError();
}

int batch_max_threads(bool digit) { return digit ? kBatchDigitThreads : kBatchMaxThreads; }

size_t batch_smem_bytes(int S_t, int n_sources, int n_sub, int max_cols, int max_nodes, int dig_words,
                        int dig_grp) {
  size_t b = (size_t)n_sources * S_t * 8 + (size_t)S_t * n_sub * 8 + (size_t)S_t * 8 + (size_t)max_nodes * S_t * 8 +
             (((size_t)max_cols * S_t + 1) & ~(size_t)1) * 12 + (size_t)n_sources * 16;
  if (dig_words > 0)   // digit form: dsel, the batch's exponents, 16-byte alignment, the table
    b += (size_t)dig_grp * 8 + (size_t)dig_grp * 16 * ((S_t + 15) / 16) * 4 + 16 + (size_t)dig_words * 4;
  return b;
}

cudaError_t launch_batch_digits(const double* ginv, const float* ginv_lo, const int64_t* mat_goff,
                                const int32_t* mat_n, const int32_t* mat_nc, const int64_t* mat_doff, int n_mats,
                                uint32_t* dig, cudaStream_t st) {
  if (n_mats <= 0) return cudaSuccess;
  batch_digits_kernel<<<n_mats, 256, 0, st>>>(ginv, ginv_lo, mat_goff, mat_n, mat_nc, mat_doff, dig);
  return cudaGetLastError();
}

void batch_graph_destroy(BatchGraph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  g->exec = nullptr;
  g->graph = nullptr;
  g->node = nullptr;
}

// One launch of batch_kernel over ceil(S / S_t) CTAs.  With `graph`, the
// launch goes through a CUDA graph that is built once per launch shape and
// whose kernel node gets this call's arguments.
cudaError_t launch_batch(const BatchParams& p, int threads, cudaStream_t st, BatchGraph* graph) {
  const size_t smem =
      batch_smem_bytes(p.S_t, p.n_sources, p.n_sub, p.max_cols, p.max_nodes, p.dig ? p.dig_words : 0, p.dig_grp);
  if (smem > 227 * 1024 || threads < 32 || threads > (p.dig != nullptr ? kBatchDigitThreads : kBatchMaxThreads) ||
      threads % 32)
    return cudaErrorInvalidValue;
  const void* fn = p.dig != nullptr ? (const void*)batch_kernel<true> : (const void*)batch_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (p.S + p.S_t - 1) / p.S_t;
  if (!graph) {
    if (p.dig != nullptr) batch_kernel<true><<<grid, threads, smem, st>>>(p);
    else batch_kernel<false><<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
  }
  BatchParams arg = p;
  void* args[] = {&arg};
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void*>(fn);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(threads);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = args;
  if (graph->exec && (graph->grid != grid || graph->threads != threads || graph->smem != smem || graph->func != fn))
    batch_graph_destroy(graph);
  if (!graph->exec) {
    e = cudaGraphCreate(&graph->graph, 0);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&graph->node, graph->graph, nullptr, 0, &kp);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&graph->exec, graph->graph, 0);
    if (e != cudaSuccess) {
      batch_graph_destroy(graph);
      return e;
    }
    graph->grid = grid;
    graph->threads = threads;
    graph->smem = smem;
    graph->func = fn;
  } else {
    e = cudaGraphExecKernelNodeSetParams(graph->exec, graph->node, &kp);
    if (e != cudaSuccess) return e;
  }
  e = cudaGraphLaunch(graph->exec, st);
  if (e == cudaSuccess) graph->launches += 1;
  return e;
}

}  // namespace emt
