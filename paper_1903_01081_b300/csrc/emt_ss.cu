// The time loop in state-space form, for networks whose subsystems are all
// small and hold the basic elements only (R/L/C branches, sources, switches
// with fixed times, lossless Bergeron lines).
//
// The EMTP step of one subsystem (Sec. III-A, processes 1-4) is linear in
// what it starts from: the history currents h(n-1) of its L and C branches,
// its sources' voltages v_src(n), and the values I_e(n) its line ends take
// from their rings.  With J(n) the per-node sums of the I_e(n),
//   v(n) = G^-1 i(n),   i(n) = A_h h(n-1) + A_s v_src(n) - A_J J(n),
//   h_b(n) = +-h_b(n-1) + e_b (v_k(n) - v_m(n)),
// so [h(n) | v(n)] = M [h(n-1) | v_src(n) | J(n)] with a fixed M per switch
// epoch, and each line end sends c_e(n) = -(2/Z_e) v_node(n) - I_e(n).  A
// step is then one matrix-vector product: the chain of dependent FP64
// operations that sets the step time on B300 (each holds its SM
// sub-partition's FP64 pipe ~64 cycles) is ceil(cols/Q) fused multiply-adds,
// log2(Q) shuffle-adds and one add, instead of the four barrier-separated
// processes of the CTA kernel (emt_kernels.cu).
//
// M is built on the device from the prefactored G^-1 = X_hi + X_lo in
// double-double arithmetic (Knuth's two-sum, the FMA two-product) and kept,
// like G^-1, as its rounding to double plus a single-precision remainder;
// the step accumulates both (the remainder on the FP32 pipe).  One CTA per
// subsystem: warps 0..6 run the product (Q lanes per row of M), warp 7
// meanwhile collects the next step's line values and source voltages, so
// the ring waits overlap the product.
#include <stdint.h>

#include <algorithm>
#include <climits>

#include <cuda_runtime.h>

#include "emt_internal.h"
#include "emt_device.cuh"

namespace emt {

namespace {

constexpr int kSsPollWarp = kSsThreads / 32 - 1;

// Phase-clock build (-DEMT_PHASE_CLOCKS): per CTA, clock cycles per step of
// 0 thread 0's part of the product, 1 the poll warp's collection of the next
// step's values (its lane 0), 2 thread 0 from its rows to the end-of-step
// barrier; 6 steps, 7 the last launch's span (see phase_clocks).
#ifdef EMT_PHASE_CLOCKS
__device__ unsigned long long g_ss_phase[kPhaseCtas][kPhaseCount];
#endif
constexpr int kSsPrefetch = 4;   // ring slots a poll lane has in flight at once

// ---------------------------------------------------------------- double-double

struct DD {
  double hi, lo;
};

__device__ __forceinline__ DD dd_norm(double s, double e) {
  const double h = s + e;
  return {h, e - (h - s)};
}

__device__ __forceinline__ DD dd_add(DD a, DD b) {   // two-sum of the high parts, then the low parts
  const double s = a.hi + b.hi, bb = s - a.hi;
  const double e = (a.hi - (s - bb)) + (b.hi - bb);
  return dd_norm(s, e + (a.lo + b.lo));
}

__device__ __forceinline__ DD dd_scale(DD a, double g) {   // two-product by FMA
  const double p = a.hi * g;
  const double e = fma(a.hi, g, -p);
  return dd_norm(p, fma(a.lo, g, e));
}

__device__ __forceinline__ DD dd_neg(DD a) { return {-a.hi, -a.lo}; }

// ---------------------------------------------------------------- building M

struct Build {
  const FwdParams& P;
  const SubDev& S;
  const SsSubDev& Q;
  int64_t goff;   // this epoch's G^-1 (n x nc, row-major)
  int nc;

  __device__ DD x(int r, int j) const {
    const int64_t i = goff + (int64_t)r * nc + j;
    return {P.ginv[i], (double)P.ginv_lo[i]};
  }
  // d v_r / d x_col, v = G^-1 i (r a local node)
  __device__ DD xa(int r, int col) const {
    if (col < S.n_lc) {
      for (int t = 0; t < S.n_str; ++t)   // a strong branch: its own column, driven by -h
        if (P.str_slot[S.str_off + t] == col) return dd_neg(x(r, S.n + t));
      const BranchDev b = P.br[P.lc_idx[S.lc_off + col]];
      DD acc{0.0, 0.0};   // i_k -= h, i_m += h
      if (b.k >= 0) acc = dd_add(acc, dd_neg(x(r, b.k)));
      if (b.m >= 0) acc = dd_add(acc, x(r, b.m));
      return acc;
    }
    col -= S.n_lc;
    if (col < S.n_src) {   // source branches of local source `col`: i_j += g v_src
      DD acc{0.0, 0.0};
      for (int t = 0; t < S.n_sb; ++t) {
        const BranchDev b = P.br[P.sb_idx[S.sb_off + t]];
        const int src = b.k <= -2 ? -2 - b.k : -2 - b.m;
        const int j = b.k <= -2 ? b.m : b.k;
        if (src == col && j >= 0) acc = dd_add(acc, dd_scale(x(r, j), b.g));
      }
      return acc;
    }
    col -= S.n_src;   // line-end node slot: i_node -= J
    return dd_neg(x(r, P.ss_lnode[Q.ln_off + col]));
  }
  __device__ DD entry(int row, int col) const {
    if (Q.compact) return xa(row, col);   // node voltages only
    if (row < S.n_lc) {   // h_b(n) = +-h_b(n-1) + e_b (v_k - v_m), a source end's voltage taken directly
      const BranchDev b = P.br[P.lc_idx[S.lc_off + row]];
      DD acc{0.0, 0.0};
      if (b.k >= 0) acc = dd_add(acc, xa(b.k, col));
      if (b.m >= 0) acc = dd_add(acc, dd_neg(xa(b.m, col)));
      acc = dd_scale(acc, b.e);
      const int s = col - S.n_lc;
      if (s >= 0 && s < S.n_src) {
        if (b.k <= -2 && -2 - b.k == s) acc = dd_add(acc, DD{b.e, 0.0});
        if (b.m <= -2 && -2 - b.m == s) acc = dd_add(acc, DD{-b.e, 0.0});
      }
      if (col == row) acc = dd_add(acc, DD{b.kind == 1 ? 1.0 : -1.0, 0.0});
      return acc;
    }
    return xa(row - S.n_lc, col);   // node voltages
  }
};

__global__ void ss_build_kernel(FwdParams P) {
  const SubDev S = P.sub[blockIdx.x];
  const SsSubDev Q = P.ss[blockIdx.x];
  const int nc = S.n + S.n_str;
  for (int te = 0; te < S.n_ep; ++te) {
    const Build B{P, S, Q, P.ep[S.ep_off + te].ginv_off, nc};
    const int64_t off = Q.m_off + (int64_t)te * Q.rows * Q.cols;
    for (int i = threadIdx.x; i < Q.rows * Q.cols; i += blockDim.x) {
      const DD v = B.entry(i / Q.cols, i % Q.cols);
      const DD r = dd_norm(v.hi, v.lo);
      const_cast<double*>(P.ss_m)[off + i] = r.hi;
      const_cast<float*>(P.ss_mlo)[off + i] = (float)r.lo;
    }
  }
}

// ---------------------------------------------------------------- the step

struct SsSmem {
  size_t mh, x, ie, ley2, leown, lefar, vv, lce;                                      // 8-byte
  size_t ml, xf, ledepth, led, rslot, wslot, lend, lnode, lptr, js, recp, srcg, lenode, lck, lcm,
      lckind;                                                                         // 4-byte
  size_t bytes;
};

__host__ __device__ inline SsSmem ss_smem(int rows, int cols, int n, int le, int src, int ln, int lc) {
  SsSmem s{};
  size_t o = 0;
  auto d = [&](size_t c) { size_t r = o; o += c * 8; return r; };
  auto w = [&](size_t c) { size_t r = o; o += c * 4; return r; };
  const size_t ldm = (size_t)(cols | 1);
  s.mh = d((size_t)rows * ldm);
  s.x = d(2 * (size_t)cols);
  s.ie = d(2 * (size_t)le);
  s.ley2 = d(le);
  s.leown = d(le);
  s.lefar = d(le);
  s.vv = d(n);
  s.lce = d(lc);
  s.ml = w((size_t)rows * ldm);
  s.xf = w(2 * (size_t)cols);
  s.ledepth = w(le);
  s.led = w(le);
  s.rslot = w(le);
  s.wslot = w(le);
  s.lend = w(le);
  s.lnode = w(ln);
  s.lptr = w((size_t)ln + 1);
  s.js = w(n);
  s.recp = w(n);
  s.srcg = w(src);
  s.lenode = w(le);
  s.lck = w(lc);
  s.lcm = w(lc);
  s.lckind = w(lc);
  s.bytes = (o + 15) & ~(size_t)15;
  return s;
}

// kCompact: every subsystem's step is the compact one (SsSubDev::compact)
template <bool kCompact>
__global__ void __launch_bounds__(kSsThreads, 4) fwd_ss_kernel(FwdParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_abort;
  const SsSmem L = ss_smem(P.ss_rows, P.ss_cols, P.lim.n, P.lim.le, P.lim.src, P.ss_ln, P.lim.lc);
  double* mh = reinterpret_cast<double*>(smem_raw + L.mh);
  double* xb = reinterpret_cast<double*>(smem_raw + L.x);
  double* ieb = reinterpret_cast<double*>(smem_raw + L.ie);
  double* ley2 = reinterpret_cast<double*>(smem_raw + L.ley2);
  long long* leown = reinterpret_cast<long long*>(smem_raw + L.leown);
  long long* lefar = reinterpret_cast<long long*>(smem_raw + L.lefar);
  float* ml = reinterpret_cast<float*>(smem_raw + L.ml);
  float* xfb = reinterpret_cast<float*>(smem_raw + L.xf);
  int* ledepth = reinterpret_cast<int*>(smem_raw + L.ledepth);
  int* led = reinterpret_cast<int*>(smem_raw + L.led);
  int* rslot = reinterpret_cast<int*>(smem_raw + L.rslot);
  int* wslot = reinterpret_cast<int*>(smem_raw + L.wslot);
  int* lend = reinterpret_cast<int*>(smem_raw + L.lend);
  int* lnode = reinterpret_cast<int*>(smem_raw + L.lnode);
  int* lptr = reinterpret_cast<int*>(smem_raw + L.lptr);
  int* js = reinterpret_cast<int*>(smem_raw + L.js);
  int* recp = reinterpret_cast<int*>(smem_raw + L.recp);
  int* srcg = reinterpret_cast<int*>(smem_raw + L.srcg);
  double* vv = reinterpret_cast<double*>(smem_raw + L.vv);
  double* lce = reinterpret_cast<double*>(smem_raw + L.lce);
  int* lenode = reinterpret_cast<int*>(smem_raw + L.lenode);
  int* lck = reinterpret_cast<int*>(smem_raw + L.lck);
  int* lcm = reinterpret_cast<int*>(smem_raw + L.lcm);
  int* lckind = reinterpret_cast<int*>(smem_raw + L.lckind);

  const int sidx = P.active != nullptr ? P.active[blockIdx.x] : (int)blockIdx.x;
  const SubDev S = P.sub[blockIdx.x];
  const SsSubDev Q = P.ss[sidx];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = S.n, n_lc = S.n_lc, n_le = S.n_le, n_src = S.n_src, n_ln = Q.n_ln;
  const int rows = Q.rows, cols = Q.cols, ldm = cols | 1, qn = Q.q;
  const int vs0 = n_lc, j0 = n_lc + n_src;   // column blocks of x
  const bool writes_lines = sidx != P.hold_sub;

  // ---- prologue: element data, the run state at step n0, the epoch's M
  // The CTAs one SM holds take their product's first warp on different SM
  // sub-partitions (a warp runs on sub-partition (hardware slot mod 4); a CTA
  // of 8 warps takes 8 consecutive slots, so its slot / 8 tells the CTAs
  // apart), so that their FP64 instructions do not queue on one pipe.
  __shared__ int s_rot;
  if (tid == 0) {
    unsigned wid;
    asm volatile("mov.u32 %0, %%warpid;" : "=r"(wid));
    s_rot = (int)((wid >> 3) & 3u);
    s_abort = 0;
  }
  const int p0 = (int)(P.n0 & 1);
  for (int b = tid; b < n_lc; b += kSsThreads) {
    const double h = P.h[EMT_CHK(P.err, S.lc_off + b, P.bnd.h, kChkHistory)];
    xb[p0 * cols + b] = h;
    xfb[p0 * cols + b] = f32_trunc(h);
    const BranchDev br = P.br[P.lc_idx[S.lc_off + b]];
    lce[b] = br.e;
    lck[b] = br.k;
    lcm[b] = br.m;
    lckind[b] = br.kind;
  }
  for (int e = tid; e < n_le; e += kSsThreads) {
    const LineEndDev le = P.le[S.le_off + e];
    ley2[e] = le.y2;
    leown[e] = le.own_ring;
    lefar[e] = le.far_ring;
    ledepth[e] = le.depth;
    led[e] = le.d;
    rslot[e] = (int)(P.n0 % le.depth);
    wslot[e] = (int)((P.n0 + le.d) % le.depth);
    lend[e] = P.ss_lend[S.le_off + e];
    lenode[e] = le.node;
  }
  for (int j = tid; j < n_ln; j += kSsThreads) lnode[j] = P.ss_lnode[Q.ln_off + j];
  for (int j = tid; j <= n_ln; j += kSsThreads) lptr[j] = P.ss_lptr[Q.ptr_off + j];
  for (int r = tid; r < n; r += kSsThreads) {
    recp[r] = P.rec != nullptr ? P.rec_pos[S.node_off + r] : -1;
    js[r] = -1;
  }
  for (int s = tid; s < n_src; s += kSsThreads) {
    srcg[s] = P.src_global[S.src_off + s];
    const double v = P.src_table[EMT_CHK(P.err, srcg[s], P.bnd.src, kChkSource)];
    xb[p0 * cols + vs0 + s] = v;
    xfb[p0 * cols + vs0 + s] = f32_trunc(v);
  }
  const int n_te = S.n_ep;
  int te = 0;
  while (te + 1 < n_te && P.ep[S.ep_off + te + 1].start <= P.n0) ++te;
  long long next_ep_start = (te + 1 < n_te) ? P.ep[S.ep_off + te + 1].start : LLONG_MAX;
  auto load_m = [&](int e) {
    const int64_t off = EMT_CHK_BLOCK(P.err, Q.m_off + (int64_t)e * rows * cols, rows * cols, P.bnd.ssm, kChkMatrix);
    for (int i = tid; i < rows * cols; i += kSsThreads) {
      const int r = i / cols, c = i - r * cols;
      mh[r * ldm + c] = P.ss_m[off + i];
      ml[r * ldm + c] = P.ss_mlo[off + i];
    }
  };
  load_m(te);
  __syncthreads();
  for (int j = tid; j < n_ln; j += kSsThreads) js[lnode[j]] = j;

  // the poll warp: step m's line values into ie / J of parity m & 1 (and
  // step m's source voltages when `src`); false if a wait ran out
  // (every load of a lane -- its source voltage, its line ends' slots, up to
  // kSsPrefetch of them -- is issued before any is looked at, so that their
  // L2 round trips overlap; a slot not yet written is then waited for)
  auto collect = [&](long long m, bool src) -> bool {
    const int pm = (int)(m & 1);
    const bool has_src = src && lane < n_src;
    double sv = 0.0;
    if (has_src) sv = __ldg(P.src_table + EMT_CHK(P.err, (m - P.n0) * P.n_sources + srcg[lane], P.bnd.src, kChkSource));
    bool ok = true;
    for (int e0 = lane; e0 < n_le && ok; e0 += 32 * kSsPrefetch) {
      unsigned long long w[kSsPrefetch][2];
#pragma unroll
      for (int k = 0; k < kSsPrefetch; ++k) {
        const int e = e0 + 32 * k;
        if (e < n_le) ld_tagged_raw(P.ring + 2 * EMT_CHK(P.err, leown[e] + rslot[e], P.bnd.ring, kChkRingRead), w[k][0], w[k][1]);
      }
#pragma unroll
      for (int k = 0; k < kSsPrefetch; ++k) {
        const int e = e0 + 32 * k;
        if (e < n_le && ok) {
          double v = 0.0;
          if (!tagged_value(w[k][0], w[k][1], (unsigned)m, v))
            ok = poll_slot(P, P.ring + 2 * EMT_CHK(P.err, leown[e] + rslot[e], P.bnd.ring, kChkRingRead), (unsigned)m,
                           sidx, e, v);
          ieb[pm * n_le + e] = v;
          const int nx = rslot[e] + 1;
          rslot[e] = nx == ledepth[e] ? 0 : nx;
        }
      }
    }
    if (has_src) {
      xb[pm * cols + vs0 + lane] = sv;
      xfb[pm * cols + vs0 + lane] = f32_trunc(sv);
    }
    if (src)
      for (int s = lane + 32; s < n_src; s += 32) {
        const double v =
            __ldg(P.src_table + EMT_CHK(P.err, (m - P.n0) * P.n_sources + srcg[s], P.bnd.src, kChkSource));
        xb[pm * cols + vs0 + s] = v;
        xfb[pm * cols + vs0 + s] = f32_trunc(v);
      }
    ok = __all_sync(0xffffffffu, ok);
    __syncwarp();
    for (int j = lane; j < n_ln; j += 32) {   // J: a node's line values summed in list order
      double a = 0.0;
      for (int t = lptr[j]; t < lptr[j + 1]; ++t) a += ieb[pm * n_le + lend[t]];
      xb[pm * cols + j0 + j] = a;
      xfb[pm * cols + j0 + j] = f32_trunc(a);
    }
    return ok;
  };
  if (warp == kSsPollWarp && !collect(P.n0, false) && lane == 0) s_abort = 1;
  const int decim = P.rec_decim > 0 ? P.rec_decim : 1;
  int dec = (int)(P.n0 % decim);
  long long rec_row = P.n0 / decim - (dec == 0 ? 1 : 0);
  __syncthreads();

  const int rpw = 32 / qn;   // rows per warp
  const int tw = (warp - s_rot + kSsPollWarp) % kSsPollWarp;   // this warp's place in the product
  const int rq = lane / qn, q = lane & (qn - 1);
  const long long n_end = P.n0 + P.n_steps;
#ifdef EMT_PHASE_CLOCKS
  __shared__ unsigned long long s_ph[kPhaseCount];
  __shared__ unsigned s_first;
  if (tid < kPhaseCount) s_ph[tid] = 0;
  __syncthreads();
#endif
  for (long long step = P.n0; step < n_end && !s_abort; ++step) {
    const int par = (int)(step & 1);
#ifdef EMT_PHASE_CLOCKS
    const unsigned c0 = (unsigned)clock();
    if (step == P.n0 && tid == 0) s_first = c0;
#endif
    if (step >= next_ep_start) {   // a switch event: the next epoch's M
      while (te + 1 < n_te && P.ep[S.ep_off + te + 1].start <= step) ++te;
      next_ep_start = (te + 1 < n_te) ? P.ep[S.ep_off + te + 1].start : LLONG_MAX;
      load_m(te);
      __syncthreads();
    }
    const double* xc = xb + par * cols;
    const float* xfc = xfb + par * cols;
    double* xn = xb + (par ^ 1) * cols;
    float* xfn = xfb + (par ^ 1) * cols;
    const double* iec = ieb + par * n_le;
    const bool rec_now = P.rec != nullptr && dec == 0 && rec_row < P.rec_rows;
    if (kCompact && warp < kSsPollWarp) {
      // one warp: v = M x (n rows of Q lanes), then from v the line outputs
      // and the history currents, as processes 1 of the CTA kernel
      if (tw == 0) {
        const int r = rq;
        double a = 0.0;
        float b = 0.f;
        if (r < n) {
          const double* row = mh + r * ldm;
          const float* rowl = ml + r * ldm;
#pragma unroll 4
          for (int j = q; j < cols; j += qn) {
            a = fma(row[j], xc[j], a);
            b = fmaf(rowl[j], xfc[j], b);
          }
        }
        for (int o = qn >> 1; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (r < n && q == 0) {
          const double y = a + f64_of(b);
          vv[r] = y;
          if (rec_now && recp[r] >= 0)
            P.rec[EMT_CHK(P.err, (rec_row - P.rec_row0) * P.n_rec + recp[r], P.bnd.rec, kChkRecord)] = y;
        }
        __syncwarp();
        for (int e = lane; e < n_le; e += 32) {
          const double c = fma(-ley2[e], vv[lenode[e]], -iec[e]);
          if (writes_lines)
            st_tagged(P.ring + 2 * EMT_CHK(P.err, lefar[e] + wslot[e], P.bnd.ring, kChkRingWrite),
                      (unsigned)(step + led[e]), c);
          const int nx = wslot[e] + 1;
          wslot[e] = nx == ledepth[e] ? 0 : nx;
        }
        for (int b2 = lane; b2 < n_lc; b2 += 32) {
          const int k = lck[b2], m = lcm[b2];
          const double vk = k >= 0 ? vv[k] : (k == -1 ? 0.0 : xc[vs0 - 2 - k]);
          const double vm = m >= 0 ? vv[m] : (m == -1 ? 0.0 : xc[vs0 - 2 - m]);
          const double hn = lckind[b2] == 1 ? fma(lce[b2], vk - vm, xc[b2]) : fma(lce[b2], vk - vm, -xc[b2]);
          xn[b2] = hn;
          xfn[b2] = f32_trunc(hn);
        }
      }
    } else if (!kCompact && warp < kSsPollWarp) {
      // y = M x: lane (row, q) over the columns q, q + Q, ...; a butterfly
      // leaves the row's sum in all Q lanes
      for (int r0 = tw * rpw; r0 < rows; r0 += kSsPollWarp * rpw) {
        const int r = r0 + rq;
        double a = 0.0;
        float b = 0.f;
        if (r < rows) {
          const double* row = mh + r * ldm;
          const float* rowl = ml + r * ldm;
#pragma unroll 4
          for (int j = q; j < cols; j += qn) {
            a = fma(row[j], xc[j], a);
            b = fmaf(rowl[j], xfc[j], b);
          }
        }
        for (int o = qn >> 1; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (r < rows) {
          const double y = a + f64_of(b);
          if (r < n_lc) {   // next step's history current
            if (q == 0) {
              xn[r] = y;
              xfn[r] = f32_trunc(y);
            }
          } else {          // node voltage: record it; its line ends send -(2/Z) v - I
            const int node = r - n_lc;
            if (q == 0 && rec_now && recp[node] >= 0)
              P.rec[EMT_CHK(P.err, (rec_row - P.rec_row0) * P.n_rec + recp[node], P.bnd.rec, kChkRecord)] = y;
            const int j = js[node];
            if (j >= 0)
              for (int t = lptr[j] + q; t < lptr[j + 1]; t += qn) {
                const int e = lend[t];
                const double c = fma(-ley2[e], y, -iec[e]);
                if (writes_lines)
                  st_tagged(P.ring + 2 * EMT_CHK(P.err, lefar[e] + wslot[e], P.bnd.ring, kChkRingWrite),
                            (unsigned)(step + led[e]), c);
                const int nx = wslot[e] + 1;
                wslot[e] = nx == ledepth[e] ? 0 : nx;
              }
          }
        }
      }
    } else if (step + 1 < n_end) {   // meanwhile: the next step's line values and source voltages
      if (!collect(step + 1, true) && lane == 0) s_abort = 1;
#ifdef EMT_PHASE_CLOCKS
      if (lane == 0) s_ph[1] += (unsigned)clock() - c0;
#endif
    }
#ifdef EMT_PHASE_CLOCKS
    const unsigned c1 = (unsigned)clock();
#endif
    if (dec == 0) ++rec_row;
    if (++dec == decim) dec = 0;
    __syncthreads();
#ifdef EMT_PHASE_CLOCKS
    if (tid == 0) {
      const unsigned c2 = (unsigned)clock();
      s_ph[0] += c1 - c0;
      s_ph[2] += c2 - c1;
      s_ph[6] += 1;
      s_ph[7] = c2 - s_first;
    }
#endif
  }
#ifdef EMT_PHASE_CLOCKS
  __syncthreads();
  if (sidx < kPhaseCtas && tid < kPhaseCount) {
    if (tid == 7) g_ss_phase[sidx][7] = s_ph[7];
    else atomicAdd(&g_ss_phase[sidx][tid], s_ph[tid]);
  }
#endif
  if (!s_abort) {
    const int pe = (int)(n_end & 1);
    for (int b = tid; b < n_lc; b += kSsThreads) P.h[EMT_CHK(P.err, S.lc_off + b, P.bnd.h, kChkHistory)] = xb[pe * cols + b];
    if (P.n_steps > 0)   // the values consumed at the last step (the CTA kernel's interpolation reads them)
      for (int e = tid; e < n_le; e += kSsThreads) P.le_prev[S.le_off + e] = ieb[(pe ^ 1) * n_le + e];
  }
}

}  // namespace

cudaError_t ss_phase_clocks(unsigned long long* out, int n, bool reset) {
#ifdef EMT_PHASE_CLOCKS
  const size_t bytes = (size_t)std::min(n, kPhaseCtas) * kPhaseCount * sizeof(unsigned long long);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && out != nullptr && bytes > 0) e = cudaMemcpyFromSymbol(out, g_ss_phase, bytes);
  if (e == cudaSuccess && reset) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_ss_phase);
    if (e == cudaSuccess) e = cudaMemset(p, 0, sizeof(g_ss_phase));
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

size_t ss_smem_bytes(int rows, int cols, int n, int le, int src, int ln, int lc) {
  return ss_smem(rows, cols, n, le, src, ln, lc).bytes;
}

cudaError_t launch_ss_build(const FwdParams& p, cudaStream_t st) {
  if (p.n_sub <= 0) return cudaSuccess;
  ss_build_kernel<<<p.n_sub, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_forward_ss(const FwdParams& p, bool compact, cudaStream_t st) {
  const void* fn = compact ? (const void*)fwd_ss_kernel<true> : (const void*)fwd_ss_kernel<false>;
  const size_t smem = ss_smem_bytes(p.ss_rows, p.ss_cols, p.lim.n, p.lim.le, p.lim.src, p.ss_ln, p.lim.lc);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = p.active != nullptr ? p.n_active : p.n_sub;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSsThreads, smem);
  if (e != cudaSuccess) return e;
  if ((long long)per_sm * n_sm < grid) return cudaErrorCooperativeLaunchTooLarge;
  FwdParams arg = p;
  void* args[] = {&arg};
  // cooperative launch: all CTAs co-resident, so every ring wait can end
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kSsThreads), args, smem, st);
}

}  // namespace emt
