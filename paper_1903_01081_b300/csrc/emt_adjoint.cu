// Discrete adjoint of the time loop for sm_103a (B300): the reverse sweep.
//
// Loss J = sum_{n=1..N} sum_k (v_n[k] - v*_n[k])^2.  Per subsystem the
// forward step is (trapezoidal companions, Bergeron lines)
//   v_n = G_n^-1 (u_n - A h_{n-1} - L I_n),    h_n = D h_{n-1} + E A^T v_n
//   I_far(n+d) = -(2/Z_c) v_near(n) - I_near(n)
// with D = +1 (L) / -1 (C), E = +2g (L) / -2g (C).  Its reverse, n = N..1,
// with hbar_N = 0 and Ibar(n) = 0 for n > N:
//   vbar_n  = 2 (v_n - v*_n) + A E hbar_n - sum_e (2/Z_c) Ibar_far(e)(n+d) e_node(e)
//   w_n     = G_n^-T vbar_n = G_n^-1 vbar_n          (G is symmetric)
//   hbar_{n-1} = D hbar_n - A^T w_n
//   Ibar_e(n)  = -w_n[node(e)] - Ibar_far(e)(n+d)
// and the parameter terms of step n
//   dJ/dg_b += -(a_b^T w_n) v_b(n) + hbar_n[b] (dE_b/dg_b) v_b(n)
//   dJ/dA_s += sin(omega t_n + phase) (g_b w_n[u] +/- E_b hbar_n[b])   (b joins source s to u)
//
// adj_kernel mirrors fwd_kernel: one CTA per subsystem, the solve matrix
// [X_hi | strong columns] and X_lo in shared memory, the same injection
// lanes assembling vbar (the lane inputs hold -E hbar for L/C slots, 0 for
// source branches and (2/Z_c) Ibar for line ends, so the forward's entry
// signs give A E hbar and -(2/Z_c) Ibar), the same matvec, and tagged rings
// carrying Ibar between subsystems with the tag N + 1 - n.  A strong branch
// enters through its extra column with the input +E hbar (the forward uses
// -h), since that column is G^-1 (e_k - e_m).  The forward tape v_n and the
// target v*_n are read one step ahead.
#include <stdint.h>

#include <algorithm>
#include <climits>

#include <cuda_runtime.h>

#include "emt_device.cuh"
#include "emt_internal.h"

namespace emt {

namespace {

constexpr int kAdjThreads = kFwdThreads;
constexpr int kAdjPollWarp = kAdjThreads / 32 - 1;
constexpr int kAdjItemThreads = kAdjThreads - 32;

struct AdjSmem {
  size_t gi, part, iv, ww, vn, ev, inp, xr, hb, lce, brg, bre, dga, dsa, ley2, leown, lefar, amp, sn, vsrc, lef,
      xmode, ceti, cetinv;                                                                               // 8-byte
  size_t gilo, ivf, partf;                                                                               // float
  size_t brk, brm, brlc, brkind, lcstr, lenode, ledepth, led, rslot, wslot, ent, ilnode, ilcnt, srcg, orig, lece,
      lemode, cele0, cenode, cecnt;                                                                      // int
  size_t bytes;
};

// doubles of the shared input vector inp
__host__ __device__ inline size_t adj_inp_len(const AdjLimits& L) {
  return (size_t)L.lc + L.sb + 2 * ((size_t)L.le + 3 * (size_t)L.ce) + 1;
}

__host__ __device__ inline AdjSmem adj_smem(const AdjLimits& L) {
  AdjSmem s{};
  size_t o = 0;
  auto d = [&](size_t count) { size_t r = o; o += count * 8; return r; };
  auto w = [&](size_t count) { size_t r = o; o += count * 4; return r; };
  const size_t ldg = (size_t)(L.nc | 1);
  s.gi = d((size_t)L.n * ldg);
  s.part = d((size_t)L.n * L.q);
  s.iv = d(L.nc);
  s.ww = d(L.n);
  s.vn = d(2 * (size_t)L.n);
  s.ev = d(2 * (size_t)L.n);
  s.inp = d(adj_inp_len(L));
  s.xr = d(2 * (size_t)L.le);
  s.hb = d(L.lc);
  s.lce = d(L.lc);
  s.brg = d(L.br);
  s.bre = d(L.br);
  s.dga = d(L.br);
  s.dsa = d(L.br);
  s.ley2 = d(L.le);
  s.leown = d(L.le);
  s.lefar = d(L.le);
  s.amp = d(L.src);
  s.sn = d(2 * (size_t)L.src);
  s.vsrc = d(2 * (size_t)L.src);
  s.lef = d(L.le);
  s.xmode = d(2 * (size_t)L.le);
  s.ceti = d(9 * (size_t)L.ce);
  s.cetinv = d(9 * (size_t)L.ce);
  s.gilo = w((size_t)L.n * ldg);
  s.ivf = w(L.nc);
  s.partf = w((size_t)L.n * L.q);
  s.brk = w(L.br);
  s.brm = w(L.br);
  s.brlc = w(L.br);
  s.brkind = w(L.br);
  s.lcstr = w(L.lc);
  s.lenode = w(L.le);
  s.ledepth = w(L.le);
  s.led = w(L.le);
  s.rslot = w(L.le);
  s.wslot = w(L.le);
  s.ent = w(4 * (size_t)L.il);
  s.ilnode = w(L.il);
  s.ilcnt = w(L.il);
  s.srcg = w(L.src);
  s.orig = w(L.n);
  s.lece = w(L.le);
  s.lemode = w(L.le);
  s.cele0 = w(L.ce);
  s.cecnt = w(L.ce);
  s.cenode = w(3 * (size_t)L.ce);
  s.bytes = (o + 15) & ~(size_t)15;
  return s;
}

// One warp collects one reverse step's adjoint line values Ibar_far(n+d)
// (raw into xr, times 2/Z_c into the lane inputs).  Bounded like the
// forward's collection: on exceeding the time budget (or seeing another
// CTA's error) it latches an error and returns false.
__device__ bool collect_adj(const AdjParams& P, int n_le, unsigned tag, int lane, int sidx, const long long* leown,
                            const int* ledepth, int* rslot, const double* ley2, double* xr, double* inp_le) {
  bool ok = true;
  for (int e = lane; e < n_le && ok; e += 32) {
    const unsigned long long* slot = P.ring + 2 * EMT_CHK(P.err, leown[e] + rslot[e], P.bnd.ring, kChkRingRead);
    double v = 0.0;
    if (!ld_tagged(slot, tag, v)) {
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (!ld_tagged(slot, tag, v)) {
        if ((++spins & 31u) == 0) {
          if (ld_volatile(P.err) != 0) { ok = false; break; }
          if (global_ns() - t0 > P.wait_budget_ns || spins > (1u << 30)) {
            if (atomicCAS(P.err, 0, 5) == 0) {
              P.err[1] = sidx;
              P.err[2] = e;
              P.err[3] = (int)tag;
            }
            ok = false;
            break;
          }
        }
      }
    }
    xr[e] = v;
    inp_le[e] = ley2[e] * v;
    const int nx = rslot[e] + 1;
    rslot[e] = nx == ledepth[e] ? 0 : nx;
  }
  return __all_sync(0xffffffffu, ok);
}

// Coupled line modes in reverse (first reverse step of a launch, after collecting): the adjoint
// of the value each mode sent, X = (1 - f) Ibar_far(n + d) + f Ibar_far(n + d
// + 1), from the values consumed at this reverse step (xr_new) and the
// previous one (xr_old); then the phase slots sum_j T_i[p][j] (2/Z_j) X_j
// that the injection entries subtract at the phase nodes.
__device__ void fold_modes_adj(int lane, int n_le, int n_ce, const int* lece, const double* lef, const double* ley2,
                               const double* xr_old, const double* xr_new, double* xmode_new, double* blk_new,
                               const int* cele0, const double* ceti) {
  for (int e = lane; e < n_le; e += 32)
    if (lece[e] >= 0) xmode_new[e] = fma(lef[e], xr_old[e], (1.0 - lef[e]) * xr_new[e]);
  __syncwarp();
  for (int x = lane; x < 3 * n_ce; x += 32) {
    const int c = x / 3, p = x - 3 * c;
    const double* ti = ceti + 9 * c + 3 * p;
    const int e0 = cele0[c];
    blk_new[n_le + x] = fma(ti[0], ley2[e0] * xmode_new[e0],
                            fma(ti[1], ley2[e0 + 1] * xmode_new[e0 + 1], ti[2] * (ley2[e0 + 2] * xmode_new[e0 + 2])));
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kAdjThreads, 4) adj_kernel(AdjParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_abort;
  const AdjSmem L = adj_smem(P.lim);
  const int inp_len = (int)adj_inp_len(P.lim);
  (void)inp_len;
  double* gi = reinterpret_cast<double*>(smem_raw + L.gi);
  double* part = reinterpret_cast<double*>(smem_raw + L.part);
  double* iv = reinterpret_cast<double*>(smem_raw + L.iv);
  double* ww = reinterpret_cast<double*>(smem_raw + L.ww);
  double* vn = reinterpret_cast<double*>(smem_raw + L.vn);     // [2][n]: v_n by tag parity
  double* ev = reinterpret_cast<double*>(smem_raw + L.ev);     // [2][n]: v_n - v*_n
  double* inp = reinterpret_cast<double*>(smem_raw + L.inp);
  double* xr = reinterpret_cast<double*>(smem_raw + L.xr);     // [2][le]
  double* hb = reinterpret_cast<double*>(smem_raw + L.hb);
  double* lce = reinterpret_cast<double*>(smem_raw + L.lce);
  double* brg = reinterpret_cast<double*>(smem_raw + L.brg);
  double* bre = reinterpret_cast<double*>(smem_raw + L.bre);
  double* dga = reinterpret_cast<double*>(smem_raw + L.dga);
  double* dsa = reinterpret_cast<double*>(smem_raw + L.dsa);
  double* ley2 = reinterpret_cast<double*>(smem_raw + L.ley2);
  long long* leown = reinterpret_cast<long long*>(smem_raw + L.leown);
  long long* lefar = reinterpret_cast<long long*>(smem_raw + L.lefar);
  double* amp = reinterpret_cast<double*>(smem_raw + L.amp);
  double* sn = reinterpret_cast<double*>(smem_raw + L.sn);     // [2][src]
  double* vsrc = reinterpret_cast<double*>(smem_raw + L.vsrc); // [2][src]
  float* gilo = reinterpret_cast<float*>(smem_raw + L.gilo);
  float* ivf = reinterpret_cast<float*>(smem_raw + L.ivf);
  float* partf = reinterpret_cast<float*>(smem_raw + L.partf);
  int* brk = reinterpret_cast<int*>(smem_raw + L.brk);
  int* brm = reinterpret_cast<int*>(smem_raw + L.brm);
  int* brlc = reinterpret_cast<int*>(smem_raw + L.brlc);
  int* brkind = reinterpret_cast<int*>(smem_raw + L.brkind);
  int* lcstr = reinterpret_cast<int*>(smem_raw + L.lcstr);
  int* lenode = reinterpret_cast<int*>(smem_raw + L.lenode);
  int* ledepth = reinterpret_cast<int*>(smem_raw + L.ledepth);
  int* led = reinterpret_cast<int*>(smem_raw + L.led);
  int* rslot = reinterpret_cast<int*>(smem_raw + L.rslot);
  int* wslot = reinterpret_cast<int*>(smem_raw + L.wslot);
  int* ent = reinterpret_cast<int*>(smem_raw + L.ent);
  int* ilnode = reinterpret_cast<int*>(smem_raw + L.ilnode);
  int* ilcnt = reinterpret_cast<int*>(smem_raw + L.ilcnt);
  int* srcg = reinterpret_cast<int*>(smem_raw + L.srcg);
  int* orig = reinterpret_cast<int*>(smem_raw + L.orig);
  double* lef = reinterpret_cast<double*>(smem_raw + L.lef);
  double* xmode = reinterpret_cast<double*>(smem_raw + L.xmode);    // [2][le]: modes' X by parity
  double* ceti = reinterpret_cast<double*>(smem_raw + L.ceti);
  double* cetinv = reinterpret_cast<double*>(smem_raw + L.cetinv);
  int* lece = reinterpret_cast<int*>(smem_raw + L.lece);
  int* lemode = reinterpret_cast<int*>(smem_raw + L.lemode);
  int* cele0 = reinterpret_cast<int*>(smem_raw + L.cele0);
  int* cecnt = reinterpret_cast<int*>(smem_raw + L.cecnt);   // per coupled end: modes collected this step
  int* cenode = reinterpret_cast<int*>(smem_raw + L.cenode);

  const int sidx = blockIdx.x;
  const SubDev S = P.sub[sidx];
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = S.n, Q = S.q, n_str = S.n_str, nc = n + n_str;
  const int blk = (nc + Q - 1) / Q;
  const int ldg = (Q * blk) | 1;   // columns nc .. Q blk - 1 are zero
  const int n_br = S.n_br, n_lc = S.n_lc, n_sb = S.n_sb, n_le = S.n_le, n_il = S.n_il, n_src = S.n_src;
  const int n_ce = S.n_ce;
  const int ie_base = n_lc + n_sb;
  const int blk_len = n_le + 3 * n_ce;   // per parity: line-end values, then coupled ends' phase slots
  const int zero_slot = ie_base + 2 * blk_len;
  const int nv = P.lim.n, sv = P.lim.src, lv = P.lim.le;   // strides of the parity-doubled arrays
  const int src_thread = T - 1 - tid;
  const int it_le = (n_br + 31) & ~31;   // branch items, then line ends on their own warps
  const int it_end = it_le + n_le;
  const long long tau0 = P.n_total + 1 - P.n_hi;
  const int64_t nn = P.n_nodes;

  // ---- prologue
  for (int x = tid; x < n_br; x += T) {
    const BranchDev b = P.br[S.br_off + x];
    brk[x] = b.k;
    brm[x] = b.m;
    brkind[x] = b.kind;
    brg[x] = b.g;
    bre[x] = b.e;
    brlc[x] = P.br_lc[S.br_off + x];
    dga[x] = P.dg[S.br_off + x];
    dsa[x] = P.dsrc[S.br_off + x];
  }
  for (int x = tid; x < n_lc; x += T) {
    const double e = P.br[P.lc_idx[S.lc_off + x]].e;
    const double h = P.hbar[S.lc_off + x];
    lce[x] = e;
    hb[x] = h;
    inp[x] = -e * h;
    lcstr[x] = -1;
  }
  for (int x = tid; x < n_sb; x += T) inp[n_lc + x] = 0.0;
  for (int x = tid; x < n_le; x += T) {
    const LineEndDev e = P.le[S.le_off + x];
    ley2[x] = e.y2;
    leown[x] = e.own_ring;
    lefar[x] = e.far_ring;
    lenode[x] = e.node;
    ledepth[x] = e.depth;
    led[x] = e.d;
    rslot[x] = (int)(tau0 % e.depth);
    wslot[x] = (int)((tau0 + e.d) % e.depth);
    lef[x] = e.f;
    lece[x] = e.ce;
    lemode[x] = e.mode;
    xr[(int)((tau0 - 1) & 1) * lv + x] = P.le_prev[S.le_off + x];   // consumed at the previous reverse step
  }
  for (int c = tid; c < n_ce; c += T) {
    const CoupledEndDev& ce = P.ce[S.ce_off + c];
    cele0[c] = ce.le0;
    cecnt[c] = 0;
    for (int k = 0; k < 3; ++k) cenode[3 * c + k] = ce.node[k];
    for (int k = 0; k < 9; ++k) {
      ceti[9 * c + k] = ce.ti[k];
      cetinv[9 * c + k] = ce.tinv[k];
    }
  }
  for (int x = tid; x < 4 * n_il; x += T) ent[x] = P.ent[4 * (size_t)S.il_off + x];
  for (int x = tid; x < n_il; x += T) {
    ilnode[x] = P.il_node[S.il_off + x];
    ilcnt[x] = P.il_cnt[S.il_off + x];
  }
  const int par0 = (int)(tau0 & 1);
  for (int x = tid; x < n_src; x += T) {
    const int g = P.src_global[S.src_off + x];
    srcg[x] = g;
    amp[x] = P.src_amp[g];
    const double s = P.sin_table[(P.n_hi - 1) * P.n_sources + g];
    sn[par0 * sv + x] = s;
    vsrc[par0 * sv + x] = P.src_amp[g] * s;
  }
  for (int r = tid; r < n; r += T) {
    const int o = P.orig_of[S.node_off + r];
    orig[r] = o;
    const double v = P.tape[EMT_CHK(P.err, (P.n_hi - 1 - P.tape_row0) * nn + S.node_off + r, P.bnd.tape, kChkTape)];
    vn[par0 * nv + r] = v;
    ev[par0 * nv + r] = v - P.target[EMT_CHK(P.err, (P.n_hi - 1) * nn + o, P.bnd.target, kChkTarget)];
  }
  if (tid == 0) {
    inp[zero_slot] = 0.0;
    s_abort = 0;
  }
  // solve matrix of step n: switch epoch te (by step) and, with runtime
  // switches, the state word the forward run had at step n (word tape)
  const int n_states = S.n_states, n_te = S.n_ep / n_states;
  const bool words = P.word_tape != nullptr && S.n_rs > 0;
  int te = 0;
  while (te + 1 < n_te && P.ep[S.ep_off + (te + 1) * n_states].start <= P.n_hi) ++te;
  long long ep_start = P.ep[S.ep_off + te * n_states].start;
  int word = words ? P.word_tape[(P.n_hi - 1 - P.tape_row0) * P.n_sub + sidx] : 0;
  {
    const int64_t off =
        EMT_CHK_BLOCK(P.err, P.ep[S.ep_off + te * n_states + word].ginv_off, n * nc, P.bnd.ginv, kChkMatrix);
    for (int i = tid; i < n * nc; i += T) {
      const int r = i / nc, c = i - r * nc;
      gi[r * ldg + c] = P.ginv[off + i];
      gilo[r * ldg + c] = P.ginv_lo[off + i];
    }
    const int pad = Q * blk - nc;   // the padding columns (reloads leave them zero)
    for (int i = tid; i < n * pad; i += T) {
      const int r = i / pad, c = nc + i - r * pad;
      gi[r * ldg + c] = 0.0;
      gilo[r * ldg + c] = 0.f;
    }
    for (int c = nc + tid; c < Q * blk; c += T) {
      iv[c] = 0.0;
      ivf[c] = 0.f;
    }
  }
  __syncthreads();
  for (int t = tid; t < n_str; t += T) {
    const int x = P.str_slot[S.str_off + t];
    lcstr[x] = t;
    const double e = lce[x] * hb[x];
    iv[n + t] = e;
    ivf[n + t] = (float)e;
  }
  if (warp == kAdjPollWarp && n_le > 0) {
    const bool ok = collect_adj(P, n_le, (unsigned)tau0, lane, sidx, leown, ledepth, rslot, ley2, xr + par0 * lv,
                                inp + ie_base + par0 * blk_len);
    if (!ok && lane == 0) s_abort = 1;
    if (n_ce > 0)
      fold_modes_adj(lane, n_le, n_ce, lece, lef, ley2, xr + (par0 ^ 1) * lv, xr + par0 * lv, xmode + par0 * lv,
                     inp + ie_base + par0 * blk_len, cele0, ceti);
  }
  double jacc = P.loss_part[(int64_t)sidx * T + tid];
  __syncthreads();

  for (long long i = 0; i < P.n_steps && !s_abort; ++i) {
    const long long nstep = P.n_hi - i;
    const long long tau = tau0 + i;
    const int par = (int)(tau & 1);
    const int parshift = par * blk_len;
    const bool more = i + 1 < P.n_steps;
    const int w_now = words ? P.word_tape[(nstep - 1 - P.tape_row0) * P.n_sub + sidx] : 0;
    if (nstep < ep_start || w_now != word) {   // an earlier epoch, or another runtime-switch state
      while (te > 0 && P.ep[S.ep_off + te * n_states].start > nstep) --te;
      ep_start = P.ep[S.ep_off + te * n_states].start;
      word = w_now;
      const int64_t off =
          EMT_CHK_BLOCK(P.err, P.ep[S.ep_off + te * n_states + word].ginv_off, n * nc, P.bnd.ginv, kChkMatrix);
      for (int x = tid; x < n * nc; x += T) {
        const int r = x / nc, c = x - r * nc;
        gi[r * ldg + c] = P.ginv[off + x];
        gilo[r * ldg + c] = P.ginv_lo[off + x];
      }
    }
    // step n-1's tape, target and source values: loads issued now, stored after the solve
    double vnx = 0.0, tnx = 0.0, snx = 0.0;
    if (more) {
      if (tid < n) {
        vnx = __ldg(P.tape + EMT_CHK(P.err, (nstep - 2 - P.tape_row0) * nn + S.node_off + tid, P.bnd.tape, kChkTape));
        tnx = __ldg(P.target + EMT_CHK(P.err, (nstep - 2) * nn + orig[tid], P.bnd.target, kChkTarget));
      }
      if (src_thread < n_src) snx = __ldg(P.sin_table + (nstep - 2) * P.n_sources + srcg[src_thread]);
    }

    // vbar_n = 2 (v_n - v*_n) + A E hbar_n - sum_e (2/Z_c) Ibar_far(n+d), by injection lanes
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
        const double vb = 2.0 * ev[par * nv + node] + acc;
        iv[node] = vb;
        ivf[node] = (float)vb;
      }
    }
    __syncthreads();

    // w_n = (X_hi + X_lo) [vbar; E hbar_strong], task (r, q) over column block q
    for (int task = tid; task < n * Q; task += T) {
      const int r = task / Q, q = task - r * Q;
      const double* row = gi + r * ldg;
      const float* rowl = gilo + r * ldg;
      double a = 0.0;
      float b = 0.f;
      for (int j = q * blk; j < (q + 1) * blk; ++j) {
        a = fma(row[j], iv[j], a);
        b = fmaf(rowl[j], ivf[j], b);
      }
      part[task] = a;
      partf[task] = b;
    }
    if (more) {
      if (tid < n) {
        vn[(par ^ 1) * nv + tid] = vnx;
        ev[(par ^ 1) * nv + tid] = vnx - tnx;
      }
      if (src_thread < n_src) {
        sn[(par ^ 1) * sv + src_thread] = snx;
        vsrc[(par ^ 1) * sv + src_thread] = amp[src_thread] * snx;
      }
    }
    __syncthreads();

    for (int r = tid; r < n; r += T) {
      double w = part[r * Q];
      float wl = partf[r * Q];
      for (int q = 1; q < Q; ++q) {
        w += part[r * Q + q];
        wl += partf[r * Q + q];
      }
      w += (double)wl;
      ww[r] = w;
      const double e = ev[par * nv + r];
      jacc = fma(e, e, jacc);
    }
    __syncthreads();

    // parameter terms, hbar_{n-1}, Ibar_e(n); then the update threads
    // collect step n-1's line values (the last warp idles)
    if (warp != kAdjPollWarp) {
      const double* vnc = vn + par * nv;
      const double* vsc = vsrc + par * sv;
      for (int it = tid; it < it_end; it += kAdjItemThreads) {
        if (it < n_br) {
          const int k = brk[it], m = brm[it];
          const double vk = k >= 0 ? vnc[k] : (k == -1 ? 0.0 : vsc[-2 - k]);
          const double vm = m >= 0 ? vnc[m] : (m == -1 ? 0.0 : vsc[-2 - m]);
          const double vb = vk - vm;
          const double aw = (k >= 0 ? ww[k] : 0.0) - (m >= 0 ? ww[m] : 0.0);
          double dg = fma(-aw, vb, dga[it]);
          const int x = brlc[it];
          const double E = bre[it];
          double hbn = 0.0;
          if (x >= 0) {
            hbn = hb[x];
            const bool is_l = brkind[it] == 1;
            dg = fma(is_l ? 2.0 * hbn : -2.0 * hbn, vb, dg);
            const double hnew = (is_l ? hbn : -hbn) - aw;
            hb[x] = hnew;
            inp[x] = -E * hnew;
            const int t = lcstr[x];
            if (t >= 0) {
              const double e = E * hnew;
              iv[n + t] = e;
              ivf[n + t] = (float)e;
            }
          }
          dga[it] = dg;
          if (k <= -2 || m <= -2) {
            const int j = k <= -2 ? -2 - k : -2 - m;
            const int u = k <= -2 ? m : k;
            double dv = brg[it] * (u >= 0 ? ww[u] : 0.0);
            if (x >= 0) dv += (k <= -2 ? E : -E) * hbn;
            dsa[it] = fma(sn[par * sv + j], dv, dsa[it]);
          }
        } else if (it >= it_le) {
          const int e = it - it_le;
          const int c = lece[e];
          double out;
          if (c < 0) {
            out = -ww[lenode[e]] - xr[par * lv + e];
          } else {   // a mode: Ibar_j(n) = -(T_i^T w)_j - X_j, T_i^T = T_v^-1
            const double* tr = cetinv + 9 * c + 3 * lemode[e];
            const int* nd = cenode + 3 * c;
            out = -fma(tr[0], ww[nd[0]], fma(tr[1], ww[nd[1]], tr[2] * ww[nd[2]])) - xmode[par * lv + e];
          }
          st_tagged(P.ring + 2 * EMT_CHK(P.err, lefar[e] + wslot[e], P.bnd.ring, kChkRingWrite),
                    (unsigned)(tau + led[e]), out);
          const int nx = wslot[e] + 1;
          wslot[e] = nx == ledepth[e] ? 0 : nx;
        }
      }
      // one update thread per line end, counted from the last thread, as in
      // the forward kernel; a coupled end's phase slots are formed by the
      // thread that collects the last of its three modes
      if (n_le > 0 && more) {
        const unsigned tag = (unsigned)(tau + 1);
        const double* xr_old = xr + par * lv;
        double* xr_new = xr + (par ^ 1) * lv;
        double* blk_new = inp + ie_base + (par ^ 1) * blk_len;
        double* xmode_new = xmode + (par ^ 1) * lv;
        bool ok = true;
        for (int e = kAdjItemThreads - 1 - tid; e < n_le && ok; e += kAdjItemThreads) {
          double v = 0.0;
          ok = poll_slot(P, P.ring + 2 * EMT_CHK(P.err, leown[e] + rslot[e], P.bnd.ring, kChkRingRead), tag, sidx,
                         e, v);
          xr_new[e] = v;
          blk_new[e] = ley2[e] * v;
          const int nx = rslot[e] + 1;
          rslot[e] = nx == ledepth[e] ? 0 : nx;
          if (!ok) break;
          const int c = lece[e];
          if (c >= 0) {
            xmode_new[e] = fma(lef[e], xr_old[e], (1.0 - lef[e]) * v);
            __threadfence_block();
            if (atomicAdd(&cecnt[c], 1) == 2) {
              __threadfence_block();
              cecnt[c] = 0;
              const int e0 = cele0[c];
              const volatile double* xm = xmode_new + e0;
              const double x0 = ley2[e0] * xm[0], x1 = ley2[e0 + 1] * xm[1], x2 = ley2[e0 + 2] * xm[2];
              for (int p = 0; p < 3; ++p) {
                const double* ti = ceti + 9 * c + 3 * p;
                blk_new[n_le + 3 * c + p] = fma(ti[0], x0, fma(ti[1], x1, ti[2] * x2));
              }
            }
          }
        }
        if (!ok) s_abort = 1;
      }
    }
    __syncthreads();
  }
  if (!s_abort) {
    for (int x = tid; x < n_lc; x += T) P.hbar[S.lc_off + x] = hb[x];
    if (P.n_steps > 0)
      for (int x = tid; x < n_le; x += T)
        P.le_prev[S.le_off + x] = xr[(int)((tau0 + P.n_steps - 1) & 1) * lv + x];
    for (int x = tid; x < n_br; x += T) {
      P.dg[S.br_off + x] = dga[x];
      P.dsrc[S.br_off + x] = dsa[x];
    }
    P.loss_part[(int64_t)sidx * T + tid] = jacc;
  }
}

// Chain rule to the element values and per-source sums, in a fixed order:
//   dJ/dR = -dJ/dg / R^2,  dJ/dL = -dJ/dg dt / (2 L^2),  dJ/dC = dJ/dg 2 / dt
//   dJ/dA_s = sum over the branches of source s (internal order) of dsrc[b]
__global__ void adj_finalize_kernel(const BranchDev* br, const int32_t* br_orig, int64_t n_br, const double* dg,
                                    const double* dsrc, const int32_t* src_br_ptr, const int32_t* src_br,
                                    int64_t n_sources, double dt, double* grad) {
  const int64_t total = n_br + n_sources;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n_br) {
      const BranchDev b = br[i];
      const double x = b.value;
      const double dgdp = b.kind == 0 ? -1.0 / (x * x) : (b.kind == 1 ? -dt / (2.0 * x * x) : 2.0 / dt);
      grad[br_orig[i]] = dg[i] * dgdp;
    } else {
      const int64_t s = i - n_br;
      double acc = 0.0;
      for (int32_t j = src_br_ptr[s]; j < src_br_ptr[s + 1]; ++j) acc += dsrc[src_br[j]];
      grad[i] = acc;
    }
  }
}

// J = sum of the per-thread partial sums: strided partial sums per thread,
// then a fixed pairwise tree (one block of kLossThreads threads).
constexpr int kLossThreads = 512;
__global__ void __launch_bounds__(kLossThreads) adj_loss_kernel(const double* part, int64_t n, double* loss) {
  __shared__ double red[kLossThreads];
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kLossThreads) acc += part[j];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kLossThreads / 2; w > 0; w /= 2) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0];
}

}  // namespace

int adjoint_threads() { return kAdjThreads; }

size_t adjoint_smem_bytes(const AdjLimits& lim) { return adj_smem(lim).bytes; }

int adjoint_blocks_per_sm(const AdjLimits& lim) {
  const size_t smem = adjoint_smem_bytes(lim);
  if (smem > 227 * 1024) return 0;
  if (cudaFuncSetAttribute(adj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_kernel, kAdjThreads, smem) != cudaSuccess) return 0;
  return per_sm;
}

cudaError_t launch_adjoint(const AdjParams& p, cudaStream_t st) {
  const size_t smem = adjoint_smem_bytes(p.lim);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(adj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_kernel, kAdjThreads, smem);
  if (e != cudaSuccess) return e;
  if ((long long)per_sm * n_sm < p.n_sub) return cudaErrorCooperativeLaunchTooLarge;
  AdjParams arg = p;
  void* args[] = {&arg};
  // cooperative launch: all CTAs co-resident, so every ring wait can end
  return cudaLaunchCooperativeKernel((const void*)adj_kernel, dim3(p.n_sub), dim3(kAdjThreads), args, smem, st);
}

cudaError_t launch_adj_finalize(const BranchDev* br, const int32_t* br_orig, int64_t n_br, const double* dg,
                                const double* dsrc, const int32_t* src_br_ptr, const int32_t* src_br, int64_t n_sources,
                                double dt, const double* loss_part, int64_t n_loss, double* grad, double* loss,
                                cudaStream_t st) {
  const int64_t total = n_br + n_sources;
  if (total > 0) {
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 4);
    adj_finalize_kernel<<<blocks, 256, 0, st>>>(br, br_orig, n_br, dg, dsrc, src_br_ptr, src_br, n_sources, dt, grad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  adj_loss_kernel<<<1, kLossThreads, 0, st>>>(loss_part, n_loss, loss);
  return cudaGetLastError();
}

}  // namespace emt
