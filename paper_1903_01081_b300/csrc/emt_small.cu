// The time loop with one warp per subsystem, for networks whose subsystems
// are all small (at most 32 nodes) and hold only the basic elements: R/L/C
// branches, sources, switches with fixed times and lossless Bergeron lines.
// Opt-in (option warp_per_subsystem): on B300 it measured no faster than the
// CTA kernel -- the step is a chain of dependent FP64 operations, each
// holding its SM sub-partition's FP64 pipe ~64 cycles, and the CTA kernel
// spreads a subsystem's chain over all four pipes while a warp keeps it on
// one (12-node network 1.78 against 1.84 us per step, 500 x 6-node
// subsystems 2.73 against 2.46).
//
// The CTA kernel (emt_kernels.cu) runs each subsystem on 256 threads and
// separates the step's processes by CTA barriers; for a subsystem of a few
// nodes its step is a chain of dependent FP64 operations and barriers that
// is much longer than the work.  Here a warp is a subsystem: lanes are its
// nodes, injection lanes, branches and line ends, the phases are separated
// by __syncwarp only, and kSmallWarps subsystems share a CTA (one warp per
// SM sub-partition, so their FP64 instructions do not queue behind each
// other).  The arithmetic is the CTA kernel's (Sec. III-A processes with the
// textbook companions and Bergeron lines): the same injection entries, the
// same X_hi + X_lo solve in contiguous column blocks (P lanes per row), the
// same history updates and tagged line rings.
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <cmath>

#include <cuda_runtime.h>

#include "emt_internal.h"
#include "emt_device.cuh"

namespace emt {

namespace {

constexpr int kSmallWarps = 4;

// One warp's shared memory, from the launch's limits.
struct SmallSmem {
  size_t gi, iv, vv, inp, vs, lce, sbg, ley2, leown, lefar;   // 8-byte
  size_t gilo, ivf, lck, lcm, lckind, lcstr, sbsrc, lenode, ledepth, led, rslot, wslot, ent, ilnode, ilcnt, srcg,
      recp;                                                   // 4-byte
  size_t bytes;
};

__host__ __device__ inline SmallSmem small_smem(const FwdLimits& L) {
  SmallSmem s{};
  size_t o = 0;
  auto d = [&](size_t count) { size_t r = o; o += count * 8; return r; };
  auto w = [&](size_t count) { size_t r = o; o += count * 4; return r; };
  const size_t ldg = (size_t)(L.nc | 1);
  s.gi = d((size_t)L.n * ldg);
  s.iv = d(L.nc);
  s.vv = d(L.n);
  s.inp = d((size_t)L.lc + L.sb + 2 * (size_t)L.le + 1);
  s.vs = d(2 * (size_t)L.src);
  s.lce = d(L.lc);
  s.sbg = d(L.sb);
  s.ley2 = d(L.le);
  s.leown = d(L.le);
  s.lefar = d(L.le);
  s.gilo = w((size_t)L.n * ldg);
  s.ivf = w(L.nc);
  s.lck = w(L.lc);
  s.lcm = w(L.lc);
  s.lckind = w(L.lc);
  s.lcstr = w(L.lc);
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
  s.bytes = (o + 15) & ~(size_t)15;
  return s;
}

__global__ void __launch_bounds__(32 * kSmallWarps) fwd_small_kernel(FwdParams P) {
  extern __shared__ __align__(16) unsigned char smem_all[];
  const SmallSmem L = small_smem(P.lim);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wi = blockIdx.x * kSmallWarps + warp;
  if (wi >= (P.active != nullptr ? P.n_active : P.n_sub)) return;   // (no CTA barrier here: a spare warp leaves)
  const int sidx = P.active != nullptr ? P.active[wi] : wi;
  unsigned char* sm = smem_all + (size_t)warp * L.bytes;
  double* gi = reinterpret_cast<double*>(sm + L.gi);
  double* iv = reinterpret_cast<double*>(sm + L.iv);
  double* vv = reinterpret_cast<double*>(sm + L.vv);
  double* inp = reinterpret_cast<double*>(sm + L.inp);
  double* vs = reinterpret_cast<double*>(sm + L.vs);
  double* lce = reinterpret_cast<double*>(sm + L.lce);
  double* sbg = reinterpret_cast<double*>(sm + L.sbg);
  double* ley2 = reinterpret_cast<double*>(sm + L.ley2);
  long long* leown = reinterpret_cast<long long*>(sm + L.leown);
  long long* lefar = reinterpret_cast<long long*>(sm + L.lefar);
  float* gilo = reinterpret_cast<float*>(sm + L.gilo);
  float* ivf = reinterpret_cast<float*>(sm + L.ivf);
  int* lck = reinterpret_cast<int*>(sm + L.lck);
  int* lcm = reinterpret_cast<int*>(sm + L.lcm);
  int* lckind = reinterpret_cast<int*>(sm + L.lckind);
  int* lcstr = reinterpret_cast<int*>(sm + L.lcstr);
  int* sbsrc = reinterpret_cast<int*>(sm + L.sbsrc);
  int* lenode = reinterpret_cast<int*>(sm + L.lenode);
  int* ledepth = reinterpret_cast<int*>(sm + L.ledepth);
  int* led = reinterpret_cast<int*>(sm + L.led);
  int* rslot = reinterpret_cast<int*>(sm + L.rslot);
  int* wslot = reinterpret_cast<int*>(sm + L.wslot);
  int* ent = reinterpret_cast<int*>(sm + L.ent);
  int* ilnode = reinterpret_cast<int*>(sm + L.ilnode);
  int* ilcnt = reinterpret_cast<int*>(sm + L.ilcnt);
  int* srcg = reinterpret_cast<int*>(sm + L.srcg);
  int* recp = reinterpret_cast<int*>(sm + L.recp);

  const SubDev S = P.sub[wi];
  const int n = S.n, n_str = S.n_str, nc = n + n_str, ldg = nc | 1;
  const int n_lc = S.n_lc, n_sb = S.n_sb, n_le = S.n_le, n_il = S.n_il, n_src = S.n_src;
  const int ie_base = n_lc + n_sb, zero_slot = ie_base + 2 * n_le;
  const int inp_len = zero_slot + 1;
  (void)inp_len;
  // P_r lanes per row of the solve, each over a contiguous block of blk columns
  const int pr = max(1, min(32 / max(n, 1), (int)lrintf(sqrtf((float)nc))));
  const int blk = (nc + pr - 1) / pr;
  const int src_vs = P.lim.src;

  // ---- prologue
  for (int x = lane; x < n_lc; x += 32) {
    const BranchDev b = P.br[P.lc_idx[S.lc_off + x]];
    inp[x] = P.h[EMT_CHK(P.err, S.lc_off + x, P.bnd.h, kChkHistory)];
    lce[x] = b.e;
    lck[x] = b.k;
    lcm[x] = b.m;
    lckind[x] = b.kind;
    lcstr[x] = -1;
  }
  for (int x = lane; x < n_sb; x += 32) {
    const BranchDev b = P.br[P.sb_idx[S.sb_off + x]];
    sbg[x] = b.g;
    sbsrc[x] = b.k <= -2 ? -2 - b.k : -2 - b.m;
  }
  for (int x = lane; x < n_le; x += 32) {
    const LineEndDev e = P.le[S.le_off + x];
    ley2[x] = e.y2;
    leown[x] = e.own_ring;
    lefar[x] = e.far_ring;
    lenode[x] = e.node;
    ledepth[x] = e.depth;
    led[x] = e.d;
    rslot[x] = (int)(P.n0 % e.depth);
    wslot[x] = (int)((P.n0 + e.d) % e.depth);
  }
  for (int r = lane; r < n; r += 32) recp[r] = P.rec != nullptr ? P.rec_pos[S.node_off + r] : -1;
  for (int x = lane; x < 4 * n_il; x += 32) ent[x] = P.ent[4 * (size_t)S.il_off + x];
  for (int x = lane; x < n_il; x += 32) {
    ilnode[x] = P.il_node[S.il_off + x];
    ilcnt[x] = P.il_cnt[S.il_off + x];
  }
  for (int x = lane; x < n_src; x += 32) {
    srcg[x] = P.src_global[S.src_off + x];
    vs[(P.n0 & 1) * src_vs + x] = P.src_table[EMT_CHK(P.err, P.src_global[S.src_off + x], P.bnd.src, kChkSource)];
  }
  if (lane == 0) inp[zero_slot] = 0.0;
  // solve matrix of the switch epoch in force at step n0
  const int n_te = S.n_ep;
  int te = 0;
  while (te + 1 < n_te && P.ep[S.ep_off + te + 1].start <= P.n0) ++te;
  long long next_ep_start = (te + 1 < n_te) ? P.ep[S.ep_off + te + 1].start : LLONG_MAX;
  auto load_matrix = [&](int e) {
    const int64_t off = EMT_CHK_BLOCK(P.err, P.ep[S.ep_off + e].ginv_off, n * nc, P.bnd.ginv, kChkMatrix);
    for (int i = lane; i < n * nc; i += 32) {
      const int r = i / nc, c = i - r * nc;
      gi[r * ldg + c] = P.ginv[off + i];
      gilo[r * ldg + c] = P.ginv_lo[off + i];
    }
  };
  load_matrix(te);
  __syncwarp();
  for (int x = lane; x < n_sb; x += 32) inp[n_lc + x] = sbg[x] * vs[(P.n0 & 1) * src_vs + sbsrc[x]];
  for (int t = lane; t < n_str; t += 32) {
    const int x = P.str_slot[S.str_off + t];
    lcstr[x] = t;
    iv[n + t] = -inp[x];
    ivf[n + t] = f32_trunc(-inp[x]);
  }
  // the first step's line values
  bool ok = true;
  {
    double* ie = inp + ie_base + (int)(P.n0 & 1) * n_le;
    for (int e = lane; e < n_le && ok; e += 32) {
      double v = 0.0;
      ok = poll_slot(P, P.ring + 2 * EMT_CHK(P.err, leown[e] + rslot[e], P.bnd.ring, kChkRingRead), (unsigned)P.n0,
                     sidx, e, v);
      ie[e] = v;
      const int nx = rslot[e] + 1;
      rslot[e] = nx == ledepth[e] ? 0 : nx;
    }
    ok = __all_sync(0xffffffffu, ok);
  }
  const int decim = P.rec_decim > 0 ? P.rec_decim : 1;
  int dec = (int)(P.n0 % decim);
  long long rec_row = P.n0 / decim - (dec == 0 ? 1 : 0);
  const bool writes_lines = sidx != P.hold_sub;
  __syncwarp();

  const long long n_end = P.n0 + P.n_steps;
  for (long long step = P.n0; step < n_end && ok; ++step) {
    const int par = (int)(step & 1);
    const double* vsc = vs + par * src_vs;
    const int parshift = par * n_le;
    if (step >= next_ep_start) {   // a switch event: the next epoch's matrix
      while (te + 1 < n_te && P.ep[S.ep_off + te + 1].start <= step) ++te;
      next_ep_start = (te + 1 < n_te) ? P.ep[S.ep_off + te + 1].start : LLONG_MAX;
      load_matrix(te);
      __syncwarp();
    }
    // next step's source voltages: loads issued now, stored after the solve
    double vnext = 0.0;
    if (lane < n_src && step + 1 < n_end)
      vnext = __ldg(P.src_table + EMT_CHK(P.err, (step + 1 - P.n0) * P.n_sources + srcg[lane], P.bnd.src, kChkSource));

    // process 2: injections, four entries per injection lane, a node's
    // first lane adding its other lanes' partial sums
    for (int base = 0; base < n_il; base += 32) {
      const int l = base + lane;
      double s = 0.0;
      int node = -1, cnt = 0;
      if (l < n_il) {
        node = ilnode[l];
        cnt = ilcnt[l];
        const int* e4 = ent + 4 * l;
        s = (signed_entry(inp, (unsigned)e4[0], ie_base, n_le, parshift, P.err, inp_len) +
             signed_entry(inp, (unsigned)e4[1], ie_base, n_le, parshift, P.err, inp_len)) +
            (signed_entry(inp, (unsigned)e4[2], ie_base, n_le, parshift, P.err, inp_len) +
             signed_entry(inp, (unsigned)e4[3], ie_base, n_le, parshift, P.err, inp_len));
      }
      const int wmax = __reduce_max_sync(0xffffffffu, cnt);
      double acc = s;
      for (int j = 1; j < wmax; ++j) {
        const double o = __shfl_down_sync(0xffffffffu, s, j);
        if (j < cnt) acc += o;
      }
      if (cnt > 0) {
        iv[node] = acc;
        ivf[node] = f32_trunc(acc);
      }
    }
    __syncwarp();

    // process 4: v = (X_hi + X_lo) i, lane (r, p) over the columns
    // [p blk, (p + 1) blk) of row r, then the row's first lane adds the others
    const int r = lane / pr, p = lane - r * pr;
    double a = 0.0;
    float b = 0.f;
    if (r < n) {
      const double* row = gi + r * ldg;
      const float* rowl = gilo + r * ldg;
      const int j1 = min(nc, (p + 1) * blk);
      for (int j = p * blk; j < j1; ++j) {
        a = fma(row[j], iv[j], a);
        b = fmaf(rowl[j], ivf[j], b);
      }
    }
    for (int q = 1; q < pr; ++q) {
      const double oa = __shfl_down_sync(0xffffffffu, a, q);
      const float ob = __shfl_down_sync(0xffffffffu, b, q);
      if (p == 0) {
        a += oa;
        b += ob;
      }
    }
    const bool rec_now = P.rec != nullptr && dec == 0 && rec_row < P.rec_rows;
    if (r < n && p == 0) {
      const double v = a + f64_of(b);
      vv[r] = v;
      if (rec_now && recp[r] >= 0)
        P.rec[EMT_CHK(P.err, (rec_row - P.rec_row0) * P.n_rec + recp[r], P.bnd.rec, kChkRecord)] = v;
    }
    if (dec == 0) ++rec_row;
    if (++dec == decim) dec = 0;
    if (lane < n_src) vs[(par ^ 1) * src_vs + lane] = vnext;
    __syncwarp();

    // process 1: history currents, line outputs, next step's source injections
    const double* ie_cur = inp + ie_base + parshift;
    const double* vs_next = vs + (par ^ 1) * src_vs;
    for (int it = lane; it < n_lc; it += 32) {
      const int k = lck[it], m = lcm[it];
      const double vk = k >= 0 ? vv[k] : (k == -1 ? 0.0 : vsc[-2 - k]);
      const double vm = m >= 0 ? vv[m] : (m == -1 ? 0.0 : vsc[-2 - m]);
      const double hn = lckind[it] == 1 ? fma(lce[it], vk - vm, inp[it]) : fma(lce[it], vk - vm, -inp[it]);
      inp[it] = hn;
      const int t = lcstr[it];
      if (t >= 0) {   // strong branch: its current drives the extra solve column
        iv[n + t] = -hn;
        ivf[n + t] = f32_trunc(-hn);
      }
    }
    for (int e = lane; e < n_le; e += 32) {
      const double out = fma(-ley2[e], vv[lenode[e]], -ie_cur[e]);
      if (writes_lines)
        st_tagged(P.ring + 2 * EMT_CHK(P.err, lefar[e] + wslot[e], P.bnd.ring, kChkRingWrite),
                  (unsigned)(step + led[e]), out);
      const int nx = wslot[e] + 1;
      wslot[e] = nx == ledepth[e] ? 0 : nx;
    }
    for (int x = lane; x < n_sb; x += 32) inp[n_lc + x] = sbg[x] * vs_next[sbsrc[x]];
    // the next step's line values
    if (n_le > 0 && step + 1 < n_end) {
      double* ie_next = inp + ie_base + (par ^ 1) * n_le;
      bool lok = true;
      for (int e = lane; e < n_le && lok; e += 32) {
        double v = 0.0;
        lok = poll_slot(P, P.ring + 2 * EMT_CHK(P.err, leown[e] + rslot[e], P.bnd.ring, kChkRingRead),
                        (unsigned)(step + 1), sidx, e, v);
        ie_next[e] = v;
        const int nx = rslot[e] + 1;
        rslot[e] = nx == ledepth[e] ? 0 : nx;
      }
      ok = __all_sync(0xffffffffu, lok);
    }
    __syncwarp();
  }
  if (ok) {
    for (int x = lane; x < n_lc; x += 32) P.h[EMT_CHK(P.err, S.lc_off + x, P.bnd.h, kChkHistory)] = inp[x];
    if (P.n_steps > 0)   // the values consumed at the last step (the CTA kernel's interpolation reads them)
      for (int x = lane; x < n_le; x += 32)
        P.le_prev[S.le_off + x] = inp[ie_base + (int)((n_end - 1) & 1) * n_le + x];
  }
}

}  // namespace

size_t small_smem_bytes(const FwdLimits& lim) { return (size_t)kSmallWarps * small_smem(lim).bytes; }

cudaError_t launch_forward_small(const FwdParams& p, cudaStream_t st) {
  const size_t smem = small_smem_bytes(p.lim);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fwd_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = ((p.active != nullptr ? p.n_active : p.n_sub) + kSmallWarps - 1) / kSmallWarps;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fwd_small_kernel, 32 * kSmallWarps, smem);
  if (e != cudaSuccess) return e;
  if ((long long)per_sm * n_sm < grid) return cudaErrorCooperativeLaunchTooLarge;
  FwdParams arg = p;
  void* args[] = {&arg};
  // cooperative launch: all CTAs co-resident, so every ring wait can end
  return cudaLaunchCooperativeKernel((const void*)fwd_small_kernel, dim3(grid), dim3(32 * kSmallWarps), args, smem, st);
}

}  // namespace emt
