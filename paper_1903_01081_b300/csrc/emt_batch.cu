// Multi-scenario time loop for sm_103a (B300).
//
// The paper's multi-scenario strategy (Sec. III-B): the scenarios of a
// study share the network structure, so every basic process becomes one
// SIMT operation over all scenarios.  Here one CTA runs the whole network
// for a tile of S_t scenarios; a warp's lanes are (item, scenario) with the
// scenario fastest, so each solve-matrix entry a warp loads serves all its
// scenarios (for a shared G^-1 the solve over the tile is a dense GEMM
// G^-1 [i^(1) ... i^(S_t)], done with DFMA: on B300 FP64 DMMA is slower).
// A scenario that changes a subsystem's G (an element removed, a switch
// closed) selects its own prefactored matrix for that subsystem and
// switch epoch.  Scenarios are independent, so CTAs never wait on each
// other.  Per step and subsystem: injections, solve, updates, three
// barriers; the work is FP64-throughput-bound, not latency-bound.
//
// Formulas as in emt_kernels.cu (trapezoidal companions, Bergeron lines;
// the paper's Sec. III-A processes with the textbook forms of its ref. [2]).
#include <stdint.h>

#include <algorithm>

#include <cuda_runtime.h>

#include "emt_internal.h"

namespace emt {

namespace {

constexpr int kBatchThreads = 512;

__device__ __forceinline__ int mat_for(const BatchParams& P, int sigma, int s, long long step) {
  const int64_t p0 = P.msel_ptr[(int64_t)sigma * P.n_sub + s], p1 = P.msel_ptr[(int64_t)sigma * P.n_sub + s + 1];
  int m = P.msel_mat[p0];
  for (int64_t x = p0 + 1; x < p1 && P.msel_start[x] <= step; ++x) m = P.msel_mat[x];
  return m;
}

__global__ void __launch_bounds__(kBatchThreads, 1) batch_kernel(BatchParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int St = P.S_t;
  const int sigma0 = blockIdx.x * St;
  const int n_here = min(St, P.S - sigma0);   // scenarios of this tile
  double* vs = reinterpret_cast<double*>(smem_raw);                  // [n_sources][St]
  double* iv = vs + (size_t)P.n_sources * St;                        // [max_nc][St]
  double* vv = iv + (size_t)P.max_nc * St;                           // [max_nc][St]
  float* ivf = reinterpret_cast<float*>(vv + (size_t)P.max_nc * St); // [max_nc][St]
  const int T = blockDim.x, tid = threadIdx.x;
  const int S = P.S;

  const int decim = P.rec_decim > 0 ? P.rec_decim : 1;
  const long long n_end = P.n0 + P.n_steps;
  for (long long step = P.n0; step < n_end; ++step) {
    const double t = (double)step * P.dt;
    // process 1 for sources: v_src(t_n) per scenario, argument (omega t) + phase
    for (int x = tid; x < P.n_sources * St; x += T) {
      const int src = x / St, sl = x - src * St;
      if (sl < n_here) {
        const int sg = sigma0 + sl;
        vs[x] = P.src_amp[(int64_t)sg * P.n_sources + src] *
                sin(__dadd_rn(__dmul_rn(P.src_omega[src], t), P.src_phase[(int64_t)sg * P.n_sources + src]));
      }
    }
    __syncthreads();
    const bool rec_now = P.rec != nullptr && step % decim == 0 && step / decim - 1 < P.rec_rows;
    const long long rec_row = step / decim - 1;

    for (int s = 0; s < P.n_sub; ++s) {
      const SubDev Sd = P.sub[s];
      const int n = Sd.n, nc = n + Sd.n_str;
      const int ie_base = Sd.n_lc + Sd.n_sb, zero_slot = ie_base + 2 * Sd.n_le;

      // process 2: nodal injections (and the strong-branch inputs -h)
      for (int x = tid; x < nc * St; x += T) {
        const int k = x / St, sl = x - k * St;
        if (sl >= n_here) continue;
        const int sg = sigma0 + sl;
        double acc = 0.0;
        if (k < n) {
          const int gk = Sd.node_off + k;
          const int l0 = P.node_l0[gk], l1 = l0 + P.node_nl[gk];
          for (int l = l0; l < l1; ++l)
            for (int u = 0; u < 4; ++u) {
              const unsigned raw = (unsigned)P.ent[4 * (int64_t)(Sd.il_off + l) + u];
              const int idx = (int)(raw & ~kEntryNeg);
              if (idx >= zero_slot) continue;
              double val;
              if (idx < Sd.n_lc) {
                const int64_t gl = Sd.lc_off + idx;
                val = P.h[gl * S + sg];
              } else if (idx < ie_base) {
                const int x2 = idx - Sd.n_lc;
                const int64_t gs = Sd.sb_off + x2;
                const BranchDev b = P.br[P.sb_idx[gs]];
                const int j = b.k <= -2 ? -2 - b.k : -2 - b.m;
                val = b.g * vs[P.src_global[Sd.src_off + j] * St + sl];
                if (P.keep_sb && !P.keep_sb[gs * S + sg]) val = 0.0;
              } else {
                const int e = idx - ie_base;
                const int64_t ge = Sd.le_off + e;
                const LineEndDev L = P.le[ge];
                val = P.ring[(P.le_bring[ge] + step % (L.d + 1)) * S + sg];
              }
              acc += (raw & kEntryNeg) ? -val : val;
            }
        } else {
          const int64_t gl = Sd.lc_off + P.str_slot[Sd.str_off + (k - n)];
          acc = -P.h[gl * S + sg];
        }
        iv[k * St + sl] = acc;
        ivf[k * St + sl] = (float)acc;
      }
      __syncthreads();

      // process 4: v = (X_hi + X_lo) [i; -h_strong] with each scenario's matrix
      for (int x = tid; x < n * St; x += T) {
        const int r = x / St, sl = x - r * St;
        if (sl >= n_here) continue;
        const int sg = sigma0 + sl;
        const EpochDev E = P.ep[mat_for(P, sg, s, step)];
        const double* row = P.ginv + E.ginv_off + (int64_t)r * nc;
        const float* rowl = P.ginv_lo + E.ginv_off + (int64_t)r * nc;
        double a = 0.0;
        float b = 0.f;
        for (int j = 0; j < nc; ++j) {
          a = fma(__ldg(row + j), iv[j * St + sl], a);
          b = fmaf(__ldg(rowl + j), ivf[j * St + sl], b);
        }
        const double v = a + (double)b;
        vv[r * St + sl] = v;
        if (rec_now) {
          const int pos = P.rec_pos[Sd.node_off + r];
          if (pos >= 0) P.rec[(rec_row * S + sg) * P.n_rec + pos] = v;
        }
      }
      __syncthreads();

      // process 1: history currents and line outputs of this subsystem
      const int n_items = Sd.n_lc + Sd.n_le;
      for (int x = tid; x < n_items * St; x += T) {
        const int it = x / St, sl = x - it * St;
        if (sl >= n_here) continue;
        const int sg = sigma0 + sl;
        if (it < Sd.n_lc) {
          const int64_t gl = Sd.lc_off + it;
          if (P.keep_lc && !P.keep_lc[gl * S + sg]) continue;   // removed: h stays 0
          const BranchDev b = P.br[P.lc_idx[gl]];
          const double vk = b.k >= 0 ? vv[b.k * St + sl]
                                     : (b.k == -1 ? 0.0 : vs[P.src_global[Sd.src_off + (-2 - b.k)] * St + sl]);
          const double vm = b.m >= 0 ? vv[b.m * St + sl]
                                     : (b.m == -1 ? 0.0 : vs[P.src_global[Sd.src_off + (-2 - b.m)] * St + sl]);
          const double hv = P.h[gl * S + sg];
          P.h[gl * S + sg] = b.kind == 1 ? fma(b.e, vk - vm, hv) : fma(b.e, vk - vm, -hv);
        } else {
          const int e = it - Sd.n_lc;
          const int64_t ge = Sd.le_off + e;
          const LineEndDev L = P.le[ge];
          const double ie = P.ring[(P.le_bring[ge] + step % (L.d + 1)) * S + sg];
          double out = fma(-L.y2, vv[L.node * St + sl], -ie);
          if (P.keep_le && !P.keep_le[ge * S + sg]) out = 0.0;   // removed line
          P.ring[(P.le_bfar[ge] + (step + L.d) % (L.d + 1)) * S + sg] = out;
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace

int batch_threads() { return kBatchThreads; }

size_t batch_smem_bytes(const BatchParams& p) {
  return (size_t)p.n_sources * p.S_t * sizeof(double) + 2 * (size_t)p.max_nc * p.S_t * sizeof(double) +
         (size_t)p.max_nc * p.S_t * sizeof(float);
}

cudaError_t launch_batch(const BatchParams& p, cudaStream_t st) {
  const size_t smem = batch_smem_bytes(p);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (p.S + p.S_t - 1) / p.S_t;
  batch_kernel<<<grid, kBatchThreads, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace emt
