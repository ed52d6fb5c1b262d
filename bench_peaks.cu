// Peaks that bench.py divides by (B300, sm_103a): FP64 throughput of the
// whole chip (DFMA alone, FP64 mma.sync alone, both mixed in one CTA), the
// per-warp issue interval and latency of DFMA, and, for context, the bf16
// mma.sync rate and latency.  Prints one JSON line.
//
// Method: every thread runs 8 independent FMA chains (or 4 independent
// m8n8k4 f64 accumulators per warp) for `iters` iterations on 148 x k CTAs
// of 256 threads (k = 1, 2, 4, 8); the kernel is timed with CUDA events
// after one warm-up launch; the best k is the peak.  Latencies come from
// clock64 around a single warp's loop.  Results go to a buffer sized by
// the grid, so the loops are not optimised away.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o bench_peaks bench_peaks.cu && ./bench_peaks
#include <cstdio>
#include <cuda_runtime.h>

#define CK(x)                                                                    \
  do {                                                                           \
    cudaError_t e_ = (x);                                                        \
    if (e_ != cudaSuccess) {                                                     \
      printf("{\"error\": \"%s at line %d\"}\n", cudaGetErrorString(e_), __LINE__); \
      return 1;                                                                  \
    }                                                                            \
  } while (0)

__global__ void dfma_chains(double* out, int iters) {
  double a[8];
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-9 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], 0.9999999, 1e-7);
  }
  double s = 0;
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__global__ void dmma_chains(double* out, int iters) {
  double d[8];
  for (int k = 0; k < 8; ++k) d[k] = 0;
  const double a = 1.0 + threadIdx.x * 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k) dmma(d[2 * k], d[2 * k + 1], a, 0.5);
  }
  double s = 0;
  for (int k = 0; k < 8; ++k) s += d[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// even warps DFMA, odd warps DMMA, same iteration count
__global__ void mixed_chains(double* out, int iters) {
  double s = 0;
  if (((threadIdx.x >> 5) & 1) == 0) {
    double a[8];
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-9 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fma(a[k], 0.9999999, 1e-7);
    }
    for (int k = 0; k < 8; ++k) s += a[k];
  } else {
    double d[8];
    for (int k = 0; k < 8; ++k) d[k] = 0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < 4; ++k) dmma(d[2 * k], d[2 * k + 1], 1.0 + threadIdx.x * 1e-9, 0.5);
    }
    for (int k = 0; k < 8; ++k) s += d[k];
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ void hmma(float* d, unsigned a0, unsigned b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%4,%4,%4}, {%5,%5}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(b0));
}

// chains independent bf16 accumulators per warp; cycles of the loop in cyc[block]
template <int chains>
__global__ void hmma_chains(float* out, long long* cyc, int iters) {
  float d[chains][4];
  for (int c = 0; c < chains; ++c) d[c][0] = d[c][1] = d[c][2] = d[c][3] = 0.f;
  const unsigned a = 0x3f803f80u ^ (threadIdx.x & 1), b = 0x3f803f80u;
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < chains; ++c) hmma(d[c], a, b);
  }
  const long long t1 = clock64();
  float s = 0;
  for (int c = 0; c < chains; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

// one warp: a dependent DFMA chain, then 8 independent chains
__global__ void dfma_latency(double* out, long long* cyc, int iters) {
  double a = threadIdx.x * 1e-9, b[8];
  for (int k = 0; k < 8; ++k) b[k] = a + k;
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) a = fma(a, 0.9999999, 1e-7);
  const long long t1 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) b[k] = fma(b[k], 0.9999999, 1e-7);
  }
  const long long t2 = clock64();
  double s = a;
  for (int k = 0; k < 8; ++k) s += b[k];
  out[threadIdx.x] = s;
  if (threadIdx.x == 0) {
    cyc[0] = t1 - t0;
    cyc[1] = t2 - t1;
  }
}

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// SM clock: clock64 ticks over 2 ms of %globaltimer
__global__ void sm_clock(long long* r) {
  const unsigned long long g0 = gtime();
  const long long c0 = clock64();
  while (gtime() - g0 < 2000000ull) {
  }
  const unsigned long long g1 = gtime();
  const long long c1 = clock64();
  r[0] = (long long)(g1 - g0);
  r[1] = c1 - c0;
}

template <class F>
static float timed(F f) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  f();
  cudaDeviceSynchronize();
  cudaEventRecord(e0);
  f();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

int main() {
  int n_sm = 0;
  CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, 0));
  const int th = 256, max_grid = n_sm * 8;
  double* dout;
  float* fout;
  long long* dcyc;
  CK(cudaMalloc(&dout, (size_t)max_grid * th * sizeof(double)));
  CK(cudaMalloc(&fout, (size_t)max_grid * th * sizeof(float)));
  CK(cudaMalloc(&dcyc, (size_t)max_grid * sizeof(long long)));
  long long hc[2];
  sm_clock<<<1, 1>>>(dcyc);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(hc, dcyc, 2 * sizeof(long long), cudaMemcpyDeviceToHost));
  const double mhz0 = 1e3 * (double)hc[1] / (double)hc[0];
  const int iters = 20000;
  double best_dfma = 0, best_dmma = 0, best_mixed = 0;
  for (int k : {1, 2, 4, 8}) {
    const int grid = n_sm * k;
    float ms = timed([&] { dfma_chains<<<grid, th>>>(dout, iters); });
    best_dfma = fmax(best_dfma, 2.0 * 8 * iters * (double)grid * th / ms / 1e6);
    ms = timed([&] { dmma_chains<<<grid, th>>>(dout, iters); });
    best_dmma = fmax(best_dmma, 512.0 * 4 * iters * (double)grid * (th / 32) / ms / 1e6);
    ms = timed([&] { mixed_chains<<<grid, th>>>(dout, iters); });
    best_mixed = fmax(best_mixed, (2.0 * 8 * iters * 32 + 512.0 * 4 * iters) * (double)grid * (th / 64) / ms / 1e6);
  }
  CK(cudaGetLastError());
  const int it2 = 4000;
  const float ms = timed([&] { hmma_chains<8><<<n_sm * 4, th>>>(fout, dcyc, it2); });
  const double hmma_tflops = 4096.0 * 8 * it2 * (double)(n_sm * 4) * (th / 32) / ms / 1e9;
  hmma_chains<1><<<1, 32>>>(fout, dcyc, 1000);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(hc, dcyc, sizeof(long long), cudaMemcpyDeviceToHost));
  const double hmma_lat = hc[0] / 1000.0;
  hmma_chains<8><<<1, 32>>>(fout, dcyc, 1000);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(hc, dcyc, sizeof(long long), cudaMemcpyDeviceToHost));
  const double hmma_issue = hc[0] / 8000.0;
  dfma_latency<<<1, 32>>>(dout, dcyc, 1000);
  CK(cudaDeviceSynchronize());
  dfma_latency<<<1, 32>>>(dout, dcyc, 1000);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(hc, dcyc, 2 * sizeof(long long), cudaMemcpyDeviceToHost));
  const double dfma_lat = hc[0] / 1000.0, dfma_issue = hc[1] / 8000.0;
  sm_clock<<<1, 1>>>(dcyc);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(hc, dcyc, 2 * sizeof(long long), cudaMemcpyDeviceToHost));
  const double mhz1 = 1e3 * (double)hc[1] / (double)hc[0];
  printf("{\"fp64_dfma_gflops\": %.1f, \"fp64_dmma_gflops\": %.1f, \"fp64_mixed_gflops\": %.1f, "
         "\"bf16_mma_sync_tflops\": %.1f, \"dfma_dependent_latency_cycles\": %.1f, "
         "\"dfma_issue_interval_cycles_one_warp\": %.1f, \"bf16_mma_sync_latency_cycles\": %.1f, "
         "\"bf16_mma_sync_issue_interval_cycles_one_warp\": %.1f, \"sm_mhz_before\": %.0f, \"sm_mhz_after\": %.0f, "
         "\"sms\": %d}\n",
         best_dfma, best_dmma, best_mixed, hmma_tflops, dfma_lat, dfma_issue, hmma_lat, hmma_issue, mhz0, mhz1, n_sm);
  return 0;
}
