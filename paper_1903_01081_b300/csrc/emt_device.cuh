// Device helpers shared by the persistent kernels (forward and adjoint).
#pragma once
#include <stdint.h>

#include <climits>

#include <cuda_runtime.h>

#include "emt_internal.h"

namespace emt {

// Checks build (compiled with -DEMT_CHECKS; the library libemt_checks.so):
// every index into a global array whose value comes from device data is
// tested against the array's length; one outside latches {kErrBounds, site,
// index, length} in the device error word (emt_sync reports it) and is
// replaced by 0, so that the access stays in bounds.  Nothing traps.  In the
// normal build the macros are the index itself.  (kErrBounds: emt_internal.h)
#ifdef EMT_CHECKS
__device__ __forceinline__ int64_t chk_index(int32_t* err, int64_t i, int64_t n, int site) {
  if (i >= 0 && i < n) return i;
  if (err != nullptr && atomicCAS(err, 0, kErrBounds) == 0) {
    err[1] = site;
    err[2] = (int)(i > INT32_MAX ? INT32_MAX : (i < INT32_MIN ? INT32_MIN : i));
    err[3] = (int)(n > INT32_MAX ? INT32_MAX : n);
  }
  return 0;
}
// a block [off, off + count) inside [0, n): off, else 0
__device__ __forceinline__ int64_t chk_block(int32_t* err, int64_t off, int64_t count, int64_t n, int site) {
  if (off >= 0 && off + count <= n) return off;
  chk_index(err, off + count - 1, n, site);
  return 0;
}
#define EMT_CHK(err, i, n, site) ::emt::chk_index((err), (int64_t)(i), (int64_t)(n), (site))
#define EMT_CHK_BLOCK(err, off, count, n, site) ::emt::chk_block((err), (int64_t)(off), (int64_t)(count), (int64_t)(n), (site))
#else
#define EMT_CHK(err, i, n, site) (i)
#define EMT_CHK_BLOCK(err, off, count, n, site) (off)
#endif
// sites reported by the checks build
enum ChkSite { kChkRingRead = 1, kChkRingWrite, kChkMatrix, kChkRecord, kChkHistory, kChkSource, kChkNlColumn,
               kChkTape, kChkTarget, kChkEntry };

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Tagged ring slot: two words (tag << 32) | low / high half of the double,
// written and read as one 16-byte single-copy-atomic access each.
__device__ __forceinline__ void st_tagged(unsigned long long* p, unsigned tag, double v) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const unsigned long long w0 = ((unsigned long long)tag << 32) | (bits & 0xffffffffull);
  const unsigned long long w1 = ((unsigned long long)tag << 32) | (bits >> 32);
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(w0), "l"(w1) : "memory");
}

__device__ __forceinline__ bool ld_tagged(const unsigned long long* p, unsigned tag, double& v) {
  unsigned long long w0, w1;
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(w0), "=l"(w1) : "l"(p) : "memory");
  if ((unsigned)(w0 >> 32) != tag || (unsigned)(w1 >> 32) != tag) return false;
  v = __longlong_as_double((long long)((w1 << 32) | (w0 & 0xffffffffull)));
  return true;
}

// double -> float by truncation, on the integer pipe (a conversion
// instruction would take the slow FP64 pipe on B300).  Only for the
// single-precision correction chains, where the truncation error (< 1 ulp
// of a float) is far below what they correct; values below 2^-126 become 0
// and finite values stay finite (|x| < 2^128 on these paths).
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const unsigned sign = hi & 0x80000000u;
  if (e <= 0) return __uint_as_float(sign);
  return __uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffull));
}

// float -> double, exact for normal floats, on the integer pipe (subnormal
// floats become 0: they only occur as corrections below 2^-126).
__device__ __forceinline__ double f64_of(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0) return __longlong_as_double((long long)sign);
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// A tagged slot's two words, loaded without looking at them (so that several
// slots' loads can be in flight at once), and the check of such a pair.
__device__ __forceinline__ void ld_tagged_raw(const unsigned long long* p, unsigned long long& w0,
                                              unsigned long long& w1) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(w0), "=l"(w1) : "l"(p) : "memory");
}

__device__ __forceinline__ bool tagged_value(unsigned long long w0, unsigned long long w1, unsigned tag, double& v) {
  if ((unsigned)(w0 >> 32) != tag || (unsigned)(w1 >> 32) != tag) return false;
  v = __longlong_as_double((long long)((w1 << 32) | (w0 & 0xffffffffull)));
  return true;
}

// Wait for a ring slot to carry `tag` and return its value.  Bounded: on
// exceeding the time budget (or seeing another CTA's error) it latches an
// error {5, subsystem, line end, tag} and returns false.  Params: the
// forward or adjoint kernel's parameters (ring-independent fields err,
// wait_budget_ns).
template <class Params>
__device__ __forceinline__ bool poll_slot(const Params& P, const unsigned long long* slot, unsigned tag, int sidx,
                                          int e, double& v) {
  if (ld_tagged(slot, tag, v)) return true;
  const unsigned long long t0 = global_ns();
  unsigned spins = 0;
  while (!ld_tagged(slot, tag, v)) {
    if ((++spins & 31u) == 0) {
      if (ld_volatile(P.err) != 0) return false;
      if (global_ns() - t0 > P.wait_budget_ns || spins > (1u << 30)) {
        if (atomicCAS(P.err, 0, 5) == 0) {
          P.err[1] = sidx;
          P.err[2] = e;
          P.err[3] = (int)tag;
        }
        return false;
      }
    }
  }
  return true;
}

// Signed injection entry (see kEntryNeg): the input value with the entry's
// sign bit applied; line-end entries are shifted to the current parity block.
__device__ __forceinline__ double signed_entry(const double* inp, unsigned raw, int ie_base, int n_le, int parshift,
                                                int32_t* err, int inp_len) {
  int idx = (int)(raw & ~kEntryNeg);
  if ((unsigned)(idx - ie_base) < (unsigned)n_le) idx += parshift;
  idx = (int)EMT_CHK(err, idx, inp_len, kChkEntry);
  (void)err;
  (void)inp_len;
  const unsigned long long bits =
      (unsigned long long)__double_as_longlong(inp[idx]) ^ ((unsigned long long)(raw & kEntryNeg) << 32);
  return __longlong_as_double((long long)bits);
}

}  // namespace emt
