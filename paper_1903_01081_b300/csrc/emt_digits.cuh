// Exact fixed-point "digit" form of the dense solve v = X i (process 4),
// for the bf16 tensor cores.
//
// B300 runs FP64 at ~2 FMA per clock per SM (a warp's DFMA holds its
// sub-partition's FP64 pipe for 64 cycles), while its bf16 tensor cores
// take a 16 x 8 x 16 product in ~8 cycles per warp.  The solve is therefore
// done as an exact integer product:
//
//   row r of X    -> M[r][k] = round(X[r][k] 2^(62 - E_r)),  |X[r][k]| < 2^E_r
//   injection i   -> N[k]    = round(i[k]    2^(62 - E_i)),  |i[k]|    < 2^E_i
//
// (62-bit two's-complement integers), each split into eight balanced base-256
// digits d_j in [-128, 127] (the top one in [-65, 64]),
//
//   M = sum_a m_a 256^a,  N = sum_b n_b 256^b.
//
// A digit is an integer of at most 8 significant bits, so bf16 holds it
// exactly, and a product of two is at most 2^14: the fp32 accumulator of a
// K <= 128 dot product of digit vectors, D_ab[r] = sum_k m_a[r][k] n_b[k],
// stays below 2^21 and is exact.  Then
//
//   sum_k M[r][k] N[k] = sum_{a,b} 256^(a+b) D_ab[r],
//
// of which the pairs a + b >= 6 are kept (the rest add less than 2^-66 of
// the largest possible value), grouped as T = sum_{s=6..14} G_s 256^(s-6),
// G_s = sum_{a+b=s} D_ab, an exact integer below 2^88, and
//
//   v[r] = T 2^(E_r + E_i - 76),
//
// rounded once to double (round to nearest even).  The errors are those of
// the two fixed-point roundings (2^-63 of the row's largest entry and of the
// largest injection) and of the dropped pairs; the explicit inverse keeps its
// 2^-77 accuracy (X = X_hi + X_lo) down to 2^-63 of each row's largest entry.
//
// Everything here is integer arithmetic, usable on the host as well (the
// CPU tests pin these helpers against exact rational arithmetic).
#pragma once
#include <stdint.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace emt {

// N' = N + kDigitBias turns the balanced digits into plain bytes: digit j of
// N (j < 7) is byte j of N' minus 128, the top digit is N' >> 56 (signed).
constexpr long long kDigitBias = 0x0080808080808080ll;
constexpr int kDigits = 8;            // base-256 digits per fixed-point value
constexpr int kDigitGroupLo = 6;      // smallest kept a + b
constexpr int kDigitMaxK = 128;       // columns of a solve matrix in digit form
constexpr int kDigitMaxRows = 64;     // rows of a solve matrix in digit form

__host__ __device__ __forceinline__ int dg_clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

__host__ __device__ __forceinline__ unsigned long long dg_bits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  union { double d; unsigned long long u; } c;
  c.d = x;
  return c.u;
#endif
}

__host__ __device__ __forceinline__ double dg_double(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  union { double d; unsigned long long u; } c;
  c.u = b;
  return c.d;
#endif
}

// Biased exponent field of x (0 for zero and subnormals, which the digit
// form treats as zero).
__host__ __device__ __forceinline__ unsigned dg_expo(double x) { return (unsigned)(dg_bits(x) >> 52) & 0x7ffu; }

// round(x 2^(62 - E)) for |x| < 2^E, E = emax - 1022 (emax = the largest
// biased exponent of the values sharing the scale, >= 1): the 53-bit
// significand shifted by expo(x) - emax + 9 <= 9, rounded half away from
// zero when bits fall off; 0 for zero or subnormal x.
__host__ __device__ __forceinline__ long long dg_fixed(double x, unsigned emax) {
  const unsigned long long b = dg_bits(x);
  const int e = (int)((b >> 52) & 0x7ffu);
  if (e == 0) return 0;
  const unsigned long long mant = (b & 0xfffffffffffffull) | 0x10000000000000ull;
  const int sh = e - (int)emax + 9;
  unsigned long long m;
  if (sh >= 0) m = mant << sh;
  else if (sh > -54) m = (mant + (1ull << (-sh - 1))) >> (-sh);
  else m = 0;
  return (b >> 63) ? -(long long)m : (long long)m;
}

// bf16 bit pattern of digit j of N, given N' = N + kDigitBias: the byte u
// (top digit: N' >> 56 plus 128) is exact in float as 2^23 + u - (2^23 +
// 128), and a float of at most 8 significant bits keeps them all in bf16.
__host__ __device__ __forceinline__ unsigned dg_digit_bf16(long long np, int j) {
  const unsigned u = (j < kDigits - 1) ? (unsigned)((unsigned long long)np >> (8 * j)) & 0xffu
                                       : (unsigned)((int)(np >> 56) + 128);
  union { unsigned i; float f; } c;
  c.i = 0x4B000000u | u;
  c.f = c.f - 8388736.0f;
  return c.i >> 16;
}

// The digit itself (for the host tests and the matrix conversion).
__host__ __device__ __forceinline__ int dg_digit(long long np, int j) {
  return (j < kDigits - 1) ? (int)(((unsigned long long)np >> (8 * j)) & 0xffu) - 128 : (int)(np >> 56);
}

// Exact integer value of an fp32 accumulator |d| < 2^22 (1.5 2^23 + d has a
// unit last place).
__host__ __device__ __forceinline__ int dg_acc_int(float d) {
  union { float f; int i; } c;
  c.f = d + 12582912.0f;
  return c.i - 0x4B400000;
}

// T = ta 2^40 + tb (ta = sum_{s>=11} G_s 256^(s-11), tb = sum_{6<=s<=10}
// G_s 256^(s-6)) times 2^xexp, rounded once to double (nearest, ties to
// even); |T| < 2^88.  Results below the normal range flush to zero.
__host__ __device__ __forceinline__ double dg_to_double(long long ta, long long tb, int xexp) {
  const unsigned long long lo_a = (unsigned long long)ta << 40;
  const unsigned long long lo_b = (unsigned long long)tb;
  unsigned long long lo = lo_a + lo_b;
  long long hi = (ta >> 24) + (tb >> 63) + (lo < lo_a ? 1 : 0);
  const unsigned long long sign = hi < 0 ? 1ull : 0ull;
  if (sign) {   // magnitude of the 128-bit two's complement
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0 ? 1 : 0);
  }
  const unsigned long long uh = (unsigned long long)hi;
  if (uh == 0 && lo == 0) return 0.0;
  const int lz = uh ? dg_clz64(uh) : 64 + dg_clz64(lo);
  unsigned long long top, rest;
  if (uh) {
    top = (uh << lz) | (lz ? (lo >> (64 - lz)) : 0ull);
    rest = lz ? (lo << lz) : lo;
  } else {
    top = lo << (lz - 64);
    rest = 0;
  }
  int p = 127 - lz;   // position of the leading one
  unsigned long long m = top >> 11;
  const unsigned long long rb = (top >> 10) & 1ull;
  const unsigned long long sticky = (top & 0x3ffull) | rest;
  if (rb && (sticky || (m & 1ull))) {
    ++m;
    if (m == (1ull << 53)) {
      m >>= 1;
      ++p;
    }
  }
  const int be = p + xexp + 1023;
  if (be <= 0) return sign ? -0.0 : 0.0;
  if (be >= 2047) return dg_double((sign << 63) | 0x7ff0000000000000ull);
  return dg_double((sign << 63) | ((unsigned long long)be << 52) | (m & 0xfffffffffffffull));
}

// Offsets (32-bit words) of a matrix in digit form: rt row tiles of 16 rows,
// ks column steps of 16; fragment (R, a, s) at ((R kDigits + a) ks + s) 128
// words, lane l's four A registers at 4 l; then 16 rt row exponents.
__host__ __device__ __forceinline__ long long dg_frag_words(int rt, int ks) { return (long long)rt * kDigits * ks * 128; }
__host__ __device__ __forceinline__ long long dg_matrix_words(int rt, int ks) { return dg_frag_words(rt, ks) + 16ll * rt; }

}  // namespace emt
