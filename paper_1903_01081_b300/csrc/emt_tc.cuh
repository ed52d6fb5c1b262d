// tcgen05 building blocks of the dense solve in the digit form of
// emt_digits.cuh on the tensor cores (the multi-scenario kernel,
// emt_batch.cu): shared-memory matrix and instruction descriptors, the MMA,
// its commit to an mbarrier, tensor-memory loads, bounded mbarrier waits,
// bulk copies, and the integer helpers of the digit tables and the
// accumulator read-back.
#pragma once
#include <stdint.h>

#include <cuda_runtime.h>

#include "emt_device.cuh"
#include "emt_digits.cuh"

namespace emt {
namespace {

// Every tensor-core wait has a time budget; past it the kernel latches
// {kErrTensorWait, subsystem, what, step} and leaves (reported by emt_sync).
constexpr unsigned long long kTensorWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05.mma, K-major without swizzle:
// start address, lbo = bytes between the two 8-column halves of a
// 16-column K slice, sbo = bytes between consecutive 8-row groups, the
// descriptor version 1 (bits 46-47), layout 0 (no swizzle).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: f32 accumulator (bits 4-5 = 1), bf16
// A and B (bits 7-9, 10-12 = 1), both K-major, N / 8 at bit 17, M / 16 at
// bit 24.
__device__ __forceinline__ uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// the MMAs issued so far by this thread arrive on the mbarrier when done
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_ld2(uint32_t taddr, uint32_t& a, uint32_t& b) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(a), "=r"(b) : "r"(taddr) : "memory");
}

__device__ __forceinline__ void tc_ld4(uint32_t taddr, uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
               : "r"(taddr)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for the mbarrier's phase `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (unsigned spins = 0;; ++spins) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((spins & 15u) == 15u && global_ns() - t0 > kTensorWaitNs) return false;
  }
}

// One bulk copy global -> shared (16-byte aligned, a multiple of 16 bytes)
// completing on the mbarrier, which expects that many bytes.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

// Exact integer value of an fp32 accumulator entry (an integer, |x| <= 2^24):
// 1.5 2^23 + x has a unit last place for |x| < 2^22 (one add on the FP32
// pipe); the rare larger ones take the conversion instruction.
__device__ __forceinline__ int acc_int(uint32_t bits) {
  const float x = __uint_as_float(bits);
  if (fabsf(x) < 4194304.0f) return __float_as_int(x + 12582912.0f) - 0x4B400000;
  return __float2int_rn(x);
}

// bf16 pair (digit of n0' in the low half, of n1' in the high half) of the
// byte `sel` of w0 and w1 (32-bit halves of N' = N + kDigitBias), as
// dg_digit_bf16: the byte u, exact in float as (2^23 + u) - (2^23 + 128),
// keeps all its bits in the high half of the float.
__device__ __forceinline__ uint32_t digit_pair(uint32_t w0, uint32_t w1, int sel) {
  const uint32_t s = 0x7540u | (uint32_t)sel;   // bytes: u, 0, 0, 0x4B
  const float f0 = __uint_as_float(__byte_perm(w0, 0x4B000000u, s)) - 8388736.0f;
  const float f1 = __uint_as_float(__byte_perm(w1, 0x4B000000u, s)) - 8388736.0f;
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// c + a b as one 64-bit multiply-add of 32-bit signed operands
__device__ __forceinline__ long long mad_wide(int a, int b, long long c) {
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

__device__ __forceinline__ long long dg_shl64(int x, int sh) {
  return (long long)((unsigned long long)(long long)x << sh);
}

}  // namespace
}  // namespace emt
