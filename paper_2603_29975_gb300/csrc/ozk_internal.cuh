// Internal device helpers of libozk: sm_103a PTX wrappers (tcgen05, TMA, mbarrier) and
// shared host-side plumbing.  Every spin-wait here is bounded; a wait that gives up sets
// a bit in the device status word instead of hanging.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ozk.h"

namespace ozk {

// ------------------------------------------------------------------ status bits
__device__ __forceinline__ void flag_error(int* status, int code) {
  if (status) atomicOr(status, 1 << code);
}

// ------------------------------------------------------------------ integer images (splits)
__device__ __forceinline__ int frexp_exponent_from_bits(unsigned long long a) {
  // a = |x| bit pattern (sign cleared), finite
  if (a == 0ull) return 0;
  const int ex = static_cast<int>(a >> 52);
  if (ex > 0) return ex - 1022;
  return -1010 - __clzll(a);          // subnormal: floor(log2 x) + 1
}

// X = trunc(x 2^(B - e)) computed exactly from the binary64 fields of x.
__device__ __forceinline__ __int128 integer_image(double x, int e, int nbits) {
  const unsigned long long u = __double_as_longlong(x);
  const bool neg = (u >> 63) != 0ull;
  const int ex = static_cast<int>((u >> 52) & 0x7FFull);
  const unsigned long long man = u & ((1ull << 52) - 1ull);
  unsigned long long M;
  int E2;
  if (ex == 0) { M = man; E2 = -1074; } else { M = man | (1ull << 52); E2 = ex - 1075; }
  const int sh = E2 + nbits - e;
  unsigned __int128 mag = 0;
  if (M != 0ull) {
    if (sh >= 0) mag = static_cast<unsigned __int128>(M) << sh;
    else if (sh > -64) mag = static_cast<unsigned __int128>(M >> (-sh));
  }
  return neg ? -static_cast<__int128>(mag) : static_cast<__int128>(mag);
}

// Next balanced base-256 digit of X (least significant first); X is advanced.
// The same with 64-bit integers, for nbits <= 62 (S <= 7): |X| < 2^nbits when |x| < 2^e.
__device__ __forceinline__ long long integer_image64(double x, int e, int nbits) {
  const unsigned long long u = __double_as_longlong(x);
  const bool neg = (u >> 63) != 0ull;
  const int ex = static_cast<int>((u >> 52) & 0x7FFull);
  const unsigned long long man = u & ((1ull << 52) - 1ull);
  const unsigned long long M = ex == 0 ? man : (man | (1ull << 52));
  const int sh = (ex == 0 ? -1074 : ex - 1075) + nbits - e;
  const unsigned long long mag = sh >= 0 ? (sh < 64 ? M << sh : 0ull) : (sh > -64 ? M >> (-sh) : 0ull);
  return neg ? -static_cast<long long>(mag) : static_cast<long long>(mag);
}

__device__ __forceinline__ int next_digit64(long long& X) {
  const int d = static_cast<int>((X + 128) & 255ll) - 128;
  X = (X - d) >> 8;
  return d;
}

__device__ __forceinline__ int next_digit(__int128& X) {
  const int d = static_cast<int>(static_cast<unsigned long long>(X + 128) & 255ull) - 128;
  X = (X - d) >> 8;
  return d;
}


// RN-even of T * 2^E as binary64, integer instructions only (subnormals and overflow handled).
__device__ __forceinline__ double round_scaled_dev(__int128 T, int E) {
  if (T == 0) return 0.0;
  const bool neg = T < 0;
  unsigned __int128 u = neg ? static_cast<unsigned __int128>(-T) : static_cast<unsigned __int128>(T);
  const unsigned long long hi0 = static_cast<unsigned long long>(u >> 64);
  const int lz = hi0 ? __clzll(hi0) : 64 + __clzll(static_cast<unsigned long long>(u));
  u <<= lz;                                           // leading one at bit 127
  const unsigned long long M = static_cast<unsigned long long>(u >> 64);
  bool sticky = static_cast<unsigned long long>(u) != 0ull;
  const int Ep = E + 64 - lz;                         // value = (M + sticky) 2^Ep
  int q = Ep + 11;                                    // ulp exponent for a 53-bit result
  if (q < -1074) q = -1074;                           // subnormal range
  const int drop = q - Ep;                            // >= 11
  unsigned long long keep, rem, half;
  if (drop < 64) {
    keep = M >> drop;
    rem = M & ((1ull << drop) - 1ull);
    half = 1ull << (drop - 1);
  } else if (drop == 64) {
    keep = 0ull; rem = M; half = 1ull << 63;
  } else {
    keep = 0ull; rem = 0ull; half = 1ull;             // below half an ulp of the smallest subnormal
  }
  keep += ((rem > half) || (rem == half && (sticky || (keep & 1ull)))) ? 1ull : 0ull;
  unsigned long long bits;
  if (keep == 0ull) {
    bits = 0ull;
  } else if (q + 1074 >= 2047) {
    bits = 0x7FF0000000000000ull;                     // overflow
  } else {
    // keep <= 2^53: ((q + 1074) << 52) + keep encodes normals and subnormals alike
    bits = (static_cast<unsigned long long>(q + 1074) << 52) + keep;
    if (bits >= 0x7FF0000000000000ull) bits = 0x7FF0000000000000ull;
  }
  if (neg) bits |= 0x8000000000000000ull;
  return __longlong_as_double(static_cast<long long>(bits));
}

// ------------------------------------------------------------------ smem / mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
               ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}

// Bounded wait: gives up after ~`budget` SM clock cycles (about one second by default),
// sets OZK_ERR_TIMEOUT in *status and the CTA-local abort flag, and returns false.
constexpr long long kWaitBudget = 2000000000LL;

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status,
                                          volatile int* abort_flag, long long budget = kWaitBudget) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > budget) {
      flag_error(status, OZK_ERR_TIMEOUT);
      *abort_flag = 1;
      return false;
    }
  }
}

// ------------------------------------------------------------------ TMA
__device__ __forceinline__ void tma_load_3d(const CUtensorMap* map, void* smem_dst, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];"
      ::"r"(smem_u32(smem_dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)),
        "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ------------------------------------------------------------------ tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t* holder_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(smem_u32(holder_smem)), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// K-major operand tile in shared memory with the 32-byte swizzle: rows of 32 bytes
// (16 fp16 = one MMA K step), 8-row groups 256 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw32(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;                 // leading byte offset (unused here)
  d |= static_cast<uint64_t>(256u >> 4) << 32;         // stride byte offset: 8 rows x 32 B
  d |= static_cast<uint64_t>(1) << 46;                 // descriptor version
  d |= static_cast<uint64_t>(6) << 61;                 // swizzle: 32 B
  return d;
}

// Instruction descriptor: kind::f16, A = B = fp16, D = f32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
  return (1u << 4) | (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------------ host plumbing
void record_launch();                          // counts kernel launches (ozk_launch_count)
ozk_status_t set_error(ozk_status_t st, const char* msg);
ozk_status_t cuda_check(cudaError_t e, const char* what);

}  // namespace ozk
