// Packed int16x2 DP primitives and TMA / mbarrier helpers shared by the
// packed kernels.  Each 32-bit register holds two independent DP cells (two
// queries against the same target residue); the DPX instructions compute
// both halves at once.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dsa {

__device__ __forceinline__ uint32_t pack2(int lo, int hi) {
  return (uint32_t)(lo & 0xFFFF) | ((uint32_t)hi << 16);
}
__device__ __forceinline__ int lo16(uint32_t v) { return (int)(int16_t)(v & 0xFFFF); }
__device__ __forceinline__ int hi16(uint32_t v) { return (int)(int16_t)(v >> 16); }

// max(a + b, c) per halfword
__device__ __forceinline__ uint32_t addmax2(uint32_t a, uint32_t b, uint32_t c) {
  return __viaddmax_s16x2(a, b, c);
}
// max(a, b, 0) per halfword
__device__ __forceinline__ uint32_t max2_relu(uint32_t a, uint32_t b) {
  return __vimax_s16x2_relu(a, b);
}
__device__ __forceinline__ uint32_t max3_2(uint32_t a, uint32_t b, uint32_t c) {
  return __vimax3_s16x2(a, b, c);
}
// Byte permute of {hi_tab, lo_tab} (bytes 0-3 from lo_tab, 4-7 from hi_tab):
// each selector nibble picks a byte with its low 3 bits and, with bit 3 set,
// replicates that byte's sign bit instead (PTX prmt, generic mode).
__device__ __forceinline__ uint32_t prmt(uint32_t lo_tab, uint32_t hi_tab, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(lo_tab), "r"(hi_tab), "r"(sel));
  return r;
}
// Offset-binary halfwords (sign bit flipped: v' = v + 0x8000 mod 2^16) order
// like unsigned numbers; DPX add-max wraps mod 2^16 in each half, so adding a
// two's-complement constant is the same in either form.
__device__ __forceinline__ uint32_t addmax2u(uint32_t a, uint32_t b, uint32_t c) {
  return __viaddmax_u16x2(a, b, c);
}
__device__ __forceinline__ uint32_t max3_2u(uint32_t a, uint32_t b, uint32_t c) {
  return __vimax3_u16x2(a, b, c);
}
// a + b per halfword (no carry between halves)
__device__ __forceinline__ uint32_t add2(uint32_t a, uint32_t b) { return __vadd2(a, b); }

// ---- shared-memory addressing, mbarrier and bulk-copy PTX ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up after `limit_ns` nanoseconds of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}
// 1-D bulk copy global -> shared, completion signalled on `bar` (tx bytes).
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// 16-, 8- and 4-byte asynchronous copies global -> shared (generic proxy,
// per thread; 16 bytes: both addresses 16-byte aligned), and their commit /
// wait-for-all-but-N groups.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem_dst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;   // 2 s

}  // namespace dsa
