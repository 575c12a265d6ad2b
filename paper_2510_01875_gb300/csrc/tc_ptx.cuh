// Device-side building blocks shared by the tcgen05 kernels: mbarriers with bounded waits,
// bulk and 8-byte asynchronous copies, proxy and tensor-memory fences, cluster addressing, shared-memory matrix
// descriptors and MMA issue (CTA pairs and single CTAs), the 128-byte-swizzled MN-major tile
// addressing, the 16-bit hi/lo split, and shared-memory loads and stores by address.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lrt {
namespace tcx {

constexpr unsigned long long kTimeoutNs = 2000000000ull;   // bound of every mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// Asynchronous 4-, 8- or 16-byte copy global -> shared (cp.async, L1-allocating); src_bytes = 0 writes
// zeros and reads nothing (src must still be a valid address).  Completion per thread by
// cp_async_wait_all; other threads see the data after a barrier.
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(n));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// try_wait with a suspend-time hint: the warp sleeps in hardware until the phase completes or
// about `hint_ns` passes, instead of spinning on the issue slots.
__device__ __forceinline__ bool mbar_try_sleep(uint64_t* b, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when this CTA is aborting or the wait ran out (then it starts the abort).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag,
                                          int* status) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = gtime();
  while (!mbar_try_sleep(b, parity, 20000u)) {
    if (*abort_flag) return false;
    if (gtime() - t0 > kTimeoutNs) {
      *abort_flag = 1;
      atomicOr(status, 2);
      return false;
    }
  }
  return true;
}
// Bounded wait used while draining: ignores the abort flag.
__device__ __forceinline__ void mbar_drain(uint64_t* b, uint32_t parity, int* status) {
  const unsigned long long t0 = gtime();
  while (!mbar_try_sleep(b, parity, 20000u)) {
    if (gtime() - t0 > kTimeoutNs) {
      atomicOr(status, 2);
      return;
    }
  }
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_u32(b)),
               "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared, completion counted in bytes on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Rank of this CTA in its cluster, and the shared::cluster address of a variable in CTA `rank`.
__device__ __forceinline__ uint32_t cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
// Arrive on an mbarrier of a CTA of the cluster (this one included).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}
// All threads of both CTAs.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: start >> 4, LBO >> 4 at bit 16, SBO >> 4 at bit 32,
// version 1 at bit 46, 128-byte swizzle (2) at bits 61-63.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46) | (2ull << 61);
}

// D (tensor memory of both CTAs) [+]= A (rows 0..127 from this CTA's shared memory, 128..255
// from the peer's, same offsets) x B (columns 0..127 here, 128..255 at the peer).
__device__ __forceinline__ void mma2(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// Arrive on barrier b in both CTAs of the pair once all prior MMAs of this thread are done.
__device__ __forceinline__ void mma_commit_pair(uint64_t* b) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
      "[%0], %1;" ::"r"(smem_u32(b)),
      "h"((uint16_t)3)
      : "memory");
}
// The same, on this CTA's barrier only.
__device__ __forceinline__ void mma_commit_local(uint64_t* b) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(b))
      : "memory");
}

// Offset of the 16-byte chunk holding MN elements [8c, 8c+8) of K index k in an MN-major,
// 128-byte-swizzled tile: [k/8][mn/64][k%8][64 elements], chunk (mn%64)/8 XOR k%8.
__device__ __forceinline__ uint32_t mn_chunk(int k, int c, int sbo) {
  return (uint32_t)((k >> 3) * sbo + (c >> 3) * 1024 + (k & 7) * 128 + (((c & 7) ^ (k & 7)) << 4));
}

template <bool BF>
struct Pack;
template <>
struct Pack<false> {
  // 8 floats -> hi and lo as 8 x f16 each
  __device__ __forceinline__ static void split(const float* v, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2 a = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
      // v - hi, exact (one rounding of an exact difference)
      const float2 rr = __ffma2_rn(__half22float2(a), make_float2(-1.f, -1.f),
                                   make_float2(v[2 * i], v[2 * i + 1]));
      __half2 b = __floats2half2_rn(rr.x, rr.y);
      h[i] = *reinterpret_cast<uint32_t*>(&a);
      l[i] = *reinterpret_cast<uint32_t*>(&b);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
  }
};
template <>
struct Pack<true> {
  __device__ __forceinline__ static void split(const float* v, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __nv_bfloat162 a = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      const float2 rr = __ffma2_rn(__bfloat1622float2(a), make_float2(-1.f, -1.f),
                                   make_float2(v[2 * i], v[2 * i + 1]));
      __nv_bfloat162 b = __floats2bfloat162_rn(rr.x, rr.y);
      h[i] = *reinterpret_cast<uint32_t*>(&a);
      l[i] = *reinterpret_cast<uint32_t*>(&b);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
  }
};

// No memory clobber: the operand tiles are read only by the tensor cores after the
// fence.proxy.async + mbarrier arrive that follow (volatile asm keeps that order), so the
// compiler may hoist the next chunk's loads above these stores.
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w));
}

// Add into global memory without a return value.
__device__ __forceinline__ void red_add_f64(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// Single-instruction approximate reciprocal (relative error about 2^-23).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// Shared-memory loads with 32-bit addresses.  They are not volatile, so the compiler may
// interleave the loads of several chunks; they are kept after the mbarrier wait that
// publishes the data by adding stage_token() (an opaque zero produced after the wait) to
// every address.
__device__ __forceinline__ uint32_t stage_token() {
  uint32_t t;
  asm volatile("mov.u32 %0, 0;" : "=r"(t)::"memory");
  return t;
}
__device__ __forceinline__ float2 lds_f2(uint32_t addr) {
  float2 v;
  asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
  return v;
}
__device__ __forceinline__ float4 lds_f4(uint32_t addr) {
  float4 v;
  asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "r"(addr));
  return v;
}

// Single-CTA forms: D (this CTA's tensor memory) [+]= A x B from this CTA's shared memory,
// and the commit that arrives on this CTA's barrier.
__device__ __forceinline__ void mma1(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma1_commit(uint64_t* b) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(b))
      : "memory");
}

}  // namespace tcx
}  // namespace lrt
