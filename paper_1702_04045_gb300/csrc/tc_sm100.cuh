// Blackwell (sm_100 family) tensor-core primitives as inline PTX: tcgen05 MMA with FP32 accumulators in
// tensor memory (TMEM), shared-memory matrix descriptors, mbarriers, and the TF32 split used by the
// "3xTF32" products (x = hi + lo with hi, lo TF32; a b ~ ah bh + ah bl + al bh, accumulated in FP32).
#pragma once

#include <cstdint>

namespace paro {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// round to TF32 (nearest, ties away from zero): the 19-bit value the tensor core consumes
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// ---- mbarrier ----
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of an mbarrier: false after max_polls unsuccessful polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t max_polls) {
  for (uint32_t i = 0; i < max_polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// one plain arrival
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// one arrival that also expects `bytes` of asynchronous copies on the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// bulk copy global -> shared (this CTA) of `bytes` (multiple of 16, both addresses 16-byte aligned),
// completing as transaction bytes on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// barrier `id` (1..15) over `count` threads (whole warps) of the CTA
__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// ---- fences ----
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---- tensor memory (one full warp executes these) ----
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor, no swizzle, K-major "interleaved" layout: core matrices of 8 rows x
// 16 bytes stored as 128 contiguous bytes; lbo = byte step between core matrices along K, sbo = byte step
// between groups of 8 rows; bits 46-47 = 1 (descriptor version of the tcgen05 family).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// The same for the 128-byte swizzled K-major layout: rows of 128 bytes (32 TF32 values), 8-row atoms of
// 1024 bytes (stride-dimension offset), the 16-byte chunk c of row r stored at chunk c ^ (r % 8); atoms
// 1024-byte aligned. A K step inside the row advances the start address by its byte width.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;            // leading-dimension offset (unused inside a 128-byte swizzle row)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride between 8-row atoms
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M x N tile.
__host__ __device__ constexpr uint32_t idesc_tf32(uint32_t M, uint32_t N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T; issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.u32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive once on `bar` when every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// 32 TMEM lanes (this warp's quarter) x 8 consecutive 32-bit columns starting at taddr
__device__ __forceinline__ void tmem_ld_x8(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4); v[5] = __uint_as_float(r5); v[6] = __uint_as_float(r6); v[7] = __uint_as_float(r7);
}

// the same lanes and columns written from registers; tmem_st_wait() before the values are used
__device__ __forceinline__ void tmem_st_x8(uint32_t taddr, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

}  // namespace tc

// ---- operand tiles of the tf32 products (shared by the tensor-core kernels) ----
// byte offset of (row, 16-byte chunk) in a K-major tile with ch chunks per row: 128-byte swizzle when a
// row is exactly 128 bytes (ch = 8: 8-row atoms of 1024 bytes, chunk c of row r at c ^ (r % 8)), else the
// no-swizzle core-matrix layout (8 rows x 16 bytes contiguous)
__host__ __device__ __forceinline__ uint32_t tc_off(int row, int chunk, int ch) {
  if (ch == 8) return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
  return (uint32_t)(((row >> 3) * ch + chunk) * 128 + (row & 7) * 16);
}

// descriptor of the K step s2 (8 TF32 values) of a tile at shared address base, layout as in tc_off
__device__ __forceinline__ uint64_t tc_desc(uint32_t base, int s2, int ch) {
  if (ch == 8) return tc::smem_desc_sw128(base + (uint32_t)s2 * 32u);
  return tc::smem_desc(base + (uint32_t)s2 * 256u, 128u, (uint32_t)ch * 128u);
}

// dynamic shared memory rounded up to the 1024-byte alignment of the swizzle atoms (1 KB extra allocated)
__device__ __forceinline__ unsigned char* tc_align1024(unsigned char* p) {
  const uint32_t a = tc::smem_addr(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// split (v0, v1) into hi and lo TF32 quadruples (re0, im0, re1, im1)
__device__ __forceinline__ void tc_split(float2 v0, float2 v1, float4& h, float4& l) {
  h.x = tc::tf32_round(v0.x); h.y = tc::tf32_round(v0.y); h.z = tc::tf32_round(v1.x); h.w = tc::tf32_round(v1.y);
  l.x = tc::tf32_round(v0.x - h.x); l.y = tc::tf32_round(v0.y - h.y);
  l.z = tc::tf32_round(v1.x - h.z); l.w = tc::tf32_round(v1.y - h.w);
}

}  // namespace paro
