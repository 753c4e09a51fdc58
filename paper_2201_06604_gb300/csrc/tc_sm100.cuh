// tc_sm100.cuh -- inline-PTX wrappers for the Blackwell (sm_100 family,
// built for sm_103a) tensor-core path: mbarriers, bulk copies into shared
// memory, tensor memory (TMEM) allocation, tcgen05.mma and tcgen05.ld.
//
// Conventions used by every kernel that includes this file:
//   * operands live in shared memory in the K-major, 128-byte-swizzled layout:
//     an "atom" is 8 rows x 128 bytes (8 rows x 64 bf16), 1024-byte aligned;
//     row r of an atom holds its 16-byte chunks c = 0..7 at chunk position
//     c ^ (r mod 8); 8-row groups follow each other 1024 bytes apart (the
//     descriptor's stride byte offset), and the two 64-element halves of a
//     128-element K extent are separate atom columns, rows x 128 bytes apart;
//   * the accumulator of an M = 128 MMA has row i in TMEM lane i and column j
//     in TMEM column (base + j), one fp32 per cell; warp w of the CTA reads
//     lanes 32w .. 32w + 31;
//   * every wait on an mbarrier is bounded by the global timer: it gives up
//     after `limit_ns` and returns false, and the caller records an error and
//     leaves without touching the operands again.
#pragma once
#include <stdint.h>

namespace mrg {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---- mbarriers -------------------------------------------------------------

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// Makes the initialised barriers visible to the async proxy (bulk copies and
// tcgen05.commit arrive on them).
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also expects `bytes` of bulk-copy transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// One plain arrival (no transaction count).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// Waits for the phase with the given parity to complete; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 15) == 0 && global_ns() - t0 > limit_ns) return false;
  }
}

// ---- bulk copy global -> shared (no tensor map: both addresses 16-byte
// aligned, size a multiple of 16), completing on an mbarrier ----------------

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ---- tensor memory -----------------------------------------------------------

// Allocates ncols TMEM columns (a power of two >= 32) for the CTA; one whole
// warp executes it.  The base address is written to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Frees them again (the same warp, once every MMA and load on them is done).
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---- descriptors -------------------------------------------------------------

// Shared-memory matrix descriptor of a K-major, 128-byte-swizzled operand
// whose 8-row groups are 1024 bytes apart; `addr` is the shared address of
// the first row's 16-byte chunk of the K slice to read (atom base + 32 bytes
// per 16 bf16 elements of K inside the atom).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);       // start address
  d |= (uint64_t)1u << 16;                       // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024u >> 4) << 32;             // stride byte offset: next 8-row group
  d |= (uint64_t)1u << 46;                       // descriptor version of this family
  d |= (uint64_t)2u << 61;                       // swizzle: 128 bytes
  return d;
}

// Instruction descriptor of kind::f16 with bf16 A and B (both K-major), fp32
// accumulation, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(uint32_t M, uint32_t N) {
  return (1u << 4)            // D format: f32
         | (1u << 7)          // A format: bf16
         | (1u << 10)         // B format: bf16
         | ((N >> 3) << 17)   // N / 8
         | ((M >> 4) << 24);  // M / 16
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The same with both descriptors given as their low words and a shared high
// word (the K-major SW128 descriptors above differ only in the start-address
// and leading-offset fields, both in the low word, and no address offset
// inside shared memory carries out of the 14-bit start field): one 32-bit
// add per operand instead of a 64-bit one.
__device__ __forceinline__ void mma_bf16_lo(uint32_t tmem_d, uint32_t alo, uint32_t blo,
                                            uint32_t hi, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t.reg .b64 da, db;\n\t"
      "setp.ne.b32 p, %5, 0;\n\t"
      "mov.b64 da, {%1, %3};\n\t"
      "mov.b64 db, {%2, %3};\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %4, p;\n\t}" ::"r"(tmem_d),
      "r"(alo), "r"(blo), "r"(hi), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrives on the mbarrier once every tcgen05 operation this thread issued
// before it has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// Eight consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Byte offset of element (r, k) of a K-major operand tile of R rows and a
// 128-element K extent in the swizzled layout above (2-byte elements).
__host__ __device__ __forceinline__ uint32_t sw128_offset(uint32_t R, uint32_t r, uint32_t k) {
  const uint32_t atom_col = k >> 6, kk = k & 63;
  const uint32_t chunk = (kk >> 3) ^ (r & 7);
  return atom_col * R * 128u + (r >> 3) * 1024u + (r & 7) * 128u + chunk * 16u + (kk & 7) * 2u;
}

}  // namespace tc
}  // namespace mrg
