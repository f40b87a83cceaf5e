// tc.cuh -- tcgen05 (5th-generation tensor core), TMEM and mbarrier primitives
// as inline PTX for sm_103a.
//
// Conventions used by the kernels:
//   * Operands A (M x K) and B (N x K) are K-major fp16 in shared memory in the
//     no-swizzle core-matrix layout: a core matrix is 8 rows x 8 elements
//     (16 bytes per row, 128 bytes contiguous); core matrices are stored
//     [k-block][row-group], so the leading byte offset (LBO) is the distance
//     between k-blocks and the stride byte offset (SBO) is 128.
//   * The accumulator D (M = 128 rows x N columns of fp32) lives in tensor
//     memory: row i in TMEM lane i.  A warp may access only its quarter of the
//     lanes, 32 * (warp % 4) .. +31.
//   * One elected thread issues the MMAs and a tcgen05.commit that arrives on
//     an mbarrier when they have completed; every wait on that barrier is
//     bounded and reports failure instead of spinning forever.
#pragma once
#include <cstdint>

namespace rsagpu {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (no swizzle, relative LBO, base offset 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor for kind::f16: fp16 A and B (K-major), fp32 D, dense.
__host__ __device__ constexpr uint32_t idesc_f16_f32(uint32_t M, uint32_t N) {
  return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// ---------------------------------------------------------------- TMEM allocation (one full warp)
__device__ __forceinline__ void tmem_alloc(uint32_t slot_saddr, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_saddr), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------- ordering
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy shared-memory writes become visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------- MMA
__device__ __forceinline__ void mma_f16(uint32_t d_taddr, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_taddr),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void commit(uint32_t mbar_saddr) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_saddr)
               : "memory");
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint32_t mbar_saddr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar_saddr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Waits for the phase with the given parity to complete; gives up after
// `limit` polls (each poll may suspend the thread for a short, hardware-defined
// time).  Returns true on completion.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar_saddr, uint32_t parity, uint32_t limit) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < limit; ++it) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(mbar_saddr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// ---------------------------------------------------------------- TMEM loads (32 lanes x 32-bit, per-thread row)
__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- L2 prefetch (bulk, asynchronous hint)
// Asks the copy engine to bring [p, p + bytes) into L2; 16-byte aligned, bytes
// a multiple of 16.  No completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Drops the L2 lines of [p, p + bytes) without writing them back (their data
// is dead); p 128-byte aligned, bytes a multiple of 128.  Thread `first` of
// `stride` threads takes every stride-th line.
__device__ __forceinline__ void discard_l2(const void *p, uint32_t bytes, uint32_t first, uint32_t stride) {
  const char *c = static_cast<const char *>(p);
  for (uint32_t i = first; i < bytes / 128u; i += stride)
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(c + (size_t)i * 128u) : "memory");
}

// ---------------------------------------------------------------- misc
// Named barrier over `nthreads` threads that also ORs a predicate across them.
__device__ __forceinline__ bool bar_red_or(int id, int nthreads, bool pred) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
      : "memory");
  return out != 0;
}
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
  return r;
}
__device__ __forceinline__ void sts128(uint32_t saddr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(saddr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ uint4 lds128(uint32_t saddr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(saddr)
               : "memory");
  return v;
}

// Two adjacent MMA output columns (bias 0x3F000000 each, sums w < 2^23) as one
// base-2^16 column: w_even + 256 w_odd < 2^31.01.  Shifting the odd word up a
// byte drops its bias (0x3F000000 << 8 = 0 mod 2^32); the even word's bias is
// subtracted.  A shift-add and an add, neither depending on a running carry.
__device__ __forceinline__ uint32_t pair_cols(uint32_t w_even, uint32_t w_odd) {
  return (w_odd << 8) + (w_even - 0x3F000000u);
}

// Base-2^16 columns y_j (< 2^32) summed as sum_j y_j 2^(16j) without a
// 16-bit ripple: with y_j = L_j + 2^16 H_j the sum is X + Y, X the string of
// the L_j and Y that of the H_j one digit up, so two permutes per pair of
// columns and one 32-bit add with carry per word.  The low halves of columns
// 2k, 2k+1 (word k of X):
__device__ __forceinline__ uint32_t lo_halves(uint32_t y_even, uint32_t y_odd) { return prmt(y_even, y_odd, 0x5410u); }
// the high halves of columns 2k-1, 2k (word k of Y):
__device__ __forceinline__ uint32_t hi_halves(uint32_t y_below, uint32_t y_even) {
  return prmt(y_below, y_even, 0x7632u);
}

// Limb p of a number as four fp16 byte digits into a K-major core-matrix row:
// digits 4p .. 4p+3 are k-block p/2, bytes (p%2)*8 .. +7 of the row's slot
// (arow: the row's address in k-block 0; kb: the k-block stride).
__device__ __forceinline__ void emit_digits(uint32_t arow, int p, uint32_t v, uint32_t kb) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(arow + (uint32_t)(p >> 1) * kb + (uint32_t)(p & 1) * 8),
               "r"(prmt(v, 0u, 0x4140u)), "r"(prmt(v, 0u, 0x4342u))
               : "memory");
}

}  // namespace tc
}  // namespace rsagpu
