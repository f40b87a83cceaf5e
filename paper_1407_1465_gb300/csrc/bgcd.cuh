// bgcd.cuh -- the binary gcd both batch-GCD forms end with (bgcd.cu: the
// scan modulus by modulus; bgcd_tree.cu: the product and remainder trees).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mont.cuh"

namespace rsagpu {

// Binary gcd of u (odd) and v: strip v's factors of two, order the pair so
// that v >= u, replace v by v - u; stops when v = 0 with the gcd in u.  Every
// pass removes at least one bit from u + v, so at most 64L passes; the loop
// runs until the last lane of the warp is done.
template <int L>
__device__ __forceinline__ void binary_gcd(uint32_t (&u)[L], uint32_t (&v)[L]) {
#pragma unroll 1
  for (;;) {
    uint32_t vor = 0;
#pragma unroll
    for (int j = 0; j < L; ++j) vor |= v[j];
    const bool act = vor != 0u;
    if (!__any_sync(0xffffffffu, act)) break;
    if (!act) continue;
    if (v[0] == 0u) {
#pragma unroll
      for (int j = 0; j < L - 1; ++j) v[j] = v[j + 1];
      v[L - 1] = 0u;
      continue;
    }
    const int z = __ffs(v[0]) - 1;
    if (z) {
#pragma unroll
      for (int j = 0; j < L - 1; ++j) v[j] = __funnelshift_r(v[j], v[j + 1], z);
      v[L - 1] >>= z;
    }
    // borrow of v - u decides the order
    (void)sub_cc(v[0], u[0]);
#pragma unroll
    for (int j = 1; j < L; ++j) (void)subc_cc(v[j], u[j]);
    const uint32_t lt = subc(0u, 0u);                 // all ones iff v < u
    if (lt) {                                         // (u, v) = (v, u - v)
      uint32_t d = sub_cc(u[0], v[0]);
      u[0] = v[0];
      v[0] = d;
#pragma unroll
      for (int j = 1; j < L; ++j) {
        d = subc_cc(u[j], v[j]);
        u[j] = v[j];
        v[j] = d;
      }
    } else {                                          // v = v - u
      v[0] = sub_cc(v[0], u[0]);
#pragma unroll
      for (int j = 1; j < L; ++j) v[j] = subc_cc(v[j], u[j]);
    }
  }
}

struct Ctx;

// The tree form (bgcd_tree.cu): device bytes it needs for `count` moduli of L
// words, and one scan enqueued on s (context lock held).
uint64_t batch_gcd_tree_bytes(uint32_t L, uint64_t count);
int batch_gcd_tree_run(Ctx *c, uint32_t nbits, uint64_t count, const uint32_t *moduli, uint32_t *gcds,
                       int32_t *flags, cudaStream_t s);

}  // namespace rsagpu
