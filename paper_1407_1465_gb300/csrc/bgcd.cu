// bgcd.cu -- batch GCD of a set of moduli (weak-key detection: the paper's
// introduction motivates RSA's security by the difficulty of factoring n; two
// moduli that share a prime are factored by one gcd).
//
// For moduli n_0 .. n_{k-1} the result is g_i = gcd(n_i, prod_{j != i} n_j).
// Since gcd(n, X) = gcd(n, X mod n) and every power of R = 2^(32L) is a unit
// modulo an odd n, it is enough to know prod_{j != i} n_j * R^(-e) mod n_i for
// some e, which Montgomery arithmetic gives without corrections.
//
// With schoolbook word arithmetic a product / remainder tree does more word
// products (its divisions alone about 4 L^2 k^2 for k moduli of L words) than
// working modulus by modulus (about L^2 k^2 here), so each thread owns one
// modulus n_i and runs over all the others:
//   * block products: a first kernel multiplies the moduli together in blocks
//     of B (8, 16 or 32) as plain integers of B*L words, one warp per block
//     (a product tree whose levels split each product over lanes);
//   * for a block that does not hold n_i the thread reduces the block product
//     word by word: q = t_0 n' mod 2^32, t = (t + q n_i) / 2^32, then the next
//     word of the block product enters at the top.  After all M words the
//     window holds P_c * 2^(-32M) mod n_i (at most n_i, one conditional
//     subtraction).  That is L word products per word of P_c -- half of a
//     Montgomery multiplication by the same words -- followed by one Montgomery
//     multiplication into the running product;
//   * the 32 moduli of the thread's own warp (the own block) go through CIOS
//     Montgomery multiplications one by one, skipping j = i;
//   * the j range is split into parts for load balance; a tree of launches
//     multiplies the parts' partial products pairwise, and a last kernel runs
//     a binary gcd.
// Moduli that are even or below 3 are invalid: they are left out of every
// product, and their own result is flagged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "bgcd.cuh"
#include "mont.cuh"
#include "rsa_gb300.h"
#include "runtime_internal.h"

namespace rsagpu {

namespace {

constexpr int kGcdThreads = 128;
constexpr int kOwn = 32;            // moduli per warp: the own block

// Scratch words per block of the product tree for blocks of B moduli: one
// level buffer of B L words and B/2 partial products of up to (B/2 + 1) L words.
__host__ __device__ constexpr size_t gcd_scratch_words(uint32_t L, uint32_t B) {
  return ((size_t)B + (size_t)(B / 2) * (B / 2 + 1)) * L;
}

struct GcdArgs {
  const uint32_t *mods;   // count rows of L words
  uint8_t *valid;         // count: 1 odd and > 1
  uint32_t *bprod;        // block c at c * blk * L words, blk * L words each
  uint32_t *bscratch;     // block c at c * gcd_scratch_words(L, blk): the product tree's buffers
  uint32_t *part;         // nparts * count rows of L words
  uint32_t *gcds;         // count rows of L words, or null
  int32_t *flags;         // count, or null
  uint32_t count, blk, nparts;
};

template <int L>
struct GcdSmem {
  static constexpr int kStageU4 = (L / 4) * 32;   // one [L/4][32] uint4 buffer per warp
  static constexpr int kBuffers = 2;              // running product, block residue
  static constexpr size_t bytes(int warps) { return (size_t)warps * kBuffers * kStageU4 * 16; }
};

template <int L>
__device__ __forceinline__ void load_n(NRegs<L> &N, const uint32_t *row) {
  const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
#pragma unroll
  for (int g = 0; g < L / 4; ++g) {
    const uint4 v = __ldg(r4 + g);
    N.n[4 * g] = v.x; N.n[4 * g + 1] = v.y; N.n[4 * g + 2] = v.z; N.n[4 * g + 3] = v.w;
  }
}

// -n^-1 mod 2^32 for odd n0: x = n0 is right to 3 bits, each step doubles them
__device__ __forceinline__ uint32_t neg_inv32(uint32_t n0) {
  uint32_t inv = n0;
#pragma unroll
  for (int k = 0; k < 4; ++k) inv *= 2u - n0 * inv;
  return 0u - inv;
}

// t = (t + b X) / 2^32, returning the low word the division drops.  Same two
// chains as reduce_step (even limbs of X, then odd limbs, results written one
// limb down), with a given multiplier instead of q.
template <int L>
__device__ __forceinline__ uint32_t mul_shift(uint32_t (&t)[L + 2], const NRegs<L> &X, uint32_t b) {
  const uint32_t out = mad_lo_cc(b, X.n[0], t[0]);
  t[0] = madc_hi_cc(b, X.n[0], t[1]);
#pragma unroll
  for (int k = 1; k < L / 2; ++k) {
    t[2 * k - 1] = madc_lo_cc(b, X.n[2 * k], t[2 * k]);
    t[2 * k] = madc_hi_cc(b, X.n[2 * k], t[2 * k + 1]);
  }
  t[L - 1] = addc_cc(t[L], 0u);
  t[L] = addc(t[L + 1], 0u);
  t[0] = mad_lo_cc(b, X.n[1], t[0]);
  t[1] = madc_hi_cc(b, X.n[1], t[1]);
#pragma unroll
  for (int k = 1; k < L / 2; ++k) {
    t[2 * k] = madc_lo_cc(b, X.n[2 * k + 1], t[2 * k]);
    t[2 * k + 1] = madc_hi_cc(b, X.n[2 * k + 1], t[2 * k + 1]);
  }
  t[L] = addc(t[L], 0u);
  t[L + 1] = 0u;
  return out;
}

// 128-bit read-only global load issued exactly where written (volatile asm is
// not hoisted or merged), so a broadcast operand read at every step of a
// multiplication is not held in registers across the steps.
__device__ __forceinline__ uint4 ldg128(const uint4 *p) {
  uint4 v;
  asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// t += b * A with A (L words) read from global memory at a warp-uniform
// address (every lane multiplies by the same modulus n_j).
template <int L>
__device__ __forceinline__ void mul_acc_bcast(uint32_t (&t)[L + 2], const uint4 *A, uint32_t b) {
  {
    const uint4 a = ldg128(A);
    t[0] = mad_lo_cc(a.x, b, t[0]);
    t[1] = madc_hi_cc(a.x, b, t[1]);
    t[2] = madc_lo_cc(a.z, b, t[2]);
    t[3] = madc_hi_cc(a.z, b, t[3]);
  }
#pragma unroll
  for (int g = 1; g < L / 4; ++g) {
    const uint4 a = ldg128(A + g);
    t[4 * g] = madc_lo_cc(a.x, b, t[4 * g]);
    t[4 * g + 1] = madc_hi_cc(a.x, b, t[4 * g + 1]);
    t[4 * g + 2] = madc_lo_cc(a.z, b, t[4 * g + 2]);
    t[4 * g + 3] = madc_hi_cc(a.z, b, t[4 * g + 3]);
  }
  t[L] = addc_cc(t[L], 0u);
  t[L + 1] = addc(t[L + 1], 0u);
  {
    const uint4 a = ldg128(A);
    t[1] = mad_lo_cc(a.y, b, t[1]);
    t[2] = madc_hi_cc(a.y, b, t[2]);
    t[3] = madc_lo_cc(a.w, b, t[3]);
    t[4] = madc_hi_cc(a.w, b, t[4]);
  }
#pragma unroll
  for (int g = 1; g < L / 4; ++g) {
    const uint4 a = ldg128(A + g);
    t[4 * g + 1] = madc_lo_cc(a.y, b, t[4 * g + 1]);
    t[4 * g + 2] = madc_hi_cc(a.y, b, t[4 * g + 2]);
    t[4 * g + 3] = madc_lo_cc(a.w, b, t[4 * g + 3]);
    t[4 * g + 4] = madc_hi_cc(a.w, b, t[4 * g + 4]);
  }
  t[L + 1] = addc(t[L + 1], 0u);
}

// acc = n_j * acc * R^-1 mod n_i: A = n_j (< R, broadcast), B = acc (< n_i,
// this lane's stage), the result written back over acc.
template <int L, int U>
__device__ __forceinline__ void mont_mul_bcast(uint4 *acc_lane, const uint4 *Aj, const NRegs<L> &N, uint32_t np) {
  uint32_t t[L + 2];
#pragma unroll
  for (int j = 0; j < L + 2; ++j) t[j] = 0u;
#pragma unroll 1
  for (int i0 = 0; i0 < L; i0 += U) {
#pragma unroll
    for (int u = 0; u < U; u += 4) {
      const uint4 b = lds128(acc_lane + ((i0 + u) >> 2) * 32);
      mul_acc_bcast<L>(t, Aj, b.x);
      reduce_step<L>(t, N, np);
      mul_acc_bcast<L>(t, Aj, b.y);
      reduce_step<L>(t, N, np);
      mul_acc_bcast<L>(t, Aj, b.z);
      reduce_step<L>(t, N, np);
      mul_acc_bcast<L>(t, Aj, b.w);
      reduce_step<L>(t, N, np);
    }
  }
  final_sub_smem<L>(acc_lane, t, N);
}

// 128-bit shared load at a 32-bit shared address plus an immediate byte
// offset, so that a stage read group by group needs one address register.
template <int OFF>
__device__ __forceinline__ uint4 lds128_at(uint32_t base) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4+%5];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(base), "n"(OFF));
  return v;
}

// t += b * A with A in this lane's stage ([L/4][32] uint4 at shared address a).
template <int L, int G = 0>
__device__ __forceinline__ void mul_acc_even(uint32_t (&t)[L + 2], uint32_t a, uint32_t b) {
  if constexpr (G < L / 4) {
    const uint4 v = lds128_at<G * 512>(a);
    if constexpr (G == 0) {
      t[0] = mad_lo_cc(v.x, b, t[0]);
    } else {
      t[4 * G] = madc_lo_cc(v.x, b, t[4 * G]);
    }
    t[4 * G + 1] = madc_hi_cc(v.x, b, t[4 * G + 1]);
    t[4 * G + 2] = madc_lo_cc(v.z, b, t[4 * G + 2]);
    t[4 * G + 3] = madc_hi_cc(v.z, b, t[4 * G + 3]);
    mul_acc_even<L, G + 1>(t, a, b);
  }
}
template <int L, int G = 0>
__device__ __forceinline__ void mul_acc_odd(uint32_t (&t)[L + 2], uint32_t a, uint32_t b) {
  if constexpr (G < L / 4) {
    const uint4 v = lds128_at<G * 512>(a);
    if constexpr (G == 0) {
      t[1] = mad_lo_cc(v.y, b, t[1]);
    } else {
      t[4 * G + 1] = madc_lo_cc(v.y, b, t[4 * G + 1]);
    }
    t[4 * G + 2] = madc_hi_cc(v.y, b, t[4 * G + 2]);
    t[4 * G + 3] = madc_lo_cc(v.w, b, t[4 * G + 3]);
    t[4 * G + 4] = madc_hi_cc(v.w, b, t[4 * G + 4]);
    mul_acc_odd<L, G + 1>(t, a, b);
  }
}
template <int L>
__device__ __forceinline__ void mul_acc_lane(uint32_t (&t)[L + 2], uint32_t a, uint32_t b) {
  mul_acc_even<L>(t, a, b);
  t[L] = addc_cc(t[L], 0u);
  t[L + 1] = addc(t[L + 1], 0u);
  mul_acc_odd<L>(t, a, b);
  t[L + 1] = addc(t[L + 1], 0u);
}

// acc = acc * r * R^-1 mod n_i, both operands in this lane's stages (< n_i).
template <int L, int U>
__device__ __forceinline__ void mont_mul_lanes(uint4 *acc_lane, const uint4 *r_lane, const NRegs<L> &N,
                                               uint32_t np) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(acc_lane);
  uint32_t t[L + 2];
#pragma unroll
  for (int j = 0; j < L + 2; ++j) t[j] = 0u;
#pragma unroll 1
  for (int i0 = 0; i0 < L; i0 += U) {
#pragma unroll
    for (int u = 0; u < U; u += 4) {
      const uint4 b = lds128(r_lane + ((i0 + u) >> 2) * 32);
      mul_acc_lane<L>(t, a, b.x);
      reduce_step<L>(t, N, np);
      mul_acc_lane<L>(t, a, b.y);
      reduce_step<L>(t, N, np);
      mul_acc_lane<L>(t, a, b.z);
      reduce_step<L>(t, N, np);
      mul_acc_lane<L>(t, a, b.w);
      reduce_step<L>(t, N, np);
    }
  }
  final_sub_smem<L>(acc_lane, t, N);
}

// One word of the block product's reduction: t = (t + q n) / 2^32, then word x
// (position L - 1 of the shifted window) enters.
template <int L>
__device__ __forceinline__ void redc_feed(uint32_t (&t)[L + 2], const NRegs<L> &N, uint32_t np, uint32_t x) {
  reduce_step<L>(t, N, np);
  t[L - 1] = add_cc(t[L - 1], x);
  t[L] = addc(t[L], 0u);
}

// r_lane = T * 2^(-32 M) mod n_i for the M-word block product T (broadcast,
// M a multiple of L).  Window t = words s .. s+L of T + Q n_i.
template <int L>
__device__ __forceinline__ void redc_block(uint4 *r_lane, const uint32_t *T, uint32_t M, const NRegs<L> &N,
                                           uint32_t np) {
  const uint4 *T4 = reinterpret_cast<const uint4 *>(T);
  uint32_t t[L + 2];
#pragma unroll
  for (int g = 0; g < L / 4; ++g) {
    const uint4 v = __ldg(T4 + g);
    t[4 * g] = v.x; t[4 * g + 1] = v.y; t[4 * g + 2] = v.z; t[4 * g + 3] = v.w;
  }
  t[L] = 0u;
  t[L + 1] = 0u;
  const uint32_t M4 = M / 4, L4 = L / 4;
  uint4 x = (L4 < M4) ? __ldg(T4 + L4) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 1
  for (uint32_t s4 = 0; s4 < M4; ++s4) {
    const uint32_t nx = s4 + 1 + L4;                 // next group, loaded one step ahead
    const uint4 xn = (nx < M4) ? ldg128(T4 + nx) : make_uint4(0u, 0u, 0u, 0u);
    redc_feed<L>(t, N, np, x.x);
    redc_feed<L>(t, N, np, x.y);
    redc_feed<L>(t, N, np, x.z);
    redc_feed<L>(t, N, np, x.w);
    x = xn;
  }
  final_sub_smem<L>(r_lane, t, N);                    // t <= n_i
}

__device__ __forceinline__ bool valid_mod(const uint32_t *row, int L) {
  uint32_t hi = 0;
  for (int j = 1; j < L; ++j) hi |= row[j];
  return (row[0] & 1u) && (hi != 0u || row[0] >= 3u);
}

// Block products, one warp per block: P_c = prod of the block's valid moduli
// (an invalid one, and a slot past the last modulus, counts as 1), B*L words,
// by a product tree.  Level l multiplies pairs of 2^(l-1) L-word numbers;
// each product A*B is split over the L-word chunks B_k of B, one lane each:
// lane (p, k) scans A's words against B_k held in registers (word a of
// A*B_k is final once row a is added), and when a product has several chunks
// one lane adds the partial products A*B_k * 2^(32 k L) with a running carry.
// The levels alternate between a scratch buffer and the block's slot of
// bprod so that the last one lands in bprod.
template <int L>
__global__ void __launch_bounds__(64) bgcd_block_kernel(GcdArgs a) {
  const uint32_t nblk = (a.count + a.blk - 1) / a.blk;
  const int lane = threadIdx.x & 31;
  const uint32_t c = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (c >= nblk) return;                               // whole warp
  const uint32_t blk = a.blk, half = blk / 2;
  const uint32_t j0 = c * blk;
  int levels = 0;
  for (uint32_t v = blk; v > 1; v >>= 1) ++levels;
  uint32_t *slot = a.bprod + (size_t)c * blk * L;
  uint32_t *scr = a.bscratch + (size_t)c * gcd_scratch_words(L, blk);
  uint32_t *part = scr + (size_t)blk * L;             // after the level buffer
  // level 0 into the buffer the parity of `levels` picks (odd: scratch)
  uint32_t *cur = (levels & 1) ? scr : slot;
  uint32_t *nxt = (levels & 1) ? slot : scr;
  for (uint32_t e = (uint32_t)lane; e < blk; e += 32) {
    const uint32_t j = j0 + e;
    bool ok = false;
    if (j < a.count) {
      ok = valid_mod(a.mods + (size_t)j * L, L);
      a.valid[j] = ok ? 1 : 0;
    }
    uint4 *dst = reinterpret_cast<uint4 *>(cur + (size_t)e * L);
    const uint4 *src = reinterpret_cast<const uint4 *>(a.mods + (size_t)j * L);
#pragma unroll 1
    for (int g = 0; g < L / 4; ++g) dst[g] = ok ? __ldg(src + g) : make_uint4(g == 0 ? 1u : 0u, 0u, 0u, 0u);
  }
  __syncwarp();
  for (int l = 1; l <= levels; ++l) {
    const uint32_t s_words = (uint32_t)L << (l - 1);   // each factor
    const uint32_t cp = 1u << (l - 1);                 // chunks of B per product
    const uint32_t np = blk >> l;                      // products at this level
    if ((uint32_t)lane < half) {
      const uint32_t p = (uint32_t)lane / cp, k = (uint32_t)lane % cp;
      const uint32_t *A = cur + (size_t)(2 * p) * s_words;
      const uint32_t *B = cur + (size_t)(2 * p + 1) * s_words + (size_t)k * L;
      uint32_t *P = cp == 1 ? nxt + (size_t)p * 2 * s_words : part + (size_t)lane * (s_words + L);
      NRegs<L> X;
      load_n<L>(X, B);
      uint32_t t[L + 2];
#pragma unroll
      for (int q = 0; q < L + 2; ++q) t[q] = 0u;
      const uint4 *A4 = reinterpret_cast<const uint4 *>(A);
      uint4 *P4 = reinterpret_cast<uint4 *>(P);
#pragma unroll 1
      for (uint32_t g = 0; g < s_words / 4; ++g) {
        uint4 v = A4[g];
        v.x = mul_shift<L>(t, X, v.x);
        v.y = mul_shift<L>(t, X, v.y);
        v.z = mul_shift<L>(t, X, v.z);
        v.w = mul_shift<L>(t, X, v.w);
        P4[g] = v;
      }
#pragma unroll
      for (int g = 0; g < L / 4; ++g)
        P4[s_words / 4 + g] = make_uint4(t[4 * g], t[4 * g + 1], t[4 * g + 2], t[4 * g + 3]);
    }
    __syncwarp();
    if (cp > 1 && (uint32_t)lane < np) {
      // out = sum_k part_k * 2^(32 k L), part_k of s_words + L words
      const uint32_t p = (uint32_t)lane, pw = s_words + L;
      const uint32_t *base = part + (size_t)p * cp * pw;
      uint32_t *out = nxt + (size_t)p * 2 * s_words;
      uint64_t carry = 0;
#pragma unroll 1
      for (uint32_t w = 0; w < 2 * s_words; ++w) {
        uint64_t acc = carry;
        const uint32_t khi = min(cp - 1, w / L);
        const uint32_t klo = w >= pw ? (w - pw) / L + 1 : 0u;
        for (uint32_t k = klo; k <= khi; ++k) acc += base[(size_t)k * pw + (w - k * L)];
        out[w] = (uint32_t)acc;
        carry = acc >> 32;
      }
    }
    __syncwarp();
    uint32_t *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
}

// Partial products: warp task (own block w, part p) multiplies, for its 32
// moduli, every valid n_j of the part's range of 32-modulus groups.
template <int L, int U, int MINB>
__global__ void __launch_bounds__(kGcdThreads, MINB) bgcd_kernel(GcdArgs a) {
  using Sm = GcdSmem<L>;
  extern __shared__ uint4 smem4[];
  const int nw = blockDim.x / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4 *acc_lane = smem4 + (size_t)warp * Sm::kBuffers * Sm::kStageU4 + lane;
  uint4 *r_lane = acc_lane + Sm::kStageU4;
  const uint32_t nsb = (a.count + kOwn - 1) / kOwn;
  const uint32_t nblk = (a.count + a.blk - 1) / a.blk;
  const uint32_t per_sb = kOwn / a.blk;
  const uint64_t ntasks = (uint64_t)nsb * a.nparts;
#pragma unroll 1
  for (uint64_t task = (uint64_t)blockIdx.x * nw + warp; task < ntasks; task += (uint64_t)gridDim.x * nw) {
    const uint32_t w = (uint32_t)(task / a.nparts), p = (uint32_t)(task % a.nparts);
    const uint32_t i = w * kOwn + (uint32_t)lane;
    const bool live = i < a.count;
    const uint32_t row = live ? i : a.count - 1;
    NRegs<L> N;
    load_n<L>(N, a.mods + (size_t)row * L);
    N.n[0] |= 1u;                                      // invalid moduli: keep the arithmetic defined
    const uint32_t np = neg_inv32(N.n[0]);
#pragma unroll
    for (int g = 0; g < L / 4; ++g) acc_lane[g * 32] = make_uint4(g == 0 ? 1u : 0u, 0u, 0u, 0u);
    const uint32_t s0 = (uint32_t)((uint64_t)nsb * p / a.nparts), s1 = (uint32_t)((uint64_t)nsb * (p + 1) / a.nparts);
#pragma unroll 1
    for (uint32_t s = s0; s < s1; ++s) {
      if (s == w) {
        const uint32_t j1 = min(a.count, (s + 1) * kOwn);
#pragma unroll 1
        for (uint32_t j = s * kOwn; j < j1; ++j) {
          if (!a.valid[j]) continue;
          if (j != i) mont_mul_bcast<L, U>(acc_lane, reinterpret_cast<const uint4 *>(a.mods + (size_t)j * L), N, np);
        }
      } else {
        const uint32_t c1 = min(nblk, (s + 1) * per_sb);
#pragma unroll 1
        for (uint32_t c = s * per_sb; c < c1; ++c) {
          const uint32_t members = min(a.count, (c + 1) * a.blk) - c * a.blk;
          redc_block<L>(r_lane, a.bprod + (size_t)c * a.blk * L, members * L, N, np);
          mont_mul_lanes<L, U>(acc_lane, r_lane, N, np);
        }
      }
    }
    if (live) {
      uint4 *dst = reinterpret_cast<uint4 *>(a.part + ((size_t)p * a.count + i) * L);
#pragma unroll
      for (int g = 0; g < L / 4; ++g) dst[g] = acc_lane[g * 32];
    }
  }
}

// One level of the tree that multiplies the parts' partial products together:
// part[p] = part[p] * part[p + half] for p < cur - half (Montgomery products,
// so each level adds a power of R^-1, a unit modulo n_i).
template <int L, int U>
__global__ void __launch_bounds__(kGcdThreads) bgcd_combine_kernel(GcdArgs a, uint32_t cur, uint32_t half) {
  using Sm = GcdSmem<L>;
  extern __shared__ uint4 smem4[];
  const int nw = blockDim.x / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4 *acc_lane = smem4 + (size_t)warp * Sm::kBuffers * Sm::kStageU4 + lane;
  uint4 *r_lane = acc_lane + Sm::kStageU4;
  const uint32_t nsb = (a.count + kOwn - 1) / kOwn, pairs = cur - half;
  const uint64_t ntasks = (uint64_t)nsb * pairs;
#pragma unroll 1
  for (uint64_t task = (uint64_t)blockIdx.x * nw + warp; task < ntasks; task += (uint64_t)gridDim.x * nw) {
    const uint32_t w = (uint32_t)(task / pairs), p = (uint32_t)(task % pairs);
    const uint32_t i = w * kOwn + (uint32_t)lane;
    const bool live = i < a.count;
    const uint32_t row = live ? i : a.count - 1;
    NRegs<L> N;
    load_n<L>(N, a.mods + (size_t)row * L);
    N.n[0] |= 1u;
    const uint32_t np = neg_inv32(N.n[0]);
    uint4 *dst = reinterpret_cast<uint4 *>(a.part + ((size_t)p * a.count + row) * L);
    const uint4 *src = reinterpret_cast<const uint4 *>(a.part + ((size_t)(p + half) * a.count + row) * L);
#pragma unroll
    for (int g = 0; g < L / 4; ++g) {
      acc_lane[g * 32] = dst[g];
      r_lane[g * 32] = src[g];
    }
    mont_mul_lanes<L, U>(acc_lane, r_lane, N, np);
    if (live) {
#pragma unroll
      for (int g = 0; g < L / 4; ++g) dst[g] = acc_lane[g * 32];
    }
  }
}

// Combine the parts' partial products, then g_i = gcd(n_i, product).
template <int L, int U>
__global__ void __launch_bounds__(kGcdThreads) bgcd_finish_kernel(GcdArgs a) {
  using Sm = GcdSmem<L>;
  extern __shared__ uint4 smem4[];
  const int nw = blockDim.x / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4 *acc_lane = smem4 + (size_t)warp * Sm::kBuffers * Sm::kStageU4 + lane;
  uint4 *r_lane = acc_lane + Sm::kStageU4;
  const uint32_t nsb = (a.count + kOwn - 1) / kOwn;
#pragma unroll 1
  for (uint32_t w = blockIdx.x * nw + warp; w < nsb; w += gridDim.x * nw) {
    const uint32_t i = w * kOwn + (uint32_t)lane;
    const bool live = i < a.count;
    const uint32_t row = live ? i : a.count - 1;
    const bool ok = live && a.valid[row];
    {
      NRegs<L> N;
      load_n<L>(N, a.mods + (size_t)row * L);
      N.n[0] |= 1u;
      const uint32_t np = neg_inv32(N.n[0]);
      const uint4 *src = reinterpret_cast<const uint4 *>(a.part + (size_t)row * L);
#pragma unroll
      for (int g = 0; g < L / 4; ++g) acc_lane[g * 32] = src[g];
#pragma unroll 1
      for (uint32_t p = 1; p < a.nparts; ++p) {
        const uint4 *sp = reinterpret_cast<const uint4 *>(a.part + ((size_t)p * a.count + row) * L);
#pragma unroll
        for (int g = 0; g < L / 4; ++g) r_lane[g * 32] = sp[g];
        mont_mul_lanes<L, U>(acc_lane, r_lane, N, np);
      }
    }
    uint32_t u[L], v[L];
    {
      const uint4 *r4 = reinterpret_cast<const uint4 *>(a.mods + (size_t)row * L);
#pragma unroll
      for (int g = 0; g < L / 4; ++g) {
        const uint4 nv = __ldg(r4 + g), av = acc_lane[g * 32];
        u[4 * g] = nv.x; u[4 * g + 1] = nv.y; u[4 * g + 2] = nv.z; u[4 * g + 3] = nv.w;
        v[4 * g] = ok ? av.x : 0u; v[4 * g + 1] = ok ? av.y : 0u;
        v[4 * g + 2] = ok ? av.z : 0u; v[4 * g + 3] = ok ? av.w : 0u;
      }
    }
    binary_gcd<L>(u, v);
    if (!live) continue;
    uint32_t hi = 0, diff = 0;
    const uint4 *r4 = reinterpret_cast<const uint4 *>(a.mods + (size_t)row * L);
#pragma unroll
    for (int g = 0; g < L / 4; ++g) {
      const uint4 nv = __ldg(r4 + g);
      diff |= (u[4 * g] ^ nv.x) | (u[4 * g + 1] ^ nv.y) | (u[4 * g + 2] ^ nv.z) | (u[4 * g + 3] ^ nv.w);
    }
#pragma unroll
    for (int j = 1; j < L; ++j) hi |= u[j];
    if (a.gcds) {
      uint4 *dst = reinterpret_cast<uint4 *>(a.gcds + (size_t)i * L);
#pragma unroll
      for (int g = 0; g < L / 4; ++g)
        dst[g] = ok ? make_uint4(u[4 * g], u[4 * g + 1], u[4 * g + 2], u[4 * g + 3]) : make_uint4(0u, 0u, 0u, 0u);
    }
    if (a.flags) a.flags[i] = !ok ? -1 : (hi == 0u && u[0] == 1u) ? 0 : (diff == 0u ? 2 : 1);
  }
}

// Resident CTAs the partial-product kernel is compiled for: 3 fits the
// 1024-bit and smaller moduli in registers; at 2048 bits the register cap of 3
// CTAs (168) forces spills, 2 CTAs (up to 255 registers) does not.
int gcd_min_blocks(uint32_t L) {
  const char *v = std::getenv("RSAGPU_GCD_MINB");
  const int m = v ? std::atoi(v) : (L >= 64 ? 2 : 3);
  return (m == 2 || m == 3) ? m : 3;
}

template <int L>
struct GcdLaunch {
  static constexpr int U = 8;
  static const void *main_fn(int minb) {
    return minb == 2 ? (const void *)bgcd_kernel<L, U, 2> : (const void *)bgcd_kernel<L, U, 3>;
  }
  // Shared-memory opt-in of the kernels above 48 KiB, set on every call: the
  // attribute belongs to the current device's context, and setting it is cheap.
  static int prepare(size_t smem) {
    cudaError_t e = cudaSuccess;
    for (int m = 2; m <= 3 && e == cudaSuccess; ++m)
      e = cudaFuncSetAttribute(main_fn(m), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(bgcd_finish_kernel<L, U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(bgcd_combine_kernel<L, U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(bgcd)");
    return 0;
  }
  static int per_sm(size_t smem, int minb) {
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, main_fn(minb), kGcdThreads, smem);
    return e == cudaSuccess ? std::max(1, n) : 1;
  }
  // Returns the number of kernels launched through *launches.
  static cudaError_t run(const GcdArgs &h, int grid_blk, int grid_main, int grid_fin, uint64_t cap, size_t smem,
                         int minb, cudaStream_t s, int *launches) {
    bgcd_block_kernel<L><<<grid_blk, 64, 0, s>>>(h);
    if (minb == 2) bgcd_kernel<L, U, 2><<<grid_main, kGcdThreads, smem, s>>>(h);
    else bgcd_kernel<L, U, 3><<<grid_main, kGcdThreads, smem, s>>>(h);
    int n = 3;
    const uint64_t nsb = (h.count + kOwn - 1) / kOwn;
    for (uint32_t cur = h.nparts; cur > 1;) {
      const uint32_t half = (cur + 1) / 2;
      const uint64_t tasks = nsb * (cur - half);
      const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((tasks + 3) / 4, cap));
      bgcd_combine_kernel<L, U><<<grid, kGcdThreads, smem, s>>>(h, cur, half);
      ++n;
      cur = half;
    }
    GcdArgs f = h;
    f.nparts = 1;
    bgcd_finish_kernel<L, U><<<grid_fin, kGcdThreads, smem, s>>>(f);
    *launches = n;
    return cudaGetLastError();
  }
};

// Moduli per block product.  Larger blocks need fewer Montgomery
// multiplications into the running product (one per block) and longer
// product trees (block kernel 1.4 ms at B = 32 for 16384 2048-bit moduli on
// GB300).  Measured for 2048-bit moduli: 32 wins from about 8192 moduli up
// (16384: 181.0 ms against 192.0 with 16 and 218.7 with 8); at 2048 moduli 8
// and 16 tie (5.4 ms) and 32 is slower (6.0 ms).
int gcd_block_size(uint64_t count) {
  const char *v = std::getenv("RSAGPU_GCD_BLOCK");
  const int def = count >= 8192 ? 32 : count >= 4096 ? 16 : 8;
  const int b = v ? std::atoi(v) : def;
  return (b == 8 || b == 16 || b == 32) ? b : def;
}

}  // namespace
}  // namespace rsagpu

using namespace rsagpu;

namespace rsagpu {
namespace {

struct GcdPlan {
  uint32_t L = 0, blk = 0;
  uint64_t nblk = 0, nsb = 0, nparts = 0;
  int per_sm = 0, minb = 3;
  size_t smem = 0;
};

int gcd_plan(const Ctx *c, uint32_t nbits, uint64_t count, GcdPlan *pl) {
  pl->L = nbits / 32;
  pl->blk = (uint32_t)gcd_block_size(count);
  pl->nblk = (count + pl->blk - 1) / pl->blk;
  pl->nsb = (count + kOwn - 1) / kOwn;
  const uint32_t L = pl->L;
  pl->smem = (L == 16)   ? GcdSmem<16>::bytes(kGcdThreads / 32)
             : (L == 32) ? GcdSmem<32>::bytes(kGcdThreads / 32)
                         : GcdSmem<64>::bytes(kGcdThreads / 32);
  int rc = (L == 16) ? GcdLaunch<16>::prepare(pl->smem) : (L == 32) ? GcdLaunch<32>::prepare(pl->smem)
                                                                    : GcdLaunch<64>::prepare(pl->smem);
  if (rc) return rc;
  pl->minb = gcd_min_blocks(L);
  pl->per_sm = (L == 16)   ? GcdLaunch<16>::per_sm(pl->smem, pl->minb)
               : (L == 32) ? GcdLaunch<32>::per_sm(pl->smem, pl->minb)
                           : GcdLaunch<64>::per_sm(pl->smem, pl->minb);
  // split the j range into parts until there are about four warp tasks per
  // resident warp; the partial products cost nparts * count * L words
  const uint64_t resident = (uint64_t)pl->per_sm * c->sm_count * (kGcdThreads / 32);
  const uint64_t row_bytes = (uint64_t)count * L * 4;
  uint64_t np = std::max<uint64_t>(1, (4 * resident + pl->nsb - 1) / pl->nsb);
  np = std::min<uint64_t>(np, pl->nsb);
  np = std::min<uint64_t>(np, std::max<uint64_t>(1, (1ull << 30) / row_bytes));
  pl->nparts = np;
  return 0;
}

int gcd_check(rsa_ctx *ctx, uint32_t nbits, uint64_t count) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  if (nbits != 512 && nbits != 1024 && nbits != 2048)
    return set_error(RSA_ERR_UNSUPPORTED, "moduli of 512, 1024 or 2048 bits");
  if (count > (1ull << 26)) return set_error(RSA_ERR_ARG, "count above 2^26");
  return RSA_OK;
}

}  // namespace
}  // namespace rsagpu

namespace rsagpu {
namespace {

// The launches of one scan on stream s: block products, reductions, the
// combine tree (one launch per level), gcd.  Context lock held.
int batch_gcd_run(Ctx *c, uint32_t nbits, uint64_t count, const uint32_t *moduli, uint32_t *gcds, int32_t *flags,
                  cudaStream_t s) {
  int rc;
  cudaSetDevice(c->device);
  Workspace &w = c->ws(s);
  NvtxRange range("rsa_batch_gcd");
  GcdPlan pl;
  if ((rc = gcd_plan(c, nbits, count, &pl))) return rc;
  const uint32_t L = pl.L;
  const size_t valid_bytes = ((size_t)count + 15) / 16 * 16;
  const size_t bprod_bytes = (size_t)pl.nblk * pl.blk * L * 4;
  const size_t scratch_bytes = (size_t)pl.nblk * gcd_scratch_words(L, pl.blk) * 4;
  if ((rc = c->ensure(w.gcd0, valid_bytes + bprod_bytes + scratch_bytes)) ||
      (rc = c->ensure(w.gcd1, (size_t)pl.nparts * count * L * 4)))
    return rc;
  uint8_t *base = static_cast<uint8_t *>(w.gcd0.ptr);
  GcdArgs h{moduli, base, reinterpret_cast<uint32_t *>(base + valid_bytes),
            reinterpret_cast<uint32_t *>(base + valid_bytes + bprod_bytes), static_cast<uint32_t *>(w.gcd1.ptr),
            gcds, flags, (uint32_t)count, pl.blk, (uint32_t)pl.nparts};
  const uint64_t cap = (uint64_t)pl.per_sm * c->sm_count;
  const int grid_blk = (int)((pl.nblk + 1) / 2);      // one warp per block, two per CTA
  const int grid_main = (int)std::max<uint64_t>(1, std::min<uint64_t>((pl.nsb * pl.nparts + 3) / 4, cap));
  const int grid_fin = (int)std::max<uint64_t>(1, std::min<uint64_t>((pl.nsb + 3) / 4, cap));
  int launches = 0;
  cudaError_t e = (L == 16)   ? GcdLaunch<16>::run(h, grid_blk, grid_main, grid_fin, cap, pl.smem, pl.minb, s, &launches)
                  : (L == 32) ? GcdLaunch<32>::run(h, grid_blk, grid_main, grid_fin, cap, pl.smem, pl.minb, s, &launches)
                              : GcdLaunch<64>::run(h, grid_blk, grid_main, grid_fin, cap, pl.smem, pl.minb, s, &launches);
  if (e != cudaSuccess) return cuda_error(e, "launch bgcd kernels");
  c->stats.kernel_launches += (uint64_t)launches;
  c->stats.ops += count;
  return RSA_OK;
}

}  // namespace
}  // namespace rsagpu

namespace rsagpu {
namespace {

// From this many modulus words (count x L) the automatic choice takes the
// trees, when their memory fits the context's budget.  Measured on GB300:
// 4096 2048-bit moduli (2^18 words) scan 15.3 ms, tree 9.3; 2048 moduli scan
// 5.4 ms.
uint64_t gcd_tree_min_words() {
  const char *v = std::getenv("RSAGPU_GCD_TREE_MIN_WORDS");
  return v ? std::strtoull(v, nullptr, 10) : (1ull << 18);
}

bool tree_fits(uint32_t L, uint64_t count) {
  uint64_t K = 2;
  while (K < count) K <<= 1;
  return K * L <= (1ull << 26);
}

int gcd_method(const Ctx *c, uint32_t nbits, uint64_t count, int method) {
  const uint32_t L = nbits / 32;
  if (method == RSA_GCD_AUTO) {
    const bool tree = count >= 2 && count * L >= gcd_tree_min_words() && tree_fits(L, count) &&
                      c->used + batch_gcd_tree_bytes(L, count) <= c->budget;
    return tree ? RSA_GCD_TREE : RSA_GCD_SCAN;
  }
  return method;
}

int gcd_dispatch(Ctx *c, uint32_t nbits, uint64_t count, const uint32_t *moduli, uint32_t *gcds, int32_t *flags,
                 int method, cudaStream_t s) {
  method = gcd_method(c, nbits, count, method);
  if (method == RSA_GCD_TREE) {
    cudaSetDevice(c->device);
    return batch_gcd_tree_run(c, nbits, count, moduli, gcds, flags, s);
  }
  return batch_gcd_run(c, nbits, count, moduli, gcds, flags, s);
}

int method_check(uint32_t nbits, uint64_t count, int method) {
  if (method != RSA_GCD_AUTO && method != RSA_GCD_SCAN && method != RSA_GCD_TREE)
    return set_error(RSA_ERR_ARG, "method must be RSA_GCD_AUTO, RSA_GCD_SCAN or RSA_GCD_TREE");
  if (method == RSA_GCD_TREE && !tree_fits(nbits / 32, count))
    return set_error(RSA_ERR_ARG, "tree form: count (rounded up to a power of two) times modulus words above 2^26");
  return RSA_OK;
}

}  // namespace
}  // namespace rsagpu

extern "C" int rsa_batch_gcd_ex(rsa_ctx *ctx, uint32_t nbits, uint64_t count, const uint32_t *moduli,
                                uint32_t *gcds, int32_t *flags, int method, void *stream) {
  int rc = gcd_check(ctx, nbits, count);
  if (rc) return rc;
  if ((rc = method_check(nbits, count, method))) return rc;
  if (count == 0) return RSA_OK;
  if (!moduli || (!gcds && !flags)) return set_error(RSA_ERR_ARG, "null pointer");
  if ((reinterpret_cast<uintptr_t>(moduli) | reinterpret_cast<uintptr_t>(gcds)) & 15u)
    return set_error(RSA_ERR_ARG, "modulus and gcd rows must be 16-byte aligned");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  return gcd_dispatch(c, nbits, count, moduli, gcds, flags, method, static_cast<cudaStream_t>(stream));
}

extern "C" int rsa_batch_gcd(rsa_ctx *ctx, uint32_t nbits, uint64_t count, const uint32_t *moduli, uint32_t *gcds,
                             int32_t *flags, void *stream) {
  return rsa_batch_gcd_ex(ctx, nbits, count, moduli, gcds, flags, RSA_GCD_AUTO, stream);
}

extern "C" int rsa_batch_gcd_method(rsa_ctx *ctx, uint32_t nbits, uint64_t count, int *method) {
  int rc = gcd_check(ctx, nbits, count);
  if (rc) return rc;
  if (!method) return set_error(RSA_ERR_ARG, "null pointer");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  *method = gcd_method(c, nbits, count, RSA_GCD_AUTO);
  return RSA_OK;
}

extern "C" int rsa_batch_gcd_tree_bytes(uint32_t nbits, uint64_t count, uint64_t *bytes) {
  if (nbits != 512 && nbits != 1024 && nbits != 2048)
    return set_error(RSA_ERR_UNSUPPORTED, "moduli of 512, 1024 or 2048 bits");
  if (!bytes) return set_error(RSA_ERR_ARG, "null pointer");
  if (!tree_fits(nbits / 32, count))
    return set_error(RSA_ERR_ARG, "tree form: count (rounded up to a power of two) times modulus words above 2^26");
  *bytes = batch_gcd_tree_bytes(nbits / 32, count);
  return RSA_OK;
}

extern "C" int rsa_batch_gcd_host(rsa_ctx *ctx, uint32_t nbits, uint64_t count, const uint32_t *moduli,
                                  uint32_t *gcds, int32_t *flags, void *stream) {
  int rc = gcd_check(ctx, nbits, count);
  if (rc) return rc;
  if (count == 0) return RSA_OK;
  if (!moduli || (!gcds && !flags)) return set_error(RSA_ERR_ARG, "null pointer");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Workspace &w = c->ws(s);
  const size_t bytes = (size_t)count * (nbits / 32) * 4;
  if ((rc = c->ensure(w.io_in, bytes)) || (gcds && (rc = c->ensure(w.io_out, bytes))) ||
      (flags && (rc = c->ensure(w.io_status, (size_t)count * 4))))
    return rc;
  cudaError_t e = cudaMemcpyAsync(w.io_in.ptr, moduli, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync H2D");
  uint32_t *dg = gcds ? static_cast<uint32_t *>(w.io_out.ptr) : nullptr;
  int32_t *df = flags ? static_cast<int32_t *>(w.io_status.ptr) : nullptr;
  if ((rc = gcd_dispatch(c, nbits, count, static_cast<const uint32_t *>(w.io_in.ptr), dg, df, RSA_GCD_AUTO, s)))
    return rc;
  if (gcds && (e = cudaMemcpyAsync(gcds, dg, bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_error(e, "cudaMemcpyAsync D2H gcds");
  if (flags && (e = cudaMemcpyAsync(flags, df, (size_t)count * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_error(e, "cudaMemcpyAsync D2H flags");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  return RSA_OK;
}

extern "C" int rsa_batch_gcd_plan(rsa_ctx *ctx, uint32_t nbits, uint64_t count, uint32_t *block, uint64_t *parts) {
  int rc = gcd_check(ctx, nbits, count);
  if (rc) return rc;
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  cudaSetDevice(c->device);
  GcdPlan pl;
  if ((rc = gcd_plan(c, nbits, std::max<uint64_t>(count, 1), &pl))) return rc;
  if (block) *block = pl.blk;
  if (parts) *parts = pl.nparts;
  return RSA_OK;
}
