// bgcd_tree.cu -- batch GCD by a product tree and a remainder tree, for scans
// of many moduli (the weak-key detection the paper's introduction motivates:
// two RSA moduli that share a prime are both factored by one gcd).
//
// g_i = gcd(n_i, prod_{j != i} n_j) for k moduli costs about L^2 k^2 word
// products modulus by modulus (bgcd.cu).  With fast multiplication the trees
// cost O(k L log^2(k L)) instead:
//   * product tree: X_0 = the moduli (1 for invalid ones and for padding up to
//     K = 2^T), X_{t+1}[v] = X_t[2v] X_t[2v+1]; a node of level t has
//     s_t = L 2^t words;
//   * remainder tree in Montgomery form, Y_t = X_t^2, mu_t = -Y_t^-1 mod
//     2^(32 k), k = 2 s_t: Z_T = X_T, Z_t[v] = (Z_{t+1}[v/2] + q Y_t[v]) /
//     2^(32k) with q = Z_{t+1}[v/2] mu_t[v] mod 2^(32k).  Z_t[v] is congruent
//     to P 2^(-e) modulo Y_t[v] (P = X_T, e a multiple of 32) and stays below
//     (T - t + 1) Y_t[v] with no subtraction, in k + 1 words;
//   * mu at the top level of the remainder tree (the root's two children) by
//     Newton's iteration from one word (mu_hi = H mu + mu mod 2^(32w), H the
//     words w..2w of Y mu); below it from the parent, one product per node:
//     mu_parent = -(Y_a Y_b)^-1, so mu_a = Y_b mu_parent mod 2^(32k);
//   * at the leaves, per modulus: Z of its level-t0 node reduced modulo n_i^2
//     word by word (Montgomery), so z = P 2^(-e') mod n_i^2, a multiple of n_i;
//     u = z / n_i (exact division, word by word from the bottom) is
//     (P / n_i) 2^(-e') mod n_i, and g_i = gcd(n_i, u) because 2 is a unit
//     modulo the odd n_i.
// Products of up to kSchoolMax words are formed schoolbook, one CTA per group
// of products; longer ones by number-theoretic transforms of the 32-bit words
// modulo three primes p = c 2^e + 1 (2013265921, 3221225473, 3489660929; every
// column of a product of operands of up to 2^26 words is below their
// product), recombined by Garner's method, with the carries resolved by a
// carry-lookahead scan.  Every multiplication takes an optional addend, an
// output slice and operand rows chosen by the node's index (its parent's or
// sibling's), which the Newton steps and the remainder steps need.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "bgcd.cuh"
#include "mont.cuh"
#include "rsa_gb300.h"
#include "runtime_internal.h"

namespace rsagpu {
namespace tree {

constexpr uint32_t kPrime[3] = {2013265921u, 3221225473u, 3489660929u};
constexpr uint32_t kMaxLog = 27;            // transforms of up to 2^27 words (2-adic order of the first prime)
constexpr uint32_t kTile = 4096;            // transform stages done in shared memory: blocks of up to 4096 words
constexpr uint32_t kSchoolMax = 512;        // products of at most this many words: schoolbook
constexpr uint32_t kCarryWords = 16;        // words per thread of the carry scan
constexpr uint32_t kCarryThreads = 256;
constexpr uint32_t kCarryBlock = kCarryWords * kCarryThreads;

// Per-prime constants of one multiplication (values in Montgomery form, R = 2^32).
struct Primes {
  uint32_t p[3], pinv[3];                   // p, p^-1 mod 2^32
  uint32_t scale[3];                        // n^-1 R^2 mod p: undoes the transform's factor n and one R^-1
  uint32_t inv12;                           // p1^-1 mod p2 (Montgomery form, modulo p2)
  uint32_t p1m3;                            // p1 mod p3 (Montgomery form, modulo p3)
  uint32_t inv123;                          // (p1 p2)^-1 mod p3 (Montgomery form, modulo p3)
  const uint32_t *tw[3], *itw[3];           // nested twiddle tables: tw[len + j] = w_(2 len)^j R mod p
};

// Operand i of a batch: row (i >> shift) ^ xr at p + row * stride (shift 1:
// the parent's row; xr = 1: the sibling's row), `words` words (zero beyond).
struct Opnd {
  const uint32_t *p;
  uint64_t stride;
  uint32_t shift, words, xr;
};

// Output of product i: words [lo, hi) of the result at p + i * stride.
struct Out {
  uint32_t *p;
  uint64_t stride;
  uint32_t lo, hi;
};

__device__ __forceinline__ uint32_t opnd_word(const Opnd &o, uint64_t i, uint32_t j) {
  if (j >= o.words) return 0u;
  return o.p[((i >> o.shift) ^ o.xr) * o.stride + j];
}

// The reductions below take the borrow of a subtraction as a mask m (0 or all
// ones) and add m * (-p) = (m ? p : 0) with one multiply-add, which keeps the
// integer-ALU pipe (the transforms' busiest) free of compares and selects.
__device__ __forceinline__ uint32_t add_masked_p(uint32_t x, uint32_t m, uint32_t p) { return x + m * (0u - p); }

// Montgomery product a b R^-1 mod p for a, b < p < 2^32: with m = lo(ab) p^-1,
// ab - mp is a multiple of 2^32 and its high word hi(ab) - hi(mp) lies in (-p, p).
__device__ __forceinline__ uint32_t mmul(uint32_t a, uint32_t b, uint32_t p, uint32_t pinv) {
  const uint64_t t = (uint64_t)a * b;
  const uint32_t m = (uint32_t)t * pinv;
  const uint32_t mh = __umulhi(m, p);
  uint32_t d, bm;
  asm("sub.cc.u32 %0, %2, %3;\n\tsubc.u32 %1, 0, 0;" : "=r"(d), "=r"(bm) : "r"((uint32_t)(t >> 32)), "r"(mh));
  return add_masked_p(d, bm, p);
}

// a + b mod p for a, b < p: s = a + b with carry c, r = s - p with borrow;
// c - borrow is all ones exactly when a + b < p (a sum that wraps 2^32 is
// above p and leaves s < p), and then s = r + p is the result.
__device__ __forceinline__ uint32_t madd(uint32_t a, uint32_t b, uint32_t p) {
  uint32_t r, bm;
  asm("{\n\t.reg .u32 s, c;\n\t"
      "add.cc.u32 s, %2, %3;\n\t"
      "addc.u32 c, 0, 0;\n\t"
      "sub.cc.u32 %0, s, %4;\n\t"
      "subc.u32 %1, c, 0;\n\t}"
      : "=r"(r), "=r"(bm)
      : "r"(a), "r"(b), "r"(p));
  return add_masked_p(r, bm, p);
}

// a - b mod p for a, b < p
__device__ __forceinline__ uint32_t msub(uint32_t a, uint32_t b, uint32_t p) {
  uint32_t d, bm;
  asm("sub.cc.u32 %0, %2, %3;\n\tsubc.u32 %1, 0, 0;" : "=r"(d), "=r"(bm) : "r"(a), "r"(b));
  return add_masked_p(d, bm, p);
}

// prime k's entry of a per-prime parameter array (selects, no local copy)
__device__ __forceinline__ uint32_t sel3(const uint32_t (&a)[3], uint32_t k) {
  return k == 0 ? a[0] : k == 1 ? a[1] : a[2];
}

__device__ __forceinline__ const uint32_t *sel3p(const uint32_t *const (&a)[3], uint32_t k) {
  return k == 0 ? a[0] : k == 1 ? a[1] : a[2];
}

// ------------------------------------------------------------------ twiddles

// tw[i] for 1 <= i < nmax: i = len + j (len the power of two below i) holds
// w_(2 len)^j = root^(j nmax / (2 len)) with root of order nmax, in
// Montgomery form; itw the same for root^-1.  One table serves every
// transform length up to nmax.
__global__ void twiddle_kernel(uint32_t *tw, uint32_t *itw, uint32_t nmax, uint32_t p, uint32_t pinv,
                               uint32_t root_m, uint32_t iroot_m, uint32_t one_m) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nmax; i += gridDim.x * blockDim.x) {
    if (i == 0) {
      tw[0] = 0u;
      itw[0] = 0u;
      continue;
    }
    const uint32_t len = 1u << (31 - __clz(i));
    uint32_t e = (i - len) * (nmax / (2u * len));
    uint32_t r = one_m, ir = one_m, b = root_m, ib = iroot_m;
    while (e) {
      if (e & 1u) {
        r = mmul(r, b, p, pinv);
        ir = mmul(ir, ib, p, pinv);
      }
      b = mmul(b, b, p, pinv);
      ib = mmul(ib, ib, p, pinv);
      e >>= 1;
    }
    tw[i] = r;
    itw[i] = ir;
  }
}

// ------------------------------------------------------------------ transforms
// Buffers hold the three primes' arrays back to back (prime k at k * E), each
// `cnt` transforms of length n, so blockIdx.y selects the prime.  Forward:
// decimation in frequency (natural order in, bit-reversed out); inverse:
// decimation in time (bit-reversed in, natural out) with the inverse roots,
// so no permutation is needed between them.

// F_k[i n + j] = word j of operand i mod p_k (zero for j >= words); prime k's
// array at k * stride.
__global__ void ntt_load_kernel(Opnd X, uint32_t *F, uint64_t E, uint64_t stride, uint32_t logn) {
  const uint32_t p0 = kPrime[0], p1 = kPrime[1], p2 = kPrime[2];
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t w = opnd_word(X, e >> logn, (uint32_t)(e & ((1ull << logn) - 1)));
    F[e] = w % p0;
    F[stride + e] = w % p1;
    F[2 * stride + e] = w % p2;
  }
}

// S decimation-in-frequency stages (distances 2^(S-1) h .. h) in one pass over
// the 2^S words x_m = F[b + m h], b = 2^S h * block + j, j < h: at distance
// d h word m pairs with m + d when m & d is clear, with twiddle
// tw[d h + j + (m mod d) h].
template <int S>
__global__ void difr_kernel(uint32_t *F, uint64_t E, uint32_t logh, Primes P) {
  constexpr int R = 1 << S;
  const uint32_t k = blockIdx.y, p = sel3(P.p, k), pinv = sel3(P.pinv, k);
  uint32_t *f = F + k * E;
  const uint32_t *tw = sel3p(P.tw, k);
  const uint32_t h = 1u << logh;
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < E / R; q += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t j = (uint32_t)(q & (h - 1));
    const uint64_t b = ((q >> logh) << (logh + S)) + j;
    uint32_t x[R];
#pragma unroll
    for (int m = 0; m < R; ++m) x[m] = f[b + (uint64_t)m * h];
#pragma unroll
    for (int d = R / 2; d >= 1; d /= 2) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        if (m & d) continue;
        const uint32_t a = x[m], c = x[m + d];
        x[m] = madd(a, c, p);
        x[m + d] = mmul(msub(a, c, p), tw[(uint32_t)d * h + j + (uint32_t)(m & (d - 1)) * h], p, pinv);
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) f[b + (uint64_t)m * h] = x[m];
  }
}

// The S decimation-in-time stages (distances h .. 2^(S-1) h) over the same words.
template <int S>
__global__ void ditr_kernel(uint32_t *F, uint64_t E, uint32_t logh, Primes P) {
  constexpr int R = 1 << S;
  const uint32_t k = blockIdx.y, p = sel3(P.p, k), pinv = sel3(P.pinv, k);
  uint32_t *f = F + k * E;
  const uint32_t *itw = sel3p(P.itw, k);
  const uint32_t h = 1u << logh;
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < E / R; q += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t j = (uint32_t)(q & (h - 1));
    const uint64_t b = ((q >> logh) << (logh + S)) + j;
    uint32_t x[R];
#pragma unroll
    for (int m = 0; m < R; ++m) x[m] = f[b + (uint64_t)m * h];
#pragma unroll
    for (int d = 1; d <= R / 2; d *= 2) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        if (m & d) continue;
        const uint32_t a = x[m], c = mmul(x[m + d], itw[(uint32_t)d * h + j + (uint32_t)(m & (d - 1)) * h], p, pinv);
        x[m] = madd(a, c, p);
        x[m + d] = msub(a, c, p);
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) f[b + (uint64_t)m * h] = x[m];
  }
}

// The twelve stages of half-length below kTile run in shared memory, one tile
// of 4096 words per CTA of 512 threads, three stages per exchange: for
// distances 4q, 2q, q (q = 512, 64, 8, 1 forward; the reverse inverse) thread
// t holds the eight words b + k q, b = (t / q) 8q + t mod q, whose butterflies
// at those three distances stay among them.  Word a lives at a + a / 32
// (padding against bank conflicts when q < 32).
constexpr uint32_t kTileThreads = 512;

__device__ __forceinline__ uint32_t pad(uint32_t a) { return a + (a >> 5); }

__device__ __forceinline__ void bf_dif(uint32_t &u, uint32_t &v, uint32_t w, uint32_t p, uint32_t pinv) {
  const uint32_t a = u, b = v;
  u = madd(a, b, p);
  v = mmul(msub(a, b, p), w, p, pinv);
}

__device__ __forceinline__ void bf_dit(uint32_t &u, uint32_t &v, uint32_t w, uint32_t p, uint32_t pinv) {
  const uint32_t a = u, b = mmul(v, w, p, pinv);
  u = madd(a, b, p);
  v = msub(a, b, p);
}

// three forward stages (distances 4q, 2q, q) on the thread's eight words;
// the first `skip` of them are left out (tiles holding several shorter
// transforms)
__device__ __forceinline__ void dif8(uint32_t (&x)[8], uint32_t q, uint32_t jp, const uint32_t *tw, uint32_t p,
                                     uint32_t pinv, uint32_t skip = 0) {
  if (skip == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) bf_dif(x[k], x[k + 4], tw[4 * q + jp + k * q], p, pinv);
  }
  if (skip <= 1) {
    const uint32_t w0 = tw[2 * q + jp], w1 = tw[2 * q + jp + q];
    bf_dif(x[0], x[2], w0, p, pinv);
    bf_dif(x[1], x[3], w1, p, pinv);
    bf_dif(x[4], x[6], w0, p, pinv);
    bf_dif(x[5], x[7], w1, p, pinv);
  }
  const uint32_t w = tw[q + jp];
#pragma unroll
  for (int k = 0; k < 8; k += 2) bf_dif(x[k], x[k + 1], w, p, pinv);
}

// three inverse stages (distances q, 2q, 4q); the last `skip` left out
__device__ __forceinline__ void dit8(uint32_t (&x)[8], uint32_t q, uint32_t jp, const uint32_t *itw, uint32_t p,
                                     uint32_t pinv, uint32_t skip = 0) {
  const uint32_t w = itw[q + jp];
#pragma unroll
  for (int k = 0; k < 8; k += 2) bf_dit(x[k], x[k + 1], w, p, pinv);
  if (skip <= 1) {
    const uint32_t w0 = itw[2 * q + jp], w1 = itw[2 * q + jp + q];
    bf_dit(x[0], x[2], w0, p, pinv);
    bf_dit(x[1], x[3], w1, p, pinv);
    bf_dit(x[4], x[6], w0, p, pinv);
    bf_dit(x[5], x[7], w1, p, pinv);
  }
  if (skip == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) bf_dit(x[k], x[k + 4], itw[4 * q + jp + k * q], p, pinv);
  }
}

__device__ __forceinline__ uint32_t tile_base(uint32_t q) {
  const uint32_t t = threadIdx.x;
  return (t / q) * 8 * q + (t & (q - 1));
}

__device__ __forceinline__ void sload8(const uint32_t *s, uint32_t b, uint32_t q, uint32_t (&x)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = s[pad(b + k * q)];
}

__device__ __forceinline__ void sstore8(uint32_t *s, uint32_t b, uint32_t q, const uint32_t (&x)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) s[pad(b + k * q)] = x[k];
}

// Forward stages below kTile of every tile (the operand that is multiplied in);
// a tile holds one 4096-word piece of a longer transform, or 2^skip
// transforms of 4096 / 2^skip words whose first `skip` stages do not exist.
__global__ void __launch_bounds__(kTileThreads) ntt_tile_fwd_kernel(uint32_t *F, uint64_t E, uint32_t skip,
                                                                    Primes P) {
  __shared__ uint32_t s[kTile + kTile / 32];
  const uint32_t k = blockIdx.y, p = sel3(P.p, k), pinv = sel3(P.pinv, k);
  const uint32_t *tw = sel3p(P.tw, k);
  uint32_t *f = F + k * E + (uint64_t)blockIdx.x * kTile;
  for (uint32_t a = threadIdx.x; a < kTile; a += kTileThreads) s[pad(a)] = f[a];
  uint32_t x[8];
  for (uint32_t q = kTile / 8; q >= 1; q /= 8) {
    __syncthreads();
    const uint32_t b = tile_base(q);
    sload8(s, b, q, x);
    dif8(x, q, threadIdx.x & (q - 1), tw, p, pinv, q == kTile / 8 ? skip : 0u);
    if (q > 1) sstore8(s, b, q, x);
  }
  // q = 1: the thread's words are 8t .. 8t+7
  uint4 *f4 = reinterpret_cast<uint4 *>(f + 8 * threadIdx.x);
  f4[0] = make_uint4(x[0], x[1], x[2], x[3]);
  f4[1] = make_uint4(x[4], x[5], x[6], x[7]);
}

// Forward stages below kTile, the pointwise product with FB (or a square;
// each product carries one factor R^-1) and the inverse stages below kTile,
// in one pass per tile: the last forward and the first inverse exchange (q =
// 1) share the thread's words, so the product happens in registers.
__global__ void __launch_bounds__(kTileThreads) ntt_tile_mul_kernel(uint32_t *FA, const uint32_t *FB, uint64_t E,
                                                                    uint32_t skip, Primes P) {
  __shared__ uint32_t s[kTile + kTile / 32];
  const uint32_t k = blockIdx.y, p = sel3(P.p, k), pinv = sel3(P.pinv, k);
  const uint32_t *tw = sel3p(P.tw, k), *itw = sel3p(P.itw, k);
  const uint64_t off = k * E + (uint64_t)blockIdx.x * kTile;
  uint32_t *f = FA + off;
  for (uint32_t a = threadIdx.x; a < kTile; a += kTileThreads) s[pad(a)] = f[a];
  uint32_t x[8];
  for (uint32_t q = kTile / 8; q >= 1; q /= 8) {
    __syncthreads();
    const uint32_t b = tile_base(q);
    sload8(s, b, q, x);
    dif8(x, q, threadIdx.x & (q - 1), tw, p, pinv, q == kTile / 8 ? skip : 0u);
    if (q > 1) sstore8(s, b, q, x);
  }
  {
    uint32_t y[8];
    if (FB) {
      const uint4 *g4 = reinterpret_cast<const uint4 *>(FB + off + 8 * threadIdx.x);
      const uint4 g0 = g4[0], g1 = g4[1];
      y[0] = g0.x; y[1] = g0.y; y[2] = g0.z; y[3] = g0.w;
      y[4] = g1.x; y[5] = g1.y; y[6] = g1.z; y[7] = g1.w;
    } else {
#pragma unroll
      for (int m = 0; m < 8; ++m) y[m] = x[m];
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = mmul(x[m], y[m], p, pinv);
  }
  for (uint32_t q = 1; q <= kTile / 8; q *= 8) {
    const uint32_t b = tile_base(q);
    if (q > 1) {
      __syncthreads();
      sload8(s, b, q, x);
    }
    dit8(x, q, threadIdx.x & (q - 1), itw, p, pinv, q == kTile / 8 ? skip : 0u);
    sstore8(s, b, q, x);
  }
  __syncthreads();
  for (uint32_t a = threadIdx.x; a < kTile; a += kTileThreads) f[a] = s[pad(a)];
}

// Pointwise product of two forward-transformed batches and the inverse stages
// below kTile, out of place (a cached transform stays intact): tile b of the
// result belongs to transform i = b 4096 / n (n >= kTile) at offset o; its
// factors are A's transform (i >> sha) ^ xra and B's transform i >> shb at
// the same offset, each batch with its own per-prime stride.
__global__ void __launch_bounds__(kTileThreads) ntt_tile_pinv_kernel(uint32_t *FO, uint64_t os, const uint32_t *FA,
                                                                     uint64_t as, uint32_t sha, uint32_t xra,
                                                                     const uint32_t *FB, uint64_t bs, uint32_t shb,
                                                                     uint32_t logn, Primes P) {
  __shared__ uint32_t s[kTile + kTile / 32];
  const uint32_t k = blockIdx.y, p = sel3(P.p, k), pinv = sel3(P.pinv, k);
  const uint32_t *itw = sel3p(P.itw, k);
  const uint64_t first = (uint64_t)blockIdx.x * kTile;
  const uint64_t i = first >> logn, o = first & ((1ull << logn) - 1);
  const uint4 *a4 = reinterpret_cast<const uint4 *>(FA + k * as + ((((i >> sha) ^ xra)) << logn) + o + 8 * threadIdx.x);
  const uint4 *b4 = reinterpret_cast<const uint4 *>(FB + k * bs + ((i >> shb) << logn) + o + 8 * threadIdx.x);
  uint32_t x[8];
  {
    const uint4 a0 = a4[0], a1 = a4[1], b0 = b4[0], b1 = b4[1];
    x[0] = mmul(a0.x, b0.x, p, pinv); x[1] = mmul(a0.y, b0.y, p, pinv);
    x[2] = mmul(a0.z, b0.z, p, pinv); x[3] = mmul(a0.w, b0.w, p, pinv);
    x[4] = mmul(a1.x, b1.x, p, pinv); x[5] = mmul(a1.y, b1.y, p, pinv);
    x[6] = mmul(a1.z, b1.z, p, pinv); x[7] = mmul(a1.w, b1.w, p, pinv);
  }
  for (uint32_t q = 1; q <= kTile / 8; q *= 8) {
    const uint32_t b = tile_base(q);
    if (q > 1) {
      __syncthreads();
      sload8(s, b, q, x);
    }
    dit8(x, q, threadIdx.x & (q - 1), itw, p, pinv);
    sstore8(s, b, q, x);
  }
  __syncthreads();
  uint32_t *f = FO + k * os + first;
  for (uint32_t a = threadIdx.x; a < kTile; a += kTileThreads) f[a] = s[pad(a)];
}

// ------------------------------------------------------------------ recombination and carries

// Column j of product i as a 96-bit integer (three words): the residues,
// scaled by n^-1 R^2, recombined by Garner's method
// x = v1 + p1 v2 + p1 p2 v3 (below p1 p2 p3 < 2^95).
__device__ __forceinline__ void column(const uint32_t *F, uint64_t E, uint64_t at, const Primes &P, uint32_t &lo,
                                       uint32_t &mid, uint32_t &hi) {
  const uint32_t p1 = P.p[0], p2 = P.p[1], p3 = P.p[2];
  const uint32_t r1 = mmul(F[at], P.scale[0], p1, P.pinv[0]);
  const uint32_t r2 = mmul(F[E + at], P.scale[1], p2, P.pinv[1]);
  const uint32_t r3 = mmul(F[2 * E + at], P.scale[2], p3, P.pinv[2]);
  const uint32_t v1 = r1;                                             // < p1 < p2 < p3
  const uint32_t v2 = mmul(msub(r2, v1, p2), P.inv12, p2, P.pinv[1]);
  const uint32_t t3 = madd(v1, mmul(v2, P.p1m3, p3, P.pinv[2]), p3);
  const uint32_t v3 = mmul(msub(r3, t3, p3), P.inv123, p3, P.pinv[2]);
  const uint64_t a = (uint64_t)p1 * v2 + v1;
  const uint64_t p12 = (uint64_t)p1 * p2;
  const uint64_t blo = p12 * v3;
  uint32_t bhi = (uint32_t)__umul64hi(p12, v3);
  const uint64_t s = blo + a;
  bhi += s < a ? 1u : 0u;
  lo = (uint32_t)s;
  mid = (uint32_t)(s >> 32);
  hi = bhi;
}

// Word c of product i before carries between words: lo(x_c) + mid(x_(c-1)) +
// hi(x_(c-2)) + d_c, below 2^34.  Columns past the transform length are 0.
struct WordSrc {
  const uint32_t *F;
  uint64_t E;
  uint32_t logn;
  Primes P;
  Opnd D;
};

// The 16 words of one thread: base value w (low 32 bits of each word sum plus
// the previous word's overflow) and the generate / propagate masks of the
// carry into the next word: g bit m set when word m overflows on its own, p
// bit m set when it is all ones (overflows only with a carry in).
__device__ __forceinline__ void thread_words(const WordSrc &S, uint64_t i, uint32_t c0, uint32_t (&w)[kCarryWords],
                                             uint32_t &g, uint32_t &pm) {
  const uint32_t n = 1u << S.logn;
  const uint64_t row = i << S.logn;
  // columns c0-3 .. c0+15
  uint32_t lo[kCarryWords + 3], mid[kCarryWords + 3], hi[kCarryWords + 3];
#pragma unroll
  for (int m = 0; m < (int)kCarryWords + 3; ++m) {
    const int64_t c = (int64_t)c0 + m - 3;
    if (c >= 0 && c < (int64_t)n) {
      column(S.F, S.E, row + (uint64_t)c, S.P, lo[m], mid[m], hi[m]);
    } else {
      lo[m] = mid[m] = hi[m] = 0u;
    }
  }
  // word sums s_c = lo_c + mid_(c-1) + hi_(c-2) + d_c for c0-1 .. c0+15
  uint32_t prev_over = 0;
  {
    const int64_t c = (int64_t)c0 - 1;
    if (c >= 0) {
      const uint64_t s = (uint64_t)lo[2] + mid[1] + hi[0] + opnd_word(S.D, i, (uint32_t)c);
      prev_over = (uint32_t)(s >> 32);
    }
  }
  g = 0u;
  pm = 0u;
#pragma unroll
  for (int m = 0; m < (int)kCarryWords; ++m) {
    const uint64_t s = (uint64_t)lo[m + 3] + mid[m + 2] + hi[m + 1] + opnd_word(S.D, i, c0 + (uint32_t)m);
    const uint64_t v = (uint64_t)(uint32_t)s + prev_over;
    prev_over = (uint32_t)(s >> 32);
    w[m] = (uint32_t)v;
    g |= (uint32_t)(v >> 32) << m;
    pm |= (v == 0xffffffffull ? 1u : 0u) << m;
  }
}

// Carry into each of the 16 words given the carry into the first, and the carry out.
__device__ __forceinline__ uint32_t apply_carries(uint32_t (&w)[kCarryWords], uint32_t g, uint32_t pm, uint32_t cin) {
  const uint64_t a = (uint64_t)(g | pm), sum = a + g + cin;
  const uint32_t into = (uint32_t)(sum ^ a ^ g);
#pragma unroll
  for (int m = 0; m < (int)kCarryWords; ++m) w[m] += (into >> m) & 1u;
  return (uint32_t)(sum >> kCarryWords) & 1u;
}

// Block-level carry functions: each thread's run of 16 words is (G, P)
// (carry out with no carry in; carry out only with one).  Lane runs combine
// like the bits of a binary addition a + b + c with a = G|P, b = G: the carry
// into bit l is bit l of (a + b + c) ^ a ^ b.
__device__ __forceinline__ void run_gp(uint32_t g, uint32_t pm, uint32_t &G, uint32_t &Pp) {
  const uint64_t a = (uint64_t)(g | pm);
  const uint32_t c0 = (uint32_t)((a + g) >> kCarryWords) & 1u;
  const uint32_t c1 = (uint32_t)((a + g + 1) >> kCarryWords) & 1u;
  G = c0;
  Pp = c1 & ~c0 & 1u;
}

// Carry into this thread's run, given the carry into the block; returns the
// block's (G, P) through gb/pb when cin_block is ignored (pass 0 and 1).
template <int NW>
__device__ __forceinline__ uint32_t block_carry_in(uint32_t G, uint32_t Pp, uint32_t cin_block, uint32_t *gb,
                                                   uint32_t *pb) {
  __shared__ uint32_t wg[NW], wp[NW];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t gm = __ballot_sync(0xffffffffu, G), pmk = __ballot_sync(0xffffffffu, Pp);
  const uint64_t a = (uint64_t)(gm | pmk);
  const uint32_t wg0 = (uint32_t)((a + gm) >> 32), wc1 = (uint32_t)((a + gm + 1) >> 32);
  if (lane == 0) {
    wg[warp] = wg0;
    wp[warp] = wc1 & ~wg0 & 1u;
  }
  __syncthreads();
  uint32_t bgm = 0, bpm = 0;
  for (uint32_t x = 0; x < (uint32_t)NW; ++x) {
    bgm |= wg[x] << x;
    bpm |= wp[x] << x;
  }
  const uint64_t ab = (uint64_t)(bgm | bpm);
  if (gb) {
    const uint32_t nw = NW;
    const uint32_t g0 = (uint32_t)((ab + bgm) >> nw) & 1u, g1 = (uint32_t)((ab + bgm + 1) >> nw) & 1u;
    *gb = g0;
    *pb = g1 & ~g0 & 1u;
  }
  const uint64_t bsum = ab + bgm + cin_block;
  const uint32_t warp_in = (uint32_t)((bsum ^ ab ^ bgm) >> warp) & 1u;
  const uint64_t wsum = a + gm + warp_in;
  return (uint32_t)((wsum ^ a ^ gm) >> lane) & 1u;
}

// ------------------------------------------------------------------ schoolbook products

// Products of nc = na + nb <= kSchoolMax words: tpp threads per product, ppb
// products per CTA of 128 threads.  Columns c = sum_j a_j b_(c-j) as 96-bit
// sums (round robin over the product's threads), then the columns' three
// words and the addend are added with their carries and words [lo, hi)
// stored: by one thread per product for products of up to 128 words, else
// by all 128 threads, each over a run of words, with carry-lookahead across
// the runs as in the transform path.
__global__ void __launch_bounds__(128) school_kernel(Opnd A, Opnd B, Opnd D, Out O, uint64_t cnt, uint32_t tpp,
                                                     uint32_t ppb) {
  extern __shared__ uint32_t sm[];
  const uint32_t na = A.words, nb = B.words, nc = na + nb;
  const uint32_t slot = threadIdx.x / tpp, lt = threadIdx.x % tpp;
  const uint64_t i = (uint64_t)blockIdx.x * ppb + slot;
  const bool live = i < cnt;
  uint32_t *sa = sm + (size_t)slot * (4 * nc);
  uint32_t *sb = sa + na;
  uint32_t *clo = sb + nb, *cmid = clo + nc, *chi = cmid + nc;
  if (live) {
    for (uint32_t j = lt; j < na; j += tpp) sa[j] = opnd_word(A, i, j);
    for (uint32_t j = lt; j < nb; j += tpp) sb[j] = opnd_word(B, i, j);
  }
  __syncthreads();
  if (live) {
    for (uint32_t c = lt; c < nc; c += tpp) {
      const uint32_t j0 = c + 1 > nb ? c + 1 - nb : 0u;
      const uint32_t j1 = c < na ? c : na - 1;
      uint64_t s0 = 0;
      uint32_t s1 = 0;
      for (uint32_t j = j0; j <= j1 && j0 <= j1; ++j) {
        const uint64_t pr = (uint64_t)sa[j] * sb[c - j];
        s0 += pr;
        s1 += s0 < pr ? 1u : 0u;
      }
      clo[c] = (uint32_t)s0;
      cmid[c] = (uint32_t)(s0 >> 32);
      chi[c] = s1;
    }
  }
  __syncthreads();
  // word sum s_c = lo_c + mid_(c-1) + hi_(c-2) + d_c (below 2^34)
  auto wsum = [&](uint32_t c) -> uint64_t {
    uint64_t v = opnd_word(D, i, c);
    if (c < nc) v += clo[c];
    if (c >= 1 && c - 1 < nc) v += cmid[c - 1];
    if (c >= 2 && c - 2 < nc) v += chi[c - 2];
    return v;
  };
  uint32_t *dst = O.p + i * O.stride;
  if (ppb == 1) {
    // one product per CTA: 128 runs of r <= 32 words, carry-lookahead across them
    const uint32_t r = (O.hi + 127) / 128, c0 = threadIdx.x * r;
    const uint32_t c1 = min(c0 + r, O.hi);
    uint32_t prev = c0 >= 1 && c0 - 1 < O.hi ? (uint32_t)(wsum(c0 - 1) >> 32) : 0u;
    uint32_t g = 0, pm = 0;
    for (uint32_t c = c0; c < c1; ++c) {
      const uint64_t sv = wsum(c);
      const uint64_t v = (uint64_t)(uint32_t)sv + prev;
      prev = (uint32_t)(sv >> 32);
      g |= (uint32_t)(v >> 32) << (c - c0);
      pm |= (v == 0xffffffffull ? 1u : 0u) << (c - c0);
    }
    const uint64_t a = (uint64_t)(g | pm);
    const uint32_t G = (uint32_t)((a + g) >> r) & 1u;
    const uint32_t Pp = (uint32_t)((a + g + 1) >> r) & 1u & ~G;
    const uint32_t cin = block_carry_in<4>(G, Pp, 0u, nullptr, nullptr);
    const uint32_t into = (uint32_t)((a + g + cin) ^ a ^ g);
    prev = c0 >= 1 && c0 - 1 < O.hi ? (uint32_t)(wsum(c0 - 1) >> 32) : 0u;
    for (uint32_t c = c0; c < c1; ++c) {
      const uint64_t sv = wsum(c);
      const uint32_t wv = (uint32_t)sv + prev + ((into >> (c - c0)) & 1u);
      prev = (uint32_t)(sv >> 32);
      if (c >= O.lo) dst[c - O.lo] = wv;
    }
    return;
  }
  if (!live || lt != 0) return;
  uint64_t carry = 0;
  for (uint32_t c = 0; c < O.hi; ++c) {
    const uint64_t v = carry + wsum(c);
    if (c >= O.lo) dst[c - O.lo] = (uint32_t)v;
    carry = v >> 32;
  }
}

// Pass 1: each thread stores its words before the carries between words
// (words [lo, hi) of the result) and its generate / propagate masks
// (masks[blockIdx.x * kCarryThreads + thread], g | p << 16); each block's carry
// function goes to flags[i * nb + b] (bit 0 generate, bit 1 propagate).  One
// CTA per (product i, block b), i = blockIdx.x / nb.
__global__ void __launch_bounds__(kCarryThreads) carry_words_kernel(WordSrc S, Out O, uint32_t nb, uint8_t *flags,
                                                                    uint32_t *masks) {
  const uint64_t i = blockIdx.x / nb;
  const uint32_t b = (uint32_t)(blockIdx.x % nb);
  const uint32_t c0 = b * kCarryBlock + threadIdx.x * kCarryWords;
  uint32_t w[kCarryWords], g = 0, pm = 0;
  if (c0 < O.hi) {
    thread_words(S, i, c0, w, g, pm);
    uint32_t *dst = O.p + i * O.stride;
#pragma unroll
    for (int m = 0; m < (int)kCarryWords; ++m) {
      const uint32_t c = c0 + (uint32_t)m;
      if (c >= O.lo && c < O.hi) dst[c - O.lo] = w[m];
    }
  }
  masks[(uint64_t)blockIdx.x * kCarryThreads + threadIdx.x] = g | (pm << 16);
  uint32_t G, Pp, gb = 0, pb = 0;
  run_gp(g, pm, G, Pp);
  (void)block_carry_in<kCarryThreads / 32>(G, Pp, 0u, &gb, &pb);
  if (threadIdx.x == 0) flags[i * nb + b] = (uint8_t)(gb | (pb << 1));
}

// Pass 2: one warp per product scans its blocks' carry functions, 32 at a
// time, and leaves the carry into each block in flags bit 2.
__global__ void carry_scan_kernel(uint8_t *flags, uint32_t nb, uint64_t cnt) {
  const uint64_t i = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (i >= cnt) return;
  const uint32_t lane = threadIdx.x & 31;
  uint8_t *f = flags + i * nb;
  uint32_t cin = 0;
  for (uint32_t base = 0; base < nb; base += 32) {
    const uint32_t b = base + lane;
    const uint32_t v = b < nb ? f[b] : 0u;
    const uint32_t gm = __ballot_sync(0xffffffffu, v & 1u), pmk = __ballot_sync(0xffffffffu, (v >> 1) & 1u);
    const uint64_t a = (uint64_t)(gm | pmk), sum = a + gm + cin;
    const uint32_t into = (uint32_t)((sum ^ a ^ gm) >> lane) & 1u;
    if (b < nb) f[b] = (uint8_t)(v | (into << 2));
    cin = (uint32_t)(sum >> 32) & 1u;
  }
}

// Pass 3: the carry into every word from the masks and the block's carry in;
// the (few) stored words that receive one are incremented.
__global__ void __launch_bounds__(kCarryThreads) carry_fix_kernel(Out O, uint32_t nb, const uint8_t *flags,
                                                                  const uint32_t *masks) {
  const uint64_t i = blockIdx.x / nb;
  const uint32_t b = (uint32_t)(blockIdx.x % nb);
  const uint32_t c0 = b * kCarryBlock + threadIdx.x * kCarryWords;
  const uint32_t mk = masks[(uint64_t)blockIdx.x * kCarryThreads + threadIdx.x];
  const uint32_t g = mk & 0xffffu, pm = mk >> 16;
  uint32_t G, Pp;
  run_gp(g, pm, G, Pp);
  const uint32_t cin_block = (flags[i * nb + b] >> 2) & 1u;
  const uint32_t cin = block_carry_in<kCarryThreads / 32>(G, Pp, cin_block, nullptr, nullptr);
  const uint64_t a = (uint64_t)(g | pm);
  uint32_t into = (uint32_t)((a + g + cin) ^ a ^ g) & 0xffffu;
  uint32_t *dst = O.p + i * O.stride;
  while (into) {
    const uint32_t m = __ffs(into) - 1;
    into &= into - 1;
    const uint32_t c = c0 + m;
    if (c >= O.lo && c < O.hi) dst[c - O.lo] += 1u;
  }
}

// ------------------------------------------------------------------ tree kernels

__device__ __forceinline__ bool valid_row(const uint32_t *row, uint32_t L) {
  uint32_t hi = 0;
  for (uint32_t j = 1; j < L; ++j) hi |= row[j];
  return (row[0] & 1u) && (hi != 0u || row[0] >= 3u);
}

// X_0: row i = n_i when valid, else 1 (also the padding rows i >= count).
__global__ void leaves_kernel(const uint32_t *mods, uint64_t count, uint64_t K, uint32_t L, uint32_t *X0) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (uint64_t)gridDim.x * blockDim.x) {
    const bool ok = i < count && valid_row(mods + i * L, L);
    for (uint32_t j = 0; j < L; ++j) X0[i * L + j] = ok ? mods[i * L + j] : (j == 0 ? 1u : 0u);
  }
}

// First word of mu: -y_0^-1 mod 2^32 (Newton's iteration on one word).
__global__ void mu_word_kernel(const uint32_t *Y, uint64_t ys, uint32_t *mu, uint64_t ms, uint64_t cnt) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t y0 = Y[i * ys];
    uint32_t inv = y0;
    for (int k = 0; k < 5; ++k) inv *= 2u - y0 * inv;
    mu[i * ms] = 0u - inv;
  }
}

// Z_T: the root X_T in a row of zs words, zero above its s words.
__global__ void root_kernel(const uint32_t *X, uint64_t s, uint32_t *Z, uint64_t zs) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < zs; j += (uint64_t)gridDim.x * blockDim.x)
    Z[j] = j < s ? X[j] : 0u;
}

constexpr int kLeafThreads = 64;

// One word of Montgomery reduction on the window t (K + 2 words) by the K-word
// N in shared memory (word j at sN[j * bd]): t = (t + q N) / 2^32, whose low
// word is zero by the choice of q.  Two carry chains, the even words of N and
// then the odd ones, each a run of multiply-adds with carry.
template <int K>
__device__ __forceinline__ void leaf_redc_step(uint32_t (&t)[K + 2], const uint32_t *sN, uint32_t bd, uint32_t q) {
  {
    const uint32_t n = sN[0];
    (void)mad_lo_cc(q, n, t[0]);
    t[0] = madc_hi_cc(q, n, t[1]);
  }
#pragma unroll
  for (int k = 1; k < K / 2; ++k) {
    const uint32_t n = sN[(2 * k) * bd];
    t[2 * k - 1] = madc_lo_cc(q, n, t[2 * k]);
    t[2 * k] = madc_hi_cc(q, n, t[2 * k + 1]);
  }
  t[K - 1] = addc_cc(t[K], 0u);
  t[K] = addc(t[K + 1], 0u);
  {
    const uint32_t n = sN[bd];
    t[0] = mad_lo_cc(q, n, t[0]);
    t[1] = madc_hi_cc(q, n, t[1]);
  }
#pragma unroll
  for (int k = 1; k < K / 2; ++k) {
    const uint32_t n = sN[(2 * k + 1) * bd];
    t[2 * k] = madc_lo_cc(q, n, t[2 * k]);
    t[2 * k + 1] = madc_hi_cc(q, n, t[2 * k + 1]);
  }
  t[K] = addc(t[K], 0u);
  t[K + 1] = 0u;
}

// Per-thread shared-memory words of the leaf kernel: n (L), N = n^2 (2L; the
// reduced value r takes its place once the reduction is done), the quotient u
// (L); column layout (word w of thread x at w * blockDim + x).
__host__ __device__ constexpr uint32_t leaf_words(uint32_t L) { return 4 * L; }

// One modulus per thread: z = Z(node of i at level t0) 2^(-32M) mod n_i^2 by
// word-serial Montgomery reduction (window of 2L + 2 words in registers),
// one conditional subtraction, u = z / n_i exactly (word by word from the
// bottom: d = r_j n_0^-1, r -= d n_i 2^(32j)), then g_i = gcd(n_i, u).
template <int L>
__global__ void __launch_bounds__(kLeafThreads) tree_leaf_kernel(const uint32_t *mods, uint64_t count,
                                                                 const uint32_t *Z, uint64_t zs, uint32_t M,
                                                                 uint32_t t0, uint32_t *gcds, int32_t *flags) {
  extern __shared__ uint32_t sm[];
  const uint32_t bd = blockDim.x, x = threadIdx.x;
  uint32_t *sn = sm + x, *sN = sm + (size_t)L * bd + x, *sr = sN;
  uint32_t *su = sm + (size_t)(3 * L) * bd + x;
  const uint64_t i = (uint64_t)blockIdx.x * bd + x;
  const bool live = i < count;
  const uint64_t row = live ? i : count - 1;
  const uint32_t *nrow = mods + row * L;
  const bool ok = live && valid_row(nrow, L);
  for (uint32_t w = 0; w < L; ++w) sn[w * bd] = ok ? nrow[w] : (w == 0 ? 1u : 0u);
  // N = n^2, rows of the schoolbook product with a running carry
  for (uint32_t w = 0; w < 2 * L; ++w) sN[w * bd] = 0u;
  for (uint32_t j = 0; j < L; ++j) {
    const uint32_t nj = sn[j * bd];
    uint32_t c = 0;
    for (uint32_t m = 0; m < L; ++m) {
      const uint64_t acc = (uint64_t)nj * sn[m * bd] + sN[(j + m) * bd] + c;
      sN[(j + m) * bd] = (uint32_t)acc;
      c = (uint32_t)(acc >> 32);
    }
    sN[(j + L) * bd] = c;
  }
  const uint32_t N0 = sN[0];
  uint32_t np = N0;
  for (int k = 0; k < 5; ++k) np *= 2u - N0 * np;
  np = 0u - np;
  // word-serial reduction of the node's M words
  const uint32_t *z = Z + (row >> t0) * zs;
  uint32_t t[2 * L + 2];
#pragma unroll
  for (int w = 0; w < 2 * L; ++w) t[w] = (uint32_t)w < M ? z[w] : 0u;
  t[2 * L] = 0u;
  t[2 * L + 1] = 0u;
  if constexpr (L <= 32) {
    // two carry chains of multiply-adds (measured faster at 512 and 1024 bits)
#pragma unroll 1
    for (uint32_t s = 0; s < M; ++s) {
      leaf_redc_step<2 * L>(t, sN, bd, t[0] * np);
      const uint32_t nx = 2 * L + s;
      if (nx < M) {
        t[2 * L - 1] = add_cc(t[2 * L - 1], z[nx]);
        t[2 * L] = addc(t[2 * L], 0u);
      }
    }
  } else {
    // 64-bit multiply-accumulate with a running carry: at 2048 bits the
    // ordered carry chains need more registers than the 130-word window leaves
    // (131072 moduli: 151 ms against 158)
#pragma unroll 1
    for (uint32_t s = 0; s < M; ++s) {
      const uint32_t q = t[0] * np;
      uint64_t acc = (uint64_t)q * sN[0] + t[0];
      uint32_t c = (uint32_t)(acc >> 32);
#pragma unroll
      for (int j = 1; j < 2 * L; ++j) {
        acc = (uint64_t)q * sN[j * bd] + t[j] + c;
        t[j - 1] = (uint32_t)acc;
        c = (uint32_t)(acc >> 32);
      }
      acc = (uint64_t)t[2 * L] + c;
      t[2 * L - 1] = (uint32_t)acc;
      t[2 * L] = t[2 * L + 1] + (uint32_t)(acc >> 32);
      t[2 * L + 1] = 0u;
      const uint32_t nx = 2 * L + s;
      if (nx < M) {
        acc = (uint64_t)t[2 * L - 1] + z[nx];
        t[2 * L - 1] = (uint32_t)acc;
        t[2 * L] += (uint32_t)(acc >> 32);
      }
    }
  }
  // t <= N: subtract N once when t >= N
  {
    uint32_t d[2 * L];
    uint32_t br = 0;
#pragma unroll
    for (int w = 0; w < 2 * L; ++w) {
      const uint32_t nw = sN[w * bd];
      const uint64_t sub = (uint64_t)nw + br;
      d[w] = t[w] - (uint32_t)sub;
      br = ((uint64_t)t[w] < sub) ? 1u : 0u;
    }
    const bool ge = t[2 * L] != 0u || br == 0u;
#pragma unroll
    for (int w = 0; w < 2 * L; ++w) sr[w * bd] = ge ? d[w] : t[w];
  }
  // u = r / n exactly
  const uint32_t n0 = sn[0];
  uint32_t inv = n0;
  for (int k = 0; k < 5; ++k) inv *= 2u - n0 * inv;
  for (uint32_t j = 0; j < L; ++j) {
    const uint32_t dj = sr[j * bd] * inv;
    su[j * bd] = dj;
    uint32_t br = 0;
    for (uint32_t m = 0; m < L; ++m) {
      const uint64_t pr = (uint64_t)dj * sn[m * bd] + br;
      const uint32_t r = sr[(j + m) * bd], lo = (uint32_t)pr;
      sr[(j + m) * bd] = r - lo;
      br = (uint32_t)(pr >> 32) + (r < lo ? 1u : 0u);
    }
    for (uint32_t m = j + L; m < 2 * L && br; ++m) {
      const uint32_t r = sr[m * bd];
      sr[m * bd] = r - br;
      br = r < br ? 1u : 0u;
    }
  }
  uint32_t a[L], b[L];
#pragma unroll
  for (int w = 0; w < L; ++w) {
    a[w] = sn[w * bd];
    b[w] = ok ? su[w * bd] : 0u;
  }
  binary_gcd<L>(a, b);
  if (!live) return;
  uint32_t hi = 0, diff = 0;
#pragma unroll
  for (int w = 0; w < L; ++w) {
    diff |= a[w] ^ nrow[w];
    if (w) hi |= a[w];
  }
  if (gcds) {
    uint32_t *dst = gcds + i * L;
#pragma unroll
    for (int w = 0; w < L; ++w) dst[w] = ok ? a[w] : 0u;
  }
  if (flags) flags[i] = !ok ? -1 : (hi == 0u && a[0] == 1u) ? 0 : (diff == 0u ? 2 : 1);
}

}  // namespace tree
}  // namespace rsagpu

// ------------------------------------------------------------------ host side

namespace rsagpu {
namespace tree {
namespace {

uint32_t powmod(uint64_t b, uint64_t e, uint32_t p) {
  uint64_t r = 1;
  b %= p;
  while (e) {
    if (e & 1) r = r * b % p;
    b = b * b % p;
    e >>= 1;
  }
  return (uint32_t)r;
}

uint32_t to_mont(uint32_t x, uint32_t p) { return (uint32_t)(((uint64_t)x << 32) % p); }

// Smallest generator of the multiplicative group mod p: g^((p-1)/f) != 1 for
// every prime factor f of p - 1 (found by trial division).
uint32_t generator(uint32_t p) {
  std::vector<uint32_t> fs;
  uint32_t m = p - 1;
  for (uint32_t f = 2; (uint64_t)f * f <= m; ++f) {
    if (m % f) continue;
    fs.push_back(f);
    while (m % f == 0) m /= f;
  }
  if (m > 1) fs.push_back(m);
  for (uint32_t g = 2;; ++g) {
    bool ok = true;
    for (uint32_t f : fs) ok = ok && powmod(g, (p - 1) / f, p) != 1;
    if (ok) return g;
  }
}

uint32_t inv32(uint32_t p) {
  uint32_t inv = p;
  for (int k = 0; k < 5; ++k) inv *= 2u - p * inv;
  return inv;
}

int ilog2(uint64_t n) {
  int l = 0;
  while ((1ull << (l + 1)) <= n) ++l;
  return l;
}

uint64_t pow2_at_least(uint64_t n) {
  uint64_t v = 1;
  while (v < n) v <<= 1;
  return v;
}

// Device buffers of one scan, as word offsets into one arena.
struct Plan {
  uint32_t L = 0, T = 0, t0 = 0;
  uint64_t K = 0, KL = 0;
  uint64_t nmax = 0;                         // longest transform
  std::vector<uint64_t> x_off;               // product tree levels
  uint64_t y_off = 0, mu_off[2] = {0, 0};    // remainder-tree level buffers
  uint64_t z_off[2] = {0, 0}, q_off = 0, h_off = 0, fa_off = 0, fb_off = 0, flags_off = 0;
  uint64_t fwords = 0;                       // per-prime capacity of the transform buffers
  uint64_t cy_off = 0, cp_off = 0;           // cached transforms of one remainder level
  uint64_t carry_blocks = 0, masks_off = 0;  // carry scan: blocks of one product batch, their masks
  uint64_t words = 0;                        // arena size in words
};

Plan make_plan(uint32_t L, uint64_t count, uint32_t t0_req) {
  Plan P;
  P.L = L;
  P.K = pow2_at_least(std::max<uint64_t>(count, 2));
  P.T = (uint32_t)ilog2(P.K);
  P.t0 = std::min(t0_req, P.T);
  P.KL = P.K * L;
  const uint64_t KL = P.KL;
  uint64_t at = 0;
  P.x_off.resize(P.T + 1);
  for (uint32_t t = 0; t <= P.T; ++t) {
    P.x_off[t] = at;
    at += KL;
  }
  // one level of the remainder tree at a time: its squares, its mu and its
  // parent's mu (both levels hold 2 KL words)
  P.y_off = at;
  at += 2 * KL;
  P.mu_off[0] = at;
  at += 2 * KL;
  P.mu_off[1] = at;
  at += 2 * KL;
  const uint64_t zwords = 2 * KL + 4 * (P.K >> P.t0) + 4;
  P.z_off[0] = at;
  at += zwords;
  P.z_off[1] = at;
  at += zwords;
  P.q_off = at;
  at += 2 * KL;
  P.h_off = at;
  at += KL;
  P.fwords = std::max<uint64_t>(4 * KL, kTile);
  P.fa_off = at;
  at += 3 * P.fwords;
  P.fb_off = at;
  at += 3 * P.fwords;
  // transforms one remainder level shares between its products: the squares
  // (one per node) and a parent-level operand (one per two nodes)
  P.cy_off = at;
  at += 3 * P.fwords;
  P.cp_off = at;
  at += 3 * (P.fwords / 2);
  // carry blocks of one transform product: cnt * ceil(hi / kCarryBlock) <=
  // cnt (n + 1) / kCarryBlock + cnt with cnt n <= fwords and n >= 1024
  P.carry_blocks = P.fwords / kCarryBlock + 2 * (P.fwords / 1024) + 2;
  P.flags_off = at;
  at += P.carry_blocks / 4 + 1;
  at = (at + 3) / 4 * 4;
  P.masks_off = at;
  at += P.carry_blocks * kCarryThreads;
  P.words = (at + 3) / 4 * 4;
  // longest transform: the remainder step and the Newton step of level T - 1 (4 s_(T-1) words)
  P.nmax = std::max<uint64_t>(2 * KL, kTile);
  return P;
}

struct Runner {
  Ctx *c;
  cudaStream_t s;
  uint32_t *base;
  const Plan &P;
  Primes pr;                                 // tables and Garner constants; scale set per product
  int launches = 0;

  uint32_t *at(uint64_t off) const { return base + off; }

  int grid_for(uint64_t work, int threads) const {
    const uint64_t want = (work + threads - 1) / threads;
    const uint64_t cap = (uint64_t)c->sm_count * 8;
    return (int)std::max<uint64_t>(1, std::min(want, cap));
  }

  // scale of the recombination for transforms of length n
  void set_scale(uint64_t n) {
    for (int k = 0; k < 3; ++k) {
      const uint32_t p = kPrime[k];
      const uint32_t ninv = p - (uint32_t)((p - 1) / n);
      const uint32_t r2 = powmod(to_mont(1, p), 2, p);
      pr.scale[k] = (uint32_t)((uint64_t)ninv * r2 % p);
    }
  }

  // global passes of up to four stages over Es words per prime: forward from
  // the top (the last pass takes the remainder), inverse from the bottom
  void pass(bool inverse, int S, uint32_t *F, uint64_t Es, uint32_t logh) {
    const dim3 grid(grid_for(Es >> S, 256), 3);
    if (inverse) {
      if (S == 1) ditr_kernel<1><<<grid, 256, 0, s>>>(F, Es, logh, pr);
      else if (S == 2) ditr_kernel<2><<<grid, 256, 0, s>>>(F, Es, logh, pr);
      else if (S == 3) ditr_kernel<3><<<grid, 256, 0, s>>>(F, Es, logh, pr);
      else ditr_kernel<4><<<grid, 256, 0, s>>>(F, Es, logh, pr);
    } else {
      if (S == 1) difr_kernel<1><<<grid, 256, 0, s>>>(F, Es, logh, pr);
      else if (S == 2) difr_kernel<2><<<grid, 256, 0, s>>>(F, Es, logh, pr);
      else if (S == 3) difr_kernel<3><<<grid, 256, 0, s>>>(F, Es, logh, pr);
      else difr_kernel<4><<<grid, 256, 0, s>>>(F, Es, logh, pr);
    }
    ++launches;
  }
  void global_forward(uint32_t *F, uint64_t Es, uint32_t logn) {
    int g = std::max((int)logn - (int)ilog2(kTile), 0);
    int logl = (int)logn - 1;                     // the next stage's half-length
    while (g > 0) {
      const int S = std::min(g, 4);
      pass(false, S, F, Es, (uint32_t)(logl - S + 1));
      logl -= S;
      g -= S;
    }
  }
  void global_inverse(uint32_t *F, uint64_t Es, uint32_t logn) {
    int g = std::max((int)logn - (int)ilog2(kTile), 0);
    int logl = (int)ilog2(kTile);
    const int first = g % 4;
    if (first) {
      pass(true, first, F, Es, (uint32_t)logl);
      logl += first;
      g -= first;
    }
    while (g > 0) {
      pass(true, 4, F, Es, (uint32_t)logl);
      logl += 4;
      g -= 4;
    }
  }

  // carry passes over the recombined columns of cnt products in F (per-prime
  // stride Es, transforms of 2^logn words): words [O.lo, O.hi) of each, plus D
  int carry(const uint32_t *F, uint64_t Es, uint32_t logn, uint64_t cnt, const Opnd &D, const Out &O) {
    set_scale(1ull << logn);
    WordSrc S{F, Es, logn, pr, D};
    const uint32_t nbk = (O.hi + kCarryBlock - 1) / kCarryBlock;
    uint8_t *flags = reinterpret_cast<uint8_t *>(at(P.flags_off));
    uint32_t *masks = at(P.masks_off);
    const uint64_t blocks = cnt * nbk;
    if (blocks > P.carry_blocks) return set_error(RSA_ERR_ARG, "batch gcd tree: carry scratch exceeded");
    carry_words_kernel<<<(unsigned)blocks, kCarryThreads, 0, s>>>(S, O, nbk, flags, masks);
    carry_scan_kernel<<<(unsigned)((cnt + 3) / 4), 128, 0, s>>>(flags, nbk, cnt);
    carry_fix_kernel<<<(unsigned)blocks, kCarryThreads, 0, s>>>(O, nbk, flags, masks);
    launches += 3;
    return 0;
  }

  // forward transforms (length 2^logn >= kTile) of cnt operands into F (per-prime
  // stride cnt 2^logn, at most cap words)
  int fwd(const Opnd &X, uint64_t cnt, uint32_t logn, uint32_t *F, uint64_t cap) {
    const uint64_t E = cnt << logn;
    if (logn < (uint32_t)ilog2(kTile) || 3 * E > cap)
      return set_error(RSA_ERR_ARG, "batch gcd tree: cached transform out of range");
    ntt_load_kernel<<<grid_for(E, 256), 256, 0, s>>>(X, F, E, E, logn);
    ++launches;
    global_forward(F, E, logn);
    ntt_tile_fwd_kernel<<<dim3((unsigned)(E / kTile), 3), kTileThreads, 0, s>>>(F, E, 0, pr);
    ++launches;
    return 0;
  }

  // FO = inverse transform of the pointwise products of A's transforms
  // (i >> sha) ^ xra (batch stride as) and B's transforms i >> shb (stride
  // bs), i < cnt; FO's per-prime stride is cnt 2^logn
  void mulinv(uint32_t *FO, const uint32_t *FA, uint64_t as, uint32_t sha, uint32_t xra, const uint32_t *FB,
              uint64_t bs, uint32_t shb, uint64_t cnt, uint32_t logn) {
    const uint64_t E = cnt << logn;
    ntt_tile_pinv_kernel<<<dim3((unsigned)(E / kTile), 3), kTileThreads, 0, s>>>(FO, E, FA, as, sha, xra, FB, bs,
                                                                                 shb, logn, pr);
    ++launches;
    global_inverse(FO, E, logn);
  }

  // out = words [O.lo, O.hi) of A_i * B_i + D_i for i < cnt (B ignored when square)
  int mul(const Opnd &A, const Opnd &B, const Opnd &D, const Out &O, uint64_t cnt, bool square) {
    if (cnt == 0) return 0;
    const uint32_t na = A.words, nb = square ? A.words : B.words, nc = na + nb;
    if (nc <= kSchoolMax) {
      uint32_t tpp = 1;
      while (tpp < 128 && 2 * tpp < nc) tpp *= 2;
      const uint32_t ppb = 128 / tpp;
      const size_t smem = (size_t)ppb * 4 * nc * 4;
      const uint64_t grid = (cnt + ppb - 1) / ppb;
      school_kernel<<<(unsigned)grid, 128, smem, s>>>(A, square ? A : B, D, O, cnt, tpp, ppb);
      ++launches;
      return 0;
    }
    const uint64_t n = pow2_at_least(nc);
    const uint32_t logn = (uint32_t)ilog2(n);
    if (logn > kMaxLog) return set_error(RSA_ERR_ARG, "batch gcd tree: product above 2^27 words");
    const uint64_t E = cnt * n;                              // words per prime
    const uint64_t Es = (E + kTile - 1) / kTile * kTile;     // per-prime stride: whole tiles
    if (Es > P.fwords) return set_error(RSA_ERR_ARG, "batch gcd tree: transform scratch exceeded");
    uint32_t *FA = at(P.fa_off), *FB = at(P.fb_off);
    const uint32_t skip = (uint32_t)std::max((int)ilog2(kTile) - (int)logn, 0);   // tiles of 2^skip transforms
    if (skip > 2) return set_error(RSA_ERR_ARG, "batch gcd tree: transform below 1024 words");
    const dim3 tiles((unsigned)(Es / kTile), 3);
    if (!square) {
      ntt_load_kernel<<<grid_for(E, 256), 256, 0, s>>>(B, FB, E, Es, logn);
      global_forward(FB, Es, logn);
      ntt_tile_fwd_kernel<<<tiles, kTileThreads, 0, s>>>(FB, Es, skip, pr);
      launches += 2;
    }
    ntt_load_kernel<<<grid_for(E, 256), 256, 0, s>>>(A, FA, E, Es, logn);
    global_forward(FA, Es, logn);
    ntt_tile_mul_kernel<<<tiles, kTileThreads, 0, s>>>(FA, square ? nullptr : FB, Es, skip, pr);
    launches += 2;
    global_inverse(FA, Es, logn);
    return carry(FA, Es, logn, cnt, D, O);
  }
};

Opnd opnd(const uint32_t *p, uint64_t stride, uint32_t words, uint32_t shift = 0, uint32_t xr = 0) {
  return Opnd{p, stride, shift, words, xr};
}

const Opnd kNone{nullptr, 0, 0, 0, 0};

}  // namespace
}  // namespace tree
}  // namespace rsagpu

namespace rsagpu {

// Lowest level of the remainder tree: its nodes hold 2^t0 moduli and the leaf
// kernel reduces a node's value modulo each n_i^2 word by word.  Nodes of
// about 1024 words measured best on GB300 (131072 2048-bit moduli: t0 = 2
// 215 ms, 3 209, 4 205, 5 207, 6 219; 1024- and 512-bit moduli: t0 = 5), so
// t0 = log2(1024 / L).
static uint32_t tree_leaf_level(uint32_t L) {
  const char *v = std::getenv("RSAGPU_GCD_TREE_T0");
  const int def = L >= 64 ? 4 : L >= 32 ? 5 : 6;
  const int t = v ? std::atoi(v) : def;
  return (uint32_t)std::min(std::max(t, 0), 6);
}

uint64_t batch_gcd_tree_bytes(uint32_t L, uint64_t count) {
  const tree::Plan P = tree::make_plan(L, count, tree_leaf_level(L));
  return P.words * 4 + 6 * P.nmax * 4;
}

int batch_gcd_tree_run(Ctx *c, uint32_t nbits, uint64_t count, const uint32_t *moduli, uint32_t *gcds,
                       int32_t *flags, cudaStream_t s) {
  using namespace tree;
  const uint32_t L = nbits / 32;
  const Plan P = make_plan(L, count, tree_leaf_level(L));
  if (P.nmax > (1ull << kMaxLog)) return set_error(RSA_ERR_ARG, "batch gcd tree: count * modulus words above 2^26");
  Workspace &w = c->ws(s);
  int rc;
  if ((rc = c->ensure(w.gcd_tree, P.words * 4)) || (rc = c->ensure(w.gcd_tw, 6 * P.nmax * 4))) return rc;
  NvtxRange range("rsa_batch_gcd(tree)");
  Runner R{c, s, static_cast<uint32_t *>(w.gcd_tree.ptr), P, {}, 0};
  uint32_t *tw = static_cast<uint32_t *>(w.gcd_tw.ptr);
  const bool rebuild = w.gcd_tw_ptr != w.gcd_tw.ptr || w.gcd_tw_n < P.nmax;
  const uint64_t tn = rebuild ? P.nmax : w.gcd_tw_n;      // table stride: the length built
  for (int k = 0; k < 3; ++k) {
    const uint32_t p = kPrime[k];
    R.pr.p[k] = p;
    R.pr.pinv[k] = inv32(p);
    R.pr.tw[k] = tw + (2 * k) * tn;
    R.pr.itw[k] = tw + (2 * k + 1) * tn;
    if (rebuild) {
      const uint32_t root = powmod(generator(p), (p - 1) / P.nmax, p);
      const uint32_t iroot = powmod(root, p - 2, p);
      twiddle_kernel<<<R.grid_for(P.nmax, 256), 256, 0, s>>>(tw + (2 * k) * tn, tw + (2 * k + 1) * tn,
                                                             (uint32_t)P.nmax, p, R.pr.pinv[k], to_mont(root, p),
                                                             to_mont(iroot, p), to_mont(1, p));
      ++R.launches;
    }
  }
  if (rebuild) {
    w.gcd_tw_ptr = w.gcd_tw.ptr;
    w.gcd_tw_n = P.nmax;
  }
  {
    const uint32_t p1 = kPrime[0], p2 = kPrime[1], p3 = kPrime[2];
    R.pr.inv12 = to_mont(powmod(p1, p2 - 2, p2), p2);
    R.pr.p1m3 = to_mont(p1 % p3, p3);
    R.pr.inv123 = to_mont(powmod((uint64_t)(p1 % p3) * (p2 % p3) % p3, p3 - 2, p3), p3);
  }
  const uint64_t K = P.K;
  const uint32_t T = P.T, t0 = P.t0;
  auto X = [&](uint32_t t) { return R.at(P.x_off[t]); };
  auto sz = [&](uint32_t t) { return (uint64_t)L << t; };
  leaves_kernel<<<R.grid_for(K, 256), 256, 0, s>>>(moduli, count, K, L, X(0));
  ++R.launches;
  // product tree
  for (uint32_t t = 0; t < T; ++t) {
    const uint64_t st = sz(t);
    if ((rc = R.mul(opnd(X(t), 2 * st, (uint32_t)st), opnd(X(t) + st, 2 * st, (uint32_t)st), kNone,
                    Out{X(t + 1), 2 * st, 0, (uint32_t)(2 * st)}, K >> (t + 1), false)))
      return rc;
  }
  // remainder tree, one level at a time from the top: Y = X_t^2; mu = -Y^-1
  // mod 2^(32k) by Newton from one word at the top level, below it from the
  // parent (mu_a = Y_b mu_parent mod 2^(32k)); then q and the quotient step
  uint32_t *H = R.at(P.h_off), *q = R.at(P.q_off), *Y = R.at(P.y_off);
  int cur = 0, mcur = 0;
  {
    const uint64_t zs = 2 * sz(T) + 4;
    root_kernel<<<R.grid_for(zs, 256), 256, 0, s>>>(X(T), sz(T), R.at(P.z_off[cur]), zs);
    ++R.launches;
  }
  for (uint32_t t = T; t-- > t0;) {
    const uint64_t st = sz(t), k = 2 * st, cnt = K >> t, zsp = 2 * sz(t + 1) + 4, zs = 2 * st + 4;
    const uint32_t k32 = (uint32_t)k;
    uint32_t *Zp = R.at(P.z_off[cur]), *Zc = R.at(P.z_off[cur ^ 1]);
    uint32_t *mu = R.at(P.mu_off[mcur]), *mup = R.at(P.mu_off[mcur ^ 1]);
    if (t + 1 < T && 2 * k >= kTile) {
      // transforms shared within the level: Y^ serves the sibling's inverse and
      // the quotient step, the parent's mu^ and Z^ serve both children.  Y is
      // carried into words first: the pointwise square of X^ would hold the
      // uncarried coefficients of X*X (up to s 2^64), and a product of those
      // with k words would pass the three primes' range
      const uint32_t logn = (uint32_t)ilog2(2 * k);
      const uint64_t E = cnt << logn, Ep = (cnt / 2) << logn;
      const uint64_t cap = 3 * P.fwords, capp = 3 * (P.fwords / 2);
      uint32_t *CY = R.at(P.cy_off), *CP = R.at(P.cp_off), *FA = R.at(P.fa_off), *FO = R.at(P.fb_off);
      if ((rc = R.mul(opnd(X(t), st, (uint32_t)st), kNone, kNone, Out{Y, k, 0, k32}, cnt, true)) ||
          (rc = R.fwd(opnd(Y, k, k32), cnt, logn, CY, cap)) ||
          (rc = R.fwd(opnd(mup, 2 * k, k32), cnt / 2, logn, CP, capp)))
        return rc;
      R.mulinv(FO, CY, E, 0, 1, CP, Ep, 1, cnt, logn);                 // Y_sibling * mu_parent
      if ((rc = R.carry(FO, E, logn, cnt, kNone, Out{mu, k, 0, k32})) ||
          (rc = R.fwd(opnd(mu, k, k32), cnt, logn, FA, cap)) ||
          (rc = R.fwd(opnd(Zp, zsp, k32), cnt / 2, logn, CP, capp)))
        return rc;
      R.mulinv(FO, FA, E, 0, 0, CP, Ep, 1, cnt, logn);                 // mu * Z_parent
      if ((rc = R.carry(FO, E, logn, cnt, kNone, Out{q, k, 0, k32})) ||
          (rc = R.fwd(opnd(q, k, k32), cnt, logn, FA, cap)))
        return rc;
      R.mulinv(FO, FA, E, 0, 0, CY, E, 0, cnt, logn);                  // q * Y
      if ((rc = R.carry(FO, E, logn, cnt, opnd(Zp, zsp, 2 * k32 + 1, 1), Out{Zc, zs, k32, 2 * k32 + 1})))
        return rc;
      cur ^= 1;
      mcur ^= 1;
      continue;
    }
    if ((rc = R.mul(opnd(X(t), st, (uint32_t)st), kNone, kNone, Out{Y, k, 0, k32}, cnt, true))) return rc;
    if (t == T - 1) {
      mu_word_kernel<<<R.grid_for(cnt, 256), 256, 0, s>>>(Y, k, mu, k, cnt);
      ++R.launches;
      for (uint64_t wd = 1; wd < k; wd *= 2) {
        const uint32_t w32 = (uint32_t)wd;
        if ((rc = R.mul(opnd(Y, k, 2 * w32), opnd(mu, k, w32), kNone, Out{H, wd, w32, 2 * w32}, cnt, false)) ||
            (rc = R.mul(opnd(H, wd, w32), opnd(mu, k, w32), opnd(mu, k, w32), Out{mu + wd, k, 0, w32}, cnt,
                        false)))
          return rc;
      }
    } else if ((rc = R.mul(opnd(Y, k, k32, 0, 1), opnd(mup, 2 * k, k32, 1), kNone, Out{mu, k, 0, k32}, cnt,
                           false))) {
      return rc;
    }
    if ((rc = R.mul(opnd(Zp, zsp, k32, 1), opnd(mu, k, k32), kNone, Out{q, k, 0, k32}, cnt, false)) ||
        (rc = R.mul(opnd(q, k, k32), opnd(Y, k, k32), opnd(Zp, zsp, 2 * k32 + 1, 1), Out{Zc, zs, k32, 2 * k32 + 1},
                    cnt, false)))
      return rc;
    cur ^= 1;
    mcur ^= 1;
  }
  // leaves
  {
    const uint64_t zs = 2 * sz(t0) + 4;
    const uint32_t M = (uint32_t)(2 * sz(t0) + 1);
    const size_t smem = (size_t)leaf_words(L) * kLeafThreads * 4;
    const unsigned grid = (unsigned)((count + kLeafThreads - 1) / kLeafThreads);
    const uint32_t *Z = R.at(P.z_off[cur]);
    cudaError_t e;
    if (L == 16) {
      e = cudaFuncSetAttribute(tree_leaf_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) tree_leaf_kernel<16><<<grid, kLeafThreads, smem, s>>>(moduli, count, Z, zs, M, t0, gcds, flags);
    } else if (L == 32) {
      e = cudaFuncSetAttribute(tree_leaf_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) tree_leaf_kernel<32><<<grid, kLeafThreads, smem, s>>>(moduli, count, Z, zs, M, t0, gcds, flags);
    } else {
      e = cudaFuncSetAttribute(tree_leaf_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) tree_leaf_kernel<64><<<grid, kLeafThreads, smem, s>>>(moduli, count, Z, zs, M, t0, gcds, flags);
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(tree_leaf)");
    ++R.launches;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "launch batch gcd tree kernels");
  c->stats.kernel_launches += (uint64_t)R.launches;
  c->stats.ops += count;
  return RSA_OK;
}

}  // namespace rsagpu
