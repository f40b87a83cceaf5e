// crt_tc4.cu -- RSA-4096 CRT decryption with the Montgomery reduction on the
// 5th-generation tensor cores (tcgen05, TMEM), for 2048-bit primes.
//
// The route is the one of crt_tc.cu (RSA-2048): M = C^d mod n as
// m_p = C^dp mod p and m_q = C^dq mod q, each a constant-time fixed-window
// exponentiation (Fig. 6 with k = W) of Montgomery products, then Garner.  A
// Montgomery product modulo a 2048-bit prime m, R = 2^2048, is done as two
// reduction rounds of r = 2^1024 (the same value: with mu = mu1 + r mu2 < R,
// (T + mu1 m + r mu2 m) / r^2 = (T + mu m) / R):
//   1. CUDA cores: T = A * B, 64 x 64 limbs, product scanning with PTX carry
//      chains (one thread per operation).  Limbs 0..31 of T leave as byte
//      digits (fp16) in the tile's A buffer, limbs 32..63 as words in the
//      tile's high stage, limbs 64..127 stay in registers.
//   2. per round: tensor core, MMA 1: the column sums of the byte convolution
//      of (T mod r) with m' = -m^-1 mod r (128 columns); CUDA cores: carry them
//      into the bytes of mu = (T mod r) m' mod r, written back as digits;
//      tensor core, MMA 2: the column sums of mu * m for positions 124..379
//      (N = 256), positions 380..382 on the CUDA cores; CUDA cores: the carry
//      out of the low 1024 bits (ceil of positions 124..127 with T's limb 31,
//      over 2^32) and T = (T + mu m) / r, the high positions carry-propagated
//      into the limbs of T above r.  After round 1 the new low 1024 bits leave
//      as digits for round 2.
//   3. one conditional subtraction of m.
// Every column of both MMAs sums at most 128 products of two bytes (K = 128
// digits of T mod r or of mu), so each sum is an integer below 2^23 and reads
// back exactly through the bias of crt_tc.cu (0x3F000000 + w).
//
// Work layout: one CTA per SM (256 threads), all of one prime, two tiles of
// 128 operations with their own A buffer, high stage, 256 TMEM columns,
// mbarrier and named barrier; thread r of a tile owns operation r and TMEM
// lane r.  One thread per operation keeps 64-limb numbers in registers (up to
// 255 registers a thread at 256 threads per CTA).
#include <cuda_runtime.h>

#include <cstdint>

#include "crt_tc.h"
#include "kernels.cuh"
#include "keyrec.h"
#include "mont.cuh"
#include "tc.cuh"

namespace rsagpu {
namespace tc4 {

// ---------------------------------------------------------------- shared memory map (bytes)
constexpr int kKb = (kRows / 8) * 128;               // k-block stride of 128-row operands (A, B1)
constexpr int kKb2 = (kN2 / 8) * 128;                // k-block stride of B2 (256 rows)
constexpr int kOffB1 = 0;
constexpr int kOffB2 = kOffB1 + (int)kImgB1;
constexpr int kOffAbias = kOffB2 + (int)kImgB2;      // 128 x 16 bias A operand
constexpr int kOffA = kOffAbias + kRows * 16 * 2;    // kTiles A buffers of 128 x 128 digits
constexpr int kABytes = kRows * kDig * 2;
constexpr int kOffHi = kOffA + kTiles * kABytes;     // kTiles high stages: [g][row] uint4, g < 8
constexpr int kHiBytes = kRows * 128;
constexpr int kOffKey = kOffHi + kTiles * kHiBytes;
// key constants (words): m, R^2, R^3, R mod m, unit, exponent (kH + 4 limbs)
constexpr int kKm = 0, kKr2 = kH, kKr3 = 2 * kH, kKone = 3 * kH, kKunit = 4 * kH, kKexp = 5 * kH;
constexpr int kKeyWords = 6 * kH + 4;
constexpr int kOffCtrl = kOffKey + kKeyWords * 4;    // kTiles mbarriers (8 B each), TMEM base at +48
constexpr int kSmem = kOffCtrl + 64;
static_assert(kOffA % 128 == 0 && kOffHi % 16 == 0 && kOffKey % 16 == 0 && kOffCtrl % 8 == 0, "layout");
static_assert(kSmem <= 227 * 1024, "shared memory");

constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kTileCols = 256;
static_assert(kTiles * kTileCols <= kTmemCols, "TMEM");
constexpr uint32_t kIdesc1 = tc::idesc_f16_f32(128, kN1);
constexpr uint32_t kIdesc2 = tc::idesc_f16_f32(128, kN2);
constexpr uint32_t kBias = 0x3F000000u;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr int kStageKb = 8;   // B limbs 0..31: k-blocks 8..15 of the thread's A row

template <int W>
struct Win {
  static constexpr int kEntries = 1 << W;
  static constexpr int kNwin = (32 * kH + W - 1) / W;            // windows of the 2048-bit exponent
  static constexpr int kTblU4 = kEntries * (kH / 4) * kRows;     // uint4 per tile slot: [entry][g][row]
};

struct Tile {
  uint32_t sb, arow, abuf, hrow, tmem, taddr, mbar, phase, pending;
  int bar_id;
  bool leader, err, dead;
};

// MMA 1 (N = 128, B1 = Toeplitz of m') or MMA 2 (N = 256, B2 = Toeplitz of m):
// the bias block, then 8 K-steps of 16 digits, then the commit; leader only.
__device__ __forceinline__ void issue_mma(const Tile &ts, bool second) {
  const uint32_t boff = second ? kOffB2 : kOffB1;
  const uint32_t bkb = second ? kKb2 : kKb;
  const uint32_t idesc = second ? kIdesc2 : kIdesc1;
  tc::fence_after_sync();
  tc::mma_f16(ts.tmem, tc::sdesc(ts.sb + kOffAbias, kKb, 128), tc::sdesc(ts.sb + boff + 16 * bkb, bkb, 128), idesc,
              0u);
#pragma unroll 1
  for (int s = 0; s < kDig / 16; ++s)
    tc::mma_f16(ts.tmem, tc::sdesc(ts.abuf + s * 2 * kKb, kKb, 128), tc::sdesc(ts.sb + boff + s * 2 * bkb, bkb, 128),
                idesc, 1u);
  tc::commit(ts.mbar);
}

__device__ __forceinline__ void wait_mma(Tile &ts, uint32_t polls) {
  if (!tc::mbar_wait(ts.mbar, ts.phase, polls)) {
    ts.err = true;
    ts.pending = ts.phase;
  }
  ts.phase ^= 1u;
  tc::fence_after_sync();
}

// The tile's digits are written: make them visible to the tensor core and
// agree (over the tile's 128 threads) whether any of them gave up a wait.
__device__ __forceinline__ bool tile_sync(Tile &ts) {
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  ts.dead = tc::bar_red_or(ts.bar_id, kRows, ts.err);
  return ts.dead;
}

// X[j0 .. j0+NL) += (4*NL column words v, carried from c in base 2^16) + cin
template <int NL, int NX>
__device__ __forceinline__ void add_columns(uint32_t (&X)[NX], int j0, const uint32_t *v, uint32_t &c, uint32_t &cin) {
  uint32_t Y[NL];
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const uint32_t y0 = tc::pair_cols(v[4 * i], v[4 * i + 1]) + c;
    c = y0 >> 16;
    const uint32_t y1 = tc::pair_cols(v[4 * i + 2], v[4 * i + 3]) + c;
    c = y1 >> 16;
    Y[i] = tc::prmt(y0, y1, 0x5410u);
  }
  (void)add_cc(cin, 0xFFFFFFFFu);
#pragma unroll
  for (int i = 0; i < NL; ++i) X[j0 + i] = addc_cc(X[j0 + i], Y[i]);
  cin = addc(0u, 0u);
}

// MMA 1's columns (TMEM columns 0..127) carried into mu's 128 digits, written
// into the tile's A buffer; returns mu's digits 124..127.
__device__ __forceinline__ uint32_t mu_pass(const Tile &ts) {
  uint32_t mu_top = 0u, c = 0u;
#pragma unroll 1
  for (int c0 = 0; c0 < kDig; c0 += 16) {
    uint32_t v[16];
    tc::ld16(ts.taddr + (uint32_t)c0, v);
    tc::wait_ld();
    uint32_t y[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      y[j] = tc::pair_cols(v[2 * j], v[2 * j + 1]) + c;
      c = y[j] >> 16;
    }
    const uint32_t ad = ts.arow + (uint32_t)(c0 >> 3) * kKb;
    tc::sts128(ad, tc::prmt(y[0], 0u, 0x4140u), tc::prmt(y[1], 0u, 0x4140u), tc::prmt(y[2], 0u, 0x4140u),
               tc::prmt(y[3], 0u, 0x4140u));
    tc::sts128(ad + kKb, tc::prmt(y[4], 0u, 0x4140u), tc::prmt(y[5], 0u, 0x4140u), tc::prmt(y[6], 0u, 0x4140u),
               tc::prmt(y[7], 0u, 0x4140u));
    mu_top = tc::prmt(y[6], y[7], 0x5410u);   // in the last chunk: digits 124..127
  }
  return mu_top;
}

// The bias-free top positions 380..383 of mu * m from mu's digits 124..127
// and m's top limb (six byte products), as column words with the bias.
__device__ __forceinline__ void top_columns(uint32_t (&tcol)[4], uint32_t mu_top, uint32_t mt) {
  const uint32_t a5 = (mu_top >> 8) & 0xFFu, a6 = (mu_top >> 16) & 0xFFu, a7 = mu_top >> 24;
  const uint32_t b5 = (mt >> 8) & 0xFFu, b6 = (mt >> 16) & 0xFFu, b7 = mt >> 24;
  tcol[0] = kBias + a5 * b7 + a6 * b6 + a7 * b5;
  tcol[1] = kBias + a6 * b7 + a7 * b6;
  tcol[2] = kBias + a7 * b7;
  tcol[3] = kBias;
}

// One reduction round on the value V whose limbs 0..31 are in the A buffer as
// digits (limb 31 also in `top`) and whose limbs 32 .. 32+NX-1 are X[0 .. NX):
// mu = (V mod r) m' mod r, then X[B0 .. B0+64) += positions 128..383 of mu * m
// with the carry out of the low half; returns the carry out of X[B0 + 63]
// (column carry + limb carry), for the caller to place.
template <int B0, int NX>
__device__ __forceinline__ uint32_t reduce_round(uint32_t (&X)[NX], uint32_t top, Tile &ts, const uint32_t *Ms,
                                                 uint32_t polls) {
  if (tile_sync(ts)) return 0u;
  if (ts.leader) issue_mma(ts, false);
  wait_mma(ts, polls);
  const uint32_t mu_top = mu_pass(ts);
  if (tile_sync(ts)) return 0u;
  if (ts.leader) issue_mma(ts, true);
  uint32_t tcol[4];
  top_columns(tcol, mu_top, Ms[kH - 1]);   // while the tensor core works
  wait_mma(ts, polls);
  uint32_t c, cin = 0u;
  {
    uint32_t v[16];
    tc::ld16(ts.taddr + 0u, v);   // positions 124..139
    tc::wait_ld();
    // carry out of the low 1024 bits: ceil of positions 124..127 (with V's limb 31) / 2^32
    const uint32_t y0 = tc::pair_cols(v[0], v[1]) + (top & 0xFFFFu);
    const uint32_t y1 = tc::pair_cols(v[2], v[3]) + (top >> 16) + (y0 >> 16);
    c = (y1 >> 16) + (((y0 | y1) & 0xFFFFu) != 0u ? 1u : 0u);
    add_columns<3>(X, B0, v + 4, c, cin);                 // positions 128..139
  }
#pragma unroll
  for (int k = 1; k < 16; ++k) {
    uint32_t v[16];
    tc::ld16(ts.taddr + (uint32_t)(16 * k), v);           // positions 124 + 16k .. +15
    tc::wait_ld();
    add_columns<4>(X, B0 + 3 + 4 * (k - 1), v, c, cin);
  }
  tc::fence_before_sync();   // this tile's TMEM reads precede its next MMA (ordered by the next barrier)
  add_columns<1>(X, B0 + 63, tcol, c, cin);               // positions 380..383
  return c + cin;
}

// ---------------------------------------------------------------- squaring
// T = A^2 = 2C + D (C: the cross products a_i a_j, i < j, each once; D: the
// squares a_k^2 at limbs 2k, 2k+1).  Row i adds a_i a_j for j > i in two carry
// chains (odd and even j - i); after row i the limbs up to 2i+2 of C are
// final, so T's limbs 2i+1 and 2i+2 are formed (the doubling shifts in the top
// bit of the limb below) and leave at once, as in the product: limbs 0..31 as
// digits, 32..63 into the high stage, 64..127 into t.
template <int I, int J0>
__device__ __forceinline__ void sq_chain(uint32_t (&c)[2 * kH], const uint32_t (&a)[kH]) {
  if constexpr (J0 < kH) {
    c[I + J0] = mad_lo_cc(a[I], a[J0], c[I + J0]);
    c[I + J0 + 1] = madc_hi_cc(a[I], a[J0], c[I + J0 + 1]);
#pragma unroll
    for (int j = J0 + 2; j < kH; j += 2) {
      c[I + j] = madc_lo_cc(a[I], a[j], c[I + j]);
      c[I + j + 1] = madc_hi_cc(a[I], a[j], c[I + j + 1]);
    }
    constexpr int last = J0 + ((kH - 1 - J0) / 2) * 2;
    c[I + last + 2] = addc(c[I + last + 2], 0u);
  }
}

template <int P>
__device__ __forceinline__ void sq_out(uint32_t v, const Tile &ts, uint32_t (&t)[kH], uint32_t &top) {
  if constexpr (P < 32) {
    tc::emit_digits(ts.arow, P, v, kKb);
    if constexpr (P == 31) top = v;
  } else if constexpr (P < 64) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(ts.hrow + (uint32_t)((P - 32) >> 2) * (kHiBytes / 8) +
                                                 (uint32_t)((P - 32) & 3) * 4u),
                 "r"(v)
                 : "memory");
  } else {
    t[P - 64] = v;
  }
}

template <int I>
__device__ __forceinline__ void sq_rows(uint32_t (&c)[2 * kH], const uint32_t (&a)[kH], uint32_t (&t)[kH],
                                        const Tile &ts, uint32_t &tc_carry, uint32_t &top) {
  if constexpr (I < kH - 1) {
    sq_chain<I, I + 1>(c, a);
    sq_chain<I, I + 2>(c, a);
    const uint32_t x0 = __funnelshift_l(c[2 * I], c[2 * I + 1], 1), x1 = __funnelshift_l(c[2 * I + 1], c[2 * I + 2], 1);
    (void)add_cc(tc_carry, 0xFFFFFFFFu);   // carry flag <- tc_carry
    const uint32_t t0 = addc_cc(x0, __umulhi(a[I], a[I]));
    const uint32_t t1 = addc_cc(x1, a[I + 1] * a[I + 1]);
    tc_carry = addc(0u, 0u);
    sq_out<2 * I + 1>(t0, ts, t, top);
    sq_out<2 * I + 2>(t1, ts, t, top);
    sq_rows<I + 1>(c, a, t, ts, tc_carry, top);
  }
}

// T = A^2 into the A buffer (limbs 0..31), the high stage (32..63) and t (64..127); returns limb 31
__device__ __forceinline__ uint32_t square(uint32_t (&t)[kH], const uint32_t (&a)[kH], const Tile &ts) {
  uint32_t c[2 * kH];
#pragma unroll
  for (int j = 0; j < 2 * kH; ++j) c[j] = 0u;
  uint32_t tc_carry = 0u, top = 0u;
  sq_out<0>(a[0] * a[0], ts, t, top);
  sq_rows<0>(c, a, t, ts, tc_carry, top);
  t[kH - 1] = __funnelshift_l(c[2 * kH - 2], c[2 * kH - 1], 1) + __umulhi(a[kH - 1], a[kH - 1]) + tc_carry;
  return top;
}

// ---------------------------------------------------------------- one Montgomery step
// A = A * B * R^-1 mod m (A < m, B < m; R = 2^2048).  B: 64 limbs in shared
// memory, groups 0..7 (limbs 0..31) at lo + g*lo_str, groups 8..15 at
// hi + (g-8)*hi_str (the thread's stage, or a key constant).
__device__ __forceinline__ void mont_step(uint32_t (&A)[kH], bool sq, uint32_t lo, uint32_t lo_str, uint32_t hi,
                                          uint32_t hi_str, Tile &ts, const uint32_t *Ms, uint32_t polls) {
  // 1. T = A * B: limbs 0..31 leave as digits (A buffer), 32..63 as words
  //    (high stage), 64..127 stay in t.  Block i0 reads B limbs i0..i0+7
  //    before it writes anything: a digit of T limb p >= 16 lands on B limbs
  //    2p-32, 2p-31 of the stage and a word of T limb p >= 32 on B limbs
  //    p - p%4 .. +3, all read by this block or an earlier one.
  uint32_t t[kH];
#pragma unroll
  for (int j = 0; j < kH; ++j) t[j] = 0u;
  uint32_t top = 0u;
  if (sq) top = square(t, A, ts);
#pragma unroll 1
  for (int i0 = 0; i0 < (sq ? 0 : kH); i0 += 8) {
    const uint32_t g = (uint32_t)(i0 >> 2);
    const uint32_t a0 = g < 8 ? lo + g * lo_str : hi + (g - 8) * hi_str;
    const uint32_t a1 = g + 1 < 8 ? lo + (g + 1) * lo_str : hi + (g - 7) * hi_str;
    const uint4 b0 = tc::lds128(a0), b1 = tc::lds128(a1);
    uint32_t e[8];
    e[0] = mul_emit<kH>(t, A, b0.x);
    e[1] = mul_emit<kH>(t, A, b0.y);
    e[2] = mul_emit<kH>(t, A, b0.z);
    e[3] = mul_emit<kH>(t, A, b0.w);
    e[4] = mul_emit<kH>(t, A, b1.x);
    e[5] = mul_emit<kH>(t, A, b1.y);
    e[6] = mul_emit<kH>(t, A, b1.z);
    e[7] = mul_emit<kH>(t, A, b1.w);
    if (i0 < 32) {
      // limbs i0..i0+7 are digits 4*i0 .. 4*i0+31: k-blocks i0/2 .. i0/2+3
      const uint32_t ad = ts.arow + (uint32_t)(i0 >> 1) * kKb;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        tc::sts128(ad + q * kKb, tc::prmt(e[2 * q], 0u, 0x4140u), tc::prmt(e[2 * q], 0u, 0x4342u),
                   tc::prmt(e[2 * q + 1], 0u, 0x4140u), tc::prmt(e[2 * q + 1], 0u, 0x4342u));
      top = e[7];   // after the block i0 = 24: limb 31
    } else {
      const uint32_t ad = ts.hrow + (uint32_t)((i0 - 32) >> 2) * kHiBytes / 8;
      tc::sts128(ad, e[0], e[1], e[2], e[3]);
      tc::sts128(ad + kHiBytes / 8, e[4], e[5], e[6], e[7]);
    }
  }
  // 2. round 1: X holds T's limbs 32..127 (the first 32 read back from the high stage)
  uint32_t X[96];
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const uint4 v = tc::lds128(ts.hrow + (uint32_t)g * (kHiBytes / 8));
    X[4 * g] = v.x; X[4 * g + 1] = v.y; X[4 * g + 2] = v.z; X[4 * g + 3] = v.w;
  }
#pragma unroll
  for (int j = 0; j < kH; ++j) X[32 + j] = t[j];
  const uint32_t c1 = reduce_round<0>(X, top, ts, Ms, polls);
  if (ts.dead) return;
  // the carry into T1's limbs 64..95 (X[64 .. 96)); T1 may carry one bit past them
  X[64] = add_cc(X[64], c1);
#pragma unroll
  for (int j = 65; j < 96; ++j) X[j] = addc_cc(X[j], 0u);
  const uint32_t x96 = addc(0u, 0u);
  // T1's limbs 0..31 leave as digits for round 2 (mu1's digits are no longer read)
#pragma unroll
  for (int p = 0; p < 32; ++p) tc::emit_digits(ts.arow, p, X[p], kKb);
  // 3. round 2: X[32 .. 96) += positions 128..383 of mu2 * m; T2 = X[32 .. 96) and the top word
  const uint32_t c2 = reduce_round<32>(X, X[31], ts, Ms, polls);
  if (ts.dead) return;
  uint32_t u[kH + 2];
#pragma unroll
  for (int j = 0; j < kH; ++j) u[j] = X[32 + j];
  u[kH] = c2 + x96;
  u[kH + 1] = 0u;
  final_sub<kH>(A, u, NSmem<kH>{Ms});
}

// ---------------------------------------------------------------- table and stage helpers
// Table of one tile slot in global memory: [entry][g][row] of uint4 (g = limb / 4).
__device__ __forceinline__ void tbl_store(uint4 *tbl, int e, const uint32_t (&A)[kH]) {
#pragma unroll
  for (int g = 0; g < kH / 4; ++g)
    tbl[(e * (kH / 4) + g) * kRows] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
}
// group g of the thread's stage: limbs 0..31 in k-blocks 8..15 of its A row, 32..63 in its high stage
__device__ __forceinline__ uint4 *stage_group(uint8_t *smem, const Tile &ts, int g) {
  const uint32_t a = g < 8 ? ts.arow + (uint32_t)(kStageKb + g) * kKb : ts.hrow + (uint32_t)(g - 8) * (kHiBytes / 8);
  return reinterpret_cast<uint4 *>(smem + (a - ts.sb));
}
// stage <- T[d], reading every entry (constant time)
template <int W>
__device__ __forceinline__ void tbl_select(uint8_t *smem, const Tile &ts, const uint4 *tbl, uint32_t d) {
#pragma unroll 1
  for (int g0 = 0; g0 < kH / 4; g0 += 2) {
    uint4 acc[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) acc[u] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int e = 0; e < (1 << W); ++e) {
      const uint32_t msk = 0u - (uint32_t)((uint32_t)e == d);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const uint4 v = tbl[(e * (kH / 4) + g0 + u) * kRows];
        acc[u].x |= v.x & msk;
        acc[u].y |= v.y & msk;
        acc[u].z |= v.z & msk;
        acc[u].w |= v.w & msk;
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) *stage_group(smem, ts, g0 + u) = acc[u];
  }
}
__device__ __forceinline__ void stage_from_table(uint8_t *smem, const Tile &ts, const uint4 *entry) {
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) *stage_group(smem, ts, g) = entry[g * kRows];
}
__device__ __forceinline__ void stage_get(uint32_t (&A)[kH], uint8_t *smem, const Tile &ts) {
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) {
    const uint4 v = *stage_group(smem, ts, g);
    A[4 * g] = v.x; A[4 * g + 1] = v.y; A[4 * g + 2] = v.z; A[4 * g + 3] = v.w;
  }
}

// ---------------------------------------------------------------- one tile's exponentiation
// x = c R mod m from the 128-limb message row (c_lo R^2 R^-1 + c_hi R^3 R^-1),
// then the constant-time fixed window over the prime's exponent (squarings by
// `square`, products with the staged B).  The q half (pi == 0) leaves
// Montgomery form.
template <int W>
__device__ __forceinline__ void exp_tile(uint32_t (&A)[kH], Tile &ts, uint8_t *smem, const uint32_t *msg, uint32_t pi,
                                         const uint32_t *kc, uint4 *tbl, uint32_t polls) {
  using Wn = Win<W>;
  const uint32_t *Ms = kc + kKm;
  const NSmem<kH> N{Ms};
  const uint32_t kca = ts.sb + kOffKey;   // key constants: groups at 16-byte stride
  const uint32_t slo = ts.arow + kStageKb * kKb, shi = ts.hrow;
  constexpr int ntab = Wn::kEntries;
  constexpr int nexp = (Wn::kNwin - 1) * (W + 1);
  const int nst = ntab + nexp + (pi == 0 ? 1 : 0);
  int k = Wn::kNwin - 2, s = 0;
#pragma unroll 1
  for (int st = 0; st < nst; ++st) {
    uint32_t lo = slo, lo_str = kKb, hi = shi, hi_str = kHiBytes / 8;
    bool sq = false;
    if (st == 0) {                      // c_lo * R mod m
      load_row<kH>(A, msg, true);
      lo = kca + 4 * kKr2; lo_str = 16; hi = lo + 128; hi_str = 16;
    } else if (st == 1) {               // c_hi * R^2 mod m
      tbl_store(tbl, 1, A);
      load_row<kH>(A, msg + kH, true);
      lo = kca + 4 * kKr3; lo_str = 16; hi = lo + 128; hi_str = 16;
    } else if (st < ntab) {             // table T[i] = x^i R, i = 2 .. ntab-1
      if (st == 2) {
        mod_add<kH>(A, SmemB{tbl + 1 * (kH / 4) * kRows, kRows}, N);   // x R = c_hi R^2 + c_lo R
        tbl_store(tbl, 1, A);
        uint32_t one[kH];
        from_uniform<kH>(one, reinterpret_cast<const uint4 *>(kc + kKone));
        tbl_store(tbl, 0, one);
        sq = true;                      // T[2] = x^2
      } else {
        tbl_store(tbl, st - 1, A);
        stage_from_table(smem, ts, tbl + 1 * (kH / 4) * kRows);   // B = x R
      }
    } else if (st < ntab + nexp) {      // windows: W squarings, then T[digit]
      if (st == ntab) {
        tbl_store(tbl, ntab - 1, A);
        tbl_select<W>(smem, ts, tbl, exp_digit<W>(kc + kKexp, (uint32_t)(Wn::kNwin - 1)));
        stage_get(A, smem, ts);
      }
      if (s < W) {
        sq = true;
        ++s;
      } else {
        tbl_select<W>(smem, ts, tbl, exp_digit<W>(kc + kKexp, (uint32_t)k));
        s = 0;
        --k;
      }
    } else {                            // q: leave Montgomery form
      lo = kca + 4 * kKunit; lo_str = 16; hi = lo + 128; hi_str = 16;
    }
    mont_step(A, sq, lo, lo_str, hi, hi_str, ts, Ms, polls);
    if (ts.dead) break;
  }
}

// ---------------------------------------------------------------- exponentiation kernel (both primes)
struct HalfArgs {
  const uint32_t *keyrec;
  const uint4 *image;       // [prime][B1 | B2], prime 0 = q, 1 = p
  const uint32_t *msgs;     // count rows of 128 limbs
  uint4 *halves;            // [prime][kH/4][count_pad]: q -> m_q, p -> m_p * R mod p
  uint32_t *herr;           // [prime][count]: 1 if a bounded wait gave up
  uint4 *tables;            // [grid * kTiles][kTblU4]
  uint32_t count, count_pad, ntiles, ctas_per_prime;
  uint32_t wait_polls;
};

template <int W>
__global__ void __launch_bounds__(kThreads, 1) crt_tc4_half_kernel(HalfArgs a) {
  using Wn = Win<W>;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slot = warp >> 2;
  const int r = ((warp & 3) << 5) | lane;
  const uint32_t pi = blockIdx.x & 1u;
  const uint32_t cta = blockIdx.x >> 1;
  const uint32_t sb = tc::smem_addr(smem);
  uint32_t *ctrl = reinterpret_cast<uint32_t *>(smem + kOffCtrl);

  if (warp == 0) tc::tmem_alloc(sb + kOffCtrl + 48, kTmemCols);
  if (tid == 0) {
    for (int t = 0; t < kTiles; ++t) tc::mbar_init(sb + kOffCtrl + 8 * t, 1u);
    tc::mbar_init_fence();
  }
  constexpr KeyLayout lay(2 * kH);
  uint32_t *kc = reinterpret_cast<uint32_t *>(smem + kOffKey);
  {
    const uint32_t om = pi ? lay.p : lay.q, or2 = pi ? lay.r2p : lay.r2q, or3 = pi ? lay.r3p : lay.r3q;
    const uint32_t oone = pi ? lay.onep : lay.oneq, oexp = pi ? lay.dp : lay.dq;
    for (int i = tid; i < kKeyWords; i += kThreads) {
      uint32_t v;
      if (i < kKr2) v = a.keyrec[om + i];
      else if (i < kKr3) v = a.keyrec[or2 + i - kKr2];
      else if (i < kKone) v = a.keyrec[or3 + i - kKr3];
      else if (i < kKunit) v = a.keyrec[oone + i - kKone];
      else if (i < kKexp) v = (i == kKunit) ? 1u : 0u;
      else v = a.keyrec[oexp + i - kKexp];
      kc[i] = v;
    }
    const uint4 *img = a.image + (size_t)pi * (kImgPrime / 16);
    uint4 *s4 = reinterpret_cast<uint4 *>(smem + kOffB1);
    for (int i = tid; i < (int)(kImgPrime / 16); i += kThreads) s4[i] = img[i];
    uint4 *ab = reinterpret_cast<uint4 *>(smem + kOffAbias);
    for (int i = tid; i < kRows * 16 * 2 / 16; i += kThreads)
      ab[i] = make_uint4(0x01000100u, 0x01000100u, 0x01000100u, 0x01000100u);
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  Tile ts;
  ts.sb = sb;
  ts.abuf = sb + kOffA + slot * kABytes;
  ts.arow = ts.abuf + (uint32_t)(r >> 3) * 128 + (uint32_t)(r & 7) * 16;
  ts.hrow = sb + kOffHi + slot * kHiBytes + (uint32_t)r * 16;
  ts.tmem = ctrl[12] + (uint32_t)slot * kTileCols;
  ts.taddr = ts.tmem + ((uint32_t)((warp & 3) * 32) << 16);
  ts.mbar = sb + kOffCtrl + 8 * slot;
  ts.phase = 0u;
  ts.pending = 2u;
  ts.bar_id = 1 + slot;
  ts.leader = (r == 0);
  ts.err = false;
  ts.dead = false;
  uint4 *tbl = a.tables + (size_t)(blockIdx.x * kTiles + slot) * Wn::kTblU4 + r;

  for (uint32_t tile = cta + a.ctas_per_prime * (uint32_t)slot; tile < a.ntiles; tile += a.ctas_per_prime * kTiles) {
    const uint32_t row = tile * kRows + (uint32_t)r;
    const bool valid = row < a.count;
    const uint32_t *msg = a.msgs + (size_t)(valid ? row : a.count - 1) * (2 * kH);
    uint32_t A[kH];
    if (!ts.dead) exp_tile<W>(A, ts, smem, msg, pi, kc, tbl, a.wait_polls);
    if (valid) {
      uint4 *h = a.halves + (size_t)pi * (kH / 4) * a.count_pad + row;
#pragma unroll
      for (int g = 0; g < kH / 4; ++g)
        h[(size_t)g * a.count_pad] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
      a.herr[(size_t)pi * a.count + row] = (ts.err || ts.dead) ? 1u : 0u;
    }
  }
  if (ts.leader && ts.pending < 2u) (void)tc::mbar_wait(ts.mbar, ts.pending, kWaitLimit);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(ctrl[12], kTmemCols);
  }
}

// ---------------------------------------------------------------- Garner recombination
// m = m_q + q * ((m_p - m_q) * qinv mod p), one thread per operation (CIOS
// Montgomery products of mont.cuh, modulus p from shared memory).
constexpr int kGThreads = 128;
constexpr int kGKeyWords = (KeyLayout(2 * kH).total + 3) / 4 * 4;
constexpr int kGSmem = kGKeyWords * 4 + (kGThreads / 32) * (kH / 4) * 32 * 16;

struct GarnerArgs {
  const uint32_t *keyrec;
  const uint4 *halves;
  const uint32_t *herr;
  const uint32_t *msgs;
  uint32_t *out;
  int32_t *status;
  uint32_t count, count_pad;
};

__global__ void __launch_bounds__(kGThreads) crt_tc4_garner_kernel(GarnerArgs a) {
  constexpr int L = 2 * kH;
  constexpr KeyLayout lay(L);
  extern __shared__ uint4 gsm[];
  uint32_t *ks = reinterpret_cast<uint32_t *>(gsm);
  for (int i = threadIdx.x; i < kGKeyWords / 4; i += kGThreads)
    gsm[i] = (i * 4 < (int)lay.total) ? reinterpret_cast<const uint4 *>(a.keyrec)[i] : make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(ks);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t row = blockIdx.x * kGThreads + threadIdx.x;
  const bool valid = row < a.count;
  const uint32_t rr = valid ? row : 0u;
  uint4 *stage_lane = gsm + kGKeyWords / 4 + warp * (kH / 4) * 32 + lane;
  const NSmem<kH> N{ks + lay.p};
  const uint4 *hq = a.halves + rr, *hp = a.halves + (size_t)(kH / 4) * a.count_pad + rr;
  uint32_t A[kH];
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) {
    const uint4 v = hq[(size_t)g * a.count_pad];
    A[4 * g] = v.x; A[4 * g + 1] = v.y; A[4 * g + 2] = v.z; A[4 * g + 3] = v.w;
  }
  mont_mul<kH, 4>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.r2p), 1}, N, hd.np_p);   // m_q * R mod p
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) stage_lane[g * 32] = hp[(size_t)g * a.count_pad];         // m_p * R mod p
  mod_rsub<kH>(A, SmemB{stage_lane, 32}, N);                                                  // (m_p - m_q) R
  mont_mul<kH, 4>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.qinv), 1}, N, hd.np_p);  // h
  uint32_t t[kH + 2];
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) {
    const uint4 v = hq[(size_t)g * a.count_pad];
    t[4 * g] = v.x; t[4 * g + 1] = v.y; t[4 * g + 2] = v.z; t[4 * g + 3] = v.w;
  }
  t[kH] = 0u;
  t[kH + 1] = 0u;
  const uint32_t *qs = ks + lay.q;
  const uint32_t *mrow = a.msgs + (size_t)rr * L;
  const bool below = row_below(mrow, ks + lay.n, L);
  const bool timed_out = a.herr[rr] != 0u || a.herr[a.count + rr] != 0u;
  const bool ok = valid && below && !timed_out;
  uint4 *orow = reinterpret_cast<uint4 *>(a.out + (size_t)rr * L);
#pragma unroll 1
  for (int i0 = 0; i0 < kH; i0 += 4) {
    uint32_t rv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      mul_acc<kH>(t, A, qs[i0 + u]);
      rv[u] = t[0];
#pragma unroll
      for (int j = 0; j < kH + 1; ++j) t[j] = t[j + 1];
      t[kH + 1] = 0u;
    }
    if (valid) orow[i0 / 4] = ok ? make_uint4(rv[0], rv[1], rv[2], rv[3]) : make_uint4(0u, 0u, 0u, 0u);
  }
#pragma unroll
  for (int g = 0; g < kH / 4; ++g)
    if (valid)
      orow[kH / 4 + g] = ok ? make_uint4(t[4 * g], t[4 * g + 1], t[4 * g + 2], t[4 * g + 3])
                            : make_uint4(0u, 0u, 0u, 0u);
  if (valid && a.status) a.status[rr] = timed_out ? -6 /* RSA_ERR_TIMEOUT */ : (below ? 0 : -3 /* RSA_ERR_RANGE */);
}

// ---------------------------------------------------------------- host side
size_t tc4_smem_bytes() { return (size_t)kSmem; }

int tc4_grid(uint32_t count, int sm_count) {
  const uint32_t ntiles = (count + kRows - 1) / kRows;
  const uint32_t want = (ntiles + kTiles - 1) / kTiles;
  const uint32_t per_prime = want < 1u ? 1u : (want < (uint32_t)(sm_count / 2) ? want : (uint32_t)(sm_count / 2));
  return (int)(2 * (per_prime ? per_prime : 1u));
}

size_t tc4_tables_bytes(int grid, int window) {
  const size_t per_slot = (window == 3) ? (size_t)Win<3>::kTblU4 : (size_t)Win<4>::kTblU4;
  return (size_t)grid * kTiles * per_slot * 16;
}

static uint32_t pad_count(uint32_t count) { return (count + 31u) & ~31u; }

size_t tc4_halves_bytes(uint32_t count) {
  return (size_t)2 * (kH / 4) * pad_count(count) * 16 + (size_t)2 * count * 4;
}

template <int W>
static cudaError_t launch_half(const HalfArgs &h, int grid, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(crt_tc4_half_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  crt_tc4_half_kernel<W><<<grid, kThreads, kSmem, s>>>(h);
  return cudaGetLastError();
}

cudaError_t launch_crt_tc4(const uint32_t *keyrec, const void *image, const uint32_t *msgs, uint32_t *out,
                           int32_t *status, uint32_t count, int grid, int window, void *tables, void *halves,
                           uint32_t wait_polls, cudaStream_t s) {
  const uint32_t cp = pad_count(count);
  HalfArgs h;
  h.keyrec = keyrec;
  h.image = static_cast<const uint4 *>(image);
  h.msgs = msgs;
  h.halves = static_cast<uint4 *>(halves);
  h.herr = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(halves) + (size_t)2 * (kH / 4) * cp * 16);
  h.tables = static_cast<uint4 *>(tables);
  h.count = count;
  h.count_pad = cp;
  h.ntiles = (count + kRows - 1) / kRows;
  h.ctas_per_prime = (uint32_t)grid / 2;
  h.wait_polls = wait_polls;
  cudaError_t e = (window == 3) ? launch_half<3>(h, grid, s) : launch_half<4>(h, grid, s);
  if (e != cudaSuccess) return e;
  GarnerArgs g;
  g.keyrec = keyrec;
  g.halves = h.halves;
  g.herr = h.herr;
  g.msgs = msgs;
  g.out = out;
  g.status = status;
  g.count = count;
  g.count_pad = cp;
  crt_tc4_garner_kernel<<<(count + kGThreads - 1) / kGThreads, kGThreads, kGSmem, s>>>(g);
  return cudaGetLastError();
}

}  // namespace tc4
}  // namespace rsagpu
