// crt_tc.cu -- RSA-2048 CRT decryption with the Montgomery reduction on the
// 5th-generation tensor cores (tcgen05, TMEM), for 1024-bit primes.
//
// Decryption follows the CRT route of the library's other kernels:
// M = C^d mod n computed as m_p = C^dp mod p and m_q = C^dq mod q, then
// recombined (Garner).  Each half is a constant-time fixed-window
// exponentiation (Fig. 6 of the paper with k = W) whose every modular
// multiplication is a Montgomery product A*B*R^-1 mod m, R = 2^1024.
//
// The Montgomery product is split between the two kinds of units:
//   1. CUDA cores: T = A * B, 32 x 32 limbs, product scanning with PTX carry
//      chains (one thread per operation).  The low half of T leaves the
//      registers as byte digits (fp16) in shared memory.
//   2. Tensor core, MMA 1: the column sums of the byte convolution of
//      T mod R with m' = -m^-1 mod R (columns 0..127).
//   3. CUDA cores: carry-propagate the columns (two at a time, as base-2^16
//      digits) into the bytes of mu = T*m' mod R, written back as fp16 digits.
//   4. Tensor core, MMA 2: the column sums of mu * m for positions 124..251;
//      positions 252..254 (six byte products) on the CUDA cores.
//   5. CUDA cores: the carry out of the low half (ceil of positions 124..127
//      with T's top bytes, over 2^32: the lower positions add less than 2^-8
//      of a unit), the high half carry-propagated and added to T_hi, one
//      conditional subtraction of m.
// m' and m are the same for every message of the batch, which is what makes
// steps 2 and 4 matrix products (messages x digits) x (digits x digits); the
// per-message product A*B (step 1) stays on the CUDA cores.  Exactness: the
// digits are bytes and a column holds at most 128 products of two bytes, so
// every column sum is an integer below 2^23 and the fp32 accumulation is exact
// (tcprep.cpp describes the bias that makes the sums readable as integers).
//
// Work layout: one CTA per SM (512 threads), all of one prime; four tiles of
// 128 operations, each with its own A buffer, 128 TMEM columns, mbarrier and
// named barrier, run independently, so one tile's MMAs and carry passes
// overlap the other tiles' multiplications.  A tile's thread r owns operation
// r of the tile and TMEM lane r.  The B operand of step 1 is staged in the
// upper half (k-blocks 8..15) of the thread's own row of the A buffer: the
// product scan reads limb group g before it overwrites k-block 8 + g.  The
// Garner recombination runs afterwards in its own kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "crt_tc.h"
#include "kernels.cuh"
#include "keyrec.h"
#include "mont.cuh"
#include "tc.cuh"

namespace rsagpu {
namespace tcr {

// ---------------------------------------------------------------- shared memory map (bytes)
constexpr int kKb = (kRows / 8) * 128;              // k-block stride of A buffers, BM and BP (2048)
static_assert(kN1 == kRows && kN2 == kRows, "all operands have 128 rows");
constexpr int kOffBm = 0;
constexpr int kOffBp = kOffBm + (int)kImgBm;
constexpr int kOffAbias = kOffBp + (int)kImgBp;     // 128 x 16 bias A operand
constexpr int kOffA = kOffAbias + kRows * 16 * 2;   // kTiles A buffers of 128 x 128 digits
constexpr int kABytes = kRows * kDig * 2;
constexpr int kOffKey = kOffA + kTiles * kABytes;
// key constants (words): m, R^2, R^3, R mod m, unit, exponent (kH + 4 limbs)
constexpr int kKm = 0, kKr2 = kH, kKr3 = 2 * kH, kKone = 3 * kH, kKunit = 4 * kH, kKexp = 5 * kH;
constexpr int kKeyWords = 6 * kH + 4;
constexpr int kOffCtrl = kOffKey + kKeyWords * 4;   // kTiles mbarriers (8 B each), TMEM base at +48
constexpr int kSmem = kOffCtrl + 64;
static_assert(kOffA % 128 == 0 && kOffKey % 16 == 0 && kOffCtrl % 8 == 0 && kTiles * 8 <= 48, "layout");
static_assert(kSmem <= 227 * 1024, "shared memory");

constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kTileCols = 128;
static_assert(kTiles * kTileCols <= kTmemCols, "TMEM");
constexpr uint32_t kIdesc = tc::idesc_f16_f32(128, 128);
constexpr uint32_t kBias = 0x3F000000u;             // fp32 bits of the column bias 1/2
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr int kStageKb = 8;                          // the stage: k-blocks 8..15 of the thread's row
// Steps ahead of a window's multiplication at which the tile's table is
// prefetched into L2 (0: no prefetch).  The tables of all tiles in flight
// exceed L2; each one is needed only at its multiplications.
#ifndef RSAGPU_TC_PREFETCH
#define RSAGPU_TC_PREFETCH 0
#endif

template <int W>
struct Win {
  static constexpr int kEntries = 1 << W;
  static constexpr int kNwin = (32 * kH + W - 1) / W;            // windows of the 1024-bit exponent
  static constexpr int kTblU4 = kEntries * (kH / 4) * kRows;     // uint4 per tile slot: [entry][g][row]
};

struct HalfArgs {
  const uint32_t *keyrec;
  const uint4 *image;       // [prime][BM | BP], prime 0 = q, 1 = p
  const uint32_t *msgs;     // count rows of 64 limbs
  uint4 *halves;            // [prime][kH/4][count_pad]: q -> m_q, p -> m_p * R mod p
  uint32_t *herr;           // [prime][count]: 1 if a bounded wait gave up
  uint4 *tables;            // [grid * kTiles][kTblU4]
  uint32_t count, count_pad, ntiles, ctas_per_prime;
  uint32_t wait_polls;      // polls of an MMA mbarrier before a tile gives up
};

struct GarnerArgs {
  const uint32_t *keyrec;
  const uint4 *halves;
  const uint32_t *herr;
  const uint32_t *msgs;
  uint32_t *out;
  int32_t *status;
  uint32_t count, count_pad;
};

// ---------------------------------------------------------------- arithmetic pieces
using tc::pair_cols;

// t[j0 .. j0+NL) += the 4*NL column words v taken as 2*NL base-2^16 columns
// (tc::lo_halves / tc::hi_halves): s = X + Y word by word with the carry cs,
// then t += s with the carry cin.  yb is the column below v[0]: its high half
// (the pending carry, < 2^16) enters word j0; the last column of v returns in
// yb.  Two carry chains of NL words, no 16-bit ripple.
template <int NL>
__device__ __forceinline__ void add_columns(uint32_t (&t)[kH], int j0, const uint32_t *v, uint32_t &yb,
                                            uint32_t &cs, uint32_t &cin) {
  uint32_t y[2 * NL];
#pragma unroll
  for (int i = 0; i < 2 * NL; ++i) y[i] = pair_cols(v[2 * i], v[2 * i + 1]);
  uint32_t x[NL];
  (void)add_cc(cs, 0xFFFFFFFFu);    // carry flag <- cs (0 or 1)
#pragma unroll
  for (int i = 0; i < NL; ++i)
    x[i] = addc_cc(tc::lo_halves(y[2 * i], y[2 * i + 1]), tc::hi_halves(i ? y[2 * i - 1] : yb, y[2 * i]));
  cs = addc(0u, 0u);
  yb = y[2 * NL - 1];
  (void)add_cc(cin, 0xFFFFFFFFu);   // carry flag <- cin
#pragma unroll
  for (int i = 0; i < NL; ++i) t[j0 + i] = addc_cc(t[j0 + i], x[i]);
  cin = addc(0u, 0u);
}

struct Tile {
  uint32_t sb;        // shared-window address of the dynamic shared memory
  uint32_t arow;      // this thread's row in its tile's A buffer (k-block 0)
  uint32_t abuf;      // the tile's A buffer
  uint32_t tmem;      // TMEM address of the tile (lane 0, first column)
  uint32_t taddr;     // TMEM address of this warp's lane quarter
  uint32_t mbar, phase, pending;
  int bar_id;
  bool leader;
  bool err;    // this thread gave up a wait (voted at the next tile barrier)
  bool dead;   // the tile voted to stop: uniform across its 128 threads
};

// Issue the nine MMAs of one product (bias block, then 8 K-steps of 16 digits)
// and the commit; leader thread only.
__device__ __forceinline__ void issue_mmas(const Tile &ts, uint32_t b_off) {
  tc::fence_after_sync();
  tc::mma_f16(ts.tmem, tc::sdesc(ts.sb + kOffAbias, kKb, 128), tc::sdesc(ts.sb + b_off + 16 * kKb, kKb, 128),
              kIdesc, 0u);
#pragma unroll 1
  for (int s = 0; s < kDig / 16; ++s)
    tc::mma_f16(ts.tmem, tc::sdesc(ts.abuf + s * 2 * kKb, kKb, 128),
                tc::sdesc(ts.sb + b_off + s * 2 * kKb, kKb, 128), kIdesc, 1u);
  tc::commit(ts.mbar);
}

__device__ __forceinline__ void wait_mmas(Tile &ts, uint32_t polls) {
  if (!tc::mbar_wait(ts.mbar, ts.phase, polls)) {
    ts.err = true;
    ts.pending = ts.phase;
  }
  ts.phase ^= 1u;
  tc::fence_after_sync();
}

__device__ __forceinline__ void emit_digits(uint32_t arow, int p, uint32_t v) { tc::emit_digits(arow, p, v, kKb); }

// T = A^2 for step 1 of the Montgomery product, with A = a_lo + a_hi r (r =
// 2^(32 HR), halves of HR = kH/2 limbs): T = a_lo^2 + 2 P r + a_hi^2 r^2,
// P = a_lo a_hi.  P runs as a rolled loop of product rows (a_lo read back
// from the thread's stage -- free in a squaring -- a_hi in registers); each
// row group's four limbs of P replace the four limbs of a_lo it read, and P's
// low half returns to registers before the square's digits overwrite the
// stage.  The half squares compute each of their cross products once
// (square_emit), and their limbs take 2P as they leave: T's limbs 0 .. HR-1
// from a_lo^2 alone, HR .. kH-1 = a_lo^2's high half + 2 P_lo (all digits of
// the thread's A row), kH .. 2kH-1 = a_hi^2 + 2 P_hi (t).  HR^2 + 2 HR(HR+1)/2
// = kH(kH+1)/2 word products, in about half the code of a square in one piece.

// a_lo^2's limbs p: T's limbs, plus (from p = HR on) 2 P_lo, whose word k is
// P_k << 1 with P_(k-1)'s top bit; all leave as digits, limb kH-1 also in top
struct LowEmit {
  uint32_t arow;
  const uint32_t (&plo)[kH / 2];
  uint32_t top, carry;
  template <int P>
  __device__ __forceinline__ void put(uint32_t v) {
    constexpr int HR = kH / 2;
    if constexpr (P >= HR) {
      constexpr int k = P - HR;
      const uint32_t d = k ? __funnelshift_l(plo[k ? k - 1 : 0], plo[k], 1) : plo[0] << 1;
      (void)add_cc(carry, 0xFFFFFFFFu);   // carry flag <- carry
      v = addc_cc(v, d);
      carry = addc(0u, 0u);
    }
    emit_digits(arow, P, v);
    if constexpr (P == kH - 1) top = v;
  }
};

// a_hi^2's limbs p become T's limbs kH + p in t: plus 2 P_hi (acc = P_hi; word
// p takes the top bit of the word below, P_lo's last for p = 0) and the carry
struct HighEmit {
  uint32_t (&t)[kH];
  const uint32_t (&acc)[kH / 2];
  uint32_t carry, plast;
  template <int P>
  __device__ __forceinline__ void put(uint32_t v) {
    constexpr int HR = kH / 2;
    uint32_t d = 0u;
    if constexpr (P == 0) d = __funnelshift_l(plast, acc[0], 1);
    else if constexpr (P < HR) d = __funnelshift_l(acc[P - 1], acc[P], 1);
    else if constexpr (P == HR) d = acc[HR - 1] >> 31;
    (void)add_cc(carry, 0xFFFFFFFFu);   // carry flag <- carry
    t[P] = addc_cc(v, d);
    carry = addc(0u, 0u);
  }
};

// Returns T limb kH-1; T_lo leaves as digits into the thread's A row, T_hi in t.
__device__ __forceinline__ uint32_t square_p(uint32_t (&t)[kH], const uint32_t (&a)[kH], uint32_t arow) {
  constexpr int HR = kH / 2;
  static_assert(HR % 4 == 0, "halves of whole limb groups");
  uint32_t alo[HR], ahi[HR];
#pragma unroll
  for (int j = 0; j < HR; ++j) {
    alo[j] = a[j];
    ahi[j] = a[HR + j];
  }
  const uint32_t st0 = arow + (uint32_t)kStageKb * kKb;   // the stage: k-blocks 8.., four raw limbs each
#pragma unroll
  for (int g = 0; g < HR / 4; ++g)
    tc::sts128(st0 + (uint32_t)g * kKb, alo[4 * g], alo[4 * g + 1], alo[4 * g + 2], alo[4 * g + 3]);
  uint32_t acc[HR];
#pragma unroll
  for (int j = 0; j < HR; ++j) acc[j] = 0u;
#pragma unroll 1
  for (int g = 0; g < HR / 4; ++g) {
    const uint32_t ad = st0 + (uint32_t)g * kKb;
    const uint4 b = tc::lds128(ad);
    const uint32_t e0 = mul_emit<HR>(acc, ahi, b.x);
    const uint32_t e1 = mul_emit<HR>(acc, ahi, b.y);
    const uint32_t e2 = mul_emit<HR>(acc, ahi, b.z);
    const uint32_t e3 = mul_emit<HR>(acc, ahi, b.w);
    tc::sts128(ad, e0, e1, e2, e3);
  }
  uint32_t plo[HR];
#pragma unroll
  for (int g = 0; g < HR / 4; ++g) {
    const uint4 v = tc::lds128(st0 + (uint32_t)g * kKb);
    plo[4 * g] = v.x; plo[4 * g + 1] = v.y; plo[4 * g + 2] = v.z; plo[4 * g + 3] = v.w;
  }
  LowEmit lo{arow, plo, 0u, 0u};
  square_emit<HR>(alo, lo);
  HighEmit hi{t, acc, lo.carry, plo[HR - 1]};
  square_emit<HR>(ahi, hi);
  return lo.top;
}

// A = A * B * R^-1 mod m (A < R, B < m; result < m).  B: kH limbs in shared
// memory at bsa, four limbs per 16 bytes, consecutive groups `bstr` bytes
// apart (the thread's stage, or a key constant).
__device__ __forceinline__ void mont_step(uint32_t (&A)[kH], bool sq, uint32_t bsa, uint32_t bstr, Tile &ts,
                                          const uint32_t *Ms, uint32_t polls) {
  // 1. T = A * B (or A^2 when sq): the low 32 limbs leave as digits, t ends
  //    as T_hi.  Block i0 of the general product reads B groups i0/4, i0/4+1
  //    (stage k-blocks 8 + i0/4 ..) before it writes k-blocks i0/2 .. i0/2+3,
  //    so the stage is never overwritten early.
  uint32_t t[kH];
#pragma unroll
  for (int j = 0; j < kH; ++j) t[j] = 0u;
  uint32_t top = 0u;
  if (sq) top = square_p(t, A, ts.arow);
#pragma unroll 1
  for (int i0 = 0; i0 < (sq ? 0 : kH); i0 += 8) {
    const uint4 b0 = tc::lds128(bsa + (uint32_t)(i0 >> 2) * bstr);
    const uint4 b1 = tc::lds128(bsa + (uint32_t)((i0 >> 2) + 1) * bstr);
    uint32_t e[8];
    e[0] = mul_emit<kH>(t, A, b0.x);
    e[1] = mul_emit<kH>(t, A, b0.y);
    e[2] = mul_emit<kH>(t, A, b0.z);
    e[3] = mul_emit<kH>(t, A, b0.w);
    e[4] = mul_emit<kH>(t, A, b1.x);
    e[5] = mul_emit<kH>(t, A, b1.y);
    e[6] = mul_emit<kH>(t, A, b1.z);
    e[7] = mul_emit<kH>(t, A, b1.w);
    // limbs i0..i0+7 are digits 4*i0 .. 4*i0+31: k-blocks i0/2 .. i0/2+3
    const uint32_t ad = ts.arow + (uint32_t)(i0 >> 1) * kKb;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      tc::sts128(ad + q * kKb, tc::prmt(e[2 * q], 0u, 0x4140u), tc::prmt(e[2 * q], 0u, 0x4342u),
                 tc::prmt(e[2 * q + 1], 0u, 0x4140u), tc::prmt(e[2 * q + 1], 0u, 0x4342u));
    top = e[7];
  }
  // 2. MMA 1: mu columns = T_lo digits x Toep(m')
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  ts.dead = tc::bar_red_or(ts.bar_id, kRows, ts.err);
  if (ts.dead) return;
  if (ts.leader) issue_mmas(ts, kOffBm);
  wait_mmas(ts, polls);
  // 3. mu = the column sums mod R (as 32-bit words: tc::lo_halves /
  //    tc::hi_halves, one carry chain), back to shared memory as digits; its
  //    top digits are kept for positions 252..254 of mu * m
  uint32_t mu_top = 0u;   // [mu_124, mu_125, mu_126, mu_127]
  {
    uint32_t yb = 0u;       // the base-2^16 column below the chunk
    uint32_t cw = 0u;       // carry between the chunks' words
#pragma unroll 1
    for (int c0 = 0; c0 < kDig; c0 += 16) {
      uint32_t v[16];
      tc::ld16(ts.taddr + (uint32_t)c0, v);
      tc::wait_ld();
      uint32_t y[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) y[j] = pair_cols(v[2 * j], v[2 * j + 1]);
      uint32_t w[4];
      (void)add_cc(cw, 0xFFFFFFFFu);   // carry flag <- cw
#pragma unroll
      for (int k = 0; k < 4; ++k)
        w[k] = addc_cc(tc::lo_halves(y[2 * k], y[2 * k + 1]), tc::hi_halves(k ? y[2 * k - 1] : yb, y[2 * k]));
      cw = addc(0u, 0u);
      yb = y[7];
      const uint32_t ad = ts.arow + (uint32_t)(c0 >> 3) * kKb;
      // [w.b0, 0, w.b1, 0], [w.b2, 0, w.b3, 0]: a word's bytes as fp16 digits
      tc::sts128(ad, tc::prmt(w[0], 0u, 0x4140u), tc::prmt(w[0], 0u, 0x4342u), tc::prmt(w[1], 0u, 0x4140u),
                 tc::prmt(w[1], 0u, 0x4342u));
      tc::sts128(ad + kKb, tc::prmt(w[2], 0u, 0x4140u), tc::prmt(w[2], 0u, 0x4342u), tc::prmt(w[3], 0u, 0x4140u),
                 tc::prmt(w[3], 0u, 0x4342u));
      mu_top = w[3];   // in the last chunk: digits 124..127
    }
  }
  // 4. MMA 2: positions 124..251 of mu * m
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  ts.dead = tc::bar_red_or(ts.bar_id, kRows, ts.err);
  if (ts.dead) return;
  if (ts.leader) issue_mmas(ts, kOffBp);
  // positions 252..255 while the tensor core works: sum of mu_i * m_j, i + j = position
  uint32_t top_cols[4];
  {
    const uint32_t mt = Ms[kH - 1];
    const uint32_t a5 = (mu_top >> 8) & 0xFFu, a6 = (mu_top >> 16) & 0xFFu, a7 = mu_top >> 24;
    const uint32_t b5 = (mt >> 8) & 0xFFu, b6 = (mt >> 16) & 0xFFu, b7 = mt >> 24;
    top_cols[0] = kBias + a5 * b7 + a6 * b6 + a7 * b5;
    top_cols[1] = kBias + a6 * b7 + a7 * b6;
    top_cols[2] = kBias + a7 * b7;
    top_cols[3] = kBias;
  }
  wait_mmas(ts, polls);
  // 5. U = T_hi + (T_lo + mu*m) / R, then one conditional subtraction.  The
  // columns are carry-propagated 4 at a time into limbs that are added to T_hi
  // right away (the carry between chunks is kept in a register: cin).
  uint32_t yb, cs = 0u, cin = 0u;
  {
    uint32_t v[16];
    tc::ld16(ts.taddr + 0u, v);   // positions 124..139
    tc::wait_ld();
    // carry out of the low half: ceil of positions 124..127 (with T's top limb)
    // / 2^32, below 2^16; it enters limb 0 as the high half of the column below
    const uint32_t y0 = pair_cols(v[0], v[1]) + (top & 0xFFFFu);
    const uint32_t y1 = pair_cols(v[2], v[3]) + (top >> 16) + (y0 >> 16);
    yb = ((y1 >> 16) + (((y0 | y1) & 0xFFFFu) != 0u ? 1u : 0u)) << 16;
    add_columns<3>(t, 0, v + 4, yb, cs, cin);         // positions 128..139: limbs 0..2
  }
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    uint32_t v[16];
    tc::ld16(ts.taddr + (uint32_t)(16 * k), v);       // positions 124 + 16k .. +15
    tc::wait_ld();
    add_columns<4>(t, 3 + 4 * (k - 1), v, yb, cs, cin);   // limbs 3 + 4(k-1) .. +3
  }
  tc::fence_before_sync();   // this tile's TMEM reads precede the next MMA (ordered by the next barrier)
  add_columns<1>(t, kH - 1, top_cols, yb, cs, cin);   // positions 252..255: limb 31
  uint32_t u[kH + 2];
#pragma unroll
  for (int j = 0; j < kH; ++j) u[j] = t[j];
  u[kH] = (yb >> 16) + cs + cin;
  u[kH + 1] = 0u;
  final_sub<kH>(A, u, NSmem<kH>{Ms});
}

// ---------------------------------------------------------------- table and stage helpers
// Table of one tile slot in global memory: [entry][g][row] of uint4 (g = limb / 4).
template <int W>
__device__ __forceinline__ void tbl_store(uint4 *tbl, int e, const uint32_t (&A)[kH]) {
#pragma unroll
  for (int g = 0; g < kH / 4; ++g)
    tbl[(e * (kH / 4) + g) * kRows] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
}
// stage <- T[d], reading every entry (constant time)
template <int W>
__device__ __forceinline__ void tbl_select(uint8_t *stage, const uint4 *tbl, uint32_t d) {
  constexpr int G = (W <= 3) ? 2 : 1;   // limb groups whose loads are in flight together
#pragma unroll 1
  for (int g0 = 0; g0 < kH / 4; g0 += G) {
    uint4 acc[G];
#pragma unroll
    for (int u = 0; u < G; ++u) acc[u] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int e = 0; e < (1 << W); ++e) {
      const uint32_t msk = 0u - (uint32_t)((uint32_t)e == d);
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const uint4 v = tbl[(e * (kH / 4) + g0 + u) * kRows];
        acc[u].x |= v.x & msk;
        acc[u].y |= v.y & msk;
        acc[u].z |= v.z & msk;
        acc[u].w |= v.w & msk;
      }
    }
#pragma unroll
    for (int u = 0; u < G; ++u) *reinterpret_cast<uint4 *>(stage + (g0 + u) * kKb) = acc[u];
  }
}
__device__ __forceinline__ void stage_from(uint8_t *stage, const uint4 *src, int src_stride) {
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) *reinterpret_cast<uint4 *>(stage + g * kKb) = src[g * src_stride];
}
__device__ __forceinline__ void stage_put(uint8_t *stage, const uint32_t (&A)[kH]) {
#pragma unroll
  for (int g = 0; g < kH / 4; ++g)
    *reinterpret_cast<uint4 *>(stage + g * kKb) = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
}
__device__ __forceinline__ void stage_get(uint32_t (&A)[kH], const uint8_t *stage) {
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) {
    const uint4 v = *reinterpret_cast<const uint4 *>(stage + g * kKb);
    A[4 * g] = v.x; A[4 * g + 1] = v.y; A[4 * g + 2] = v.z; A[4 * g + 3] = v.w;
  }
}

// ---------------------------------------------------------------- one tile's exponentiation
// x = c * R mod m from the message row, then the constant-time fixed window
// over the prime's exponent (T[0] = R mod m, T[1] = x, T[i] = T[i-1] x; each
// window W squarings and one product by T[digit]); the q half (pi == 0) leaves
// Montgomery form, the p half stays in it for the recombination.  A is the
// thread's result.
template <int W>
__device__ __forceinline__ void exp_tile(uint32_t (&A)[kH], Tile &ts, const uint32_t *msg, uint32_t pi,
                                         const uint32_t *kc, uint8_t *stage, uint32_t stage_sa, uint4 *tbl,
                                         int r, uint32_t polls) {
  using Wn = Win<W>;
  const uint32_t *Ms = kc + kKm;
  const NSmem<kH> N{Ms};
  const uint32_t sb = ts.sb;
  constexpr int ntab = Wn::kEntries;                  // steps 2 .. ntab-1 build T[2 .. ntab-1]
  constexpr int nexp = (Wn::kNwin - 1) * (W + 1);
  const int nst = ntab + nexp + (pi == 0 ? 1 : 0);
  int k = Wn::kNwin - 2, s = 0;
#pragma unroll 1
  for (int st = 0; st < nst; ++st) {
    uint32_t bsa = stage_sa, bstr = kKb;
    bool sq = false;
    if (st == 0) {                      // c_lo * R mod m
      load_row<kH>(A, msg, true);
      bsa = sb + kOffKey + 4 * kKr2;
      bstr = 16;
    } else if (st == 1) {               // c_hi * R^2 mod m
      tbl_store<W>(tbl, 1, A);
      load_row<kH>(A, msg + kH, true);
      bsa = sb + kOffKey + 4 * kKr3;
      bstr = 16;
    } else if (st < ntab) {             // table T[i] = x^i * R, i = 2 .. ntab-1
      if (st == 2) {
        stage_from(stage, tbl + 1 * (kH / 4) * kRows, kRows);   // c_lo * R
        mod_add<kH>(A, SmemB{reinterpret_cast<const uint4 *>(stage), kKb / 16}, N);   // x R = c R mod m
        tbl_store<W>(tbl, 1, A);
        uint32_t one[kH];
        from_uniform<kH>(one, reinterpret_cast<const uint4 *>(kc + kKone));
        tbl_store<W>(tbl, 0, one);
        sq = true;                        // T[2] = x^2
      } else {
        tbl_store<W>(tbl, st - 1, A);
      }
      stage_from(stage, tbl + 1 * (kH / 4) * kRows, kRows);     // B = x R
    } else if (st < ntab + nexp) {      // windows: W squarings, then T[digit]
      if (st == ntab) {
        tbl_store<W>(tbl, ntab - 1, A);
        tbl_select<W>(stage, tbl, exp_digit<W>(kc + kKexp, (uint32_t)(Wn::kNwin - 1)));
        stage_get(A, stage);
      }
      if (s < W) {
        sq = true;
        ++s;
        if (RSAGPU_TC_PREFETCH > 0 && s == W + 1 - RSAGPU_TC_PREFETCH && ts.leader) {
          const uint4 *tb = tbl - r;   // the slot's table: one contiguous block
#pragma unroll 1
          for (int e = 0; e < Wn::kEntries; ++e)
            tc::prefetch_l2(tb + (size_t)e * (kH / 4) * kRows, (kH / 4) * kRows * 16);
        }
      } else {
        tbl_select<W>(stage, tbl, exp_digit<W>(kc + kKexp, (uint32_t)k));
        s = 0;
        --k;
      }
    } else {                            // q: leave Montgomery form
      bsa = sb + kOffKey + 4 * kKunit;
      bstr = 16;
    }
    mont_step(A, sq, bsa, bstr, ts, Ms, polls);
    if (ts.dead) break;
  }
}

// key constants of prime pi (0: q, 1: p) into shared memory
__device__ __forceinline__ void load_prime_consts(uint32_t *kc, const uint32_t *keyrec, uint32_t pi, int tid) {
  constexpr KeyLayout lay(2 * kH);
  const uint32_t om = pi ? lay.p : lay.q, or2 = pi ? lay.r2p : lay.r2q, or3 = pi ? lay.r3p : lay.r3q;
  const uint32_t oone = pi ? lay.onep : lay.oneq, oexp = pi ? lay.dp : lay.dq;
  for (int i = tid; i < kKeyWords; i += kThreads) {
    uint32_t v;
    if (i < kKr2) v = keyrec[om + i];
    else if (i < kKr3) v = keyrec[or2 + i - kKr2];
    else if (i < kKone) v = keyrec[or3 + i - kKr3];
    else if (i < kKunit) v = keyrec[oone + i - kKone];
    else if (i < kKexp) v = (i == kKunit) ? 1u : 0u;
    else v = keyrec[oexp + i - kKexp];
    kc[i] = v;
  }
}

// B images of prime pi into shared memory
__device__ __forceinline__ void load_prime_image(uint8_t *smem, const uint4 *image, uint32_t pi, int tid) {
  const uint4 *img = image + (size_t)pi * (kImgPrime / 16);
  uint4 *s4 = reinterpret_cast<uint4 *>(smem + kOffBm);
  for (int i = tid; i < (int)(kImgPrime / 16); i += kThreads) s4[i] = img[i];
}

// A tile's window table is dead once its exponentiation returns (its last
// read, the final multiplication's select, precedes that step's tile
// barriers): drop its lines from L2 instead of letting them be written back
// to DRAM; the slot's next tile writes it afresh after its own barriers.
template <int W>
__device__ __forceinline__ void drop_table(const uint4 *tbl, int r) {
  const uint4 *tb = tbl - r;   // the slot's table: one contiguous block
  if ((reinterpret_cast<uintptr_t>(tb) & 127u) == 0u) tc::discard_l2(tb, Win<W>::kTblU4 * 16u, (uint32_t)r, kRows);
}

// ---------------------------------------------------------------- exponentiation kernel (both primes)
// Uniform batches (RAGGED = false): one key; CTA 2c + pi runs prime pi, its
// four tile slots take tiles round-robin.  Ragged batches (RAGGED = true): the
// CTA repeatedly takes a work item (chunk, prime) from a counter, loads that
// key's constants and operands, and runs the chunk's tiles in its slots.
template <int W, bool RAGGED>
__device__ __forceinline__ void half_body(const HalfArgs &a, const RaggedTcArgs &ra) {
  using Wn = Win<W>;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slot = warp >> 2;                   // tile slot 0 .. kTiles-1
  const int r = ((warp & 3) << 5) | lane;       // operation within the tile = TMEM lane
  const uint32_t sb = tc::smem_addr(smem);
  uint32_t *ctrl = reinterpret_cast<uint32_t *>(smem + kOffCtrl);
  if constexpr (RAGGED) {
    // CTAs beyond the planned work items leave before touching TMEM
    if (blockIdx.x >= 2u * ra.ctl[kCtlTcChunks]) return;
  }

  if (warp == 0) tc::tmem_alloc(sb + kOffCtrl + 48, kTmemCols);
  if (tid == 0) {
    for (int t = 0; t < kTiles; ++t) tc::mbar_init(sb + kOffCtrl + 8 * t, 1u);
    tc::mbar_init_fence();
  }
  uint32_t *kc = reinterpret_cast<uint32_t *>(smem + kOffKey);
  if constexpr (!RAGGED) {
    load_prime_consts(kc, a.keyrec, blockIdx.x & 1u, tid);
    load_prime_image(smem, a.image, blockIdx.x & 1u, tid);
  }
  {
    // the constant bias A block (2^-16 = fp16 0x0100)
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
  ts.tmem = ctrl[12] + (uint32_t)slot * kTileCols;
  ts.taddr = ts.tmem + ((uint32_t)((warp & 3) * 32) << 16);
  ts.mbar = sb + kOffCtrl + 8 * slot;
  ts.phase = 0u;
  ts.pending = 2u;
  ts.bar_id = 1 + slot;
  ts.leader = (r == 0);
  ts.err = false;
  ts.dead = false;

  uint8_t *stage = smem + (ts.arow - sb) + kStageKb * kKb;   // this thread's stage (generic pointer)
  const uint32_t stage_sa = ts.arow + kStageKb * kKb;
  uint4 *tbl = (RAGGED ? static_cast<uint4 *>(ra.tables) : a.tables) +
               (size_t)(blockIdx.x * kTiles + slot) * Wn::kTblU4 + r;

  if constexpr (!RAGGED) {
    const uint32_t pi = blockIdx.x & 1u;          // 0: q, 1: p
    const uint32_t cta = blockIdx.x >> 1;
    for (uint32_t tile = cta + a.ctas_per_prime * (uint32_t)slot; tile < a.ntiles;
         tile += a.ctas_per_prime * kTiles) {
      const uint32_t row = tile * kRows + (uint32_t)r;
      const bool valid = row < a.count;
      const uint32_t *msg = a.msgs + (size_t)(valid ? row : a.count - 1) * (2 * kH);
      uint32_t A[kH];
      if (!ts.dead) exp_tile<W>(A, ts, msg, pi, kc, stage, stage_sa, tbl, r, a.wait_polls);
      drop_table<W>(tbl, r);
      if (valid) {
        uint4 *h = a.halves + (size_t)pi * (kH / 4) * a.count_pad + row;
#pragma unroll
        for (int g = 0; g < kH / 4; ++g)
          h[(size_t)g * a.count_pad] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
        a.herr[(size_t)pi * a.count + row] = (ts.err || ts.dead) ? 1u : 0u;
      }
    }
  } else {
    const uint32_t nitems = 2u * ra.ctl[kCtlTcChunks];
    const uint32_t cpad = (ra.count + 31u) & ~31u;
    uint4 *halves = static_cast<uint4 *>(ra.halves);
    uint32_t *herr = reinterpret_cast<uint32_t *>(halves + (size_t)2 * (kH / 4) * cpad);
#pragma unroll 1
    for (;;) {
      // every slot is done with the previous item's constants and operands (its
      // MMAs have completed: each slot waited for them), so they may be replaced
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) ctrl[8] = atomicAdd(&ra.ctl[kCtlTcNext], 1u);
      __syncthreads();
      const uint32_t item = ctrl[8];
      if (item >= nitems) break;
      const TcChunk ch = ra.chunks[item >> 1];
      const uint32_t pi = item & 1u;
      load_prime_consts(kc, ch.keyrec, pi, tid);
      load_prime_image(smem, static_cast<const uint4 *>(ch.image), pi, tid);
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (slot < ch.ntiles) {
        // rows past the chunk's operations (a bucket's partial last tile)
        // compute on its first operation and store nothing
        const uint32_t row = (uint32_t)slot * kRows + (uint32_t)r;
        const bool valid = row < (uint32_t)ch.nops;
        const uint32_t pos = (uint32_t)ch.op_start + (valid ? row : 0u);
        const uint32_t op = (uint32_t)ra.sorted[pos];
        const uint32_t *msg = ra.msgs + ra.offsets[op];
        uint32_t A[kH];
        if (!ts.dead) exp_tile<W>(A, ts, msg, pi, kc, stage, stage_sa, tbl, r, ra.wait_polls);
        drop_table<W>(tbl, r);
        if (valid) {
          uint4 *h = halves + (size_t)pi * (kH / 4) * cpad + pos;
#pragma unroll
          for (int g = 0; g < kH / 4; ++g)
            h[(size_t)g * cpad] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
          herr[(size_t)pi * ra.count + pos] = (ts.err || ts.dead) ? 1u : 0u;
        }
      }
    }
  }
  // a tile that gave up may still have an MMA in flight: wait for it (bounded,
  // with the full poll budget whatever the steps used) before freeing TMEM
  if (ts.leader && ts.pending < 2u) (void)tc::mbar_wait(ts.mbar, ts.pending, kWaitLimit);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(ctrl[12], kTmemCols);
  }
}

template <int W>
__global__ void __launch_bounds__(kThreads, 1) crt_tc_half_kernel(HalfArgs a) {
  half_body<W, false>(a, RaggedTcArgs{});
}
template <int W>
__global__ void __launch_bounds__(kThreads, 1) crt_tc_ragged_half_kernel(RaggedTcArgs ra) {
  half_body<W, true>(HalfArgs{}, ra);
}

// ---------------------------------------------------------------- Garner recombination
// m = m_q + q * ((m_p - m_q) * qinv mod p), one thread per operation, with the
// CIOS Montgomery product of mont.cuh (modulus p from shared memory).
constexpr int kGThreads = 256;
constexpr int kGKeyWords = (KeyLayout(2 * kH).total + 3) / 4 * 4;
constexpr int kGSmem = kGKeyWords * 4 + (kGThreads / 32) * (kH / 4) * 32 * 16;
constexpr int kRGSmem = kGKeyWords * 4 + (kRaggedGarnerThreads / 32) * (kH / 4) * 32 * 16;

// One operation: hq / hp are its m_q and m_p * R mod p (kH/4 uint4, `hstride`
// apart); ks the key record in shared memory; stage_lane the thread's slot of
// a [kH/4][32] uint4 stage.  Writes the L-limb row at orow (zeros unless ok)
// and returns the status (0, RSA_ERR_RANGE -3 or RSA_ERR_TIMEOUT -6).
__device__ __forceinline__ int32_t garner_op(const uint32_t *ks, uint4 *stage_lane, const uint4 *hq, const uint4 *hp,
                                             size_t hstride, bool timed_out, const uint32_t *mrow, uint4 *orow,
                                             bool valid) {
  constexpr int L = 2 * kH;
  constexpr KeyLayout lay(L);
  const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(ks);
  const NSmem<kH> N{ks + lay.p};
  uint32_t A[kH];
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) {
    const uint4 v = hq[(size_t)g * hstride];
    A[4 * g] = v.x; A[4 * g + 1] = v.y; A[4 * g + 2] = v.z; A[4 * g + 3] = v.w;
  }
  mont_mul<kH, 8>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.r2p), 1}, N, hd.np_p);   // m_q * R mod p
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) stage_lane[g * 32] = hp[(size_t)g * hstride];            // m_p * R mod p
  mod_rsub<kH>(A, SmemB{stage_lane, 32}, N);                                                  // (m_p - m_q) R
  mont_mul<kH, 8>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.qinv), 1}, N, hd.np_p);  // h
  uint32_t t[kH + 2];
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) {
    const uint4 v = hq[(size_t)g * hstride];
    t[4 * g] = v.x; t[4 * g + 1] = v.y; t[4 * g + 2] = v.z; t[4 * g + 3] = v.w;
  }
  t[kH] = 0u;
  t[kH + 1] = 0u;
  const uint32_t *qs = ks + lay.q;
  const bool below = row_below(mrow, ks + lay.n, L);
  const bool ok = valid && below && !timed_out;
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
  return timed_out ? -6 /* RSA_ERR_TIMEOUT */ : (below ? 0 : -3 /* RSA_ERR_RANGE */);
}

__global__ void __launch_bounds__(kGThreads) crt_tc_garner_kernel(GarnerArgs a) {
  constexpr KeyLayout lay(2 * kH);
  extern __shared__ uint4 gsm[];
  uint32_t *ks = reinterpret_cast<uint32_t *>(gsm);
  for (int i = threadIdx.x; i < kGKeyWords / 4; i += kGThreads)
    gsm[i] = (i * 4 < (int)lay.total) ? reinterpret_cast<const uint4 *>(a.keyrec)[i] : make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t row = blockIdx.x * kGThreads + threadIdx.x;
  const bool valid = row < a.count;
  const uint32_t rr = valid ? row : 0u;
  uint4 *stage_lane = gsm + kGKeyWords / 4 + warp * (kH / 4) * 32 + lane;
  const bool timed_out = a.herr[rr] != 0u || a.herr[a.count + rr] != 0u;
  const int32_t st = garner_op(ks, stage_lane, a.halves + rr, a.halves + (size_t)(kH / 4) * a.count_pad + rr,
                               a.count_pad, timed_out, a.msgs + (size_t)rr * 2 * kH,
                               reinterpret_cast<uint4 *>(a.out + (size_t)rr * 2 * kH), valid);
  if (valid && a.status) a.status[rr] = st;
}

// Ragged batches: block b takes the (chunk, slot) tiles b, b + grid, ... of the
// planned chunks; one thread per operation of the tile, the tile's key record
// in shared memory.  Timeouts are also flagged in the batch's error word.
__global__ void __launch_bounds__(kRaggedGarnerThreads) crt_tc_ragged_garner_kernel(RaggedTcArgs ra) {
  constexpr KeyLayout lay(2 * kH);
  extern __shared__ uint4 gsm[];
  uint32_t *ks = reinterpret_cast<uint32_t *>(gsm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4 *stage_lane = gsm + kGKeyWords / 4 + warp * (kH / 4) * 32 + lane;
  const uint32_t ntile_slots = (uint32_t)kTiles * ra.ctl[kCtlTcChunks];
  const uint32_t cpad = (ra.count + 31u) & ~31u;
  const uint4 *halves = static_cast<const uint4 *>(ra.halves);
  const uint32_t *herr = reinterpret_cast<const uint32_t *>(halves + (size_t)2 * (kH / 4) * cpad);
#pragma unroll 1
  for (uint32_t t = blockIdx.x; t < ntile_slots; t += gridDim.x) {
    const TcChunk ch = ra.chunks[t / kTiles];
    const int s = (int)(t % kTiles);
    if (s >= ch.ntiles) continue;   // uniform over the block
    __syncthreads();                // the previous tile's key record is no longer read
    for (int i = threadIdx.x; i < kGKeyWords / 4; i += kRaggedGarnerThreads)
      gsm[i] = (i * 4 < (int)lay.total) ? reinterpret_cast<const uint4 *>(ch.keyrec)[i] : make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const uint32_t row = (uint32_t)s * kRows + threadIdx.x;
    if (row >= (uint32_t)ch.nops) continue;   // past a partial last tile; rejoins at the next tile's barrier
    const uint32_t pos = (uint32_t)ch.op_start + row;
    const uint32_t op = (uint32_t)ra.sorted[pos];
    const size_t off = (size_t)ra.offsets[op];
    const bool timed_out = herr[pos] != 0u || herr[ra.count + pos] != 0u;
    const int32_t st = garner_op(ks, stage_lane, halves + pos, halves + (size_t)(kH / 4) * cpad + pos, cpad,
                                 timed_out, ra.msgs + off, reinterpret_cast<uint4 *>(ra.out + off), true);
    if (ra.status) ra.status[op] = st;
    if (timed_out) atomicOr(&ra.ctl[2], 1u << 6);   // RSA_ERR_TIMEOUT for rsa_sync
  }
}

// ---------------------------------------------------------------- host side
size_t tc_smem_bytes() { return (size_t)kSmem; }

int tc_grid(uint32_t count, int sm_count) {
  const uint32_t ntiles = (count + kRows - 1) / kRows;
  const uint32_t want = (ntiles + kTiles - 1) / kTiles;   // CTAs per prime so every slot has a tile
  const uint32_t per_prime =
      std::max<uint32_t>(1u, std::min<uint32_t>(want, (uint32_t)std::max(1, sm_count / 2)));
  return (int)(2 * per_prime);
}

size_t tc_tables_bytes(int grid, int window) {
  const size_t per_slot = (window == 3) ? (size_t)Win<3>::kTblU4 : (size_t)Win<4>::kTblU4;
  return (size_t)grid * kTiles * per_slot * 16;
}

static uint32_t pad_count(uint32_t count) { return (count + 31u) & ~31u; }

size_t tc_halves_bytes(uint32_t count) {
  return (size_t)2 * (kH / 4) * pad_count(count) * 16 + (size_t)2 * count * 4;
}

template <int W>
static cudaError_t launch_half(const HalfArgs &h, int grid, cudaStream_t s) {
  // set on every call: the attribute belongs to the current device's context
  cudaError_t e = cudaFuncSetAttribute(crt_tc_half_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  crt_tc_half_kernel<W><<<grid, kThreads, kSmem, s>>>(h);
  return cudaGetLastError();
}

const void *ragged_tc_half_fn(int window) {
  if (window == 3) return reinterpret_cast<const void *>(&crt_tc_ragged_half_kernel<3>);
  if (window == 4) return reinterpret_cast<const void *>(&crt_tc_ragged_half_kernel<4>);
  return nullptr;
}
const void *ragged_tc_garner_fn() { return reinterpret_cast<const void *>(&crt_tc_ragged_garner_kernel); }
size_t ragged_tc_garner_smem() { return (size_t)kRGSmem; }

cudaError_t launch_crt_tc(const uint32_t *keyrec, const void *image, const uint32_t *msgs, uint32_t *out,
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
  crt_tc_garner_kernel<<<(count + kGThreads - 1) / kGThreads, kGThreads, kGSmem, s>>>(g);
  return cudaGetLastError();
}

}  // namespace tcr
}  // namespace rsagpu
