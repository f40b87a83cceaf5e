// crt_tc4.cu -- RSA-3072 and RSA-4096 CRT decryption with the Montgomery
// reduction on the 5th-generation tensor cores (tcgen05, TMEM), for primes of
// H = 48 or 64 limbs (1536 or 2048 bits).
//
// The route is the one of crt_tc.cu (RSA-2048): M = C^d mod n as
// m_p = C^dp mod p and m_q = C^dq mod q, each a constant-time fixed-window
// exponentiation (Fig. 6 with k = W) of Montgomery products, then Garner.  A
// Montgomery product modulo a prime m of H limbs, R = 2^(32H), is done as two
// reduction rounds of r = 2^(16H) (the same value: with mu = mu1 + r mu2 < R,
// (T + mu1 m + r mu2 m) / r^2 = (T + mu m) / R).  With D = 2H byte digits per
// round:
//   1. CUDA cores: T = A * B, H x H limbs, product scanning with PTX carry
//      chains (one thread per operation); squarings add each cross product
//      once.  Limbs 0 .. H/2-1 of T leave as byte digits (fp16) in the tile's A
//      buffer, limbs H/2 .. H-1 as words in the tile's high stage, limbs
//      H .. 2H-1 stay in registers.
//   2. per round: tensor core, MMA 1: the column sums of the byte convolution
//      of (T mod r) with m' = -m^-1 mod r (D columns); CUDA cores: carry them
//      into the bytes of mu = (T mod r) m' mod r, written back as digits;
//      tensor core, MMA 2: the column sums of mu * m for positions D-4 .. 3D-5
//      (N = 2D), positions 3D-4 .. 3D-2 on the CUDA cores; CUDA cores: the carry
//      out of the low half (ceil of positions D-4 .. D-1 with T's limb H/2-1,
//      over 2^32) and T = (T + mu m) / r, the high positions carry-propagated
//      into T's limbs above r.  After round 1 the new low limbs leave as digits
//      for round 2.
//   3. one conditional subtraction of m.
// Every column of both MMAs sums at most D <= 128 products of two bytes, so
// each sum is an integer below 2^23 and reads back exactly through the bias of
// crt_tc.cu (0x3F000000 + w).
//
// Work layout: one CTA per SM (256 threads), all of one prime, two tiles of
// 128 operations with their own A buffer, high stage, 2D TMEM columns,
// mbarrier and named barrier; thread r of a tile owns operation r and TMEM
// lane r.  One thread per operation keeps H-limb numbers in registers (up to
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

constexpr int kHiG = kRows * 16;                     // group stride of a high stage: [g][row] uint4
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kBias = 0x3F000000u;
constexpr uint32_t kWaitLimit = 1u << 22;

// Sizes and the shared-memory map (bytes) of the kernel for primes of H limbs.
template <int H_>
struct Shape {
  static constexpr int H = H_;                       // limbs per prime
  static constexpr int HR = H / 2;                   // limbs per reduction round
  static constexpr int D = 2 * H;                    // byte digits per round
  static constexpr int N1 = D, N2 = 2 * D, N2First = D - 4;
  static constexpr int KS = D / 16;                  // MMA K-steps of 16 digits (without the bias block)
  static constexpr int Kb = (kRows / 8) * 128;       // k-block stride of 128-row operands (the A buffers)
  static constexpr int Kb1 = (N1 / 8) * 128, Kb2 = (N2 / 8) * 128;
  static constexpr int ImgB1 = (int)img_b1_bytes(H), ImgB2 = (int)img_b2_bytes(H);
  static constexpr int OffB1 = 0;
  static constexpr int OffB2 = OffB1 + ImgB1;
  static constexpr int OffAbias = OffB2 + ImgB2;     // 128 x 16 bias A operand
  static constexpr int OffA = (OffAbias + kRows * 16 * 2 + 127) / 128 * 128;
  static constexpr int ABytes = kRows * D * 2;
  static constexpr int OffHi = OffA + kTiles * ABytes;
  static constexpr int HiGroups = HR / 4;
  static constexpr int HiBytes = HiGroups * kHiG;
  static constexpr int OffKey = OffHi + kTiles * HiBytes;
  // key constants (words): m, R^2, R^3, R mod m, unit, exponent (H + 4 limbs)
  static constexpr int Km = 0, Kr2 = H, Kr3 = 2 * H, Kone = 3 * H, Kunit = 4 * H, Kexp = 5 * H;
  static constexpr int KeyWords = 6 * H + 4;
  static constexpr int OffCtrl = OffKey + KeyWords * 4;   // kTiles mbarriers (8 B each), TMEM base at +48
  static constexpr int Smem = OffCtrl + 64;
  static constexpr int StageKb = KS;                 // B limbs 0 .. HR-1: k-blocks KS .. 2KS-1 of the A row
  static constexpr int NX = 3 * HR;                  // X: the value's limbs HR .. 2H-1
  static constexpr uint32_t TileCols = N2;
  static constexpr uint32_t Idesc1 = tc::idesc_f16_f32(128, N1);
  static constexpr uint32_t Idesc2 = tc::idesc_f16_f32(128, N2);
  static_assert(OffB2 % 16 == 0 && OffAbias % 16 == 0 && OffHi % 16 == 0 && OffKey % 16 == 0 && OffCtrl % 8 == 0,
                "layout");
  static_assert(Smem <= 227 * 1024, "shared memory");
  static_assert(kTiles * TileCols <= kTmemCols, "TMEM");
  static_assert(HR % 8 == 0 && D % 16 == 0 && N2 <= 256, "shape");
};

template <int H, int W>
struct Win {
  static constexpr int kEntries = 1 << W;
  static constexpr int kNwin = (32 * H + W - 1) / W;             // windows of the prime-size exponent
  static constexpr int kTblU4 = kEntries * (H / 4) * kRows;      // uint4 per tile slot: [entry][g][row]
};

struct Tile {
  uint32_t sb, arow, abuf, hrow, tmem, taddr, mbar, phase, pending;
  int bar_id;
  bool leader, err, dead;
};

// MMA 1 (N = D, B1 = Toeplitz of m') or MMA 2 (N = 2D, B2 = Toeplitz of m):
// the bias block, then D/16 K-steps of 16 digits, then the commit; leader only.
template <int H>
__device__ __forceinline__ void issue_mma(const Tile &ts, bool second) {
  using S = Shape<H>;
  const uint32_t boff = second ? S::OffB2 : S::OffB1;
  const uint32_t bkb = second ? S::Kb2 : S::Kb1;
  const uint32_t idesc = second ? S::Idesc2 : S::Idesc1;
  tc::fence_after_sync();
  tc::mma_f16(ts.tmem, tc::sdesc(ts.sb + S::OffAbias, S::Kb, 128), tc::sdesc(ts.sb + boff + 2 * S::KS * bkb, bkb, 128),
              idesc, 0u);
#pragma unroll 1
  for (int s = 0; s < S::KS; ++s)
    tc::mma_f16(ts.tmem, tc::sdesc(ts.abuf + s * 2 * S::Kb, S::Kb, 128), tc::sdesc(ts.sb + boff + s * 2 * bkb, bkb, 128),
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

// X[j0 .. j0+NL) += the 4*NL column words v taken as 2*NL base-2^16 columns
// (tc::lo_halves / tc::hi_halves): s = X' + Y' word by word with the carry
// cs, then X += s with the carry cin.  yb is the column below v[0] (its high
// half, the pending carry, enters word j0); the last column of v returns in yb.
template <int NL, int NX>
__device__ __forceinline__ void add_columns(uint32_t (&X)[NX], int j0, const uint32_t *v, uint32_t &yb, uint32_t &cs,
                                            uint32_t &cin) {
  uint32_t s[NL];
  (void)add_cc(cs, 0xFFFFFFFFu);    // carry flag <- cs (0 or 1)
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const uint32_t y0 = tc::pair_cols(v[4 * i], v[4 * i + 1]), y1 = tc::pair_cols(v[4 * i + 2], v[4 * i + 3]);
    s[i] = addc_cc(tc::lo_halves(y0, y1), tc::hi_halves(yb, y0));
    yb = y1;
  }
  cs = addc(0u, 0u);
  (void)add_cc(cin, 0xFFFFFFFFu);   // carry flag <- cin
#pragma unroll
  for (int i = 0; i < NL; ++i) X[j0 + i] = addc_cc(X[j0 + i], s[i]);
  cin = addc(0u, 0u);
}

// MMA 1's columns (TMEM columns 0 .. D-1) summed into mu's D digits (32-bit
// words from tc::lo_halves / tc::hi_halves, one carry chain), written into the
// tile's A buffer; returns mu's digits D-4 .. D-1.
template <int H>
__device__ __forceinline__ uint32_t mu_pass(const Tile &ts) {
  using S = Shape<H>;
  uint32_t mu_top = 0u, yb = 0u, cw = 0u;
#pragma unroll 1
  for (int c0 = 0; c0 < S::D; c0 += 16) {
    uint32_t v[16];
    tc::ld16(ts.taddr + (uint32_t)c0, v);
    tc::wait_ld();
    uint32_t y[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) y[j] = tc::pair_cols(v[2 * j], v[2 * j + 1]);
    uint32_t w[4];
    (void)add_cc(cw, 0xFFFFFFFFu);   // carry flag <- cw
#pragma unroll
    for (int k = 0; k < 4; ++k)
      w[k] = addc_cc(tc::lo_halves(y[2 * k], y[2 * k + 1]), tc::hi_halves(k ? y[2 * k - 1] : yb, y[2 * k]));
    cw = addc(0u, 0u);
    yb = y[7];
    const uint32_t ad = ts.arow + (uint32_t)(c0 >> 3) * S::Kb;
    tc::sts128(ad, tc::prmt(w[0], 0u, 0x4140u), tc::prmt(w[0], 0u, 0x4342u), tc::prmt(w[1], 0u, 0x4140u),
               tc::prmt(w[1], 0u, 0x4342u));
    tc::sts128(ad + S::Kb, tc::prmt(w[2], 0u, 0x4140u), tc::prmt(w[2], 0u, 0x4342u), tc::prmt(w[3], 0u, 0x4140u),
               tc::prmt(w[3], 0u, 0x4342u));
    mu_top = w[3];   // in the last chunk: digits D-4 .. D-1
  }
  return mu_top;
}

// Positions 3D-4 .. 3D-1 of mu * m from mu's digits D-3 .. D-1 and m's top
// limb (six byte products), as column words with the bias.
__device__ __forceinline__ void top_columns(uint32_t (&tcol)[4], uint32_t mu_top, uint32_t mt) {
  const uint32_t a5 = (mu_top >> 8) & 0xFFu, a6 = (mu_top >> 16) & 0xFFu, a7 = mu_top >> 24;
  const uint32_t b5 = (mt >> 8) & 0xFFu, b6 = (mt >> 16) & 0xFFu, b7 = mt >> 24;
  tcol[0] = kBias + a5 * b7 + a6 * b6 + a7 * b5;
  tcol[1] = kBias + a6 * b7 + a7 * b6;
  tcol[2] = kBias + a7 * b7;
  tcol[3] = kBias;
}

// One reduction round on the value V whose limbs 0 .. HR-1 are in the A
// buffer as digits (limb HR-1 also in `top`) and whose limbs from HR up are in
// X: mu = (V mod r) m' mod r, then X[B0 .. B0+H) += positions D .. 3D-1 of
// mu * m with the carry out of the low half; returns the carry out of
// X[B0 + H - 1] (column carry + limb carry), for the caller to place.
template <int H, int B0, int NX>
__device__ __forceinline__ uint32_t reduce_round(uint32_t (&X)[NX], uint32_t top, Tile &ts, const uint32_t *Ms,
                                                 uint32_t polls) {
  using S = Shape<H>;
  if (tile_sync(ts)) return 0u;
  if (ts.leader) issue_mma<H>(ts, false);
  wait_mma(ts, polls);
  const uint32_t mu_top = mu_pass<H>(ts);
  if (tile_sync(ts)) return 0u;
  if (ts.leader) issue_mma<H>(ts, true);
  uint32_t tcol[4];
  top_columns(tcol, mu_top, Ms[H - 1]);   // while the tensor core works
  wait_mma(ts, polls);
  uint32_t yb, cs = 0u, cin = 0u;
  {
    uint32_t v[16];
    tc::ld16(ts.taddr + 0u, v);   // positions D-4 .. D+11
    tc::wait_ld();
    // carry out of the low half: ceil of positions D-4 .. D-1 (with V's limb
    // HR-1) / 2^32, below 2^16; it enters as the high half of the column below
    const uint32_t y0 = tc::pair_cols(v[0], v[1]) + (top & 0xFFFFu);
    const uint32_t y1 = tc::pair_cols(v[2], v[3]) + (top >> 16) + (y0 >> 16);
    yb = ((y1 >> 16) + (((y0 | y1) & 0xFFFFu) != 0u ? 1u : 0u)) << 16;
    add_columns<3>(X, B0, v + 4, yb, cs, cin);            // positions D .. D+11
  }
#pragma unroll
  for (int k = 1; k < S::N2 / 16; ++k) {
    uint32_t v[16];
    tc::ld16(ts.taddr + (uint32_t)(16 * k), v);           // positions D-4 + 16k .. +15
    tc::wait_ld();
    add_columns<4>(X, B0 + 3 + 4 * (k - 1), v, yb, cs, cin);
  }
  tc::fence_before_sync();   // this tile's TMEM reads precede its next MMA (ordered by the next barrier)
  add_columns<1>(X, B0 + H - 1, tcol, yb, cs, cin);      // positions 3D-4 .. 3D-1
  return (yb >> 16) + cs + cin;
}

// ---------------------------------------------------------------- squaring
// T = A^2 with A = a_lo + a_hi r (r = 2^(32 HR), halves of HR = H/2 limbs):
// T = a_lo^2 + 2 P r + a_hi^2 r^2, P = a_lo a_hi.  The cross product P runs
// as a rolled loop of product rows (a_lo read back from the thread's high
// stage, a_hi in registers); the half squares compute each of their cross
// products once (square_emit).  T's limbs come out in increasing order:
// 0 .. HR-1 from a_lo^2 alone (digits into the A buffer), HR .. H-1 =
// a_lo^2's high half + 2 P_lo (high stage), H .. 2H-1 = a_hi^2 + 2 P_hi (t).
// Word products: HR^2 + 2 HR(HR+1)/2 = H(H+1)/2, as for a square in one
// piece, in about half the code (the unrolled rows of two HR-limb squares
// and one rolled row loop, instead of the rows of an H-limb square).
__device__ __forceinline__ uint32_t lds32(uint32_t saddr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr) : "memory");
  return v;
}
__device__ __forceinline__ void sts32(uint32_t saddr, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}

// a_lo^2's limbs p: below HR they are T's final limbs (digits; limb HR-1 also
// in `top`), from HR on they add 2 P_lo (P_lo in the high stage, doubled as it
// is read: word k of 2P is P_k << 1 with P_(k-1)'s top bit) and replace it
// there as T's limbs.  `carry` and `pprev` continue into the next emitter.
template <int H>
struct LowEmit {
  const Tile &ts;
  uint32_t top, carry, pprev;
  template <int P>
  __device__ __forceinline__ void put(uint32_t v) {
    using S = Shape<H>;
    if constexpr (P < S::HR) {
      tc::emit_digits(ts.arow, P, v, S::Kb);
      if constexpr (P == S::HR - 1) top = v;
    } else {
      constexpr int k = P - S::HR;
      const uint32_t ad = ts.hrow + (uint32_t)(k >> 2) * kHiG + (uint32_t)(k & 3) * 4u;
      const uint32_t pk = lds32(ad);
      const uint32_t d = __funnelshift_l(pprev, pk, 1);
      pprev = pk;
      (void)add_cc(carry, 0xFFFFFFFFu);   // carry flag <- carry
      const uint32_t w = addc_cc(v, d);
      carry = addc(0u, 0u);
      sts32(ad, w);
    }
  }
};

// a_hi^2's limbs p become T's limbs H + p in t: plus 2 P_hi (acc = P_hi; word
// p of it takes the top bit of the word below, P_lo's last word for p = 0),
// plus the carry out of the limbs below.
template <int H>
struct HighEmit {
  uint32_t (&t)[H];
  const uint32_t (&acc)[H / 2];
  uint32_t carry, plast;
  template <int P>
  __device__ __forceinline__ void put(uint32_t v) {
    constexpr int HR = H / 2;
    uint32_t d = 0u;
    if constexpr (P == 0) d = __funnelshift_l(plast, acc[0], 1);
    else if constexpr (P < HR) d = __funnelshift_l(acc[P - 1], acc[P], 1);
    else if constexpr (P == HR) d = acc[HR - 1] >> 31;
    (void)add_cc(carry, 0xFFFFFFFFu);   // carry flag <- carry
    t[P] = addc_cc(v, d);
    carry = addc(0u, 0u);
  }
};

// T = A^2 into the A buffer (limbs 0 .. HR-1 as digits), the high stage
// (HR .. H-1) and t (H .. 2H-1); returns limb HR-1.  The high stage is free:
// a squaring has no B operand.
template <int H>
__device__ __forceinline__ uint32_t square(uint32_t (&t)[H], const uint32_t (&a)[H], const Tile &ts) {
  constexpr int HR = H / 2;
  static_assert(HR % 4 == 0, "halves of whole limb groups");
  uint32_t alo[HR], ahi[HR];
#pragma unroll
  for (int j = 0; j < HR; ++j) {
    alo[j] = a[j];
    ahi[j] = a[HR + j];
  }
  // 1. P = a_lo a_hi: a_lo to the high stage, then rows of four limbs of
  //    a_lo (read back) times a_hi; each row group's four emitted limbs of P
  //    replace the four a_lo limbs it read
#pragma unroll
  for (int g = 0; g < HR / 4; ++g)
    tc::sts128(ts.hrow + (uint32_t)g * kHiG, alo[4 * g], alo[4 * g + 1], alo[4 * g + 2], alo[4 * g + 3]);
  uint32_t acc[HR];
#pragma unroll
  for (int j = 0; j < HR; ++j) acc[j] = 0u;
#pragma unroll 1
  for (int g = 0; g < HR / 4; ++g) {
    const uint32_t ad = ts.hrow + (uint32_t)g * kHiG;
    const uint4 b = tc::lds128(ad);
    const uint32_t e0 = mul_emit<HR>(acc, ahi, b.x);
    const uint32_t e1 = mul_emit<HR>(acc, ahi, b.y);
    const uint32_t e2 = mul_emit<HR>(acc, ahi, b.z);
    const uint32_t e3 = mul_emit<HR>(acc, ahi, b.w);
    tc::sts128(ad, e0, e1, e2, e3);
  }
  // 2. a_lo^2 with 2 P_lo: T's limbs 0 .. H-1
  LowEmit<H> lo{ts, 0u, 0u, 0u};
  square_emit<HR>(alo, lo);
  // 3. a_hi^2 with 2 P_hi and the carry: T's limbs H .. 2H-1 (T < 2^(64H): no carry out)
  HighEmit<H> hi{t, acc, lo.carry, lo.pprev};
  square_emit<HR>(ahi, hi);
  return lo.top;
}

// ---------------------------------------------------------------- one Montgomery step
// A = A * B * R^-1 mod m (A < m, B < m).  B: H limbs in shared memory, groups
// 0 .. HR/4-1 at lo + g*lo_str, the others at hi + (g - HR/4)*hi_str (the
// thread's stage, or a key constant); sq: B = A.
template <int H>
__device__ __forceinline__ void mont_step(uint32_t (&A)[H], bool sq, uint32_t lo, uint32_t lo_str, uint32_t hi,
                                          uint32_t hi_str, Tile &ts, const uint32_t *Ms, uint32_t polls) {
  using S = Shape<H>;
  constexpr int HR = S::HR, LG = S::HR / 4;
  // 1. T = A * B: limbs 0 .. HR-1 leave as digits (A buffer), HR .. H-1 as
  //    words (high stage), H .. 2H-1 stay in t.  Block i0 reads B limbs
  //    i0 .. i0+7 before it writes anything: a digit of T limb p >= HR/2 lands
  //    on B limbs 2p-HR, 2p-HR+1 of the stage and a word of T limb p >= HR on
  //    B limbs p - p%4 .. +3, all read by this block or an earlier one.
  uint32_t t[H];
#pragma unroll
  for (int j = 0; j < H; ++j) t[j] = 0u;
  uint32_t top = 0u;
  if (sq) top = square<H>(t, A, ts);
#pragma unroll 1
  for (int i0 = 0; i0 < (sq ? 0 : H); i0 += 8) {
    const uint32_t g = (uint32_t)(i0 >> 2);
    const uint32_t a0 = g < LG ? lo + g * lo_str : hi + (g - LG) * hi_str;
    const uint32_t a1 = g + 1 < LG ? lo + (g + 1) * lo_str : hi + (g + 1 - LG) * hi_str;
    const uint4 b0 = tc::lds128(a0), b1 = tc::lds128(a1);
    uint32_t e[8];
    e[0] = mul_emit<H>(t, A, b0.x);
    e[1] = mul_emit<H>(t, A, b0.y);
    e[2] = mul_emit<H>(t, A, b0.z);
    e[3] = mul_emit<H>(t, A, b0.w);
    e[4] = mul_emit<H>(t, A, b1.x);
    e[5] = mul_emit<H>(t, A, b1.y);
    e[6] = mul_emit<H>(t, A, b1.z);
    e[7] = mul_emit<H>(t, A, b1.w);
    if (i0 < HR) {
      // limbs i0..i0+7 are digits 4*i0 .. 4*i0+31: k-blocks i0/2 .. i0/2+3
      const uint32_t ad = ts.arow + (uint32_t)(i0 >> 1) * S::Kb;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        tc::sts128(ad + q * S::Kb, tc::prmt(e[2 * q], 0u, 0x4140u), tc::prmt(e[2 * q], 0u, 0x4342u),
                   tc::prmt(e[2 * q + 1], 0u, 0x4140u), tc::prmt(e[2 * q + 1], 0u, 0x4342u));
      top = e[7];   // after the block i0 = HR - 8: limb HR - 1
    } else {
      const uint32_t ad = ts.hrow + (uint32_t)((i0 - HR) >> 2) * kHiG;
      tc::sts128(ad, e[0], e[1], e[2], e[3]);
      tc::sts128(ad + kHiG, e[4], e[5], e[6], e[7]);
    }
  }
  // 2. round 1: X holds T's limbs HR .. 2H-1 (the first HR read back from the high stage)
  uint32_t X[S::NX];
#pragma unroll
  for (int g = 0; g < LG; ++g) {
    const uint4 v = tc::lds128(ts.hrow + (uint32_t)g * kHiG);
    X[4 * g] = v.x; X[4 * g + 1] = v.y; X[4 * g + 2] = v.z; X[4 * g + 3] = v.w;
  }
#pragma unroll
  for (int j = 0; j < H; ++j) X[HR + j] = t[j];
  const uint32_t c1 = reduce_round<H, 0>(X, top, ts, Ms, polls);
  if (ts.dead) return;
  // the carry into T1's limbs H .. 3HR-1 (X[H .. NX)); T1 may carry one bit past them
  X[H] = add_cc(X[H], c1);
#pragma unroll
  for (int j = H + 1; j < S::NX; ++j) X[j] = addc_cc(X[j], 0u);
  const uint32_t xtop = addc(0u, 0u);
  // T1's limbs 0 .. HR-1 leave as digits for round 2 (mu1's digits are no longer read)
#pragma unroll
  for (int p = 0; p < HR; ++p) tc::emit_digits(ts.arow, p, X[p], S::Kb);
  // 3. round 2: X[HR .. NX) += positions D .. 3D-1 of mu2 * m; T2 = X[HR .. NX) and the top word
  const uint32_t c2 = reduce_round<H, HR>(X, X[HR - 1], ts, Ms, polls);
  if (ts.dead) return;
  uint32_t u[H + 2];
#pragma unroll
  for (int j = 0; j < H; ++j) u[j] = X[HR + j];
  u[H] = c2 + xtop;
  u[H + 1] = 0u;
  final_sub<H>(A, u, NSmem<H>{Ms});
}

// ---------------------------------------------------------------- table and stage helpers
// Table of one tile slot in global memory: [entry][g][row] of uint4 (g = limb / 4).
template <int H>
__device__ __forceinline__ void tbl_store(uint4 *tbl, int e, const uint32_t (&A)[H]) {
#pragma unroll
  for (int g = 0; g < H / 4; ++g)
    tbl[(e * (H / 4) + g) * kRows] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
}
// group g of the thread's stage: limbs 0 .. HR-1 in the upper k-blocks of its A row, the rest in its high stage
template <int H>
__device__ __forceinline__ uint4 *stage_group(uint8_t *smem, const Tile &ts, int g) {
  using S = Shape<H>;
  const uint32_t a = g < S::HR / 4 ? ts.arow + (uint32_t)(S::StageKb + g) * S::Kb
                                   : ts.hrow + (uint32_t)(g - S::HR / 4) * kHiG;
  return reinterpret_cast<uint4 *>(smem + (a - ts.sb));
}
// stage <- T[d], reading every entry (constant time)
template <int H, int W>
__device__ __forceinline__ void tbl_select(uint8_t *smem, const Tile &ts, const uint4 *tbl, uint32_t d) {
#pragma unroll 1
  for (int g0 = 0; g0 < H / 4; g0 += 2) {
    uint4 acc[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) acc[u] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int e = 0; e < (1 << W); ++e) {
      const uint32_t msk = 0u - (uint32_t)((uint32_t)e == d);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const uint4 v = tbl[(e * (H / 4) + g0 + u) * kRows];
        acc[u].x |= v.x & msk;
        acc[u].y |= v.y & msk;
        acc[u].z |= v.z & msk;
        acc[u].w |= v.w & msk;
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) *stage_group<H>(smem, ts, g0 + u) = acc[u];
  }
}
template <int H>
__device__ __forceinline__ void stage_from_table(uint8_t *smem, const Tile &ts, const uint4 *entry) {
#pragma unroll
  for (int g = 0; g < H / 4; ++g) *stage_group<H>(smem, ts, g) = entry[g * kRows];
}
template <int H>
__device__ __forceinline__ void stage_get(uint32_t (&A)[H], uint8_t *smem, const Tile &ts) {
#pragma unroll
  for (int g = 0; g < H / 4; ++g) {
    const uint4 v = *stage_group<H>(smem, ts, g);
    A[4 * g] = v.x; A[4 * g + 1] = v.y; A[4 * g + 2] = v.z; A[4 * g + 3] = v.w;
  }
}

// ---------------------------------------------------------------- one tile's exponentiation
// x = c R mod m from the 2H-limb message row (c_lo R^2 R^-1 + c_hi R^3 R^-1),
// then the constant-time fixed window over the prime's exponent (squarings by
// `square`, products with the staged B).  The q half (pi == 0) leaves
// Montgomery form.
template <int H, int W>
__device__ __forceinline__ void exp_tile(uint32_t (&A)[H], Tile &ts, uint8_t *smem, const uint32_t *msg, uint32_t pi,
                                         const uint32_t *kc, uint4 *tbl, uint32_t polls) {
  using S = Shape<H>;
  using Wn = Win<H, W>;
  const uint32_t *Ms = kc + S::Km;
  const NSmem<H> N{Ms};
  const uint32_t kca = ts.sb + S::OffKey;   // key constants: groups at 16-byte stride
  const uint32_t slo = ts.arow + S::StageKb * S::Kb, shi = ts.hrow;
  constexpr int ntab = Wn::kEntries;
  constexpr int nexp = (Wn::kNwin - 1) * (W + 1);
  const int nst = ntab + nexp + (pi == 0 ? 1 : 0);
  int k = Wn::kNwin - 2, s = 0;
#pragma unroll 1
  for (int st = 0; st < nst; ++st) {
    uint32_t lo = slo, lo_str = S::Kb, hi = shi, hi_str = kHiG;
    bool sq = false;
    if (st == 0) {                      // c_lo * R mod m
      load_row<H>(A, msg, true);
      lo = kca + 4 * S::Kr2; lo_str = 16; hi = lo + 16 * (S::HR / 4); hi_str = 16;
    } else if (st == 1) {               // c_hi * R^2 mod m
      tbl_store<H>(tbl, 1, A);
      load_row<H>(A, msg + H, true);
      lo = kca + 4 * S::Kr3; lo_str = 16; hi = lo + 16 * (S::HR / 4); hi_str = 16;
    } else if (st < ntab) {             // table T[i] = x^i R, i = 2 .. ntab-1
      if (st == 2) {
        mod_add<H>(A, SmemB{tbl + 1 * (H / 4) * kRows, kRows}, N);   // x R = c_hi R^2 + c_lo R
        tbl_store<H>(tbl, 1, A);
        uint32_t one[H];
        from_uniform<H>(one, reinterpret_cast<const uint4 *>(kc + S::Kone));
        tbl_store<H>(tbl, 0, one);
        sq = true;                      // T[2] = x^2
      } else {
        tbl_store<H>(tbl, st - 1, A);
        stage_from_table<H>(smem, ts, tbl + 1 * (H / 4) * kRows);   // B = x R
      }
    } else if (st < ntab + nexp) {      // windows: W squarings, then T[digit]
      if (st == ntab) {
        tbl_store<H>(tbl, ntab - 1, A);
        tbl_select<H, W>(smem, ts, tbl, exp_digit<W>(kc + S::Kexp, (uint32_t)(Wn::kNwin - 1)));
        stage_get<H>(A, smem, ts);
      }
      if (s < W) {
        sq = true;
        ++s;
      } else {
        tbl_select<H, W>(smem, ts, tbl, exp_digit<W>(kc + S::Kexp, (uint32_t)k));
        s = 0;
        --k;
      }
    } else {                            // q: leave Montgomery form
      lo = kca + 4 * S::Kunit; lo_str = 16; hi = lo + 16 * (S::HR / 4); hi_str = 16;
    }
    mont_step<H>(A, sq, lo, lo_str, hi, hi_str, ts, Ms, polls);
    if (ts.dead) break;
  }
}

// A tile's window table (or the public path's multiplier slot) is dead once
// its exponentiation returns: its last read precedes that step's tile
// barriers.  Drop its lines from L2 instead of letting them be written back
// to DRAM; the slot's next tile writes it afresh after its own barriers.
__device__ __forceinline__ void drop_slot(const uint4 *tbl, int r, uint32_t u4) {
  const uint4 *tb = tbl - r;   // the slot's block
  if ((reinterpret_cast<uintptr_t>(tb) & 127u) == 0u) tc::discard_l2(tb, u4 * 16u, (uint32_t)r, kRows);
}

// ---------------------------------------------------------------- exponentiation kernel (both primes)
struct HalfArgs {
  const uint32_t *keyrec;
  const uint4 *image;       // [prime][B1 | B2], prime 0 = q, 1 = p
  const uint32_t *msgs;     // count rows of 2H limbs
  uint4 *halves;            // [prime][H/4][count_pad]: q -> m_q, p -> m_p * R mod p
  uint32_t *herr;           // [prime][count]: 1 if a bounded wait gave up
  uint4 *tables;            // [grid * kTiles][kTblU4]
  uint32_t count, count_pad, ntiles, ctas_per_prime;
  uint32_t wait_polls;
};

// key constants of prime pi (0: q, 1: p) and its two B operands into shared memory
template <int H>
__device__ __forceinline__ void load_prime(uint8_t *smem, const uint32_t *keyrec, const uint4 *image, uint32_t pi,
                                           int tid) {
  using S = Shape<H>;
  constexpr KeyLayout lay(2 * H);
  uint32_t *kc = reinterpret_cast<uint32_t *>(smem + S::OffKey);
  const uint32_t om = pi ? lay.p : lay.q, or2 = pi ? lay.r2p : lay.r2q, or3 = pi ? lay.r3p : lay.r3q;
  const uint32_t oone = pi ? lay.onep : lay.oneq, oexp = pi ? lay.dp : lay.dq;
  for (int i = tid; i < S::KeyWords; i += kThreads) {
    uint32_t v;
    if (i < S::Kr2) v = keyrec[om + i];
    else if (i < S::Kr3) v = keyrec[or2 + i - S::Kr2];
    else if (i < S::Kone) v = keyrec[or3 + i - S::Kr3];
    else if (i < S::Kunit) v = keyrec[oone + i - S::Kone];
    else if (i < S::Kexp) v = (i == S::Kunit) ? 1u : 0u;
    else v = keyrec[oexp + i - S::Kexp];
    kc[i] = v;
  }
  constexpr int img_u4 = (S::ImgB1 + S::ImgB2) / 16;
  const uint4 *img = image + (size_t)pi * img_u4;
  uint4 *s4 = reinterpret_cast<uint4 *>(smem + S::OffB1);
  for (int i = tid; i < img_u4; i += kThreads) s4[i] = img[i];
}

// Uniform batches (RAGGED = false): one key; CTA 2c + pi runs prime pi, its two
// tile slots take tiles round-robin.  Ragged batches (RAGGED = true): the CTA
// repeatedly takes a work item (chunk, prime) from the counter
// ctl[ra.ctl_word + 1], loads that key's constants and operands, and runs the
// chunk's tiles (up to two) in its slots.
template <int H, int W, bool RAGGED>
__device__ __forceinline__ void half_body(const HalfArgs &a, const tcr::RaggedTcArgs &ra) {
  using S = Shape<H>;
  using Wn = Win<H, W>;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slot = warp >> 2;
  const int r = ((warp & 3) << 5) | lane;
  const uint32_t sb = tc::smem_addr(smem);
  uint32_t *ctrl = reinterpret_cast<uint32_t *>(smem + S::OffCtrl);
  if constexpr (RAGGED) {
    // CTAs beyond the planned work items leave before touching TMEM
    if (blockIdx.x >= 2u * ra.ctl[ra.ctl_word]) return;
  }

  if (warp == 0) tc::tmem_alloc(sb + S::OffCtrl + 48, kTmemCols);
  if (tid == 0) {
    for (int t = 0; t < kTiles; ++t) tc::mbar_init(sb + S::OffCtrl + 8 * t, 1u);
    tc::mbar_init_fence();
  }
  uint32_t *kc = reinterpret_cast<uint32_t *>(smem + S::OffKey);
  if constexpr (!RAGGED) load_prime<H>(smem, a.keyrec, a.image, blockIdx.x & 1u, tid);
  {
    uint4 *ab = reinterpret_cast<uint4 *>(smem + S::OffAbias);
    for (int i = tid; i < kRows * 16 * 2 / 16; i += kThreads)
      ab[i] = make_uint4(0x01000100u, 0x01000100u, 0x01000100u, 0x01000100u);
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  Tile ts;
  ts.sb = sb;
  ts.abuf = sb + S::OffA + slot * S::ABytes;
  ts.arow = ts.abuf + (uint32_t)(r >> 3) * 128 + (uint32_t)(r & 7) * 16;
  ts.hrow = sb + S::OffHi + slot * S::HiBytes + (uint32_t)r * 16;
  ts.tmem = ctrl[12] + (uint32_t)slot * S::TileCols;
  ts.taddr = ts.tmem + ((uint32_t)((warp & 3) * 32) << 16);
  ts.mbar = sb + S::OffCtrl + 8 * slot;
  ts.phase = 0u;
  ts.pending = 2u;
  ts.bar_id = 1 + slot;
  ts.leader = (r == 0);
  ts.err = false;
  ts.dead = false;
  uint4 *tbl = (RAGGED ? static_cast<uint4 *>(ra.tables) : a.tables) + (size_t)(blockIdx.x * kTiles + slot) * Wn::kTblU4 + r;

  if constexpr (!RAGGED) {
    const uint32_t pi = blockIdx.x & 1u;
    const uint32_t cta = blockIdx.x >> 1;
    for (uint32_t tile = cta + a.ctas_per_prime * (uint32_t)slot; tile < a.ntiles;
         tile += a.ctas_per_prime * kTiles) {
      const uint32_t row = tile * kRows + (uint32_t)r;
      const bool valid = row < a.count;
      const uint32_t *msg = a.msgs + (size_t)(valid ? row : a.count - 1) * (2 * H);
      uint32_t A[H];
      if (!ts.dead) exp_tile<H, W>(A, ts, smem, msg, pi, kc, tbl, a.wait_polls);
      drop_slot(tbl, r, Wn::kTblU4);
      if (valid) {
        uint4 *h = a.halves + (size_t)pi * (H / 4) * a.count_pad + row;
#pragma unroll
        for (int g = 0; g < H / 4; ++g)
          h[(size_t)g * a.count_pad] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
        a.herr[(size_t)pi * a.count + row] = (ts.err || ts.dead) ? 1u : 0u;
      }
    }
  } else {
    const uint32_t nitems = 2u * ra.ctl[ra.ctl_word];
    const uint32_t cpad = (ra.count + 31u) & ~31u;
    uint4 *halves = static_cast<uint4 *>(ra.halves);
    uint32_t *herr = reinterpret_cast<uint32_t *>(halves + (size_t)2 * (H / 4) * cpad);
#pragma unroll 1
    for (;;) {
      // every slot is done with the previous item's constants and operands
      // (its MMAs have completed: each slot waited for them)
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) ctrl[8] = atomicAdd(&ra.ctl[ra.ctl_word + 1], 1u);
      __syncthreads();
      const uint32_t item = ctrl[8];
      if (item >= nitems) break;
      const tcr::TcChunk ch = ra.chunks[item >> 1];
      const uint32_t pi = item & 1u;
      load_prime<H>(smem, ch.keyrec, static_cast<const uint4 *>(ch.image), pi, tid);
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
        uint32_t A[H];
        if (!ts.dead) exp_tile<H, W>(A, ts, smem, msg, pi, kc, tbl, ra.wait_polls);
        drop_slot(tbl, r, Wn::kTblU4);
        if (valid) {
          uint4 *h = halves + (size_t)pi * (H / 4) * cpad + pos;
#pragma unroll
          for (int g = 0; g < H / 4; ++g)
            h[(size_t)g * cpad] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
          herr[(size_t)pi * ra.count + pos] = (ts.err || ts.dead) ? 1u : 0u;
        }
      }
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

template <int H, int W>
__global__ void __launch_bounds__(kThreads, 1) crt_tc4_half_kernel(HalfArgs a) {
  half_body<H, W, false>(a, tcr::RaggedTcArgs{});
}
template <int H, int W>
__global__ void __launch_bounds__(kThreads, 1) crt_tc4_ragged_half_kernel(tcr::RaggedTcArgs ra) {
  half_body<H, W, true>(HalfArgs{}, ra);
}

// ---------------------------------------------------------------- public exponent of 2048-bit keys
// C = M^e mod n for a 2048-bit n: the modulus has the shape of an RSA-4096
// prime (H = 64 limbs), so every Montgomery product mod n (R = 2^2048) runs
// the same two reduction rounds on the tensor cores.  e is the key's public
// exponent, the same for every operation and not secret: left-to-right binary
// method (Fig. 5) over its bits below the top one.  One CTA per SM, the key's
// n operands loaded once; tiles round-robin over the CTAs' two slots.
struct PubArgs {
  const uint32_t *keyrec;   // the key record (an L = H-limb key)
  const uint4 *image;       // n's two B operands (build_tc4_image)
  const uint32_t *msgs;     // count rows of H limbs
  uint32_t *out;            // count rows of H limbs
  int32_t *status;          // per operation (may be null)
  uint4 *tables;            // [grid * kTiles][H/4][kRows]: the multiplier x R per tile slot
  uint32_t count, ntiles, wait_polls;
};

// key constants of n (Km: n, Kr2: R^2 mod n, Kone: R mod n, Kunit: 1, Kexp: e)
// and its two B operands into shared memory
template <int H>
__device__ __forceinline__ void load_modulus(uint8_t *smem, const uint32_t *keyrec, const uint4 *image, int tid) {
  using S = Shape<H>;
  constexpr KeyLayout lay(H);
  uint32_t *kc = reinterpret_cast<uint32_t *>(smem + S::OffKey);
  for (int i = tid; i < S::KeyWords; i += kThreads) {
    uint32_t v;
    if (i < S::Kr2) v = keyrec[lay.n + i];
    else if (i < S::Kr3) v = keyrec[lay.r2n + i - S::Kr2];
    else if (i < S::Kone) v = 0u;
    else if (i < S::Kunit) v = keyrec[lay.onen + i - S::Kone];
    else if (i < S::Kexp) v = (i == S::Kunit) ? 1u : 0u;
    else v = keyrec[lay.e + i - S::Kexp];
    kc[i] = v;
  }
  constexpr int img_u4 = (S::ImgB1 + S::ImgB2) / 16;
  uint4 *s4 = reinterpret_cast<uint4 *>(smem + S::OffB1);
  for (int i = tid; i < img_u4; i += kThreads) s4[i] = image[i];
}

// One tile: A = x^e mod n for the thread's row x (< n checked by the caller).
// The multiplier x R waits in the slot's table entry and is staged before each
// multiplication (a product's digits overwrite the stage).
template <int H>
__device__ __forceinline__ void pub_exp_tile(uint32_t (&A)[H], Tile &ts, uint8_t *smem, const uint32_t *msg,
                                             const uint32_t *kc, uint4 *tbl, uint32_t ebits, uint32_t polls) {
  using S = Shape<H>;
  const uint32_t *Ms = kc + S::Km;
  const uint32_t *E = kc + S::Kexp;
  const uint32_t kca = ts.sb + S::OffKey;
  const uint32_t slo = ts.arow + S::StageKb * S::Kb, shi = ts.hrow;
  load_row<H>(A, msg, true);
  // x R mod n = x * R^2 * R^-1
  mont_step<H>(A, false, kca + 4 * S::Kr2, 16, kca + 4 * S::Kr2 + 16 * (S::HR / 4), 16, ts, Ms, polls);
  if (ts.dead) return;
  tbl_store<H>(tbl, 0, A);
#pragma unroll 1
  for (int bit = (int)ebits - 2; bit >= 0; --bit) {
    mont_step<H>(A, true, slo, S::Kb, shi, kHiG, ts, Ms, polls);
    if (ts.dead) return;
    if ((E[bit >> 5] >> (bit & 31)) & 1u) {   // uniform over the tile: the key's exponent
      stage_from_table<H>(smem, ts, tbl);
      mont_step<H>(A, false, slo, S::Kb, shi, kHiG, ts, Ms, polls);
      if (ts.dead) return;
    }
  }
  // leave Montgomery form: A * 1 * R^-1
  mont_step<H>(A, false, kca + 4 * S::Kunit, 16, kca + 4 * S::Kunit + 16 * (S::HR / 4), 16, ts, Ms, polls);
}

template <int H>
__global__ void __launch_bounds__(kThreads, 1) pub_tc4_kernel(PubArgs a) {
  using S = Shape<H>;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slot = warp >> 2;
  const int r = ((warp & 3) << 5) | lane;
  const uint32_t sb = tc::smem_addr(smem);
  uint32_t *ctrl = reinterpret_cast<uint32_t *>(smem + S::OffCtrl);
  if (warp == 0) tc::tmem_alloc(sb + S::OffCtrl + 48, kTmemCols);
  if (tid == 0) {
    for (int t = 0; t < kTiles; ++t) tc::mbar_init(sb + S::OffCtrl + 8 * t, 1u);
    tc::mbar_init_fence();
  }
  const uint32_t *kc = reinterpret_cast<const uint32_t *>(smem + S::OffKey);
  load_modulus<H>(smem, a.keyrec, a.image, tid);
  {
    uint4 *ab = reinterpret_cast<uint4 *>(smem + S::OffAbias);
    for (int i = tid; i < kRows * 16 * 2 / 16; i += kThreads)
      ab[i] = make_uint4(0x01000100u, 0x01000100u, 0x01000100u, 0x01000100u);
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  Tile ts;
  ts.sb = sb;
  ts.abuf = sb + S::OffA + slot * S::ABytes;
  ts.arow = ts.abuf + (uint32_t)(r >> 3) * 128 + (uint32_t)(r & 7) * 16;
  ts.hrow = sb + S::OffHi + slot * S::HiBytes + (uint32_t)r * 16;
  ts.tmem = ctrl[12] + (uint32_t)slot * S::TileCols;
  ts.taddr = ts.tmem + ((uint32_t)((warp & 3) * 32) << 16);
  ts.mbar = sb + S::OffCtrl + 8 * slot;
  ts.phase = 0u;
  ts.pending = 2u;
  ts.bar_id = 1 + slot;
  ts.leader = (r == 0);
  ts.err = false;
  ts.dead = false;
  uint4 *tbl = a.tables + (size_t)(blockIdx.x * kTiles + slot) * (H / 4) * kRows + r;
  constexpr KeyLayout lay(H);
  const uint32_t ebits = reinterpret_cast<const KeyHeader *>(a.keyrec)->e_bits;
  for (uint32_t tile = blockIdx.x + gridDim.x * (uint32_t)slot; tile < a.ntiles; tile += gridDim.x * kTiles) {
    const uint32_t row = tile * kRows + (uint32_t)r;
    const bool valid = row < a.count;
    const uint32_t *msg = a.msgs + (size_t)(valid ? row : a.count - 1) * H;
    uint32_t A[H];
    if (!ts.dead) pub_exp_tile<H>(A, ts, smem, msg, kc, tbl, ebits, a.wait_polls);
    drop_slot(tbl, r, (H / 4) * kRows);
    if (valid) {
      const bool below = row_below(msg, a.keyrec + lay.n, H);
      const bool timed_out = ts.err || ts.dead;
      const bool ok = below && !timed_out;
      uint4 *orow = reinterpret_cast<uint4 *>(a.out + (size_t)row * H);
#pragma unroll
      for (int g = 0; g < H / 4; ++g)
        orow[g] = ok ? make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]) : make_uint4(0u, 0u, 0u, 0u);
      if (a.status) a.status[row] = timed_out ? -6 /* RSA_ERR_TIMEOUT */ : (below ? 0 : -3 /* RSA_ERR_RANGE */);
    }
  }
  // a tile that gave up may still have an MMA in flight: wait for it (bounded)
  // before freeing TMEM
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
template <int H>
struct GarnerSmem {
  static constexpr int KeyWords = (KeyLayout(2 * H).total + 3) / 4 * 4;
  static constexpr int Bytes = KeyWords * 4 + (kGThreads / 32) * (H / 4) * 32 * 16;
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

// One operation: hq / hp are its m_q and m_p * R mod p (H/4 uint4, `hstride`
// apart); ks the key record in shared memory; stage_lane the thread's slot of
// an [H/4][32] uint4 stage.  Writes the 2H-limb row at orow (zeros unless ok)
// and returns the status (0, RSA_ERR_RANGE -3 or RSA_ERR_TIMEOUT -6).
template <int H>
__device__ __forceinline__ int32_t garner_op(const uint32_t *ks, uint4 *stage_lane, const uint4 *hq, const uint4 *hp,
                                             size_t hstride, bool timed_out, const uint32_t *mrow, uint4 *orow,
                                             bool valid) {
  constexpr int L = 2 * H;
  constexpr KeyLayout lay(L);
  const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(ks);
  const NSmem<H> N{ks + lay.p};
  uint32_t A[H];
#pragma unroll
  for (int g = 0; g < H / 4; ++g) {
    const uint4 v = hq[(size_t)g * hstride];
    A[4 * g] = v.x; A[4 * g + 1] = v.y; A[4 * g + 2] = v.z; A[4 * g + 3] = v.w;
  }
  mont_mul<H, 4>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.r2p), 1}, N, hd.np_p);   // m_q * R mod p
#pragma unroll
  for (int g = 0; g < H / 4; ++g) stage_lane[g * 32] = hp[(size_t)g * hstride];             // m_p * R mod p
  mod_rsub<H>(A, SmemB{stage_lane, 32}, N);                                                  // (m_p - m_q) R
  mont_mul<H, 4>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.qinv), 1}, N, hd.np_p);  // h
  uint32_t t[H + 2];
#pragma unroll
  for (int g = 0; g < H / 4; ++g) {
    const uint4 v = hq[(size_t)g * hstride];
    t[4 * g] = v.x; t[4 * g + 1] = v.y; t[4 * g + 2] = v.z; t[4 * g + 3] = v.w;
  }
  t[H] = 0u;
  t[H + 1] = 0u;
  const uint32_t *qs = ks + lay.q;
  const bool below = row_below(mrow, ks + lay.n, L);
  const bool ok = valid && below && !timed_out;
#pragma unroll 1
  for (int i0 = 0; i0 < H; i0 += 4) {
    uint32_t rv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      mul_acc<H>(t, A, qs[i0 + u]);
      rv[u] = t[0];
#pragma unroll
      for (int j = 0; j < H + 1; ++j) t[j] = t[j + 1];
      t[H + 1] = 0u;
    }
    if (valid) orow[i0 / 4] = ok ? make_uint4(rv[0], rv[1], rv[2], rv[3]) : make_uint4(0u, 0u, 0u, 0u);
  }
#pragma unroll
  for (int g = 0; g < H / 4; ++g)
    if (valid)
      orow[H / 4 + g] = ok ? make_uint4(t[4 * g], t[4 * g + 1], t[4 * g + 2], t[4 * g + 3])
                           : make_uint4(0u, 0u, 0u, 0u);
  return timed_out ? -6 /* RSA_ERR_TIMEOUT */ : (below ? 0 : -3 /* RSA_ERR_RANGE */);
}

template <int H>
__device__ __forceinline__ void load_key_record(uint4 *gsm, const uint32_t *keyrec) {
  constexpr KeyLayout lay(2 * H);
  for (int i = threadIdx.x; i < GarnerSmem<H>::KeyWords / 4; i += blockDim.x)
    gsm[i] = (i * 4 < (int)lay.total) ? reinterpret_cast<const uint4 *>(keyrec)[i] : make_uint4(0u, 0u, 0u, 0u);
}

template <int H>
__global__ void __launch_bounds__(kGThreads) crt_tc4_garner_kernel(GarnerArgs a) {
  extern __shared__ uint4 gsm[];
  load_key_record<H>(gsm, a.keyrec);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t row = blockIdx.x * kGThreads + threadIdx.x;
  const bool valid = row < a.count;
  const uint32_t rr = valid ? row : 0u;
  uint4 *stage_lane = gsm + GarnerSmem<H>::KeyWords / 4 + warp * (H / 4) * 32 + lane;
  const bool timed_out = a.herr[rr] != 0u || a.herr[a.count + rr] != 0u;
  const int32_t st = garner_op<H>(reinterpret_cast<const uint32_t *>(gsm), stage_lane, a.halves + rr,
                                  a.halves + (size_t)(H / 4) * a.count_pad + rr, a.count_pad, timed_out,
                                  a.msgs + (size_t)rr * 2 * H, reinterpret_cast<uint4 *>(a.out + (size_t)rr * 2 * H),
                                  valid);
  if (valid && a.status) a.status[rr] = st;
}

// Ragged batches: block b takes the (chunk, slot) tiles b, b + grid, ... of the
// group's planned chunks; one thread per operation of the tile, the tile's key
// record in shared memory.  Timeouts are also flagged in the batch's error word.
template <int H>
__global__ void __launch_bounds__(kGThreads) crt_tc4_ragged_garner_kernel(tcr::RaggedTcArgs ra) {
  extern __shared__ uint4 gsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4 *stage_lane = gsm + GarnerSmem<H>::KeyWords / 4 + warp * (H / 4) * 32 + lane;
  const uint32_t ntile_slots = (uint32_t)kTiles * ra.ctl[ra.ctl_word];
  const uint32_t cpad = (ra.count + 31u) & ~31u;
  const uint4 *halves = static_cast<const uint4 *>(ra.halves);
  const uint32_t *herr = reinterpret_cast<const uint32_t *>(halves + (size_t)2 * (H / 4) * cpad);
#pragma unroll 1
  for (uint32_t t = blockIdx.x; t < ntile_slots; t += gridDim.x) {
    const tcr::TcChunk ch = ra.chunks[t / kTiles];
    const int s = (int)(t % kTiles);
    if (s >= ch.ntiles) continue;   // uniform over the block
    __syncthreads();                // the previous tile's key record is no longer read
    load_key_record<H>(gsm, ch.keyrec);
    __syncthreads();
    const uint32_t row = (uint32_t)s * kRows + threadIdx.x;
    if (row >= (uint32_t)ch.nops) continue;   // past a partial last tile; rejoins at the next tile's barrier
    const uint32_t pos = (uint32_t)ch.op_start + row;
    const uint32_t op = (uint32_t)ra.sorted[pos];
    const size_t off = (size_t)ra.offsets[op];
    const bool timed_out = herr[pos] != 0u || herr[ra.count + pos] != 0u;
    const int32_t st = garner_op<H>(reinterpret_cast<const uint32_t *>(gsm), stage_lane, halves + pos,
                                    halves + (size_t)(H / 4) * cpad + pos, cpad, timed_out, ra.msgs + off,
                                    reinterpret_cast<uint4 *>(ra.out + off), true);
    if (ra.status) ra.status[op] = st;
    if (timed_out) atomicOr(&ra.ctl[2], 1u << 6);   // RSA_ERR_TIMEOUT for rsa_sync
  }
}

// ---------------------------------------------------------------- host side
int tc4_grid(uint32_t count, int sm_count) {
  const uint32_t ntiles = (count + kRows - 1) / kRows;
  const uint32_t want = (ntiles + kTiles - 1) / kTiles;
  const uint32_t cap = (uint32_t)(sm_count / 2 > 0 ? sm_count / 2 : 1);
  const uint32_t per_prime = want < 1u ? 1u : (want < cap ? want : cap);
  return (int)(2 * per_prime);
}

template <int H>
static size_t tables_bytes_h(int grid, int window) {
  const size_t per_slot = (window == 3) ? (size_t)Win<H, 3>::kTblU4 : (size_t)Win<H, 4>::kTblU4;
  return (size_t)grid * kTiles * per_slot * 16;
}
size_t tc4_tables_bytes(int H, int grid, int window) {
  return H == 48 ? tables_bytes_h<48>(grid, window) : tables_bytes_h<64>(grid, window);
}

static uint32_t pad_count(uint32_t count) { return (count + 31u) & ~31u; }

size_t tc4_halves_bytes(int H, uint32_t count) {
  return (size_t)2 * (H / 4) * pad_count(count) * 16 + (size_t)2 * count * 4;
}

template <int H, int W>
static cudaError_t launch_half(const HalfArgs &h, int grid, cudaStream_t s) {
  constexpr int smem = Shape<H>::Smem;
  cudaError_t e = cudaFuncSetAttribute(crt_tc4_half_kernel<H, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  crt_tc4_half_kernel<H, W><<<grid, kThreads, smem, s>>>(h);
  return cudaGetLastError();
}

template <int H>
static cudaError_t launch_h(const uint32_t *keyrec, const void *image, const uint32_t *msgs, uint32_t *out,
                            int32_t *status, uint32_t count, int grid, int window, void *tables, void *halves,
                            uint32_t wait_polls, cudaStream_t s) {
  const uint32_t cp = pad_count(count);
  HalfArgs h;
  h.keyrec = keyrec;
  h.image = static_cast<const uint4 *>(image);
  h.msgs = msgs;
  h.halves = static_cast<uint4 *>(halves);
  h.herr = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(halves) + (size_t)2 * (H / 4) * cp * 16);
  h.tables = static_cast<uint4 *>(tables);
  h.count = count;
  h.count_pad = cp;
  h.ntiles = (count + kRows - 1) / kRows;
  h.ctas_per_prime = (uint32_t)grid / 2;
  h.wait_polls = wait_polls;
  cudaError_t e = (window == 3) ? launch_half<H, 3>(h, grid, s) : launch_half<H, 4>(h, grid, s);
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
  crt_tc4_garner_kernel<H><<<(count + kGThreads - 1) / kGThreads, kGThreads, GarnerSmem<H>::Bytes, s>>>(g);
  return cudaGetLastError();
}

const void *ragged_tc4_half_fn(int H, int window) {
  if (H == 48) return window == 3 ? reinterpret_cast<const void *>(&crt_tc4_ragged_half_kernel<48, 3>)
                                  : reinterpret_cast<const void *>(&crt_tc4_ragged_half_kernel<48, 4>);
  if (H == 64) return window == 3 ? reinterpret_cast<const void *>(&crt_tc4_ragged_half_kernel<64, 3>)
                                  : reinterpret_cast<const void *>(&crt_tc4_ragged_half_kernel<64, 4>);
  return nullptr;
}
const void *ragged_tc4_garner_fn(int H) {
  if (H == 48) return reinterpret_cast<const void *>(&crt_tc4_ragged_garner_kernel<48>);
  if (H == 64) return reinterpret_cast<const void *>(&crt_tc4_ragged_garner_kernel<64>);
  return nullptr;
}
// ---- public exponent of 2048-bit keys
int pub_tc4_grid(uint32_t count, int sm_count) {
  const uint32_t ntiles = (count + kRows - 1) / kRows;
  const uint32_t want = (ntiles + kTiles - 1) / kTiles;
  const uint32_t cap = (uint32_t)(sm_count > 0 ? sm_count : 1);
  return (int)(want < 1u ? 1u : (want < cap ? want : cap));
}
size_t pub_tc4_tables_bytes(int grid) { return (size_t)grid * kTiles * (kPubH / 4) * kRows * 16; }
cudaError_t launch_pub_tc4(const uint32_t *keyrec, const void *image, const uint32_t *msgs, uint32_t *out,
                           int32_t *status, uint32_t count, int grid, void *tables, uint32_t wait_polls,
                           cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  PubArgs a{keyrec, static_cast<const uint4 *>(image), msgs, out, status, static_cast<uint4 *>(tables), count,
            (count + kRows - 1) / kRows, wait_polls};
  const int smem = Shape<kPubH>::Smem;
  cudaError_t e = cudaFuncSetAttribute(pub_tc4_kernel<kPubH>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  pub_tc4_kernel<kPubH><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

size_t tc4_smem_bytes(int H) { return H == 48 ? (size_t)Shape<48>::Smem : (size_t)Shape<64>::Smem; }
size_t ragged_tc4_garner_smem(int H) {
  return H == 48 ? (size_t)GarnerSmem<48>::Bytes : (size_t)GarnerSmem<64>::Bytes;
}

cudaError_t launch_crt_tc4(int H, const uint32_t *keyrec, const void *image, const uint32_t *msgs, uint32_t *out,
                           int32_t *status, uint32_t count, int grid, int window, void *tables, void *halves,
                           uint32_t wait_polls, cudaStream_t s) {
  if (H == 48)
    return launch_h<48>(keyrec, image, msgs, out, status, count, grid, window, tables, halves, wait_polls, s);
  if (H == 64)
    return launch_h<64>(keyrec, image, msgs, out, status, count, grid, window, tables, halves, wait_polls, s);
  return cudaErrorInvalidValue;
}

}  // namespace tc4
}  // namespace rsagpu
