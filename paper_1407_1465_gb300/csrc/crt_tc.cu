// crt_tc.cu -- RSA-2048 CRT decryption with the Montgomery reduction on the
// 5th-generation tensor cores (tcgen05, TMEM), for 1024-bit primes.
//
// Decryption follows the CRT route of the library's other kernels:
// M = C^d mod n computed as m_p = C^dp mod p and m_q = C^dq mod q, then
// recombined (Garner).  Each half is a constant-time fixed-window
// exponentiation (Fig. 6 of the paper with k = 4) whose every modular
// multiplication is a Montgomery product A*B*R^-1 mod m, R = 2^1024.
//
// The Montgomery product is split between the two kinds of units:
//   1. CUDA cores: T = A * B, 32 x 32 limbs, product scanning with PTX carry
//      chains (one thread per operation).  The low half of T leaves the
//      registers as byte digits (fp16) in shared memory.
//   2. Tensor core, MMA 1: mu_cols = T_lo * Toep(m'), the column sums of the
//      byte convolution of T mod R with m' = -m^-1 mod R (only columns < 128).
//   3. CUDA cores: carry-propagate the columns into the bytes of
//      mu = T*m' mod R, written back as fp16 digits.
//   4. Tensor core, MMA 2: the column sums of mu * m for positions 112..255.
//   5. CUDA cores: the carry out of the low half (ceil of the top four low
//      columns; the lower ones add less than 2^-8 of a unit), the high half
//      carry-propagated and added to T_hi, one conditional subtraction of m.
// m' and m are the same for every message of the batch, which is what makes
// steps 2 and 4 matrix products (messages x digits) x (digits x digits); the
// per-message product A*B (step 1) stays on the CUDA cores.  Exactness: the
// digits are bytes and a column holds at most 128 products of two bytes, so
// every column sum is an integer below 2^23 and the fp32 accumulation is exact
// (tcprep.cpp describes the bias that makes the sums readable as integers).
//
// Work layout: one CTA per SM (384 threads), all of one prime; three tiles of
// 128 operations, each with its own A buffer, 160 TMEM columns, mbarrier and
// named barrier, run independently, so one tile's MMAs overlap the other
// tiles' CUDA-core work.  A tile's thread r owns operation r of the tile and
// TMEM lane r.  The Garner recombination runs afterwards in its own kernel.
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
constexpr int kKbA = (kRows / 8) * 128;            // k-block stride of an A buffer (2048)
constexpr int kKbM = (kN1 / 8) * 128;              // k-block stride of BM (2048)
constexpr int kKbP = (kN2 / 8) * 128;              // k-block stride of BP (2304)
constexpr int kOffBm = 0;
constexpr int kOffBp = kOffBm + (int)kImgBm;
constexpr int kOffAbias = kOffBp + (int)kImgBp;     // 128 x 16 bias A operand
constexpr int kOffA = kOffAbias + kRows * 16 * 2;   // kTiles A buffers of 128 x 128 digits
constexpr int kABytes = kRows * kDig * 2;
constexpr int kOffStage = kOffA + kTiles * kABytes; // [kH/4][kThreads] uint4
constexpr int kOffKey = kOffStage + kThreads * kH * 4;
// key constants (words): m, R^2, R^3, R mod m, unit, exponent (kH + 4 limbs)
constexpr int kKm = 0, kKr2 = kH, kKr3 = 2 * kH, kKone = 3 * kH, kKunit = 4 * kH, kKexp = 5 * kH;
constexpr int kKeyWords = 6 * kH + 4;
constexpr int kOffCtrl = kOffKey + kKeyWords * 4;   // 3 mbarriers (8 B each), TMEM base at +32
constexpr int kSmem = kOffCtrl + 64;
static_assert(kOffA % 128 == 0 && kOffStage % 16 == 0 && kOffCtrl % 8 == 0, "alignment");
static_assert(kSmem <= 227 * 1024, "shared memory");

constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kTileCols = 160;                 // >= kN2, per tile
constexpr uint32_t kIdesc1 = tc::idesc_f16_f32(128, kN1);
constexpr uint32_t kIdesc2 = tc::idesc_f16_f32(128, kN2);
constexpr int kNwin = 32 * kH / kWin;               // windows of the 1024-bit exponent
constexpr int kTblU4 = (1 << kWin) * (kH / 4) * kRows;   // uint4 per tile slot: [entry][g][row]
constexpr uint32_t kBias = 0x3F000000u;             // fp32 bits of the column bias 1/2
constexpr uint32_t kWaitLimit = 1u << 22;

struct HalfArgs {
  const uint32_t *keyrec;
  const uint4 *image;       // [prime][BM | BP], prime 0 = q, 1 = p
  const uint32_t *msgs;     // count rows of 64 limbs
  uint4 *halves;            // [prime][kH/4][count_pad]: q -> m_q, p -> m_p * R mod p
  uint32_t *herr;           // [prime][count]: 1 if a bounded wait gave up
  uint4 *tables;            // [grid * kTiles][kTblU4]
  uint32_t count, count_pad, ntiles, ctas_per_prime;
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
// One row of the product scan: t + a*b, the lowest limb returned and the rest
// shifted down one limb (t[j] <- position j+1).  t < 2^(32L) on entry, so the
// sum fits in L+1 limbs.  Even and odd limbs of a in two carry chains as in
// mul_acc (mont.cuh).
template <int L>
__device__ __forceinline__ uint32_t mul_emit(uint32_t (&t)[L], const uint32_t (&a)[L], uint32_t b) {
  const uint32_t out = mad_lo_cc(a[0], b, t[0]);
  t[0] = madc_hi_cc(a[0], b, t[1]);
#pragma unroll
  for (int k = 1; k < L / 2; ++k) {
    t[2 * k - 1] = madc_lo_cc(a[2 * k], b, t[2 * k]);
    t[2 * k] = madc_hi_cc(a[2 * k], b, t[2 * k + 1]);
  }
  t[L - 1] = addc(0u, 0u);
  t[0] = mad_lo_cc(a[1], b, t[0]);
  t[1] = madc_hi_cc(a[1], b, t[1]);
#pragma unroll
  for (int k = 1; k < L / 2; ++k) {
    t[2 * k] = madc_lo_cc(a[2 * k + 1], b, t[2 * k]);
    t[2 * k + 1] = madc_hi_cc(a[2 * k + 1], b, t[2 * k + 1]);
  }
  return out;
}

__device__ __forceinline__ uint4 lds128a(uint32_t saddr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(saddr) : "memory");
  return v;
}

// carry of a column word x = 0x3F000000 + x' (x' < 2^24): x' >> 8
__device__ __forceinline__ uint32_t ccarry(uint32_t x) { return tc::prmt(x, 0u, 0x4421u); }

// t[j0 .. j0+NL) += (4*NL column words v, carry-propagated from the running
// column state x) + cin; the carry out returns in cin.  Each group of four
// columns becomes one limb of byte digits.
template <int NL>
__device__ __forceinline__ void add_columns(uint32_t (&t)[kH], int j0, const uint32_t *v, uint32_t &x, uint32_t &cin) {
  uint32_t X[NL];
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const uint32_t x0 = v[4 * i] + ccarry(x);
    const uint32_t x1 = v[4 * i + 1] + ccarry(x0);
    const uint32_t x2 = v[4 * i + 2] + ccarry(x1);
    const uint32_t x3 = v[4 * i + 3] + ccarry(x2);
    X[i] = tc::prmt(tc::prmt(x0, x1, 0x0040u), tc::prmt(x2, x3, 0x4000u), 0x7610u);
    x = x3;
  }
  (void)add_cc(cin, 0xFFFFFFFFu);   // carry flag <- cin (0 or 1)
#pragma unroll
  for (int i = 0; i < NL; ++i) t[j0 + i] = addc_cc(t[j0 + i], X[i]);
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

// A = A * B * R^-1 mod m (A < R, B < m; result < m).  B: kH limbs in shared
// memory at bsa, four limbs per 16 bytes, consecutive groups `bstr` bytes apart.
__device__ __forceinline__ void mont_step(uint32_t (&A)[kH], uint32_t bsa, uint32_t bstr, Tile &ts,
                                          const uint32_t *Ms) {
  // 1. T = A * B: the low 32 limbs leave as digits, t ends as T_hi
  uint32_t t[kH];
#pragma unroll
  for (int j = 0; j < kH; ++j) t[j] = 0u;
  uint32_t top = 0u;
#pragma unroll 1
  for (int i0 = 0; i0 < kH; i0 += 8) {
    const uint4 b0 = lds128a(bsa + (uint32_t)(i0 >> 2) * bstr);
    const uint4 b1 = lds128a(bsa + (uint32_t)((i0 >> 2) + 1) * bstr);
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
    const uint32_t ad = ts.arow + (uint32_t)(i0 >> 1) * kKbA;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      tc::sts128(ad + q * kKbA, tc::prmt(e[2 * q], 0u, 0x4140u), tc::prmt(e[2 * q], 0u, 0x4342u),
                 tc::prmt(e[2 * q + 1], 0u, 0x4140u), tc::prmt(e[2 * q + 1], 0u, 0x4342u));
    top = e[7];
  }
  // 2. MMA 1: mu columns = T_lo digits x Toep(m')
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  ts.dead = tc::bar_red_or(ts.bar_id, kRows, ts.err);
  if (ts.dead) return;
  if (ts.leader) {
    tc::fence_after_sync();
    tc::mma_f16(ts.tmem, tc::sdesc(ts.sb + kOffAbias, kKbA, 128), tc::sdesc(ts.sb + kOffBm + 16 * kKbM, kKbM, 128),
                kIdesc1, 0u);
#pragma unroll 1
    for (int s = 0; s < kDig / 16; ++s)
      tc::mma_f16(ts.tmem, tc::sdesc(ts.abuf + s * 2 * kKbA, kKbA, 128),
                  tc::sdesc(ts.sb + kOffBm + s * 2 * kKbM, kKbM, 128), kIdesc1, 1u);
    tc::commit(ts.mbar);
  }
  if (!tc::mbar_wait(ts.mbar, ts.phase, kWaitLimit)) {
    ts.err = true;
    ts.pending = ts.phase;
  }
  ts.phase ^= 1u;
  tc::fence_after_sync();
  // 3. mu = carry-propagated columns mod R, back to shared memory as digits
  {
    uint32_t x = kBias;
#pragma unroll 1
    for (int c0 = 0; c0 < kDig; c0 += 32) {
      uint32_t v[32];
      tc::ld32(ts.taddr + (uint32_t)c0, v);
      tc::wait_ld();
      uint32_t w[16];
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const uint32_t x0 = v[j] + ccarry(x);
        const uint32_t x1 = v[j + 1] + ccarry(x0);
        w[j >> 1] = tc::prmt(x0, x1, 0xB4B0u);   // [x0.b0, 0, x1.b0, 0]: two fp16 digits
        x = x1;
      }
      const uint32_t ad = ts.arow + (uint32_t)(c0 >> 3) * kKbA;
#pragma unroll
      for (int q = 0; q < 4; ++q) tc::sts128(ad + q * kKbA, w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    }
  }
  // 4. MMA 2: columns 112..255 of mu * m
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  ts.dead = tc::bar_red_or(ts.bar_id, kRows, ts.err);
  if (ts.dead) return;
  if (ts.leader) {
    tc::fence_after_sync();
    tc::mma_f16(ts.tmem, tc::sdesc(ts.sb + kOffAbias, kKbA, 128), tc::sdesc(ts.sb + kOffBp + 16 * kKbP, kKbP, 128),
                kIdesc2, 0u);
#pragma unroll 1
    for (int s = 0; s < kDig / 16; ++s)
      tc::mma_f16(ts.tmem, tc::sdesc(ts.abuf + s * 2 * kKbA, kKbA, 128),
                  tc::sdesc(ts.sb + kOffBp + s * 2 * kKbP, kKbP, 128), kIdesc2, 1u);
    tc::commit(ts.mbar);
  }
  if (!tc::mbar_wait(ts.mbar, ts.phase, kWaitLimit)) {
    ts.err = true;
    ts.pending = ts.phase;
  }
  ts.phase ^= 1u;
  tc::fence_after_sync();
  // 5. U = T_hi + (T_lo + mu*m) / R, then one conditional subtraction.  The
  // columns are carry-propagated 4 at a time into limbs that are added to T_hi
  // right away (the carry between chunks is kept in a register: cin).
  uint32_t x, cin = 0u;
  {
    uint32_t v[32];
    tc::ld32(ts.taddr + 0u, v);   // positions 112..143
    tc::wait_ld();
    // carry out of the low half: ceil of positions 124..127 (with T's top limb) / 2^32
    const uint32_t y0 = v[12] + (top & 0xFFu);
    const uint32_t y1 = v[13] + ((top >> 8) & 0xFFu) + ccarry(y0);
    const uint32_t y2 = v[14] + ((top >> 16) & 0xFFu) + ccarry(y1);
    const uint32_t y3 = v[15] + (top >> 24) + ccarry(y2);
    const uint32_t low = (y0 | y1 | y2 | y3) & 0xFFu;
    x = (ccarry(y3) + (low != 0u ? 1u : 0u)) << 8;   // so that ccarry(x) is that carry
    add_columns<4>(t, 0, v + 16, x, cin);
  }
#pragma unroll
  for (int c = 1; c < 4; ++c) {
    uint32_t v[32];
    tc::ld32(ts.taddr + (uint32_t)(32 * c), v);
    tc::wait_ld();
    add_columns<8>(t, 4 + 8 * (c - 1), v, x, cin);
  }
  {
    uint32_t v[16];
    tc::ld16(ts.taddr + 128u, v);   // positions 240..255
    tc::wait_ld();
    add_columns<4>(t, 28, v, x, cin);
  }
  tc::fence_before_sync();   // this tile's TMEM reads precede the next MMA (ordered by the next barrier)
  uint32_t u[kH + 2];
#pragma unroll
  for (int j = 0; j < kH; ++j) u[j] = t[j];
  u[kH] = ccarry(x) + cin;
  u[kH + 1] = 0u;
  final_sub<kH>(A, u, NSmem<kH>{Ms});
}

// ---------------------------------------------------------------- table helpers (global, per tile slot)
__device__ __forceinline__ void tbl_store(uint4 *tbl, int e, const uint32_t (&A)[kH]) {
#pragma unroll
  for (int g = 0; g < kH / 4; ++g)
    tbl[(e * (kH / 4) + g) * kRows] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
}
// stage <- T[d], reading every entry (constant time)
__device__ __forceinline__ void tbl_select(uint4 *stage, const uint4 *tbl, uint32_t d) {
#pragma unroll 1
  for (int g = 0; g < kH / 4; ++g) {
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int e = 0; e < (1 << kWin); ++e) {
      const uint4 v = tbl[(e * (kH / 4) + g) * kRows];
      const uint32_t msk = 0u - (uint32_t)((uint32_t)e == d);
      acc.x |= v.x & msk;
      acc.y |= v.y & msk;
      acc.z |= v.z & msk;
      acc.w |= v.w & msk;
    }
    stage[g * kThreads] = acc;
  }
}
__device__ __forceinline__ void stage_put(uint4 *stage, const uint32_t (&A)[kH]) {
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) stage[g * kThreads] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
}
__device__ __forceinline__ void stage_get(uint32_t (&A)[kH], const uint4 *stage) {
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) {
    const uint4 v = stage[g * kThreads];
    A[4 * g] = v.x; A[4 * g + 1] = v.y; A[4 * g + 2] = v.z; A[4 * g + 3] = v.w;
  }
}

// ---------------------------------------------------------------- exponentiation kernel (both primes)
__global__ void __launch_bounds__(kThreads, 1) crt_tc_half_kernel(HalfArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slot = warp >> 2;                   // tile slot 0 .. kTiles-1
  const int r = ((warp & 3) << 5) | lane;       // operation within the tile = TMEM lane
  const uint32_t pi = blockIdx.x & 1u;          // 0: q, 1: p
  const uint32_t cta = blockIdx.x >> 1;
  const uint32_t sb = tc::smem_addr(smem);
  uint32_t *ctrl = reinterpret_cast<uint32_t *>(smem + kOffCtrl);

  if (warp == 0) tc::tmem_alloc(sb + kOffCtrl + 32, kTmemCols);
  if (tid == 0) {
    for (int t = 0; t < kTiles; ++t) tc::mbar_init(sb + kOffCtrl + 8 * t, 1u);
    tc::mbar_init_fence();
  }
  // key constants of this prime
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
  }
  // B images of this prime and the constant bias A block (2^-16 = fp16 0x0100)
  {
    const uint4 *img = a.image + (size_t)pi * (kImgPrime / 16);
    uint4 *s4 = reinterpret_cast<uint4 *>(smem + kOffBm);
    for (int i = tid; i < (int)(kImgPrime / 16); i += kThreads) s4[i] = img[i];
    uint4 *ab = reinterpret_cast<uint4 *>(smem + kOffAbias);
    for (int i = tid; i < kRows * 16 * 2 / 16; i += kThreads) ab[i] = make_uint4(0x01000100u, 0x01000100u, 0x01000100u, 0x01000100u);
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  Tile ts;
  ts.sb = sb;
  ts.abuf = sb + kOffA + slot * kABytes;
  ts.arow = ts.abuf + (uint32_t)(r >> 3) * 128 + (uint32_t)(r & 7) * 16;
  ts.tmem = ctrl[8] + (uint32_t)slot * kTileCols;
  ts.taddr = ts.tmem + ((uint32_t)((warp & 3) * 32) << 16);
  ts.mbar = sb + kOffCtrl + 8 * slot;
  ts.phase = 0u;
  ts.pending = 2u;
  ts.bar_id = 1 + slot;
  ts.leader = (r == 0);
  ts.err = false;
  ts.dead = false;

  const uint32_t *Ms = kc + kKm;
  const NSmem<kH> N{Ms};
  uint4 *stage = reinterpret_cast<uint4 *>(smem + kOffStage) + tid;
  const uint32_t stage_sa = sb + kOffStage + (uint32_t)tid * 16;
  const uint32_t stage_str = kThreads * 16;
  uint4 *tbl = a.tables + (size_t)(blockIdx.x * kTiles + slot) * kTblU4 + r;

  for (uint32_t tile = cta + a.ctas_per_prime * (uint32_t)slot; tile < a.ntiles;
       tile += a.ctas_per_prime * kTiles) {
    const uint32_t row = tile * kRows + (uint32_t)r;
    const bool valid = row < a.count;
    const uint32_t *msg = a.msgs + (size_t)(valid ? row : a.count - 1) * (2 * kH);
    uint32_t A[kH];
    if (!ts.dead) {
      const int nexp = (kNwin - 1) * (kWin + 1);
      const int nst = 16 + nexp + (pi == 0 ? 1 : 0);
      int k = kNwin - 2, s = 0;
#pragma unroll 1
      for (int st = 0; st < nst; ++st) {
        uint32_t bsa = stage_sa, bstr = stage_str;
        if (st == 0) {                      // c_lo * R mod m
          load_row<kH>(A, msg, true);
          bsa = sb + kOffKey + 4 * kKr2;
          bstr = 16;
        } else if (st == 1) {               // c_hi * R^2 mod m
          tbl_store(tbl, 1, A);
          load_row<kH>(A, msg + kH, true);
          bsa = sb + kOffKey + 4 * kKr3;
          bstr = 16;
        } else if (st < 16) {               // table T[i] = x^i * R, i = 2 .. 15
          if (st == 2) {
#pragma unroll
            for (int g = 0; g < kH / 4; ++g) stage[g * kThreads] = tbl[(1 * (kH / 4) + g) * kRows];   // c_lo * R
            mod_add<kH>(A, SmemB{stage, kThreads}, N);   // x * R = c * R mod m
            tbl_store(tbl, 1, A);
            uint32_t one[kH];
            from_uniform<kH>(one, reinterpret_cast<const uint4 *>(kc + kKone));
            tbl_store(tbl, 0, one);
            stage_put(stage, A);
          } else {
            tbl_store(tbl, st - 1, A);
          }
        } else if (st < 16 + nexp) {        // windows: kWin squarings, then T[digit]
          if (st == 16) {
            tbl_store(tbl, 15, A);
            tbl_select(stage, tbl, exp_digit<kWin>(kc + kKexp, (uint32_t)(kNwin - 1)));
            stage_get(A, stage);
          }
          if (s < kWin) {
            stage_put(stage, A);
            ++s;
          } else {
            tbl_select(stage, tbl, exp_digit<kWin>(kc + kKexp, (uint32_t)k));
            s = 0;
            --k;
          }
        } else {                            // q: leave Montgomery form
          bsa = sb + kOffKey + 4 * kKunit;
          bstr = 16;
        }
        mont_step(A, bsa, bstr, ts, Ms);
        if (ts.dead) break;
      }
    }
    if (valid) {
      uint4 *h = a.halves + (size_t)pi * (kH / 4) * a.count_pad + row;
#pragma unroll
      for (int g = 0; g < kH / 4; ++g)
        h[(size_t)g * a.count_pad] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
      a.herr[(size_t)pi * a.count + row] = (ts.err || ts.dead) ? 1u : 0u;
    }
  }
  // a tile that gave up may still have an MMA in flight: wait for it (bounded) before freeing TMEM
  if (ts.leader && ts.pending < 2u) (void)tc::mbar_wait(ts.mbar, ts.pending, kWaitLimit);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(ctrl[8], kTmemCols);
  }
}

// ---------------------------------------------------------------- Garner recombination
// m = m_q + q * ((m_p - m_q) * qinv mod p), one thread per operation, with the
// CIOS Montgomery product of mont.cuh (modulus p from shared memory).
constexpr int kGThreads = 256;
constexpr int kGKeyWords = (KeyLayout(2 * kH).total + 3) / 4 * 4;
constexpr int kGSmem = kGKeyWords * 4 + (kGThreads / 32) * (kH / 4) * 32 * 16;

__global__ void __launch_bounds__(kGThreads) crt_tc_garner_kernel(GarnerArgs a) {
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
  mont_mul<kH, 8>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.r2p), 1}, N, hd.np_p);   // m_q * R mod p
#pragma unroll
  for (int g = 0; g < kH / 4; ++g) stage_lane[g * 32] = hp[(size_t)g * a.count_pad];         // m_p * R mod p
  mod_rsub<kH>(A, SmemB{stage_lane, 32}, N);                                                  // (m_p - m_q) R
  mont_mul<kH, 8>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.qinv), 1}, N, hd.np_p);  // h
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
  const bool ok = valid && row_below(mrow, ks + lay.n, L) && a.herr[rr] == 0u && a.herr[a.count + rr] == 0u;
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
    if (valid) orow[kH / 4 + g] = ok ? make_uint4(t[4 * g], t[4 * g + 1], t[4 * g + 2], t[4 * g + 3]) : make_uint4(0u, 0u, 0u, 0u);
  if (valid && a.status) {
    int32_t st = 0;
    if (a.herr[rr] != 0u || a.herr[a.count + rr] != 0u) st = -6;        // RSA_ERR_TIMEOUT
    else if (!row_below(mrow, ks + lay.n, L)) st = -3;                  // RSA_ERR_RANGE
    a.status[rr] = st;
  }
}

// ---------------------------------------------------------------- host side
size_t tc_smem_bytes() { return (size_t)kSmem; }

int tc_grid(uint32_t count, int sm_count) {
  const uint32_t ntiles = (count + kRows - 1) / kRows;
  const uint32_t want = (ntiles + kTiles - 1) / kTiles;            // CTAs per prime to give every slot a tile
  const uint32_t per_prime = std::max<uint32_t>(1u, std::min<uint32_t>(want, (uint32_t)std::max(1, sm_count / 2)));
  return (int)(2 * per_prime);
}

size_t tc_tables_bytes(int grid) { return (size_t)grid * kTiles * kTblU4 * 16; }

static uint32_t pad_count(uint32_t count) { return (count + 31u) & ~31u; }

size_t tc_halves_bytes(uint32_t count) {
  return (size_t)2 * (kH / 4) * pad_count(count) * 16 + (size_t)2 * count * 4;
}

cudaError_t launch_crt_tc(const uint32_t *keyrec, const void *image, const uint32_t *msgs, uint32_t *out,
                          int32_t *status, uint32_t count, int grid, void *tables, void *halves,
                          cudaStream_t s) {
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(crt_tc_half_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
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
  crt_tc_half_kernel<<<grid, kThreads, kSmem, s>>>(h);
  cudaError_t e = cudaGetLastError();
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
