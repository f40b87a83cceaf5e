// kernels.cuh -- batched RSA modular exponentiation kernels (one operation per
// thread, 32 operations per warp = one tile).
//
// Paper: C = M^e mod n, M = C^d mod n (Sec. 2, Sec. 3.2-3.3); the data-parallel
// decomposition is one message per thread (Sec. 6, Algorithm 1).  The paper's
// modulo routine (Algorithm 2) is replaced by Montgomery multiplication on
// 32-bit limbs (mont.cuh) and its O(e) loop by:
//   - public exponent: left-to-right binary square-and-multiply (Fig. 5);
//   - private exponent: left-to-right k-ary with k = W (Fig. 6) made
//     constant-time: a fixed number of windows for the modulus size, W
//     squarings and always one multiplication per window (digit 0 multiplies
//     by the Montgomery one, T[0]), and the table entry chosen by reading every
//     entry and masking, so the memory access pattern does not depend on d;
//   - CRT decryption: c mod p and c mod q, two half-size exponentiations with
//     dp, dq, and Garner's recombination m = m_q + q * (qinv (m_p - m_q) mod p).
//
// Work layout.  A CRT tile is handled by a warp pair: the even warp runs the
// q half and the odd warp the p half of the same 32 messages; the q warp hands
// m_q to the p warp through a double-buffered shared-memory slot and a named
// barrier.  Tables of 2^W entries live in a global-memory scratch slot per
// warp, interleaved [entry][limb/4][lane] so every table access is a
// coalesced 128-bit load or store.  Grids are persistent: each warp (pair)
// walks tiles with a stride of the grid's warp (pair) count.
#pragma once
#include <cstdint>
#include <type_traits>

#include "keyrec.h"
#include "mont.cuh"

namespace rsagpu {

// Named barrier of a warp pair (64 threads).  The warp is reconverged first and
// the non-aligned form is used, so the barrier never meets a diverged warp.
__device__ __forceinline__ void pair_barrier(int bar_id) {
  __syncwarp();
  asm volatile("barrier.sync %0, 64;" ::"r"(bar_id) : "memory");
}

// Message/result row loads and stores (rows are 16-byte aligned: L % 4 == 0).
template <int L>
__device__ __forceinline__ void load_row(uint32_t (&A)[L], const uint32_t *row, bool valid) {
  const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
#pragma unroll
  for (int g = 0; g < L / 4; ++g) {
    uint4 v = valid ? __ldg(r4 + g) : make_uint4(0u, 0u, 0u, 0u);
    A[4 * g] = v.x; A[4 * g + 1] = v.y; A[4 * g + 2] = v.z; A[4 * g + 3] = v.w;
  }
}

// Is the row (nl limbs, global) below m (nl limbs, shared)?  Compared from the top.
__device__ __forceinline__ bool row_below(const uint32_t *row, const uint32_t *m, int nl) {
  int res = 0;  // -1 row < m, +1 row > m, 0 equal so far
  for (int j = nl - 1; j >= 0; --j) {
    const uint32_t a = row[j], b = m[j];
    if (res == 0 && a != b) res = a < b ? -1 : 1;
  }
  return res < 0;
}

// W-bit digit k of an exponent held in shared memory (padded by >= 1 limb).
template <int W>
__device__ __forceinline__ uint32_t exp_digit(const uint32_t *e, uint32_t k) {
  const uint32_t bit = k * W;
  const uint32_t lo = e[bit >> 5], hi = e[(bit >> 5) + 1];
  return __funnelshift_r(lo, hi, bit & 31u) & ((1u << W) - 1u);
}

// stage <- T[d], reading all 2^W entries and keeping the one selected by a mask.
template <int L, int W>
__device__ __forceinline__ void table_select(uint4 *stage_lane, const uint4 *table_lane, uint32_t d) {
#pragma unroll 1
  for (int g = 0; g < L / 4; ++g) {
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 8
    for (int e = 0; e < (1 << W); ++e) {
      const uint4 v = table_lane[(e * (L / 4) + g) * 32];
      const uint32_t m = 0u - (uint32_t)((uint32_t)e == d);
      acc.x |= v.x & m;
      acc.y |= v.y & m;
      acc.z |= v.z & m;
      acc.w |= v.w & m;
    }
    stage_lane[g * 32] = acc;
  }
}

template <int L>
__device__ __forceinline__ void table_store(uint4 *table_lane, int e, const uint32_t (&A)[L]) {
#pragma unroll
  for (int g = 0; g < L / 4; ++g)
    table_lane[(e * (L / 4) + g) * 32] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
}
template <int L>
__device__ __forceinline__ void table_store_uniform(uint4 *table_lane, int e, const uint4 *s) {
#pragma unroll
  for (int g = 0; g < L / 4; ++g) table_lane[(e * (L / 4) + g) * 32] = s[g];
}

// N operand selection: registers for small L with CIOS squarings, shared
// memory otherwise (the separated squaring needs the registers for its
// 2L-limb product).
template <int L, bool SQR> struct NPick { static constexpr bool reg = (L <= 32) && !SQR; };

// Constant-time fixed-window exponentiation (Fig. 6 with k = W).
// In: A = x * R mod N (Montgomery form).  Out: A = x^E * R mod N.
// ebits is the number of exponent bit positions processed: a fixed count for
// the modulus size, not E's own length.  SQR selects the separated squaring
// (mont_sqr) for the W squarings of each window; otherwise squarings run
// through the general CIOS multiply with A staged as the B operand.
template <int L, int W, int U, bool SQR, class NS>
__device__ __forceinline__ void fixed_window_exp(uint32_t (&A)[L], const uint32_t *E, int ebits,
                                                 const uint4 *one, uint4 *stage_lane,
                                                 uint4 *table_lane, const NS &N, uint32_t np) {
  constexpr int NE = 1 << W;
  const SmemB st{stage_lane, 32};
  // table: T[0] = R mod N (Montgomery one), T[1] = x, T[i] = T[i-1] * x
  table_store_uniform<L>(table_lane, 0, one);
  table_store<L>(table_lane, 1, A);
  to_stage<L>(stage_lane, A);
#pragma unroll 1
  for (int i = 2; i < NE; ++i) {
    mont_mul<L, U>(A, st, N, np);
    table_store<L>(table_lane, i, A);
  }
  const int nwin = (ebits + W - 1) / W;
  // leading window
  table_select<L, W>(stage_lane, table_lane, exp_digit<W>(E, (uint32_t)(nwin - 1)));
  from_stage<L>(A, stage_lane);
  // remaining windows: W squarings, then one multiplication by T[digit]
  if constexpr (SQR) {
#pragma unroll 1
    for (int k = nwin - 2; k >= 0; --k) {
#pragma unroll 1
      for (int s = 0; s < W; ++s) mont_sqr_h<L, U>(A, N, np, stage_lane);
      table_select<L, W>(stage_lane, table_lane, exp_digit<W>(E, (uint32_t)k));
      mont_mul<L, U>(A, st, N, np);
    }
  } else {
    // one call site of mont_mul for every step keeps the hot code small
    const int nsteps = (nwin - 1) * (W + 1);
    int k = nwin - 2, s = 0;
#pragma unroll 1
    for (int step = 0; step < nsteps; ++step) {
      if (s < W) {
        to_stage<L>(stage_lane, A);
        ++s;
      } else {
        table_select<L, W>(stage_lane, table_lane, exp_digit<W>(E, (uint32_t)k));
        s = 0;
        --k;
      }
      mont_mul<L, U>(A, st, N, np);
    }
  }
}

// ------------------------------------------------------------------ tile addressing
// A tile is up to 32 operations handled by one warp (one lane each).  Dense
// batches address operation `base + lane` at row msgs + op*L; ragged batches
// take the operation index from a sorted list and its row from an offset table.
struct TileIO {
  const uint32_t *msgs;
  uint32_t *out;
  int32_t *status;          // may be null
  const int32_t *op_index;  // null: op = base + lane
  const uint64_t *offsets;  // null: row at op * L limbs
  uint32_t base, nops;      // first slot and number of live lanes
};

struct LaneOp {
  bool valid;
  uint32_t op;
  const uint32_t *row;
  uint32_t *orow;
};

__device__ __forceinline__ LaneOp lane_op(const TileIO &io, int lane, int L) {
  LaneOp r;
  r.valid = (uint32_t)lane < io.nops;
  const uint32_t slot = io.base + (uint32_t)lane;
  r.op = r.valid ? (io.op_index ? (uint32_t)io.op_index[slot] : slot) : 0u;
  const size_t off = io.offsets ? (size_t)io.offsets[r.op] : (size_t)r.op * (size_t)L;
  r.row = io.msgs + off;
  r.orow = io.out + off;
  return r;
}

// ------------------------------------------------------------------ CRT decryption (warp pairs)
struct CrtArgs {
  const uint32_t *keyrec;   // device key record
  const uint32_t *msgs;     // count rows of L = 2H limbs
  uint32_t *out;
  int32_t *status;          // may be null
  uint32_t count;
  uint4 *tables;            // scratch: per warp 2^W * H/4 * 32 uint4
};

template <int H, int W>
struct CrtSmem {
  static constexpr int kKeyWords = (KeyLayout(2 * H).total + 3) / 4 * 4;
  static constexpr int kStageU4 = (H / 4) * 32;   // one [H/4][32] uint4 buffer
  // bytes for P pairs: key record + per pair 2 exchange buffers + per warp 1 stage
  static constexpr size_t bytes(int P) {
    return kKeyWords * 4 + (size_t)P * 2 * kStageU4 * 16 + (size_t)2 * P * kStageU4 * 16;
  }
};

// One CRT tile on a warp pair.  ks: key record in shared memory; isP selects
// the p half (odd warp) or the q half (even warp); xb: this tile's exchange
// slot (+lane); bar_id: the pair's named barrier (64 threads).
template <int H, int W, int U, bool SQR>
__device__ __forceinline__ void crt_tile(const uint32_t *ks, bool isP, int lane, uint4 *stage_lane, uint4 *xb,
                                         uint4 *table_lane, int bar_id, const TileIO &io) {
  constexpr int L = 2 * H;
  constexpr KeyLayout lay(L);
  const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(ks);
  const uint32_t *Ms = ks + (isP ? lay.p : lay.q);
  const uint4 *r2 = reinterpret_cast<const uint4 *>(ks + (isP ? lay.r2p : lay.r2q));
  const uint4 *r3 = reinterpret_cast<const uint4 *>(ks + (isP ? lay.r3p : lay.r3q));
  const uint4 *one = reinterpret_cast<const uint4 *>(ks + (isP ? lay.onep : lay.oneq));
  const uint32_t *E = ks + (isP ? lay.dp : lay.dq);
  const uint32_t np = isP ? hd.np_p : hd.np_q;
  using NS = typename std::conditional<NPick<H, SQR>::reg, NRegs<H>, NSmem<H>>::type;
  NS N;
  if constexpr (NPick<H, SQR>::reg) N.load(reinterpret_cast<const uint4 *>(Ms)); else N.s = Ms;

  const LaneOp lo = lane_op(io, lane, L);
  uint32_t A[H];
  // CRT split in Montgomery form: x = c_lo*R + c_hi*R^2 = c*R mod m
  load_row<H>(A, lo.row, lo.valid);
  mont_mul<H, U>(A, SmemB{r2, 1}, N, np);
  to_stage<H>(stage_lane, A);
  load_row<H>(A, lo.row + H, lo.valid);
  mont_mul<H, U>(A, SmemB{r3, 1}, N, np);
  mod_add<H>(A, SmemB{stage_lane, 32}, N);
  // x^(d mod (m-1)) in Montgomery form
  fixed_window_exp<H, W, U, SQR>(A, E, 32 * H, one, stage_lane, table_lane, N, np);
  if (!isP) {
    // m_q = from-Montgomery; hand it to the p warp
    mont_mul<H, U>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.unitH), 1}, N, np);
    to_stage<H>(xb, A);
    pair_barrier(bar_id);
    return;
  }
  pair_barrier(bar_id);
  to_stage<H>(stage_lane, A);                      // A_p = m_p * R mod p
  from_stage<H>(A, xb);                            // m_q
  mont_mul<H, U>(A, SmemB{r2, 1}, N, np);          // m_q * R mod p
  mod_rsub<H>(A, SmemB{stage_lane, 32}, N);        // (m_p - m_q) * R mod p
  mont_mul<H, U>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.qinv), 1}, N, np);  // h
  // m = m_q + h * q, operand scanning over the limbs of q; one result limb per step
  uint32_t t[H + 2];
#pragma unroll
  for (int g = 0; g < H / 4; ++g) {
    const uint4 v = xb[g * 32];
    t[4 * g] = v.x; t[4 * g + 1] = v.y; t[4 * g + 2] = v.z; t[4 * g + 3] = v.w;
  }
  t[H] = 0u;
  t[H + 1] = 0u;
  const uint32_t *qs = ks + lay.q;
  const bool ok = lo.valid && row_below(lo.row, ks + lay.n, L);
  uint4 *orow = reinterpret_cast<uint4 *>(lo.orow);
#pragma unroll 1
  for (int i0 = 0; i0 < H; i0 += 4) {
    uint32_t r[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      mul_acc<H>(t, A, qs[i0 + u]);
      r[u] = t[0];
#pragma unroll
      for (int j = 0; j < H + 1; ++j) t[j] = t[j + 1];
      t[H + 1] = 0u;
    }
    if (lo.valid) orow[i0 / 4] = ok ? make_uint4(r[0], r[1], r[2], r[3]) : make_uint4(0u, 0u, 0u, 0u);
  }
#pragma unroll
  for (int g = 0; g < H / 4; ++g)
    if (lo.valid)
      orow[H / 4 + g] = ok ? make_uint4(t[4 * g], t[4 * g + 1], t[4 * g + 2], t[4 * g + 3])
                           : make_uint4(0u, 0u, 0u, 0u);
  if (lo.valid && io.status) io.status[lo.op] = ok ? 0 : -3;
}

template <int H, int W, int U, bool SQR>
__global__ void __launch_bounds__(256, 1) crt_kernel(CrtArgs a) {
  constexpr int L = 2 * H;
  constexpr KeyLayout lay(L);
  using Sm = CrtSmem<H, W>;
  extern __shared__ uint4 smem4[];
  uint32_t *ks = reinterpret_cast<uint32_t *>(smem4);
  for (int i = threadIdx.x; i < Sm::kKeyWords / 4; i += blockDim.x)
    smem4[i] = (i * 4 < (int)lay.total) ? reinterpret_cast<const uint4 *>(a.keyrec)[i]
                                         : make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  const int P = blockDim.x / 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = warp >> 1;
  const bool isP = (warp & 1) != 0;
  uint4 *xchg = smem4 + Sm::kKeyWords / 4 + (size_t)pair * 2 * Sm::kStageU4;
  uint4 *stage_lane = smem4 + Sm::kKeyWords / 4 + (size_t)P * 2 * Sm::kStageU4 + (size_t)warp * Sm::kStageU4 + lane;
  uint4 *table_lane = a.tables + ((size_t)blockIdx.x * (2 * P) + warp) * ((size_t)(1 << W) * (H / 4) * 32) + lane;
  const uint32_t ntiles = (a.count + 31) / 32;
  uint32_t iter = 0;
#pragma unroll 1
  for (uint32_t tile = blockIdx.x * P + pair; tile < ntiles; tile += gridDim.x * P, ++iter) {
    const uint32_t base = tile * 32;
    const TileIO io{a.msgs, a.out, a.status, nullptr, nullptr, base, min(32u, a.count - base)};
    crt_tile<H, W, U, SQR>(ks, isP, lane, stage_lane, xchg + (iter & 1) * Sm::kStageU4 + lane, table_lane,
                           1 + pair, io);
  }
}

// ------------------------------------------------------------------ single-limb keys
// The paper's own setting (Sec. 10: 8-bit-class keys, n = 131*137 = 17947):
// each thread computes one message's x^E mod m with 64-bit products reduced by
// "%" (Fig. 3), by left-to-right binary square-and-multiply (Fig. 5) over all
// 32 exponent bit positions with the multiplication always performed and kept
// by a mask, so the work does not depend on the exponent.
__device__ __forceinline__ uint32_t pow_mod32(uint32_t x, uint32_t E, uint32_t m) {
  uint64_t r = 1u % m;
  const uint64_t xm = x % m;
#pragma unroll 4
  for (int b = 31; b >= 0; --b) {
    r = (r * r) % m;
    const uint64_t rx = (r * xm) % m;
    const uint64_t keep = 0ull - (uint64_t)((E >> b) & 1u);
    r = (rx & keep) | (r & ~keep);
  }
  return (uint32_t)r;
}

// kind 0: x^e mod n; 2: x^d mod n; 1: CRT (m_p = x^dp mod p, m_q = x^dq mod q,
// h = qinv (m_p - m_q) mod p, m = m_q + h q) with p, q, dp, dq, qinv in the header.
__device__ __forceinline__ uint32_t toy_op(const uint32_t *rec, const KeyHeader &hd, int kind, uint32_t x) {
  const KeyLayout lay(1);
  const uint32_t n = rec[lay.n];
  if (kind == 0) return pow_mod32(x, rec[lay.e], n);
  if (kind == 2) return pow_mod32(x, rec[lay.d], n);
  const uint32_t p = hd.reserved[0], q = hd.reserved[1];
  const uint32_t mp = pow_mod32(x, hd.reserved[2], p);
  const uint32_t mq = pow_mod32(x, hd.reserved[3], q);
  const uint64_t diff = ((uint64_t)mp + p - (mq % p)) % p;
  const uint64_t h = (diff * hd.reserved[4]) % p;
  return (uint32_t)(mq + h * q);
}

struct ToyArgs {
  const uint32_t *keyrec;
  const uint32_t *msgs;
  uint32_t *out;
  int32_t *status;
  uint32_t count;
  int32_t kind;  // 0 public, 1 CRT, 2 plain private
};

// ------------------------------------------------------------------ plain private exponent (mod n)
struct ExpArgs {
  const uint32_t *keyrec;
  const uint32_t *msgs;
  uint32_t *out;
  int32_t *status;
  uint32_t count;
  uint4 *tables;            // PLAIN only: per warp 2^W * L/4 * 32 uint4
};

template <int L>
struct ExpSmem {
  static constexpr int kKeyWords = (KeyLayout(L).total + 3) / 4 * 4;
  static constexpr int kStageU4 = (L / 4) * 32;
  static constexpr size_t bytes(int warps) { return kKeyWords * 4 + (size_t)warps * 2 * kStageU4 * 16; }
};

template <int L>
__device__ __forceinline__ void load_key_smem(uint4 *smem4, const uint32_t *keyrec) {
  constexpr KeyLayout lay(L);
  constexpr int kw = ExpSmem<L>::kKeyWords;
  for (int i = threadIdx.x; i < kw / 4; i += blockDim.x)
    smem4[i] = (i * 4 < (int)lay.total) ? reinterpret_cast<const uint4 *>(keyrec)[i]
                                         : make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
}

// One tile of plain private-exponent operations on one warp.
template <int L, int W, int U, bool SQR>
__device__ __forceinline__ void plain_tile(const uint32_t *ks, int lane, uint4 *stage_lane, uint4 *table_lane,
                                           const TileIO &io) {
  constexpr KeyLayout lay(L);
  const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(ks);
  using NS = typename std::conditional<NPick<L, SQR>::reg, NRegs<L>, NSmem<L>>::type;
  NS N;
  if constexpr (NPick<L, SQR>::reg) N.load(reinterpret_cast<const uint4 *>(ks + lay.n)); else N.s = ks + lay.n;
  const LaneOp lo = lane_op(io, lane, L);
  uint32_t A[L];
  load_row<L>(A, lo.row, lo.valid);
  mont_mul<L, U>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.r2n), 1}, N, hd.np_n);
  fixed_window_exp<L, W, U, SQR>(A, ks + lay.d, 32 * L, reinterpret_cast<const uint4 *>(ks + lay.onen),
                                 stage_lane, table_lane, N, hd.np_n);
  mont_mul<L, U>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.unitL), 1}, N, hd.np_n);
  const bool ok = lo.valid && row_below(lo.row, ks + lay.n, L);
  if (lo.valid) {
    uint4 *orow = reinterpret_cast<uint4 *>(lo.orow);
#pragma unroll
    for (int g = 0; g < L / 4; ++g)
      orow[g] = ok ? make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]) : make_uint4(0u, 0u, 0u, 0u);
    if (io.status) io.status[lo.op] = ok ? 0 : -3;
  }
}

template <int L, int W, int U, bool SQR>
__global__ void __launch_bounds__(256) plain_kernel(ExpArgs a) {
  using Sm = ExpSmem<L>;
  extern __shared__ uint4 smem4[];
  load_key_smem<L>(smem4, a.keyrec);
  const uint32_t *ks = reinterpret_cast<const uint32_t *>(smem4);
  const int nw = blockDim.x / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4 *stage_lane = smem4 + Sm::kKeyWords / 4 + (size_t)warp * 2 * Sm::kStageU4 + lane;
  uint4 *table_lane = a.tables + ((size_t)blockIdx.x * nw + warp) * ((size_t)(1 << W) * (L / 4) * 32) + lane;
  const uint32_t ntiles = (a.count + 31) / 32;
#pragma unroll 1
  for (uint32_t tile = blockIdx.x * nw + warp; tile < ntiles; tile += gridDim.x * nw) {
    const uint32_t base = tile * 32;
    const TileIO io{a.msgs, a.out, a.status, nullptr, nullptr, base, min(32u, a.count - base)};
    plain_tile<L, W, U, SQR>(ks, lane, stage_lane, table_lane, io);
  }
}

// ------------------------------------------------------------------ public exponent (binary, Fig. 5)
// One tile of public-exponent operations on one warp; sq_lane, x_lane: two
// per-lane staging buffers.
template <int L, int U>
__device__ __forceinline__ void pub_tile(const uint32_t *ks, int lane, uint4 *sq_lane, uint4 *x_lane,
                                         const TileIO &io) {
  constexpr KeyLayout lay(L);
  const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(ks);
  using NS = typename std::conditional<NPick<L, false>::reg, NRegs<L>, NSmem<L>>::type;
  NS N;
  if constexpr (NPick<L, false>::reg) N.load(reinterpret_cast<const uint4 *>(ks + lay.n)); else N.s = ks + lay.n;
  const uint32_t *E = ks + lay.e;
  const int ebits = (int)hd.e_bits;
  const LaneOp lo = lane_op(io, lane, L);
  uint32_t A[L];
  load_row<L>(A, lo.row, lo.valid);
  mont_mul<L, U>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.r2n), 1}, N, hd.np_n);
  to_stage<L>(x_lane, A);
  // left-to-right binary over the bits below the top one; one call site
  int bit = ebits - 2;
  bool mul_next = false;
#pragma unroll 1
  while (bit >= 0 || mul_next) {
    const uint4 *b;
    if (mul_next) {
      b = x_lane;
      mul_next = false;
      --bit;
    } else {
      to_stage<L>(sq_lane, A);
      b = sq_lane;
      mul_next = (E[bit >> 5] >> (bit & 31)) & 1u;
      if (!mul_next) --bit;
    }
    mont_mul<L, U>(A, SmemB{b, 32}, N, hd.np_n);
  }
  mont_mul<L, U>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.unitL), 1}, N, hd.np_n);
  const bool ok = lo.valid && row_below(lo.row, ks + lay.n, L);
  if (lo.valid) {
    uint4 *orow = reinterpret_cast<uint4 *>(lo.orow);
#pragma unroll
    for (int g = 0; g < L / 4; ++g)
      orow[g] = ok ? make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]) : make_uint4(0u, 0u, 0u, 0u);
    if (io.status) io.status[lo.op] = ok ? 0 : -3;
  }
}

template <int L, int U>
__global__ void __launch_bounds__(256) pub_kernel(ExpArgs a) {
  using Sm = ExpSmem<L>;
  extern __shared__ uint4 smem4[];
  load_key_smem<L>(smem4, a.keyrec);
  const uint32_t *ks = reinterpret_cast<const uint32_t *>(smem4);
  const int nw = blockDim.x / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4 *sq_lane = smem4 + Sm::kKeyWords / 4 + (size_t)warp * 2 * Sm::kStageU4 + lane;
  uint4 *x_lane = sq_lane + Sm::kStageU4;
  const uint32_t ntiles = (a.count + 31) / 32;
#pragma unroll 1
  for (uint32_t tile = blockIdx.x * nw + warp; tile < ntiles; tile += gridDim.x * nw) {
    const uint32_t base = tile * 32;
    const TileIO io{a.msgs, a.out, a.status, nullptr, nullptr, base, min(32u, a.count - base)};
    pub_tile<L, U>(ks, lane, sq_lane, x_lane, io);
  }
}

// ------------------------------------------------------------------ public exponent, sliding windows
// Fig. 7 (sliding window method) for long public, i.e. non-secret, exponents.
// The exponent is scanned from its top bit: a 0 bit costs one squaring; a 1
// bit opens the longest window of at most W bits that ends in a 1 bit (an odd
// value v), which costs its squarings and one multiplication by x^v from a
// table of the odd powers x, x^3, ..., x^(2^W - 1).  The leading window is a
// table read.  The exponent is the key's (the same for every lane and not
// secret), so the control flow and the table index may depend on it; every
// product goes through one mont_mul call site.
template <int L>
__device__ __forceinline__ void table_load(uint32_t (&A)[L], const uint4 *table_lane, int e) {
#pragma unroll
  for (int g = 0; g < L / 4; ++g) {
    const uint4 v = table_lane[(e * (L / 4) + g) * 32];
    A[4 * g] = v.x; A[4 * g + 1] = v.y; A[4 * g + 2] = v.z; A[4 * g + 3] = v.w;
  }
}

// Bits i down to the lowest 1 bit at or above max(i - W + 1, 0), as a value; *j gets that bit's index.
template <int W>
__device__ __forceinline__ uint32_t slide_window(const uint32_t *E, int i, int *j) {
  int lo = i - W + 1 > 0 ? i - W + 1 : 0;
  while (!((E[lo >> 5] >> (lo & 31)) & 1u)) ++lo;
  uint32_t v = 0;
  for (int b = i; b >= lo; --b) v = (v << 1) | ((E[b >> 5] >> (b & 31)) & 1u);
  *j = lo;
  return v;
}

template <int L, int U, int W>
__device__ __forceinline__ void pub_slide_tile(const uint32_t *ks, int lane, uint4 *sq_lane, uint4 *x2_lane,
                                               uint4 *table_lane, const TileIO &io) {
  constexpr KeyLayout lay(L);
  constexpr int NT = 1 << (W - 1);   // table entries: x^(2t+1), t < NT
  const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(ks);
  using NS = typename std::conditional<NPick<L, false>::reg, NRegs<L>, NSmem<L>>::type;
  NS N;
  if constexpr (NPick<L, false>::reg) N.load(reinterpret_cast<const uint4 *>(ks + lay.n)); else N.s = ks + lay.n;
  const uint32_t *E = ks + lay.e;
  const LaneOp lo = lane_op(io, lane, L);
  uint32_t A[L];
  load_row<L>(A, lo.row, lo.valid);
  int i = (int)hd.e_bits - 1;   // highest exponent bit not yet consumed
  int nsq = 0, tidx = 0, step = 0;
  bool mul_pending = false, started = false, finished = false;
#pragma unroll 1
  while (true) {
    SmemB B{sq_lane, 32};
    if (step == 0) {
      B = SmemB{reinterpret_cast<const uint4 *>(ks + lay.r2n), 1};   // x R
    } else if (step == 1) {
      to_stage<L>(sq_lane, A);                                       // x^2 R
    } else if (step <= NT) {
      B = SmemB{x2_lane, 32};                                        // x^(2(step-1)+1) R
    } else {
      if (!started) {                                                // leading window
        int j;
        const uint32_t v = slide_window<W>(E, i, &j);
        table_load<L>(A, table_lane, (int)(v >> 1));
        i = j - 1;
        started = true;
      }
      if (nsq == 0 && !mul_pending) {
        if (i < 0) {
          if (finished) break;
          B = SmemB{reinterpret_cast<const uint4 *>(ks + lay.unitL), 1};   // leave Montgomery form
          finished = true;
        } else if (!((E[i >> 5] >> (i & 31)) & 1u)) {
          nsq = 1;
          --i;
        } else {
          int j;
          const uint32_t v = slide_window<W>(E, i, &j);
          nsq = i - j + 1;
          tidx = (int)(v >> 1);
          mul_pending = true;
          i = j - 1;
        }
      }
      if (!finished) {
        if (nsq > 0) {
          to_stage<L>(sq_lane, A);
          --nsq;
        } else {
#pragma unroll
          for (int g = 0; g < L / 4; ++g) sq_lane[g * 32] = table_lane[(tidx * (L / 4) + g) * 32];
          mul_pending = false;
        }
      }
    }
    mont_mul<L, U>(A, B, N, hd.np_n);
    if (step == 0) {
      table_store<L>(table_lane, 0, A);
    } else if (step == 1) {
      to_stage<L>(x2_lane, A);
      table_load<L>(A, table_lane, 0);
    } else if (step <= NT) {
      table_store<L>(table_lane, step - 1, A);
    }
    ++step;
  }
  const bool ok = lo.valid && row_below(lo.row, ks + lay.n, L);
  if (lo.valid) {
    uint4 *orow = reinterpret_cast<uint4 *>(lo.orow);
#pragma unroll
    for (int g = 0; g < L / 4; ++g)
      orow[g] = ok ? make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]) : make_uint4(0u, 0u, 0u, 0u);
    if (io.status) io.status[lo.op] = ok ? 0 : -3;
  }
}

// tables: per warp 2^(W-1) * L/4 * 32 uint4
template <int L, int U, int W>
__global__ void __launch_bounds__(256) pub_slide_kernel(ExpArgs a) {
  using Sm = ExpSmem<L>;
  extern __shared__ uint4 smem4[];
  load_key_smem<L>(smem4, a.keyrec);
  const uint32_t *ks = reinterpret_cast<const uint32_t *>(smem4);
  const int nw = blockDim.x / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4 *sq_lane = smem4 + Sm::kKeyWords / 4 + (size_t)warp * 2 * Sm::kStageU4 + lane;
  uint4 *x2_lane = sq_lane + Sm::kStageU4;
  uint4 *table_lane = a.tables + (size_t)(blockIdx.x * nw + warp) * (1 << (W - 1)) * (L / 4) * 32 + lane;
  const uint32_t ntiles = (a.count + 31) / 32;
#pragma unroll 1
  for (uint32_t tile = blockIdx.x * nw + warp; tile < ntiles; tile += gridDim.x * nw) {
    const uint32_t base = tile * 32;
    const TileIO io{a.msgs, a.out, a.status, nullptr, nullptr, base, min(32u, a.count - base)};
    pub_slide_tile<L, U, W>(ks, lane, sq_lane, x2_lane, table_lane, io);
  }
}

// ------------------------------------------------------------------ public exponent, wide moduli
// L = 96 or 128 limbs: A, the base x and the key constants stay in shared
// memory (mont_mul_smemA); same binary method as pub_tile.
template <int L, int U>
__device__ __forceinline__ void pub_wide_tile(const uint32_t *ks, int lane, uint4 *A_lane, uint4 *x_lane,
                                              const TileIO &io) {
  constexpr KeyLayout lay(L);
  const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(ks);
  NSmem<L> N;
  N.s = ks + lay.n;
  const uint32_t *E = ks + lay.e;
  const int ebits = (int)hd.e_bits;
  const LaneOp lo = lane_op(io, lane, L);
  const uint4 *r4 = reinterpret_cast<const uint4 *>(lo.row);
#pragma unroll 4
  for (int g = 0; g < L / 4; ++g) A_lane[g * 32] = lo.valid ? __ldg(r4 + g) : make_uint4(0u, 0u, 0u, 0u);
  mont_mul_smemA<L, U>(A_lane, SmemB{reinterpret_cast<const uint4 *>(ks + lay.r2n), 1}, N, hd.np_n);
#pragma unroll 4
  for (int g = 0; g < L / 4; ++g) x_lane[g * 32] = A_lane[g * 32];
  int bit = ebits - 2;
  bool mul_next = false;
#pragma unroll 1
  while (bit >= 0 || mul_next) {
    const uint4 *b;
    if (mul_next) {
      b = x_lane;
      mul_next = false;
      --bit;
    } else {
      b = A_lane;
      mul_next = (E[bit >> 5] >> (bit & 31)) & 1u;
      if (!mul_next) --bit;
    }
    mont_mul_smemA<L, U>(A_lane, SmemB{b, 32}, N, hd.np_n);
  }
  mont_mul_smemA<L, U>(A_lane, SmemB{reinterpret_cast<const uint4 *>(ks + lay.unitL), 1}, N, hd.np_n);
  const bool ok = lo.valid && row_below(lo.row, ks + lay.n, L);
  if (lo.valid) {
    uint4 *orow = reinterpret_cast<uint4 *>(lo.orow);
#pragma unroll 4
    for (int g = 0; g < L / 4; ++g) orow[g] = ok ? A_lane[g * 32] : make_uint4(0u, 0u, 0u, 0u);
    if (io.status) io.status[lo.op] = ok ? 0 : -3;
  }
}

template <int L, int U>
__global__ void __launch_bounds__(128) pub_wide_kernel(ExpArgs a) {
  using Sm = ExpSmem<L>;
  extern __shared__ uint4 smem4[];
  load_key_smem<L>(smem4, a.keyrec);
  const uint32_t *ks = reinterpret_cast<const uint32_t *>(smem4);
  const int nw = blockDim.x / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4 *A_lane = smem4 + Sm::kKeyWords / 4 + (size_t)warp * 2 * Sm::kStageU4 + lane;
  uint4 *x_lane = A_lane + Sm::kStageU4;
  const uint32_t ntiles = (a.count + 31) / 32;
#pragma unroll 1
  for (uint32_t tile = blockIdx.x * nw + warp; tile < ntiles; tile += gridDim.x * nw) {
    const uint32_t base = tile * 32;
    const TileIO io{a.msgs, a.out, a.status, nullptr, nullptr, base, min(32u, a.count - base)};
    pub_wide_tile<L, U>(ks, lane, A_lane, x_lane, io);
  }
}

}  // namespace rsagpu
