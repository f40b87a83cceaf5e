// kernels_t.cuh -- kernels with T lanes per operation (threads per operation
// T = 2 or 4): a warp holds 32/T operations.  Same methods as kernels.cuh
// (CRT with Garner recombination on warp pairs, constant-time fixed window,
// binary public exponent); every number is sliced over the group's ranks
// (mont_t.cuh).  Fewer limbs per thread means fewer registers per thread and
// a shorter dependency chain per operation (lower latency per operation), at
// the cost of shuffles and carry resolution per Montgomery product.
#pragma once
#include <cstdint>

#include "kernels.cuh"
#include "mont_t.cuh"

namespace rsagpu {

// stage <- T[d] for this rank's slice (all 2^W entries read and masked)
template <int K, int W>
__device__ __forceinline__ void table_select_to(uint4 *out, int ostride, const uint4 *table_lane, uint32_t d) {
#pragma unroll 1
  for (int gg = 0; gg < K / 4; ++gg) {
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 8
    for (int e = 0; e < (1 << W); ++e) {
      const uint4 v = table_lane[(e * (K / 4) + gg) * 32];
      const uint32_t m = 0u - (uint32_t)((uint32_t)e == d);
      acc.x |= v.x & m;
      acc.y |= v.y & m;
      acc.z |= v.z & m;
      acc.w |= v.w & m;
    }
    out[gg * ostride] = acc;
  }
}

template <int K, int T>
__device__ __forceinline__ void slice_of_uniform(uint32_t (&A)[K], const uint32_t *full, const Group<T> &g) {
  from_uniform<K>(A, reinterpret_cast<const uint4 *>(full + g.r * K));
}

// fixed_window_exp (kernels.cuh) for a group: A in, A = x^E out (Montgomery form)
template <int K, int T, int W, int U, class NS>
__device__ __forceinline__ void fixed_window_exp_t(uint32_t (&A)[K], const uint32_t *E, int ebits,
                                                   const uint32_t *one_full, uint4 *stage_op, uint4 *table_lane,
                                                   const NS &N, uint32_t np, const Group<T> &g) {
  constexpr int NE = 1 << W;
  constexpr int OS = 32 / T;
  const SmemB st{stage_op, OS};
  uint4 *sel_out = stage_op + g.r * (K / 4) * OS;
  {
    uint32_t one[K];
    slice_of_uniform<K, T>(one, one_full, g);
    table_store<K>(table_lane, 0, one);
  }
  table_store<K>(table_lane, 1, A);
  __syncwarp();
  to_stage_t<K, T>(stage_op, A, g);
  __syncwarp();
#pragma unroll 1
  for (int i = 2; i < NE; ++i) {
    mont_mul_t<K, T, U>(A, st, N, np, g);
    table_store<K>(table_lane, i, A);
  }
  const int nwin = (ebits + W - 1) / W;
  __syncwarp();
  table_select_to<K, W>(sel_out, OS, table_lane, exp_digit<W>(E, (uint32_t)(nwin - 1)));
  __syncwarp();
  from_stage_t<K, T>(A, stage_op, g);
  const int nsteps = (nwin - 1) * (W + 1);
  int k = nwin - 2, s = 0;
#pragma unroll 1
  for (int step = 0; step < nsteps; ++step) {
    __syncwarp();
    if (s < W) {
      to_stage_t<K, T>(stage_op, A, g);
      ++s;
    } else {
      table_select_to<K, W>(sel_out, OS, table_lane, exp_digit<W>(E, (uint32_t)k));
      s = 0;
      --k;
    }
    __syncwarp();
    mont_mul_t<K, T, U>(A, st, N, np, g);
  }
}

// load this rank's slice (K limbs at word offset `off` of the row)
template <int K>
__device__ __forceinline__ void load_slice(uint32_t (&A)[K], const uint32_t *row, int off, bool valid) {
  load_row<K>(A, row + off, valid);
}

// ------------------------------------------------------------------ CRT on warp pairs, T lanes per operation
template <int H, int T, int W, int U>
__device__ __forceinline__ void crt_tile_t(const uint32_t *ks, bool isP, const Group<T> &g, uint4 *stage_op,
                                           uint4 *xb_op, uint4 *table_lane, int bar_id, const TileIO &io) {
  constexpr int L = 2 * H;
  constexpr int K = H / T;
  constexpr int OS = 32 / T;
  constexpr KeyLayout lay(L);
  const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(ks);
  const uint32_t *Ms = ks + (isP ? lay.p : lay.q);
  const uint4 *r2 = reinterpret_cast<const uint4 *>(ks + (isP ? lay.r2p : lay.r2q));
  const uint4 *r3 = reinterpret_cast<const uint4 *>(ks + (isP ? lay.r3p : lay.r3q));
  const uint32_t *one = ks + (isP ? lay.onep : lay.oneq);
  const uint32_t *E = ks + (isP ? lay.dp : lay.dq);
  const uint32_t np = isP ? hd.np_p : hd.np_q;
  using NS = typename std::conditional<(K <= 16), NRegs<K>, NSmem<K>>::type;
  NS N;
  if constexpr (K <= 16) N.load(reinterpret_cast<const uint4 *>(Ms + g.r * K)); else N.s = Ms + g.r * K;

  const bool valid = (uint32_t)g.opi < io.nops;
  const uint32_t slot = io.base + (uint32_t)g.opi;
  const uint32_t op = valid ? (io.op_index ? (uint32_t)io.op_index[slot] : slot) : 0u;
  const size_t off = io.offsets ? (size_t)io.offsets[op] : (size_t)op * L;
  const uint32_t *row = io.msgs + off;
  uint32_t *orow = io.out + off;
  const SmemB st{stage_op, OS};

  uint32_t A[K];
  load_slice<K>(A, row, g.r * K, valid);                   // c_lo slice
  mont_mul_t<K, T, U>(A, SmemB{r2, 1}, N, np, g);
  __syncwarp();
  to_stage_t<K, T>(stage_op, A, g);
  __syncwarp();
  load_slice<K>(A, row, H + g.r * K, valid);               // c_hi slice
  mont_mul_t<K, T, U>(A, SmemB{r3, 1}, N, np, g);
  mod_add_t<K, T>(A, st, N, g);
  fixed_window_exp_t<K, T, W, U>(A, E, 32 * H, one, stage_op, table_lane, N, np, g);
  if (!isP) {
    mont_mul_t<K, T, U>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.unitH), 1}, N, np, g);
    to_stage_t<K, T>(xb_op, A, g);
    pair_barrier(bar_id);
    return;
  }
  pair_barrier(bar_id);
  __syncwarp();
  to_stage_t<K, T>(stage_op, A, g);                        // A_p = m_p * R mod p
  __syncwarp();
  uint32_t mq[K];
  from_stage_t<K, T>(mq, xb_op, g);
#pragma unroll
  for (int j = 0; j < K; ++j) A[j] = mq[j];
  mont_mul_t<K, T, U>(A, SmemB{r2, 1}, N, np, g);         // m_q * R mod p
  mod_rsub_t<K, T>(A, st, N, g);                           // (m_p - m_q) * R mod p
  mont_mul_t<K, T, U>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.qinv), 1}, N, np, g);  // h
  // m = m_q + h * q: operand scanning over the limbs of q; rank 0 emits one limb per step
  uint32_t t[K + 2];
#pragma unroll
  for (int j = 0; j < K; ++j) t[j] = mq[j];
  uint32_t pend = 0u;
  const uint32_t *qs = ks + lay.q;
  // both halves compared by every lane (cmp_t holds warp-wide ballots, so it must
  // never sit under a condition that differs between the warp's operations)
  const int cmp_hi = cmp_t<K, T>(row + H + g.r * K, ks + lay.n + H + g.r * K, g);
  const int cmp_lo = cmp_t<K, T>(row + g.r * K, ks + lay.n + g.r * K, g);
  const int cmp = cmp_hi != 0 ? cmp_hi : cmp_lo;
  const bool ok = valid && cmp < 0;
#pragma unroll 1
  for (int i = 0; i < H; ++i) {
    t[K] = pend;
    t[K + 1] = 0u;
    mul_acc<K>(t, A, qs[i]);
    const bool emit = (g.r == 0) & valid;
    if (emit) orow[i] = ok ? t[0] : 0u;
    const uint32_t up = g.from_above(t[0]);
#pragma unroll
    for (int j = 0; j < K - 1; ++j) t[j] = t[j + 1];
    t[K - 1] = add_cc(t[K], up);
    pend = addc(t[K + 1], 0u);
  }
  uint32_t s[K];
#pragma unroll
  for (int j = 0; j < K; ++j) s[j] = t[j];
  uint32_t top;
  carry_resolve_t<K, T>(s, pend, &top, g);
  if (valid) {
    uint4 *o4 = reinterpret_cast<uint4 *>(orow + H + g.r * K);
#pragma unroll
    for (int gg = 0; gg < K / 4; ++gg)
      o4[gg] = ok ? make_uint4(s[4 * gg], s[4 * gg + 1], s[4 * gg + 2], s[4 * gg + 3]) : make_uint4(0u, 0u, 0u, 0u);
    if (g.r == 0 && io.status) io.status[op] = ok ? 0 : -3;
  }
}

template <int H, int T>
struct CrtSmemT {
  static constexpr int kKeyWords = (KeyLayout(2 * H).total + 3) / 4 * 4;
  static constexpr int kStageU4 = (H / 4) * (32 / T);   // [H/4][32/T] uint4 per warp
  static constexpr size_t bytes(int P) {
    return kKeyWords * 4 + (size_t)P * 2 * kStageU4 * 16 + (size_t)2 * P * kStageU4 * 16;
  }
};

template <int H, int T, int W, int U>
__global__ void __launch_bounds__(256, 1) crt_kernel_t(CrtArgs a) {
  constexpr int L = 2 * H;
  constexpr KeyLayout lay(L);
  using Sm = CrtSmemT<H, T>;
  constexpr int OPW = 32 / T;   // operations per warp
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
  const Group<T> g(lane);
  uint4 *xchg = smem4 + Sm::kKeyWords / 4 + (size_t)pair * 2 * Sm::kStageU4;
  uint4 *stage = smem4 + Sm::kKeyWords / 4 + (size_t)P * 2 * Sm::kStageU4 + (size_t)warp * Sm::kStageU4;
  uint4 *table_lane = a.tables + ((size_t)blockIdx.x * (2 * P) + warp) * ((size_t)(1 << W) * (H / T / 4) * 32) + lane;
  const uint32_t ntiles = (a.count + OPW - 1) / OPW;
  uint32_t iter = 0;
#pragma unroll 1
  for (uint32_t tile = blockIdx.x * P + pair; tile < ntiles; tile += gridDim.x * P, ++iter) {
    const uint32_t base = tile * OPW;
    const TileIO io{a.msgs, a.out, a.status, nullptr, nullptr, base, min((uint32_t)OPW, a.count - base)};
    crt_tile_t<H, T, W, U>(ks, isP, g, stage + g.opi, xchg + (iter & 1) * Sm::kStageU4 + g.opi, table_lane,
                           1 + pair, io);
  }
}

// ------------------------------------------------------------------ public exponent, T lanes per operation
template <int L, int T, int U>
__device__ __forceinline__ void pub_tile_t(const uint32_t *ks, const Group<T> &g, uint4 *sq_op, uint4 *x_op,
                                           const TileIO &io) {
  constexpr int K = L / T;
  constexpr int OS = 32 / T;
  constexpr KeyLayout lay(L);
  const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(ks);
  using NS = typename std::conditional<(K <= 16), NRegs<K>, NSmem<K>>::type;
  NS N;
  if constexpr (K <= 16) N.load(reinterpret_cast<const uint4 *>(ks + lay.n + g.r * K)); else N.s = ks + lay.n + g.r * K;
  const uint32_t *E = ks + lay.e;
  const int ebits = (int)hd.e_bits;
  const bool valid = (uint32_t)g.opi < io.nops;
  const uint32_t slot = io.base + (uint32_t)g.opi;
  const uint32_t op = valid ? (io.op_index ? (uint32_t)io.op_index[slot] : slot) : 0u;
  const size_t off = io.offsets ? (size_t)io.offsets[op] : (size_t)op * L;
  const uint32_t *row = io.msgs + off;
  uint32_t A[K];
  load_slice<K>(A, row, g.r * K, valid);
  mont_mul_t<K, T, U>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.r2n), 1}, N, hd.np_n, g);
  __syncwarp();
  to_stage_t<K, T>(x_op, A, g);
  int bit = ebits - 2;
  bool mul_next = false;
#pragma unroll 1
  while (bit >= 0 || mul_next) {
    const uint4 *b;
    __syncwarp();
    if (mul_next) {
      b = x_op;
      mul_next = false;
      --bit;
    } else {
      to_stage_t<K, T>(sq_op, A, g);
      b = sq_op;
      mul_next = (E[bit >> 5] >> (bit & 31)) & 1u;
      if (!mul_next) --bit;
    }
    __syncwarp();
    mont_mul_t<K, T, U>(A, SmemB{b, OS}, N, hd.np_n, g);
  }
  mont_mul_t<K, T, U>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.unitL), 1}, N, hd.np_n, g);
  const int cmp = cmp_t<K, T>(row + g.r * K, ks + lay.n + g.r * K, g);  // every lane, see crt_tile_t
  const bool ok = valid && cmp < 0;
  if (valid) {
    uint4 *o4 = reinterpret_cast<uint4 *>(io.out + off + g.r * K);
#pragma unroll
    for (int gg = 0; gg < K / 4; ++gg)
      o4[gg] = ok ? make_uint4(A[4 * gg], A[4 * gg + 1], A[4 * gg + 2], A[4 * gg + 3]) : make_uint4(0u, 0u, 0u, 0u);
    if (g.r == 0 && io.status) io.status[op] = ok ? 0 : -3;
  }
}

template <int L, int T, int U>
__global__ void __launch_bounds__(256) pub_kernel_t(ExpArgs a) {
  using Sm = ExpSmem<L>;
  constexpr int OPW = 32 / T;
  constexpr int kStage = (L / 4) * OPW;   // [L/4][32/T] uint4 per buffer
  extern __shared__ uint4 smem4[];
  load_key_smem<L>(smem4, a.keyrec);
  const uint32_t *ks = reinterpret_cast<const uint32_t *>(smem4);
  const int nw = blockDim.x / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Group<T> g(lane);
  uint4 *sq = smem4 + Sm::kKeyWords / 4 + (size_t)warp * 2 * kStage;
  const uint32_t ntiles = (a.count + OPW - 1) / OPW;
#pragma unroll 1
  for (uint32_t tile = blockIdx.x * nw + warp; tile < ntiles; tile += gridDim.x * nw) {
    const uint32_t base = tile * OPW;
    const TileIO io{a.msgs, a.out, a.status, nullptr, nullptr, base, min((uint32_t)OPW, a.count - base)};
    pub_tile_t<L, T, U>(ks, g, sq + g.opi, sq + kStage + g.opi, io);
  }
}


// ------------------------------------------------------------------ plain private exponent, T lanes per operation
// x^d mod n without the CRT split (d of the full key length): to Montgomery
// form, the constant-time fixed window of fixed_window_exp_t over all 32L bits
// of d, back out of Montgomery form.  For 3072/4096-bit moduli, whose full-size
// numbers do not fit one thread's registers.
template <int L, int T, int W, int U>
__device__ __forceinline__ void plain_tile_t(const uint32_t *ks, const Group<T> &g, uint4 *stage_op,
                                             uint4 *table_lane, const TileIO &io) {
  constexpr int K = L / T;
  constexpr KeyLayout lay(L);
  const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(ks);
  using NS = typename std::conditional<(K <= 16), NRegs<K>, NSmem<K>>::type;
  NS N;
  if constexpr (K <= 16) N.load(reinterpret_cast<const uint4 *>(ks + lay.n + g.r * K)); else N.s = ks + lay.n + g.r * K;
  const bool valid = (uint32_t)g.opi < io.nops;
  const uint32_t slot = io.base + (uint32_t)g.opi;
  const uint32_t op = valid ? (io.op_index ? (uint32_t)io.op_index[slot] : slot) : 0u;
  const size_t off = io.offsets ? (size_t)io.offsets[op] : (size_t)op * L;
  const uint32_t *row = io.msgs + off;
  uint32_t A[K];
  load_slice<K>(A, row, g.r * K, valid);
  mont_mul_t<K, T, U>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.r2n), 1}, N, hd.np_n, g);
  fixed_window_exp_t<K, T, W, U>(A, ks + lay.d, 32 * L, ks + lay.onen, stage_op, table_lane, N, hd.np_n, g);
  mont_mul_t<K, T, U>(A, SmemB{reinterpret_cast<const uint4 *>(ks + lay.unitL), 1}, N, hd.np_n, g);
  const int cmp = cmp_t<K, T>(row + g.r * K, ks + lay.n + g.r * K, g);  // every lane, see crt_tile_t
  const bool ok = valid && cmp < 0;
  if (valid) {
    uint4 *o4 = reinterpret_cast<uint4 *>(io.out + off + g.r * K);
#pragma unroll
    for (int gg = 0; gg < K / 4; ++gg)
      o4[gg] = ok ? make_uint4(A[4 * gg], A[4 * gg + 1], A[4 * gg + 2], A[4 * gg + 3]) : make_uint4(0u, 0u, 0u, 0u);
    if (g.r == 0 && io.status) io.status[op] = ok ? 0 : -3;
  }
}

// one warp per 32/T operations; per warp one stage of [L/4][32/T] uint4 in
// shared memory and a window table of 2^W entries x (L/T/4) x 32 uint4
template <int L, int T, int W, int U>
__global__ void __launch_bounds__(256) plain_kernel_t(ExpArgs a) {
  using Sm = ExpSmem<L>;
  constexpr int OPW = 32 / T;
  constexpr int kStage = (L / 4) * OPW;
  extern __shared__ uint4 smem4[];
  load_key_smem<L>(smem4, a.keyrec);
  const uint32_t *ks = reinterpret_cast<const uint32_t *>(smem4);
  const int nw = blockDim.x / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Group<T> g(lane);
  uint4 *stage = smem4 + Sm::kKeyWords / 4 + (size_t)warp * kStage;
  uint4 *table_lane = a.tables + ((size_t)blockIdx.x * nw + warp) * ((size_t)(1 << W) * (L / T / 4) * 32) + lane;
  const uint32_t ntiles = (a.count + OPW - 1) / OPW;
#pragma unroll 1
  for (uint32_t tile = blockIdx.x * nw + warp; tile < ntiles; tile += gridDim.x * nw) {
    const uint32_t base = tile * OPW;
    const TileIO io{a.msgs, a.out, a.status, nullptr, nullptr, base, min((uint32_t)OPW, a.count - base)};
    plain_tile_t<L, T, W, U>(ks, g, stage + g.opi, table_lane, io);
  }
}

}  // namespace rsagpu
