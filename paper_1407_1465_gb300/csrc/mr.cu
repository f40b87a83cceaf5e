// mr.cu -- batch Miller-Rabin probable-prime tests (key generation, Fig. 1:
// "choose two large primes"; the paper names no test, this is the standard one).
//
// One candidate per thread, 32 per warp (512/1024 bits; 2048-bit candidates
// run on four lanes each, mr_kernel_t below).  Every candidate is its own
// modulus, so its Montgomery constants are derived in the kernel:
//   n' = -n^-1 mod 2^32   Newton's iteration on one word,
//   R mod n               32L modular doublings of 1 (R = 2^(32L)),
//   R^2 mod n             64 more doublings give 2^64 R mod n, then log2(L/2)
//                         Montgomery squarings, each (2^k R)^2 / R = 2^(2k) R.
// A round with base a: n - 1 = d 2^s with d odd; x = a^d mod n by the
// constant-time fixed-window method with this lane's own exponent d (the
// candidates are future secret primes), then up to s - 1 squarings looking for
// n - 1.  In Montgomery form 1 is R mod n and n - 1 is n - (R mod n).  Loop
// counts are the same for the whole warp (windows over 32L bits, squarings up
// to the warp's largest s), so nothing diverges.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"
#include "kernels_t.cuh"
#include "mont.cuh"
#include "rsa_gb300.h"
#include "runtime_internal.h"

namespace rsagpu {

namespace {

constexpr int kMrWindow = 4;
constexpr int kMrThreads = 128;

struct MrArgs {
  const uint32_t *cands;    // count rows of L limbs
  const uint32_t *bases;    // count * rounds rows of L limbs, row i * rounds + r
  int32_t *verdict;         // count: 1 probable prime, 0 composite, -1 invalid candidate
  uint4 *tables;            // per warp 2^W * L/4 * 32 uint4, then kLaneBufs stages
  uint32_t count, rounds;
};

// Per-warp [L/4][32] uint4 buffers.  The B operand of every multiplication
// sits in shared memory; R^2, the Montgomery forms of 1 and n - 1 and the
// exponent d are read once per round or per window and live in global memory
// next to the window table (coalesced, L2-resident), which keeps shared memory
// from limiting the resident warps.
template <int L>
struct MrSmem {
  static constexpr int kStageU4 = (L / 4) * 32;   // one [L/4][32] uint4 buffer per warp
  static constexpr int kBuffers = 1;              // B operand
  static constexpr int kLaneBufs = 4;             // global: R^2, one, minus one, exponent d
  static constexpr size_t bytes(int warps) { return (size_t)warps * kBuffers * kStageU4 * 16; }
  template <int W>
  __host__ __device__ static constexpr size_t global_u4_per_warp() { return ((size_t)1 << W) * (L / 4) * 32 + (size_t)kLaneBufs * kStageU4; }
};

// x = 2x mod n for x < n: the doubled value has L limbs plus a top bit; one
// conditional subtraction (2x < 2n), selected without a branch.
template <int L>
__device__ __forceinline__ void dbl_mod(uint32_t (&x)[L], const NRegs<L> &N) {
  uint32_t y[L], t[L];
  const uint32_t top = x[L - 1] >> 31;
  y[0] = x[0] << 1;
#pragma unroll
  for (int j = 1; j < L; ++j) y[j] = __funnelshift_l(x[j - 1], x[j], 1);
  t[0] = sub_cc(y[0], N.n[0]);
#pragma unroll
  for (int j = 1; j < L; ++j) t[j] = subc_cc(y[j], N.n[j]);
  const uint32_t keep = subc(top, 0u);   // all ones iff 2x < n
#pragma unroll
  for (int j = 0; j < L; ++j) x[j] = (y[j] & keep) | (t[j] & ~keep);
}

// word j of a lane's number in a [L/4][32] stage (0 beyond the top)
template <int L>
__device__ __forceinline__ uint32_t stage_word(const uint4 *lane, int j) {
  if (j >= L) return 0u;
  const uint4 v = lane[(j >> 2) * 32];
  const int c = j & 3;
  return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}

template <int L>
__device__ __forceinline__ bool stage_equal(const uint32_t (&A)[L], const uint4 *lane) {
  uint32_t diff = 0;
#pragma unroll
  for (int g = 0; g < L / 4; ++g) {
    const uint4 v = lane[g * 32];
    diff |= (A[4 * g] ^ v.x) | (A[4 * g + 1] ^ v.y) | (A[4 * g + 2] ^ v.z) | (A[4 * g + 3] ^ v.w);
  }
  return diff == 0;
}

template <int L, int W>
__device__ __forceinline__ uint32_t lane_digit(const uint4 *d_lane, int k) {
  const int bit = k * W;
  const uint32_t lo = stage_word<L>(d_lane, bit >> 5), hi = stage_word<L>(d_lane, (bit >> 5) + 1);
  return __funnelshift_r(lo, hi, bit & 31) & ((1u << W) - 1u);
}

template <int L, int W, int U>
__global__ void __launch_bounds__(kMrThreads) mr_kernel(MrArgs a) {
  using Sm = MrSmem<L>;
  extern __shared__ uint4 smem4[];
  const int nw = blockDim.x / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4 *b_lane = smem4 + (size_t)warp * Sm::kBuffers * Sm::kStageU4 + lane;
  uint4 *table_lane = a.tables + (size_t)(blockIdx.x * nw + warp) * Sm::template global_u4_per_warp<W>() + lane;
  uint4 *r2_lane = table_lane + ((size_t)1 << W) * (L / 4) * 32;
  uint4 *one_lane = r2_lane + Sm::kStageU4, *m1_lane = r2_lane + 2 * Sm::kStageU4, *d_lane = r2_lane + 3 * Sm::kStageU4;
  const uint32_t ntiles = (a.count + 31) / 32;
  constexpr int kSqToR2 = (L == 16) ? 3 : (L == 32) ? 4 : 5;    // log2(L / 2)
  static_assert(L == 16 || L == 32 || L == 64, "candidate sizes");
  constexpr int kNwin = (32 * L + W - 1) / W;
#pragma unroll 1
  for (uint32_t tile = blockIdx.x * nw + warp; tile < ntiles; tile += gridDim.x * nw) {
    const uint32_t i = tile * 32 + (uint32_t)lane;
    const bool live = i < a.count;
    const uint32_t row = live ? i : a.count - 1;
    NRegs<L> N;
    {
      const uint4 *r4 = reinterpret_cast<const uint4 *>(a.cands + (size_t)row * L);
#pragma unroll
      for (int g = 0; g < L / 4; ++g) {
        const uint4 v = r4[g];
        N.n[4 * g] = v.x; N.n[4 * g + 1] = v.y; N.n[4 * g + 2] = v.z; N.n[4 * g + 3] = v.w;
      }
    }
    uint32_t hi_or = 0;
#pragma unroll
    for (int j = 1; j < L; ++j) hi_or |= N.n[j];
    const bool valid = (N.n[0] & 1u) && (hi_or != 0u || N.n[0] >= 5u);
    if (!valid) N.n[0] |= 1u;                // keep the arithmetic defined; the verdict is -1 anyway
    // n' = -n^-1 mod 2^32: x = n is right to 3 bits, each step doubles them
    uint32_t inv = N.n[0];
#pragma unroll
    for (int k = 0; k < 4; ++k) inv *= 2u - N.n[0] * inv;
    const uint32_t np = 0u - inv;
    uint32_t x[L];
    // R mod n, and n - R mod n (the Montgomery forms of 1 and n - 1)
#pragma unroll
    for (int j = 0; j < L; ++j) x[j] = 0u;
    x[0] = 1u;
#pragma unroll 1
    for (int k = 0; k < 32 * L; ++k) dbl_mod<L>(x, N);
    to_stage<L>(one_lane, x);
    {
      uint32_t m1[L];
      m1[0] = sub_cc(N.n[0], x[0]);
#pragma unroll
      for (int j = 1; j < L; ++j) m1[j] = subc_cc(N.n[j], x[j]);
      to_stage<L>(m1_lane, m1);
    }
    // R^2 mod n
#pragma unroll 1
    for (int k = 0; k < 64; ++k) dbl_mod<L>(x, N);
#pragma unroll 1
    for (int k = 0; k < kSqToR2; ++k) {
      to_stage<L>(b_lane, x);
      mont_mul<L, U>(x, SmemB{b_lane, 32}, N, np);
    }
    to_stage<L>(r2_lane, x);
    // n - 1 = d 2^s, d odd (n - 1 is n with bit 0 cleared)
    int s = 0;
    {
      N.n[0] &= ~1u;
      to_stage<L>(d_lane, N.n);
      int j = 0;
      while (j < L - 1 && stage_word<L>(d_lane, j) == 0u) ++j;
      const uint32_t w = stage_word<L>(d_lane, j);
      s = 32 * j + (w ? __ffs(w) - 1 : 0);
      uint32_t d[L];
      const int q = s >> 5, r = s & 31;
#pragma unroll
      for (int k = 0; k < L; ++k)
        d[k] = __funnelshift_r(stage_word<L>(d_lane, k + q), stage_word<L>(d_lane, k + q + 1), r);
      to_stage<L>(d_lane, d);
      N.n[0] |= 1u;
    }
    const int s_max = __reduce_max_sync(0xffffffffu, s);
    int verdict = 1;
#pragma unroll 1
    for (uint32_t rd = 0; rd < a.rounds; ++rd) {
      uint32_t A[L];
      load_row<L>(A, a.bases + ((size_t)row * a.rounds + rd) * L, true);
      mont_mul<L, U>(A, SmemB{r2_lane, 32}, N, np);            // a R
      // table T[e] = a^e R, e < 2^W (T[0] = R mod n), then the fixed windows
#pragma unroll
      for (int g = 0; g < L / 4; ++g) table_lane[g * 32] = one_lane[g * 32];   // T[0] = R mod n
      table_store<L>(table_lane, 1, A);
      to_stage<L>(b_lane, A);
#pragma unroll 1
      for (int e = 2; e < (1 << W); ++e) {
        mont_mul<L, U>(A, SmemB{b_lane, 32}, N, np);
        table_store<L>(table_lane, e, A);
      }
      table_select<L, W>(b_lane, table_lane, lane_digit<L, W>(d_lane, kNwin - 1));
      from_stage<L>(A, b_lane);
      int k = kNwin - 2, sq = 0;
      const int nsteps = (kNwin - 1) * (W + 1);
#pragma unroll 1
      for (int st = 0; st < nsteps; ++st) {
        if (sq < W) {
          to_stage<L>(b_lane, A);
          ++sq;
        } else {
          table_select<L, W>(b_lane, table_lane, lane_digit<L, W>(d_lane, k));
          sq = 0;
          --k;
        }
        mont_mul<L, U>(A, SmemB{b_lane, 32}, N, np);
      }
      bool pass = stage_equal<L>(A, one_lane) || stage_equal<L>(A, m1_lane);
#pragma unroll 1
      for (int j = 1; j < s_max; ++j) {
        to_stage<L>(b_lane, A);
        mont_mul<L, U>(A, SmemB{b_lane, 32}, N, np);
        if (j < s && stage_equal<L>(A, m1_lane)) pass = true;
      }
      if (!pass) verdict = 0;
    }
    if (live) a.verdict[i] = valid ? verdict : -1;
  }
}

// ---------------------------------------------------------------- 2048-bit candidates, T lanes each
// The same test with every number sliced over T lanes (mont_t.cuh): 64-limb
// candidates need 255 registers on one lane (two CTAs of 128 threads per SM);
// on four lanes a thread holds 16 limbs and more warps hide the carry chains'
// latency.  Each candidate's own constants live contiguously in the warp's
// global scratch (words): d = (n - 1) / 2^s zero padded to L + 4, R mod n,
// n - R mod n and R^2 mod n, L each; the fixed-window exponentiation of
// kernels_t.cuh reads its exponent digits and its 1 from there.
template <int L>
struct MrT {
  static constexpr int kOpWords = 4 * L + 4;   // d (L + 4), one, minus one, R^2
  static constexpr int kD = 0, kOne = L + 4, kM1 = 2 * L + 4, kR2 = 3 * L + 4;
  template <int T, int W>
  __host__ __device__ static constexpr size_t table_u4() { return ((size_t)1 << W) * (L / T / 4) * 32; }
  template <int T, int W>
  __host__ __device__ static constexpr size_t per_warp_u4() { return table_u4<T, W>() + (size_t)(32 / T) * kOpWords / 4; }
};

// every rank's slice of A equals that of the L-limb number at w (contiguous)
template <int K, int T>
__device__ __forceinline__ bool group_equal(const uint32_t (&A)[K], const uint32_t *w, const Group<T> &g) {
  uint32_t diff = 0u;
#pragma unroll
  for (int j = 0; j < K; ++j) diff |= A[j] ^ w[g.r * K + j];
  return g.bits(diff == 0u) == (1u << T) - 1u;
}

template <int L, int T, int W, int U>
__device__ __forceinline__ void mr_tile_t(const MrArgs &a, uint32_t base, const Group<T> &g, uint4 *stage_op,
                                          uint4 *table_lane, uint32_t *opw) {
  constexpr int K = L / T, OS = 32 / T;
  constexpr int kSqToR2 = (L == 16) ? 3 : (L == 32) ? 4 : 5;    // log2(L / 2)
  const uint32_t idx = base + (uint32_t)g.opi;
  const bool live = idx < a.count;
  const uint32_t row = live ? idx : a.count - 1;
  NRegs<K> N;
  load_row<K>(N.n, a.cands + (size_t)row * L + g.r * K, true);
  uint32_t above = 0u;   // any limb above limb 0 nonzero
#pragma unroll
  for (int j = 0; j < K; ++j) above |= (g.r == 0 && j == 0) ? 0u : N.n[j];
  const uint32_t n0 = g.from_rank(N.n[0], 0);
  const uint32_t above_any = g.bits(above != 0u);   // a collective: every lane, before any condition
  const bool valid = (n0 & 1u) && (above_any != 0u || n0 >= 5u);
  if (g.r == 0 && !valid) N.n[0] |= 1u;   // keep the arithmetic defined; the verdict is -1 anyway
  uint32_t inv = g.from_rank(N.n[0], 0);  // n' = -n^-1 mod 2^32 (Newton, as mr_kernel)
  const uint32_t n0f = inv;
#pragma unroll
  for (int k = 0; k < 4; ++k) inv *= 2u - n0f * inv;
  const uint32_t np = 0u - inv;
  uint32_t *dw = opw + MrT<L>::kD, *onew = opw + MrT<L>::kOne, *m1w = opw + MrT<L>::kM1, *r2w = opw + MrT<L>::kR2;
  // n - 1 = d 2^s: n - 1 (n odd: bit 0 cleared) into the d area, s from the
  // lowest rank with a nonzero slice, then every rank shifts its words down
  int s;
  {
    uint32_t w0 = 0u;
    int j0 = -1;
#pragma unroll
    for (int j = K - 1; j >= 0; --j) {
      const uint32_t v = (g.r == 0 && j == 0) ? (N.n[0] & ~1u) : N.n[j];
      dw[g.r * K + j] = v;
      if (v) { w0 = v; j0 = j; }
    }
    if (g.r == T - 1) {
#pragma unroll
      for (int j = 0; j < 4; ++j) dw[L + j] = 0u;
    }
    const uint32_t nz = g.bits(j0 >= 0);
    const int r0 = nz ? __ffs(nz) - 1 : 0;
    const int mine = j0 >= 0 ? 32 * (g.r * K + j0) + __ffs(w0) - 1 : 0;
    s = (int)g.from_rank((uint32_t)mine, r0);
    __syncwarp();
    uint32_t dd[K];
    const int q = s >> 5, sh = s & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = g.r * K + k + q;
      dd[k] = __funnelshift_r(i < L ? dw[i] : 0u, i + 1 < L ? dw[i + 1] : 0u, sh);
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < K; ++k) dw[g.r * K + k] = dd[k];
  }
  // R mod n by 32L doublings of 1, n - R mod n, then R^2 mod n: 64 more
  // doublings (2^64 R) and log2(L/2) Montgomery squarings
  uint32_t x[K];
#pragma unroll
  for (int j = 0; j < K; ++j) x[j] = 0u;
  if (g.r == 0) x[0] = 1u;
  const SmemB st{stage_op, OS};
#pragma unroll 1
  for (int k = 0; k < 32 * L; ++k) {
    to_stage_t<K, T>(stage_op, x, g);   // mod_add_t reads this rank's own slice only
    mod_add_t<K, T>(x, st, N, g);
  }
#pragma unroll
  for (int j = 0; j < K; ++j) onew[g.r * K + j] = x[j];
  {
    uint32_t m1[K];
#pragma unroll
    for (int j = 0; j < K; ++j) m1[j] = x[j];
    to_stage_t<K, T>(stage_op, N.n, g);
    mod_rsub_t<K, T>(m1, st, N, g);       // n - (R mod n)
#pragma unroll
    for (int j = 0; j < K; ++j) m1w[g.r * K + j] = m1[j];
  }
#pragma unroll 1
  for (int k = 0; k < 64; ++k) {
    to_stage_t<K, T>(stage_op, x, g);
    mod_add_t<K, T>(x, st, N, g);
  }
#pragma unroll 1
  for (int k = 0; k < kSqToR2; ++k) {
    __syncwarp();
    to_stage_t<K, T>(stage_op, x, g);
    __syncwarp();
    mont_mul_t<K, T, U>(x, st, N, np, g);
  }
#pragma unroll
  for (int j = 0; j < K; ++j) r2w[g.r * K + j] = x[j];
  __syncwarp();
  const int s_max = __reduce_max_sync(0xffffffffu, s);
  int verdict = 1;
#pragma unroll 1
  for (uint32_t rd = 0; rd < a.rounds; ++rd) {
    uint32_t A[K];
    load_row<K>(A, a.bases + ((size_t)row * a.rounds + rd) * L + g.r * K, true);
    mont_mul_t<K, T, U>(A, SmemB{reinterpret_cast<const uint4 *>(r2w), 1}, N, np, g);   // a R
    fixed_window_exp_t<K, T, W, U>(A, dw, 32 * L, onew, stage_op, table_lane, N, np, g);
    bool pass = group_equal<K, T>(A, onew, g);
    pass = group_equal<K, T>(A, m1w, g) || pass;
#pragma unroll 1
    for (int j = 1; j < s_max; ++j) {
      __syncwarp();
      to_stage_t<K, T>(stage_op, A, g);
      __syncwarp();
      mont_mul_t<K, T, U>(A, st, N, np, g);
      const bool m1 = group_equal<K, T>(A, m1w, g);   // every lane: a collective
      if (j < s && m1) pass = true;
    }
    if (!pass) verdict = 0;
  }
  if (live && g.r == 0) a.verdict[idx] = valid ? verdict : -1;
}

template <int L, int T, int W, int U>
__global__ void __launch_bounds__(kMrThreads) mr_kernel_t(MrArgs a) {
  constexpr int OPW = 32 / T;
  extern __shared__ uint4 smem4[];
  const int nw = blockDim.x / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Group<T> g(lane);
  uint4 *stage = smem4 + (size_t)warp * (L / 4) * OPW;   // [L/4][32/T] uint4 per warp
  uint4 *wbase = a.tables + (size_t)(blockIdx.x * nw + warp) * MrT<L>::template per_warp_u4<T, W>();
  uint4 *table_lane = wbase + lane;
  uint32_t *opw = reinterpret_cast<uint32_t *>(wbase + MrT<L>::template table_u4<T, W>()) +
                  (size_t)g.opi * MrT<L>::kOpWords;
  const uint32_t ntiles = (a.count + OPW - 1) / OPW;
#pragma unroll 1
  for (uint32_t tile = blockIdx.x * nw + warp; tile < ntiles; tile += gridDim.x * nw)
    mr_tile_t<L, T, W, U>(a, tile * OPW, g, stage + g.opi, table_lane, opw);
}

template <int L>
cudaError_t launch_mr(const MrArgs &h, int grid, cudaStream_t s) {
  const size_t smem = MrSmem<L>::bytes(kMrThreads / 32);
  // set on every call: the attribute belongs to the current device's context
  cudaError_t e = cudaFuncSetAttribute(mr_kernel<L, kMrWindow, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  mr_kernel<L, kMrWindow, 8><<<grid, kMrThreads, smem, s>>>(h);
  return cudaGetLastError();
}


// T lanes per candidate (mr_kernel_t), as many CTAs as fit
template <int L, int T>
int launch_mr_t(Ctx *c, Workspace &w, const uint32_t *cands, const uint32_t *bases, int32_t *verdicts, uint64_t count,
                uint32_t rounds, cudaStream_t s) {
  const int per_cta = kMrThreads / 32;
  const void *fn = reinterpret_cast<const void *>(&mr_kernel_t<L, T, kMrWindow, 8>);
  const size_t smem = (size_t)per_cta * (L / 4) * (32 / T) * 16;
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kMrThreads, smem);
  if (e != cudaSuccess) return cuda_error(e, "occupancy of mr_kernel_t");
  const uint64_t warps_needed = (count + 32 / T - 1) / (32 / T);
  const int grid = (int)std::max<uint64_t>(
      1, std::min<uint64_t>((warps_needed + per_cta - 1) / per_cta, (uint64_t)c->sm_count * std::max(occ, 1)));
  const size_t tbytes = (size_t)grid * per_cta * MrT<L>::template per_warp_u4<T, kMrWindow>() * 16;
  int rc = c->ensure(w.tables, tbytes);
  if (rc) return rc;
  MrArgs h{cands, bases, verdicts, static_cast<uint4 *>(w.tables.ptr), (uint32_t)count, rounds};
  void *args[] = {&h};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(kMrThreads), args, smem, s);
  if (e != cudaSuccess) return cuda_error(e, "launch mr_kernel_t");
  c->stats.kernel_launches++;
  c->stats.ops += count;
  return RSA_OK;
}
}  // namespace
}  // namespace rsagpu

using namespace rsagpu;

extern "C" int rsa_mr_batch(rsa_ctx *ctx, uint32_t nbits, uint64_t count, const uint32_t *cands, uint32_t rounds,
                            const uint32_t *bases, int32_t *verdicts, void *stream) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  if (nbits != 512 && nbits != 1024 && nbits != 2048)
    return set_error(RSA_ERR_UNSUPPORTED, "candidates of 512, 1024 or 2048 bits");
  if (count == 0) return RSA_OK;
  if (!cands || !verdicts || (rounds > 0 && !bases)) return set_error(RSA_ERR_ARG, "null pointer");
  if (count > 0x7fffffffull || rounds > 256) return set_error(RSA_ERR_ARG, "count or rounds out of range");
  if ((reinterpret_cast<uintptr_t>(cands) | reinterpret_cast<uintptr_t>(bases)) & 15u)
    return set_error(RSA_ERR_ARG, "candidate and base rows must be 16-byte aligned");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NvtxRange range("rsa_mr_batch");
  Workspace &w = c->ws(s);
  const int L = (int)nbits / 32;
  const int per_cta = kMrThreads / 32;
  // 2048-bit candidates on four lanes each (GB300: 252 K against 189 K rounds/s on
  // one); 1024-bit ones stay on one lane (2.10 M rounds/s against 1.91 M on two
  // lanes and 1.95 M on four)
  if (L == 64) return launch_mr_t<64, 4>(c, w, cands, bases, verdicts, count, rounds, s);
  const uint64_t warps_needed = (count + 31) / 32;
  const int grid = (int)std::max<uint64_t>(
      1, std::min<uint64_t>((warps_needed + per_cta - 1) / per_cta, (uint64_t)c->sm_count * 4));
  const size_t per_warp_u4 = (L == 16) ? MrSmem<16>::global_u4_per_warp<kMrWindow>()
                                        : MrSmem<32>::global_u4_per_warp<kMrWindow>();
  const size_t tbytes = (size_t)grid * per_cta * per_warp_u4 * 16;
  int rc = c->ensure(w.tables, tbytes);
  if (rc) return rc;
  MrArgs h{cands, bases, verdicts, static_cast<uint4 *>(w.tables.ptr), (uint32_t)count, rounds};
  cudaError_t e = (L == 16) ? launch_mr<16>(h, grid, s) : launch_mr<32>(h, grid, s);
  if (e != cudaSuccess) return cuda_error(e, "launch mr_kernel");
  c->stats.kernel_launches++;
  c->stats.ops += count;
  return RSA_OK;
}
