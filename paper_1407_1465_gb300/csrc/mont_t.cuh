// mont_t.cuh -- Montgomery arithmetic with one operation spread over T lanes.
//
// T consecutive lanes of a warp (a "group") hold one operation: rank r = lane % T
// holds limbs [rK, rK+K) of every L-limb number (K = L/T).  A CIOS step adds
// b_i * A and q * N slice by slice; q = t_0 * n' is computed by rank 0 (the only
// rank whose low limb is exact) and broadcast with a shuffle.  Carries between
// ranks are kept lazily: each rank carries a small pending word that sits just
// above its slice; the division by 2^32 of every step moves the next rank's low
// limb (a shuffle) plus that pending word into the rank's top limb, so pending
// words stay below 4.  At the end of a multiplication the pending words are
// added into the rank above and the remaining single-bit carries are resolved
// for all ranks at once with a ballot carry-lookahead: with generate bits G and
// propagate bits P (bit j = rank j), the carries into the ranks are the carries
// of the integer sum G + (G | P), i.e. (G + (G|P)) ^ G ^ (G|P).
#pragma once
#include <cstdint>

#include "mont.cuh"

namespace rsagpu {

// Every member function below is a warp-wide collective (full-mask shuffle or
// ballot): all 32 lanes must call it together, never under a lane-dependent
// condition.
template <int T>
struct Group {
  int lane, r, base, opi;  // opi: operation index of the group within the warp
  __device__ __forceinline__ explicit Group(int lane_)
      : lane(lane_), r(lane_ % T), base(lane_ - lane_ % T), opi(lane_ / T) {}
  __device__ __forceinline__ uint32_t from_rank(uint32_t v, int src) const {
    return __shfl_sync(0xffffffffu, v, base + src);
  }
  // next rank's value (0 for the top rank)
  __device__ __forceinline__ uint32_t from_above(uint32_t v) const {
    const uint32_t x = __shfl_down_sync(0xffffffffu, v, 1);
    return r == T - 1 ? 0u : x;
  }
  // previous rank's value (0 for rank 0)
  __device__ __forceinline__ uint32_t from_below(uint32_t v) const {
    const uint32_t x = __shfl_up_sync(0xffffffffu, v, 1);
    return r == 0 ? 0u : x;
  }
  // this group's ballot bits, bit j = rank j
  __device__ __forceinline__ uint32_t bits(bool pred) const {
    const uint32_t m = __ballot_sync(0xffffffffu, pred);
    return (m >> base) & ((1u << T) - 1u);
  }
};

// carry (or borrow) into each rank, and out of the top rank at bit T
__device__ __forceinline__ uint32_t lookahead(uint32_t G, uint32_t P) {
  const uint32_t Y = G | P;
  return (G + Y) ^ G ^ Y;
}

// t[0..K+1] += q * N (N: this rank's slice), no shift
template <int K, class NS>
__device__ __forceinline__ void mul_acc_ns(uint32_t (&t)[K + 2], const NS &N, uint32_t q) {
  t[0] = mad_lo_cc(N.get(0), q, t[0]);
  t[1] = madc_hi_cc(N.get(0), q, t[1]);
#pragma unroll
  for (int k = 1; k < K / 2; ++k) {
    t[2 * k] = madc_lo_cc(N.get(2 * k), q, t[2 * k]);
    t[2 * k + 1] = madc_hi_cc(N.get(2 * k), q, t[2 * k + 1]);
  }
  t[K] = addc_cc(t[K], 0u);
  t[K + 1] = addc(t[K + 1], 0u);
  t[1] = mad_lo_cc(N.get(1), q, t[1]);
  t[2] = madc_hi_cc(N.get(1), q, t[2]);
#pragma unroll
  for (int k = 1; k < K / 2; ++k) {
    t[2 * k + 1] = madc_lo_cc(N.get(2 * k + 1), q, t[2 * k + 1]);
    t[2 * k + 2] = madc_hi_cc(N.get(2 * k + 1), q, t[2 * k + 2]);
  }
  t[K + 1] = addc(t[K + 1], 0u);
}

// One CIOS step on a group: t += b*A + q*N, then divide by 2^32 across ranks.
template <int K, int T, class NS>
__device__ __forceinline__ void step_t(uint32_t (&t)[K + 2], uint32_t &pend, const uint32_t (&A)[K], uint32_t b,
                                       const NS &N, uint32_t np, const Group<T> &g) {
  t[K] = pend;
  t[K + 1] = 0u;
  mul_acc<K>(t, A, b);
  const uint32_t q = g.from_rank(t[0] * np, 0);
  mul_acc_ns<K>(t, N, q);
  const uint32_t up = g.from_above(t[0]);
#pragma unroll
  for (int j = 0; j < K - 1; ++j) t[j] = t[j + 1];
  t[K - 1] = add_cc(t[K], up);
  pend = addc(t[K + 1], 0u);
}

// s (value with pending words) -> fully carried slice; returns this rank's
// slice in s and the group's top word (limb L) in *top.
template <int K, int T>
__device__ __forceinline__ void carry_resolve_t(uint32_t (&s)[K], uint32_t pend, uint32_t *top, const Group<T> &g) {
  const uint32_t pin = g.from_below(pend);
  s[0] = add_cc(s[0], pin);
#pragma unroll
  for (int j = 1; j < K; ++j) s[j] = addc_cc(s[j], 0u);
  const uint32_t c = addc(0u, 0u);
  uint32_t ones = 0xffffffffu;  // branch-free: every predicate is plain arithmetic
#pragma unroll
  for (int j = 0; j < K; ++j) ones &= s[j];
  const uint32_t cin_bits = lookahead(g.bits(c != 0u), g.bits(ones == 0xffffffffu));
  const uint32_t cin = (cin_bits >> g.r) & 1u;
  s[0] = add_cc(s[0], cin);
#pragma unroll
  for (int j = 1; j < K; ++j) s[j] = addc_cc(s[j], 0u);
  (void)addc(0u, 0u);
  *top = g.from_rank(pend, T - 1) + ((cin_bits >> T) & 1u);
}

// A = s - N if (top, s) >= N else s, for a value below 2N; all ranks agree.
template <int K, int T, class NS>
__device__ __forceinline__ void cond_sub_t(uint32_t (&A)[K], const uint32_t (&s)[K], uint32_t top, const NS &N,
                                           const Group<T> &g) {
  uint32_t d[K];
  d[0] = sub_cc(s[0], N.get(0));
#pragma unroll
  for (int j = 1; j < K; ++j) d[j] = subc_cc(s[j], N.get(j));
  const uint32_t bo = subc(0u, 0u) & 1u;
  uint32_t any = 0u;
#pragma unroll
  for (int j = 0; j < K; ++j) any |= d[j];
  const uint32_t bin_bits = lookahead(g.bits(bo != 0u), g.bits(any == 0u));
  const uint32_t bin = (bin_bits >> g.r) & 1u;
  const uint32_t bout = (bin_bits >> T) & 1u;
  d[0] = sub_cc(d[0], bin);
#pragma unroll
  for (int j = 1; j < K; ++j) d[j] = subc_cc(d[j], 0u);
  (void)subc(0u, 0u);
  const uint32_t keep = 0u - (((top == 0u) ? 1u : 0u) & bout);  // value < N
#pragma unroll
  for (int j = 0; j < K; ++j) A[j] = (s[j] & keep) | (d[j] & ~keep);
}

// A = A * B * R^-1 mod N, R = 2^(32 K T); B streamed from the group's stage.
template <int K, int T, int U, class NS>
__device__ __forceinline__ void mont_mul_t(uint32_t (&A)[K], const SmemB &B, const NS &N, uint32_t np,
                                           const Group<T> &g) {
  constexpr int L = K * T;
  static_assert(K % 4 == 0 && U % 4 == 0 && L % U == 0, "limb blocking");
  uint32_t t[K + 2];
#pragma unroll
  for (int j = 0; j < K + 2; ++j) t[j] = 0u;
  uint32_t pend = 0u;
#pragma unroll 1
  for (int i0 = 0; i0 < L; i0 += U) {
#pragma unroll
    for (int u = 0; u < U; u += 4) {
      const uint4 b = B.get4((i0 + u) >> 2);
      step_t<K, T>(t, pend, A, b.x, N, np, g);
      step_t<K, T>(t, pend, A, b.y, N, np, g);
      step_t<K, T>(t, pend, A, b.z, N, np, g);
      step_t<K, T>(t, pend, A, b.w, N, np, g);
    }
  }
  uint32_t s[K];
#pragma unroll
  for (int j = 0; j < K; ++j) s[j] = t[j];
  uint32_t top;
  carry_resolve_t<K, T>(s, pend, &top, g);
  cond_sub_t<K, T>(A, s, top, N, g);
}

// A = (A + B) mod N, B from the group's stage (slice of this rank), A, B < N.
template <int K, int T, class NS>
__device__ __forceinline__ void mod_add_t(uint32_t (&A)[K], const SmemB &B, const NS &N, const Group<T> &g) {
  uint32_t s[K];
#pragma unroll
  for (int gg = 0; gg < K / 4; ++gg) {
    const uint4 b = B.get4(g.r * (K / 4) + gg);
    if (gg == 0) s[0] = add_cc(A[0], b.x); else s[4 * gg] = addc_cc(A[4 * gg], b.x);
    s[4 * gg + 1] = addc_cc(A[4 * gg + 1], b.y);
    s[4 * gg + 2] = addc_cc(A[4 * gg + 2], b.z);
    s[4 * gg + 3] = addc_cc(A[4 * gg + 3], b.w);
  }
  const uint32_t c = addc(0u, 0u);
  uint32_t top;
  carry_resolve_t<K, T>(s, c, &top, g);   // the carry out of each rank is its pending word
  cond_sub_t<K, T>(A, s, top, N, g);
}

// A = (B - A) mod N, B from the group's stage, A, B < N.
template <int K, int T, class NS>
__device__ __forceinline__ void mod_rsub_t(uint32_t (&A)[K], const SmemB &B, const NS &N, const Group<T> &g) {
  uint32_t d[K];
#pragma unroll
  for (int gg = 0; gg < K / 4; ++gg) {
    const uint4 b = B.get4(g.r * (K / 4) + gg);
    if (gg == 0) d[0] = sub_cc(b.x, A[0]); else d[4 * gg] = subc_cc(b.x, A[4 * gg]);
    d[4 * gg + 1] = subc_cc(b.y, A[4 * gg + 1]);
    d[4 * gg + 2] = subc_cc(b.z, A[4 * gg + 2]);
    d[4 * gg + 3] = subc_cc(b.w, A[4 * gg + 3]);
  }
  const uint32_t bo = subc(0u, 0u) & 1u;
  uint32_t any = 0u;
#pragma unroll
  for (int j = 0; j < K; ++j) any |= d[j];
  const uint32_t bin_bits = lookahead(g.bits(bo != 0u), g.bits(any == 0u));
  const uint32_t bin = (bin_bits >> g.r) & 1u;
  const uint32_t neg = 0u - ((bin_bits >> T) & 1u);  // B < A: add N
  d[0] = sub_cc(d[0], bin);
#pragma unroll
  for (int j = 1; j < K; ++j) d[j] = subc_cc(d[j], 0u);
  (void)subc(0u, 0u);
  // d + (N & neg) with carries across ranks; the carry out of the top rank is dropped
  uint32_t s[K];
  s[0] = add_cc(d[0], N.get(0) & neg);
#pragma unroll
  for (int j = 1; j < K; ++j) s[j] = addc_cc(d[j], N.get(j) & neg);
  const uint32_t c = addc(0u, 0u);
  uint32_t top;
  carry_resolve_t<K, T>(s, c, &top, g);
#pragma unroll
  for (int j = 0; j < K; ++j) A[j] = s[j];
}

// Write this rank's slice of A into the group's stage ([L/4][32/T] of uint4).
template <int K, int T>
__device__ __forceinline__ void to_stage_t(uint4 *stage_op, const uint32_t (&A)[K], const Group<T> &g) {
#pragma unroll
  for (int gg = 0; gg < K / 4; ++gg)
    stage_op[(g.r * (K / 4) + gg) * (32 / T)] = make_uint4(A[4 * gg], A[4 * gg + 1], A[4 * gg + 2], A[4 * gg + 3]);
}
template <int K, int T>
__device__ __forceinline__ void from_stage_t(uint32_t (&A)[K], const uint4 *stage_op, const Group<T> &g) {
#pragma unroll
  for (int gg = 0; gg < K / 4; ++gg) {
    const uint4 v = stage_op[(g.r * (K / 4) + gg) * (32 / T)];
    A[4 * gg] = v.x; A[4 * gg + 1] = v.y; A[4 * gg + 2] = v.z; A[4 * gg + 3] = v.w;
  }
}

// Compare an L-limb row held as rank slices (lo: limbs [rK, rK+K) of the value)
// with m (same slices): -1, 0, +1 for the whole group.
template <int K, int T>
__device__ __forceinline__ int cmp_t(const uint32_t *row_slice, const uint32_t *m_slice, const Group<T> &g) {
  // branch-free: lt/gt of the first differing limb from the top
  uint32_t lt = 0u, gt = 0u, decided = 0u;
#pragma unroll
  for (int j = K - 1; j >= 0; --j) {
    const uint32_t a = row_slice[j], b = m_slice[j];
    const uint32_t fresh = (a != b ? 1u : 0u) & ~decided;
    lt |= fresh & (a < b ? 1u : 0u);
    gt |= fresh & (a > b ? 1u : 0u);
    decided |= fresh;
  }
  const uint32_t L_ = g.bits(lt != 0u), G_ = g.bits(gt != 0u);
  const uint32_t any = L_ | G_;
  const int topr = 31 - __clz(any | 1u);
  const int sign = ((L_ >> topr) & 1u) ? -1 : 1;
  return any ? sign : 0;
}

}  // namespace rsagpu
