// mont.cuh -- multi-limb Montgomery arithmetic for one operation per thread.
//
// The paper computes g^e mod n with built-in integers (Algorithm 2, Fig. 12)
// and reduces every product with the identity of Fig. 3,
// (u*v) mod m = ((u mod m)*(v mod m)) mod m.  For moduli of 1024-4096 bits this
// library keeps numbers as L little-endian 32-bit limbs and replaces "mod m" by
// Montgomery multiplication (operand-scanning CIOS form):
//     mont_mul(A, B) = A * B * R^-1 mod N,   R = 2^(32L), N odd,
// valid for A < R and B < N; the result is fully reduced (< N).
//
// Each CIOS step i adds b_i * A into the accumulator t and then adds q * N with
// q = t_0 * n' mod 2^32 (n' = -N^-1 mod 2^32), which clears t_0, and shifts t
// down one limb.  The products are issued as PTX carry chains
// (mad.lo.cc / madc.hi.cc / madc.lo.cc ... alternating, addc to close a
// chain), one chain over the even limbs and one over the odd limbs; a chain
// cannot interleave with another because all share the single carry flag.
//
// Operand placement: A (the register operand) lives in registers; B is streamed
// four limbs at a time from shared memory (a per-lane staging buffer or a
// warp-uniform constant); N either sits in registers (NREG) or is read from
// shared memory as warp-uniform 128-bit loads.
#pragma once
#include <cstdint>

namespace rsagpu {

// ------------------------------------------------------------------ PTX carry-chain primitives
__device__ __forceinline__ uint32_t mad_lo_cc(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("mad.lo.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t madc_lo_cc(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("madc.lo.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t mad_hi_cc(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("mad.hi.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t madc_hi_cc(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("madc.hi.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t add_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t addc_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t addc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("addc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t sub_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t subc_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t subc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("subc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

// ------------------------------------------------------------------ operand sources
// B operand: four limbs (b_{4g} .. b_{4g+3}) per get4(g).
// SmemB{stage + lane, 32}: per-lane staging buffer, layout [L/4][32] of uint4;
// SmemB{konst, 1}: warp-uniform constant, layout [L/4] of uint4.
struct SmemB {
  const uint4 *base;
  int stride;
  __device__ __forceinline__ uint4 get4(int g) const { return base[g * stride]; }
};

// N operand
template <int L>
struct NRegs {             // N in registers
  uint32_t n[L];
  __device__ __forceinline__ void load(const uint4 *s) {
#pragma unroll
    for (int g = 0; g < L / 4; ++g) {
      uint4 v = s[g];
      n[4 * g] = v.x; n[4 * g + 1] = v.y; n[4 * g + 2] = v.z; n[4 * g + 3] = v.w;
    }
  }
  __device__ __forceinline__ uint32_t get(int j) const { return n[j]; }
};
template <int L>
struct NSmem {             // N read from shared memory (warp-uniform address)
  const uint32_t *s;
  __device__ __forceinline__ uint32_t get(int j) const { return s[j]; }
};

// ------------------------------------------------------------------ CIOS pieces
// t[0 .. L+1] += b * a   (t < 2N on entry, so the sum fits in L+2 limbs).
// Two carry chains: the even limbs of a (products land on limbs 2k, 2k+1) and
// the odd limbs (limbs 2k+1, 2k+2).  Inside a chain the low and high halves of
// each product are consumed back to back, so no product stays live.
template <int L>
__device__ __forceinline__ void mul_acc(uint32_t (&t)[L + 2], const uint32_t (&a)[L], uint32_t b) {
  t[0] = mad_lo_cc(a[0], b, t[0]);
  t[1] = madc_hi_cc(a[0], b, t[1]);
#pragma unroll
  for (int k = 1; k < L / 2; ++k) {
    t[2 * k] = madc_lo_cc(a[2 * k], b, t[2 * k]);
    t[2 * k + 1] = madc_hi_cc(a[2 * k], b, t[2 * k + 1]);
  }
  t[L] = addc_cc(t[L], 0u);
  t[L + 1] = addc(t[L + 1], 0u);
  t[1] = mad_lo_cc(a[1], b, t[1]);
  t[2] = madc_hi_cc(a[1], b, t[2]);
#pragma unroll
  for (int k = 1; k < L / 2; ++k) {
    t[2 * k + 1] = madc_lo_cc(a[2 * k + 1], b, t[2 * k + 1]);
    t[2 * k + 2] = madc_hi_cc(a[2 * k + 1], b, t[2 * k + 2]);
  }
  t[L + 1] = addc(t[L + 1], 0u);
}

// One row of a product scan: t + a*b, the lowest limb returned and the rest
// shifted down one limb (t[j] <- position j+1).  t < 2^(32L) on entry, so the
// sum fits in L+1 limbs.  Even and odd limbs of a in two carry chains as in
// mul_acc.
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

// q = t_0 * n'; t = (t + q*N) / 2^32.  Same even/odd chains as mul_acc; every
// result is written one limb down (position p goes to t[p-1]), which is the
// division by 2^32, done in place in increasing position order.
template <int L, class NS>
__device__ __forceinline__ void reduce_step(uint32_t (&t)[L + 2], const NS &N, uint32_t np) {
  const uint32_t q = t[0] * np;
  // even limbs of N: positions 2k, 2k+1
  (void)mad_lo_cc(q, N.get(0), t[0]);  // position 0: = 0 mod 2^32, only the carry matters
  t[0] = madc_hi_cc(q, N.get(0), t[1]);
#pragma unroll
  for (int k = 1; k < L / 2; ++k) {
    t[2 * k - 1] = madc_lo_cc(q, N.get(2 * k), t[2 * k]);
    t[2 * k] = madc_hi_cc(q, N.get(2 * k), t[2 * k + 1]);
  }
  t[L - 1] = addc_cc(t[L], 0u);
  t[L] = addc(t[L + 1], 0u);
  // odd limbs of N: positions 2k+1, 2k+2, now held at t[2k], t[2k+1]
  t[0] = mad_lo_cc(q, N.get(1), t[0]);
  t[1] = madc_hi_cc(q, N.get(1), t[1]);
#pragma unroll
  for (int k = 1; k < L / 2; ++k) {
    t[2 * k] = madc_lo_cc(q, N.get(2 * k + 1), t[2 * k]);
    t[2 * k + 1] = madc_hi_cc(q, N.get(2 * k + 1), t[2 * k + 1]);
  }
  t[L] = addc(t[L], 0u);
  t[L + 1] = 0u;
}

// A = t - N if t >= N else t, without a branch (t < 2N, t[L] in {0,1}).
template <int L, class NS>
__device__ __forceinline__ void final_sub(uint32_t (&A)[L], const uint32_t (&t)[L + 2], const NS &N) {
  uint32_t u[L];
  u[0] = sub_cc(t[0], N.get(0));
#pragma unroll
  for (int j = 1; j < L; ++j) u[j] = subc_cc(t[j], N.get(j));
  const uint32_t keep_t = subc(t[L], 0u);  // all ones iff t < N
#pragma unroll
  for (int j = 0; j < L; ++j) A[j] = (t[j] & keep_t) | (u[j] & ~keep_t);
}

template <int L>
__device__ __forceinline__ void reduce_step_smem(uint32_t (&t)[L + 2], const uint4 *N4, uint32_t np);

template <class NS> struct IsNSmem { static constexpr bool value = false; };
template <int L> struct IsNSmem<NSmem<L>> { static constexpr bool value = true; };

// One reduction step with the modulus from registers, or from shared memory
// with 128-bit loads issued next to their use.
template <int L, class NS>
__device__ __forceinline__ void reduce_any(uint32_t (&t)[L + 2], const NS &N, uint32_t np) {
  if constexpr (IsNSmem<NS>::value) reduce_step_smem<L>(t, reinterpret_cast<const uint4 *>(N.s), np);
  else reduce_step<L>(t, N, np);
}

// A = A * B * R^-1 mod N.  The outer loop runs over B in blocks of U limbs
// (U a multiple of 4 dividing L): fully unrolled inside a block, a runtime
// loop across blocks to bound the code size.
template <int L, int U, class BS, class NS>
__device__ __forceinline__ void mont_mul(uint32_t (&A)[L], const BS &B, const NS &N, uint32_t np) {
  static_assert(L % 4 == 0 && U % 4 == 0 && L % U == 0, "limb blocking");
  uint32_t t[L + 2];
#pragma unroll
  for (int j = 0; j < L + 2; ++j) t[j] = 0u;
#pragma unroll 1
  for (int i0 = 0; i0 < L; i0 += U) {
#pragma unroll
    for (int u = 0; u < U; u += 4) {
      const uint4 b = B.get4((i0 + u) >> 2);
      mul_acc<L>(t, A, b.x);
      reduce_any<L>(t, N, np);
      mul_acc<L>(t, A, b.y);
      reduce_any<L>(t, N, np);
      mul_acc<L>(t, A, b.z);
      reduce_any<L>(t, N, np);
      mul_acc<L>(t, A, b.w);
      reduce_any<L>(t, N, np);
    }
  }
  final_sub<L>(A, t, N);
}

// A = A^2 * R^-1 mod N (A < N), separated form: the square A^2 first, then a
// Montgomery reduction of the 2L-limb product.  The square needs each cross
// product a_i a_j (i < j) once, doubled, plus the diagonal a_i^2:
// L(L+1)/2 word products instead of L^2; the reduction costs L^2 + L like the
// second half of CIOS.  Every index is a compile-time constant (fully
// unrolled), so the 2L-limb product lives in registers.
template <int L, class NS>
__device__ __forceinline__ void mont_sqr(uint32_t (&A)[L], const NS &N, uint32_t np) {
  uint32_t t[2 * L];
#pragma unroll
  for (int k = 0; k < 2 * L; ++k) t[k] = 0u;
  // cross products, row i: t[i+j .. i+j+1] += a_i * a_j for j > i, two chains
  // (j - i odd, j - i even), each closed by propagating its carry two limbs up
#pragma unroll
  for (int i = 0; i < L - 1; ++i) {
#pragma unroll
    for (int par = 0; par < 2; ++par) {
      const int j0 = i + 1 + par;
      if (j0 <= L - 1) {
        t[i + j0] = mad_lo_cc(A[i], A[j0], t[i + j0]);
        t[i + j0 + 1] = madc_hi_cc(A[i], A[j0], t[i + j0 + 1]);
        int last = i + j0 + 1;
#pragma unroll
        for (int j = j0 + 2; j < L; j += 2) {
          t[i + j] = madc_lo_cc(A[i], A[j], t[i + j]);
          t[i + j + 1] = madc_hi_cc(A[i], A[j], t[i + j + 1]);
          last = i + j + 1;
        }
        if (last + 2 < 2 * L) {
          t[last + 1] = addc_cc(t[last + 1], 0u);
          t[last + 2] = addc(t[last + 2], 0u);
        } else if (last + 1 < 2 * L) {
          t[last + 1] = addc(t[last + 1], 0u);
        }
      }
    }
  }
  // double (the cross sum is below 2^(64L-1), so nothing leaves the top limb)
#pragma unroll
  for (int k = 2 * L - 1; k > 0; --k) t[k] = __funnelshift_l(t[k - 1], t[k], 1);
  t[0] <<= 1;
  // diagonal squares a_i^2 at limbs 2i, 2i+1
  t[0] = mad_lo_cc(A[0], A[0], t[0]);
  t[1] = madc_hi_cc(A[0], A[0], t[1]);
#pragma unroll
  for (int i = 1; i < L; ++i) {
    t[2 * i] = madc_lo_cc(A[i], A[i], t[2 * i]);
    t[2 * i + 1] = madc_hi_cc(A[i], A[i], t[2 * i + 1]);
  }
  // Montgomery reduction: step i clears limb i by adding q*N*2^(32i); the
  // carry leaving limb i+L waits in c and enters at the next step's top limb.
  uint32_t c = 0u;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const uint32_t q = t[i] * np;
    (void)mad_lo_cc(q, N.get(0), t[i]);
    t[i + 1] = madc_hi_cc(q, N.get(0), t[i + 1]);
#pragma unroll
    for (int k = 1; k < L / 2; ++k) {
      t[i + 2 * k] = madc_lo_cc(q, N.get(2 * k), t[i + 2 * k]);
      t[i + 2 * k + 1] = madc_hi_cc(q, N.get(2 * k), t[i + 2 * k + 1]);
    }
    t[i + L] = addc_cc(t[i + L], c);
    const uint32_t c1 = addc(0u, 0u);
    t[i + 1] = mad_lo_cc(q, N.get(1), t[i + 1]);
    t[i + 2] = madc_hi_cc(q, N.get(1), t[i + 2]);
#pragma unroll
    for (int k = 1; k < L / 2; ++k) {
      t[i + 2 * k + 1] = madc_lo_cc(q, N.get(2 * k + 1), t[i + 2 * k + 1]);
      t[i + 2 * k + 2] = madc_hi_cc(q, N.get(2 * k + 1), t[i + 2 * k + 2]);
    }
    c = addc(c1, 0u);
  }
  uint32_t r[L + 2];
#pragma unroll
  for (int j = 0; j < L; ++j) r[j] = t[L + j];
  r[L] = c;
  r[L + 1] = 0u;
  final_sub<L>(A, r, N);
}

// A = A^2 * R^-1 mod N (A < N), separated form with a compact reduction: the
// square's cross products (each a_i a_j, i < j, once), doubled, plus the
// diagonal, fully unrolled (L(L+1)/2 word products); its upper L limbs go to
// the per-lane stage and the Montgomery reduction runs as the same U-blocked
// loop as mont_mul, taking one upper limb per step:
//   t = low L limbs; for each i: t[L] += upper_i, then reduce_step (q, + q*N, / 2^32).
template <int L, int U, class NS>
__device__ __forceinline__ void mont_sqr_h(uint32_t (&A)[L], const NS &N, uint32_t np, uint4 *stage_lane) {
  static_assert(L % 4 == 0 && U % 4 == 0 && L % U == 0, "limb blocking");
  uint32_t t2[2 * L];
#pragma unroll
  for (int k = 0; k < 2 * L; ++k) t2[k] = 0u;
#pragma unroll
  for (int i = 0; i < L - 1; ++i) {
#pragma unroll
    for (int par = 0; par < 2; ++par) {
      const int j0 = i + 1 + par;
      if (j0 <= L - 1) {
        t2[i + j0] = mad_lo_cc(A[i], A[j0], t2[i + j0]);
        t2[i + j0 + 1] = madc_hi_cc(A[i], A[j0], t2[i + j0 + 1]);
        int last = i + j0 + 1;
#pragma unroll
        for (int j = j0 + 2; j < L; j += 2) {
          t2[i + j] = madc_lo_cc(A[i], A[j], t2[i + j]);
          t2[i + j + 1] = madc_hi_cc(A[i], A[j], t2[i + j + 1]);
          last = i + j + 1;
        }
        if (last + 2 < 2 * L) {
          t2[last + 1] = addc_cc(t2[last + 1], 0u);
          t2[last + 2] = addc(t2[last + 2], 0u);
        } else if (last + 1 < 2 * L) {
          t2[last + 1] = addc(t2[last + 1], 0u);
        }
      }
    }
  }
#pragma unroll
  for (int k = 2 * L - 1; k > 0; --k) t2[k] = __funnelshift_l(t2[k - 1], t2[k], 1);
  t2[0] <<= 1;
  t2[0] = mad_lo_cc(A[0], A[0], t2[0]);
  t2[1] = madc_hi_cc(A[0], A[0], t2[1]);
#pragma unroll
  for (int i = 1; i < L; ++i) {
    t2[2 * i] = madc_lo_cc(A[i], A[i], t2[2 * i]);
    t2[2 * i + 1] = madc_hi_cc(A[i], A[i], t2[2 * i + 1]);
  }
#pragma unroll
  for (int g = 0; g < L / 4; ++g)
    stage_lane[g * 32] = make_uint4(t2[L + 4 * g], t2[L + 4 * g + 1], t2[L + 4 * g + 2], t2[L + 4 * g + 3]);
  uint32_t t[L + 2];
#pragma unroll
  for (int j = 0; j < L; ++j) t[j] = t2[j];
  t[L] = 0u;
  t[L + 1] = 0u;
#pragma unroll 1
  for (int i0 = 0; i0 < L; i0 += U) {
#pragma unroll
    for (int u = 0; u < U; u += 4) {
      const uint4 up = stage_lane[((i0 + u) >> 2) * 32];
      t[L] = add_cc(t[L], up.x);
      t[L + 1] = addc(t[L + 1], 0u);
      reduce_any<L>(t, N, np);
      t[L] = add_cc(t[L], up.y);
      t[L + 1] = addc(t[L + 1], 0u);
      reduce_any<L>(t, N, np);
      t[L] = add_cc(t[L], up.z);
      t[L + 1] = addc(t[L + 1], 0u);
      reduce_any<L>(t, N, np);
      t[L] = add_cc(t[L], up.w);
      t[L + 1] = addc(t[L + 1], 0u);
      reduce_any<L>(t, N, np);
    }
  }
  final_sub<L>(A, t, N);
}

// ------------------------------------------------------------------ wide operands (L = 96, 128)
// 128-bit shared-memory load issued exactly where written (volatile asm is not
// reordered against the carry-chain asm), so operands are not hoisted into
// registers ahead of their use.
__device__ __forceinline__ uint4 lds128(const uint4 *p) {
  uint4 v;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}

// For moduli too wide to keep A in registers next to the accumulator, A lives
// in a per-lane staging buffer (layout [L/4][32] of uint4) and is streamed
// like B; only t stays in registers.  Same CIOS steps and chains as mul_acc.

// t += b * A with A read from shared memory (even limbs, then odd limbs)
template <int L>
__device__ __forceinline__ void mul_acc_smem(uint32_t (&t)[L + 2], const uint4 *A_lane, uint32_t b) {
  {
    const uint4 a = lds128(A_lane);
    t[0] = mad_lo_cc(a.x, b, t[0]);
    t[1] = madc_hi_cc(a.x, b, t[1]);
    t[2] = madc_lo_cc(a.z, b, t[2]);
    t[3] = madc_hi_cc(a.z, b, t[3]);
  }
#pragma unroll
  for (int g = 1; g < L / 4; ++g) {
    const uint4 a = lds128(A_lane + g * 32);
    t[4 * g] = madc_lo_cc(a.x, b, t[4 * g]);
    t[4 * g + 1] = madc_hi_cc(a.x, b, t[4 * g + 1]);
    t[4 * g + 2] = madc_lo_cc(a.z, b, t[4 * g + 2]);
    t[4 * g + 3] = madc_hi_cc(a.z, b, t[4 * g + 3]);
  }
  t[L] = addc_cc(t[L], 0u);
  t[L + 1] = addc(t[L + 1], 0u);
  {
    const uint4 a = lds128(A_lane);
    t[1] = mad_lo_cc(a.y, b, t[1]);
    t[2] = madc_hi_cc(a.y, b, t[2]);
    t[3] = madc_lo_cc(a.w, b, t[3]);
    t[4] = madc_hi_cc(a.w, b, t[4]);
  }
#pragma unroll
  for (int g = 1; g < L / 4; ++g) {
    const uint4 a = lds128(A_lane + g * 32);
    t[4 * g + 1] = madc_lo_cc(a.y, b, t[4 * g + 1]);
    t[4 * g + 2] = madc_hi_cc(a.y, b, t[4 * g + 2]);
    t[4 * g + 3] = madc_lo_cc(a.w, b, t[4 * g + 3]);
    t[4 * g + 4] = madc_hi_cc(a.w, b, t[4 * g + 4]);
  }
  t[L + 1] = addc(t[L + 1], 0u);
}

// reduce_step with N read from shared memory four limbs at a time next to its
// use (the even chain takes .x/.z, the odd chain .y/.w of each group).
template <int L>
__device__ __forceinline__ void reduce_step_smem(uint32_t (&t)[L + 2], const uint4 *N4, uint32_t np) {
  const uint32_t q = t[0] * np;
  {
    const uint4 n = lds128(N4);
    (void)mad_lo_cc(q, n.x, t[0]);
    t[0] = madc_hi_cc(q, n.x, t[1]);
    t[1] = madc_lo_cc(q, n.z, t[2]);
    t[2] = madc_hi_cc(q, n.z, t[3]);
  }
#pragma unroll
  for (int g = 1; g < L / 4; ++g) {
    const uint4 n = lds128(N4 + g);
    t[4 * g - 1] = madc_lo_cc(q, n.x, t[4 * g]);
    t[4 * g] = madc_hi_cc(q, n.x, t[4 * g + 1]);
    t[4 * g + 1] = madc_lo_cc(q, n.z, t[4 * g + 2]);
    t[4 * g + 2] = madc_hi_cc(q, n.z, t[4 * g + 3]);
  }
  t[L - 1] = addc_cc(t[L], 0u);
  t[L] = addc(t[L + 1], 0u);
  {
    const uint4 n = lds128(N4);
    t[0] = mad_lo_cc(q, n.y, t[0]);
    t[1] = madc_hi_cc(q, n.y, t[1]);
    t[2] = madc_lo_cc(q, n.w, t[2]);
    t[3] = madc_hi_cc(q, n.w, t[3]);
  }
#pragma unroll
  for (int g = 1; g < L / 4; ++g) {
    const uint4 n = lds128(N4 + g);
    t[4 * g] = madc_lo_cc(q, n.y, t[4 * g]);
    t[4 * g + 1] = madc_hi_cc(q, n.y, t[4 * g + 1]);
    t[4 * g + 2] = madc_lo_cc(q, n.w, t[4 * g + 2]);
    t[4 * g + 3] = madc_hi_cc(q, n.w, t[4 * g + 3]);
  }
  t[L] = addc(t[L], 0u);
  t[L + 1] = 0u;
}

// A_lane = t - N if t >= N else t (t < 2N), written back in groups of four.
// First pass finds the borrow of t - N, second pass recomputes the difference
// limb by limb and selects, so no L-limb temporary is needed.
template <int L, class NS>
__device__ __forceinline__ void final_sub_smem(uint4 *A_lane, const uint32_t (&t)[L + 2], const NS &N) {
  uint32_t d = sub_cc(t[0], N.get(0));
#pragma unroll
  for (int j = 1; j < L; ++j) d = subc_cc(t[j], N.get(j));
  const uint32_t keep_t = subc(t[L], 0u);  // all ones iff t < N
  (void)d;
  uint32_t u0 = sub_cc(t[0], N.get(0));
#pragma unroll
  for (int g = 0; g < L / 4; ++g) {
    uint32_t u1, u2, u3;
    if (g > 0) u0 = subc_cc(t[4 * g], N.get(4 * g));
    u1 = subc_cc(t[4 * g + 1], N.get(4 * g + 1));
    u2 = subc_cc(t[4 * g + 2], N.get(4 * g + 2));
    u3 = subc_cc(t[4 * g + 3], N.get(4 * g + 3));
    A_lane[g * 32] = make_uint4((t[4 * g] & keep_t) | (u0 & ~keep_t), (t[4 * g + 1] & keep_t) | (u1 & ~keep_t),
                                (t[4 * g + 2] & keep_t) | (u2 & ~keep_t), (t[4 * g + 3] & keep_t) | (u3 & ~keep_t));
  }
}

// A_lane = A * B * R^-1 mod N with A in shared memory (B may alias A).
template <int L, int U, class NS>
__device__ __forceinline__ void mont_mul_smemA(uint4 *A_lane, const SmemB &B, const NS &N, uint32_t np) {
  static_assert(L % 4 == 0 && U % 4 == 0 && L % U == 0, "limb blocking");
  const uint4 *N4 = reinterpret_cast<const uint4 *>(N.s);
  uint32_t t[L + 2];
#pragma unroll
  for (int j = 0; j < L + 2; ++j) t[j] = 0u;
#pragma unroll 1
  for (int i0 = 0; i0 < L; i0 += U) {
#pragma unroll
    for (int u = 0; u < U; u += 4) {
      const uint4 b = B.get4((i0 + u) >> 2);
      mul_acc_smem<L>(t, A_lane, b.x);
      reduce_step_smem<L>(t, N4, np);
      mul_acc_smem<L>(t, A_lane, b.y);
      reduce_step_smem<L>(t, N4, np);
      mul_acc_smem<L>(t, A_lane, b.z);
      reduce_step_smem<L>(t, N4, np);
      mul_acc_smem<L>(t, A_lane, b.w);
      reduce_step_smem<L>(t, N4, np);
    }
  }
  final_sub_smem<L>(A_lane, t, N);
}

// ------------------------------------------------------------------ modular add / sub
// A = (A + B) mod N for A, B < N (B from a per-lane stage).
template <int L, class NS>
__device__ __forceinline__ void mod_add(uint32_t (&A)[L], const SmemB &B, const NS &N) {
  uint32_t s[L];
#pragma unroll
  for (int g = 0; g < L / 4; ++g) {
    const uint4 b = B.get4(g);
    if (g == 0) s[0] = add_cc(A[0], b.x); else s[4 * g] = addc_cc(A[4 * g], b.x);
    s[4 * g + 1] = addc_cc(A[4 * g + 1], b.y);
    s[4 * g + 2] = addc_cc(A[4 * g + 2], b.z);
    s[4 * g + 3] = addc_cc(A[4 * g + 3], b.w);
  }
  uint32_t t[L + 2];
#pragma unroll
  for (int j = 0; j < L; ++j) t[j] = s[j];
  t[L] = addc(0u, 0u);
  t[L + 1] = 0u;
  final_sub<L>(A, t, N);
}

// A = (B - A) mod N for A, B < N (B from a per-lane stage): B - A, plus N on borrow.
template <int L, class NS>
__device__ __forceinline__ void mod_rsub(uint32_t (&A)[L], const SmemB &B, const NS &N) {
  uint32_t s[L];
#pragma unroll
  for (int g = 0; g < L / 4; ++g) {
    const uint4 b = B.get4(g);
    if (g == 0) s[0] = sub_cc(b.x, A[0]); else s[4 * g] = subc_cc(b.x, A[4 * g]);
    s[4 * g + 1] = subc_cc(b.y, A[4 * g + 1]);
    s[4 * g + 2] = subc_cc(b.z, A[4 * g + 2]);
    s[4 * g + 3] = subc_cc(b.w, A[4 * g + 3]);
  }
  const uint32_t neg = subc(0u, 0u);  // all ones iff B < A
  A[0] = add_cc(s[0], N.get(0) & neg);
#pragma unroll
  for (int j = 1; j < L; ++j) A[j] = addc_cc(s[j], N.get(j) & neg);
}

// ------------------------------------------------------------------ staging helpers
template <int L>
__device__ __forceinline__ void to_stage(uint4 *stage_lane, const uint32_t (&A)[L]) {
#pragma unroll
  for (int g = 0; g < L / 4; ++g)
    stage_lane[g * 32] = make_uint4(A[4 * g], A[4 * g + 1], A[4 * g + 2], A[4 * g + 3]);
}
template <int L>
__device__ __forceinline__ void from_stage(uint32_t (&A)[L], const uint4 *stage_lane) {
#pragma unroll
  for (int g = 0; g < L / 4; ++g) {
    const uint4 v = stage_lane[g * 32];
    A[4 * g] = v.x; A[4 * g + 1] = v.y; A[4 * g + 2] = v.z; A[4 * g + 3] = v.w;
  }
}
template <int L>
__device__ __forceinline__ void from_uniform(uint32_t (&A)[L], const uint4 *s) {
#pragma unroll
  for (int g = 0; g < L / 4; ++g) {
    const uint4 v = s[g];
    A[4 * g] = v.x; A[4 * g + 1] = v.y; A[4 * g + 2] = v.z; A[4 * g + 3] = v.w;
  }
}

// ---------------------------------------------------------------- squares, each cross product once
// The square of an N-limb a is T = 2C + D, C the cross products a_i a_j
// (i < j), D the squares a_k^2 at limbs 2k, 2k+1.  Row I adds a_I a_j for
// j > I in two carry chains (odd and even j - I); after row I the limbs of C
// up to 2I+2 are final, so T's limbs 2I+1 and 2I+2 are formed (the doubling
// shifts in the top bit of the limb below) and handed on at once, which keeps
// the live part of C short.  N(N+1)/2 word products.
//
// One chain of row I: a_I a_j for j = J0, J0+2, ... < H, added at positions
// I+j (low) and I+j+1 (high); its carry lands after its last high word.
template <int H, int I, int J0>
__device__ __forceinline__ void sq_chain(uint32_t (&c)[2 * H], const uint32_t (&a)[H]) {
  if constexpr (J0 < H) {
    c[I + J0] = mad_lo_cc(a[I], a[J0], c[I + J0]);
    c[I + J0 + 1] = madc_hi_cc(a[I], a[J0], c[I + J0 + 1]);
#pragma unroll
    for (int j = J0 + 2; j < H; j += 2) {
      c[I + j] = madc_lo_cc(a[I], a[j], c[I + j]);
      c[I + j + 1] = madc_hi_cc(a[I], a[j], c[I + j + 1]);
    }
    constexpr int last = J0 + ((H - 1 - J0) / 2) * 2;
    c[I + last + 2] = addc(c[I + last + 2], 0u);
  }
}

// Rows I .. N-2; limb p of T goes to emit.put<p>() (in increasing p).
template <int N, int I, class E>
__device__ __forceinline__ void sq_rows(uint32_t (&c)[2 * N], const uint32_t (&a)[N], uint32_t &tc_carry, E &emit) {
  if constexpr (I < N - 1) {
    sq_chain<N, I, I + 1>(c, a);
    sq_chain<N, I, I + 2>(c, a);
    const uint32_t x0 = __funnelshift_l(c[2 * I], c[2 * I + 1], 1), x1 = __funnelshift_l(c[2 * I + 1], c[2 * I + 2], 1);
    (void)add_cc(tc_carry, 0xFFFFFFFFu);   // carry flag <- tc_carry
    const uint32_t t0 = addc_cc(x0, __umulhi(a[I], a[I]));
    const uint32_t t1 = addc_cc(x1, a[I + 1] * a[I + 1]);
    tc_carry = addc(0u, 0u);
    emit.template put<2 * I + 1>(t0);
    emit.template put<2 * I + 2>(t1);
    sq_rows<N, I + 1>(c, a, tc_carry, emit);
  }
}

// T = a^2 for an N-limb a, its 2N limbs handed to emit in increasing order
template <int N, class E>
__device__ __forceinline__ void square_emit(const uint32_t (&a)[N], E &emit) {
  uint32_t c[2 * N];
#pragma unroll
  for (int j = 0; j < 2 * N; ++j) c[j] = 0u;
  uint32_t tc_carry = 0u;
  emit.template put<0>(a[0] * a[0]);
  sq_rows<N, 0>(c, a, tc_carry, emit);
  emit.template put<2 * N - 1>(__funnelshift_l(c[2 * N - 2], c[2 * N - 1], 1) + __umulhi(a[N - 1], a[N - 1]) +
                               tc_carry);
}

}  // namespace rsagpu
