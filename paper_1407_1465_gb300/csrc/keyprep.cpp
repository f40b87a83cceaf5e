// keyprep.cpp -- host precomputation of the per-key constants (see keyprep.h).
#include "keyprep.h"

#include <algorithm>

#include "keyrec.h"

namespace rsagpu {
namespace {

using Nat = std::vector<uint32_t>;

bool is_zero(const Nat &a) {
  for (uint32_t w : a)
    if (w) return false;
  return true;
}
bool is_one(const Nat &a) {
  if (a.empty() || a[0] != 1u) return false;
  for (size_t i = 1; i < a.size(); ++i)
    if (a[i]) return false;
  return true;
}
// compare a and b as numbers (any lengths)
int cmp(const Nat &a, const Nat &b) {
  size_t n = std::max(a.size(), b.size());
  for (size_t i = n; i-- > 0;) {
    uint32_t x = i < a.size() ? a[i] : 0u, y = i < b.size() ? b[i] : 0u;
    if (x != y) return x < y ? -1 : 1;
  }
  return 0;
}
// a -= b (b no longer than a, a >= b)
void sub_in(Nat &a, const Nat &b) {
  uint64_t borrow = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    uint64_t y = (i < b.size() ? b[i] : 0u) + borrow;
    uint64_t x = a[i];
    a[i] = (uint32_t)(x - y);
    borrow = x < y ? 1 : 0;
  }
}
// a += b, returns the carry out of a's top limb
uint32_t add_in(Nat &a, const Nat &b) {
  uint64_t carry = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    uint64_t s = (uint64_t)a[i] + (i < b.size() ? b[i] : 0u) + carry;
    a[i] = (uint32_t)s;
    carry = s >> 32;
  }
  return (uint32_t)carry;
}
void shl1_in(Nat &a, uint32_t bit_in) {
  for (size_t i = 0; i < a.size(); ++i) {
    uint32_t out = a[i] >> 31;
    a[i] = (a[i] << 1) | bit_in;
    bit_in = out;
  }
}
void shr1_in(Nat &a, uint32_t bit_in_top) {
  for (size_t i = a.size(); i-- > 0;) {
    uint32_t out = a[i] & 1u;
    a[i] = (a[i] >> 1) | (bit_in_top << 31);
    bit_in_top = out;
  }
}
uint32_t bitlen(const Nat &a) {
  for (size_t i = a.size(); i-- > 0;)
    if (a[i]) return (uint32_t)(32 * i + 32 - __builtin_clz(a[i]));
  return 0;
}
// x = (x + y) / 2 mod m style helper: halve x modulo odd m (x < m)
void half_mod(Nat &x, const Nat &m) {
  if (x[0] & 1u) {
    uint32_t c = add_in(x, m);
    shr1_in(x, c);
  } else {
    shr1_in(x, 0u);
  }
}
// x = (x - y) mod m for x, y < m
void sub_mod(Nat &x, const Nat &y, const Nat &m) {
  if (cmp(x, y) >= 0) {
    sub_in(x, y);
  } else {
    uint32_t c = add_in(x, m);  // x + m < 2m; may carry out of the top limb
    (void)c;
    sub_in(x, y);               // wraps correctly modulo 2^(32*len)
  }
}
Nat mul(const Nat &a, const Nat &b) {
  Nat r(a.size() + b.size(), 0u);
  for (size_t i = 0; i < a.size(); ++i) {
    uint64_t carry = 0;
    for (size_t j = 0; j < b.size(); ++j) {
      uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
    r[i + b.size()] = (uint32_t)carry;
  }
  return r;
}
Nat minus_one(const Nat &a) {
  Nat r = a;
  sub_in(r, Nat{1u});
  return r;
}
void put(std::vector<uint32_t> &rec, uint32_t off, const Nat &v, size_t len) {
  for (size_t i = 0; i < len; ++i) rec[off + i] = i < v.size() ? v[i] : 0u;
}

}  // namespace

uint32_t neg_inv32(uint32_t n0) {
  uint32_t x = n0;                       // n0 * n0 = 1 mod 8 for odd n0
  for (int i = 0; i < 4; ++i) x *= 2u - n0 * x;  // Newton: doubles the correct bits
  return 0u - x;
}

void pow2_mod(Nat &out, const Nat &m, uint64_t k) {
  const size_t lm = m.size();
  Nat r(lm + 1, 0u), mm(m);
  mm.push_back(0u);
  if (cmp(m, Nat{1u}) > 0) r[0] = 1u;
  for (uint64_t i = 0; i < k; ++i) {
    shl1_in(r, 0u);
    if (cmp(r, mm) >= 0) sub_in(r, mm);
  }
  out.assign(r.begin(), r.begin() + lm);
}

void mod_bitserial(Nat &out, const Nat &a, const Nat &m) {
  const size_t lm = m.size();
  Nat r(lm + 1, 0u), mm(m);
  mm.push_back(0u);
  for (uint32_t i = bitlen(a); i-- > 0;) {
    shl1_in(r, (a[i / 32] >> (i % 32)) & 1u);
    if (cmp(r, mm) >= 0) sub_in(r, mm);
  }
  out.assign(r.begin(), r.begin() + lm);
}

bool inv_mod(Nat &out, const Nat &a, const Nat &m) {
  // binary extended Euclid for odd m: x1*a = u, x2*a = v (mod m) throughout
  Nat u, v(m), x1(m.size(), 0u), x2(m.size(), 0u);
  mod_bitserial(u, a, m);
  x1[0] = 1u;
  if (is_zero(u) || !(m[0] & 1u)) return false;
  while (!is_one(u) && !is_one(v)) {
    while (!(u[0] & 1u)) {
      shr1_in(u, 0u);
      half_mod(x1, m);
    }
    while (!(v[0] & 1u)) {
      shr1_in(v, 0u);
      half_mod(x2, m);
    }
    if (cmp(u, v) >= 0) {
      sub_in(u, v);
      sub_mod(x1, x2, m);
    } else {
      sub_in(v, u);
      sub_mod(x2, x1, m);
    }
    if (is_zero(u) || is_zero(v)) return false;  // gcd(a, m) > 1
  }
  out = is_one(u) ? x1 : x2;
  return true;
}

std::string build_key_record(const KeyInput &in, std::vector<uint32_t> &rec, uint32_t &flags,
                             char *err_class) {
  auto fail = [&](char c, const char *msg) {
    *err_class = c;
    return std::string(msg);
  };
  const uint32_t nbits = in.nbits;
  if (!(nbits == 32 || nbits == 1024 || nbits == 2048 || nbits == 3072 || nbits == 4096))
    return fail('U', "key size must be 32 (single limb) or 1024, 2048, 3072, 4096 bits");
  const uint32_t L = nbits / 32, H = L / 2;
  if (in.n.size() != L) return fail('A', "n must have nbits/32 limbs");
  if (!(in.n[0] & 1u)) return fail('K', "modulus must be odd");
  if (cmp(in.n, Nat{1u}) <= 0) return fail('K', "modulus must exceed 1");
  if (L > 1 && in.n[L - 1] == 0u) return fail('K', "modulus must have exactly nbits bits (top limb nonzero)");
  if (in.e.empty() || in.e.size() > L || is_zero(in.e)) return fail('K', "public exponent must be 1..L limbs and nonzero");
  const bool has_d = !in.d.empty();
  if (has_d && (in.d.size() != L || is_zero(in.d))) return fail('K', "private exponent must have L limbs and be nonzero");
  const bool has_pq = !in.p.empty() || !in.q.empty();
  const uint32_t hl = (L == 1) ? 1u : H;
  if (has_pq) {
    if (in.p.size() != hl || in.q.size() != hl) return fail('A', "p and q must have L/2 limbs each (1 for 32-bit keys)");
    if (!has_d) return fail('K', "p and q given without d");
    if (!(in.p[0] & 1u) || !(in.q[0] & 1u)) return fail('K', "p and q must be odd");
    if (cmp(in.p, Nat{1u}) <= 0 || cmp(in.q, Nat{1u}) <= 0) return fail('K', "p and q must exceed 1");
    if (cmp(mul(in.p, in.q), in.n) != 0) return fail('K', "p*q != n");
  }
  const KeyLayout lay(L);
  rec.assign(lay.total, 0u);
  KeyHeader hd{};
  hd.nbits = nbits;
  hd.L = L;
  hd.H = H;
  hd.np_n = neg_inv32(in.n[0]);
  hd.e_bits = bitlen(in.e);
  hd.d_bits = has_d ? bitlen(in.d) : 0u;
  flags = has_d ? KEY_HAS_D : 0u;

  Nat t;
  put(rec, lay.n, in.n, L);
  pow2_mod(t, in.n, 64ull * L);
  put(rec, lay.r2n, t, L);
  pow2_mod(t, in.n, 32ull * L);
  put(rec, lay.onen, t, L);
  put(rec, lay.unitL, Nat{1u}, L);
  put(rec, lay.e, in.e, L + 4);
  if (has_d) put(rec, lay.d, in.d, L + 4);

  if (has_pq) {
    Nat qinv, dp, dq;
    if (!inv_mod(qinv, in.q, in.p)) return fail('K', "q has no inverse mod p (gcd(p, q) != 1)");
    mod_bitserial(dp, in.d, minus_one(in.p));
    mod_bitserial(dq, in.d, minus_one(in.q));
    // d = 0 mod (p-1): use p-1 itself so that c = 0 mod p still maps to 0
    if (is_zero(dp)) dp = minus_one(in.p);
    if (is_zero(dq)) dq = minus_one(in.q);
    hd.np_p = neg_inv32(in.p[0]);
    hd.np_q = neg_inv32(in.q[0]);
    flags |= KEY_HAS_CRT;
    if (L == 1) {
      // single-limb keys keep p, q, dp, dq, qinv in the header
      hd.reserved[0] = in.p[0];
      hd.reserved[1] = in.q[0];
      hd.reserved[2] = dp[0];
      hd.reserved[3] = dq[0];
      hd.reserved[4] = qinv[0];
    } else {
      put(rec, lay.p, in.p, H);
      put(rec, lay.q, in.q, H);
      pow2_mod(t, in.p, 64ull * H);
      put(rec, lay.r2p, t, H);
      pow2_mod(t, in.p, 96ull * H);
      put(rec, lay.r3p, t, H);
      pow2_mod(t, in.q, 64ull * H);
      put(rec, lay.r2q, t, H);
      pow2_mod(t, in.q, 96ull * H);
      put(rec, lay.r3q, t, H);
      pow2_mod(t, in.p, 32ull * H);
      put(rec, lay.onep, t, H);
      pow2_mod(t, in.q, 32ull * H);
      put(rec, lay.oneq, t, H);
      put(rec, lay.qinv, qinv, H);
      put(rec, lay.unitH, Nat{1u}, H);
      put(rec, lay.dp, dp, H + 4);
      put(rec, lay.dq, dq, H + 4);
    }
  }
  hd.flags = flags;
  const uint32_t *hw = reinterpret_cast<const uint32_t *>(&hd);
  std::copy(hw, hw + 16, rec.begin());
  return std::string();
}

}  // namespace rsagpu
