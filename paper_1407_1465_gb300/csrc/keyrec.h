// keyrec.h -- layout of the device-resident key record (host and device).
//
// One record per loaded key, built on the host at key load (per-key
// precomputation) and copied once to device memory.  Every limb array starts
// on a 16-byte boundary so the kernels read it with 128-bit loads.
//
//   words 0..15   header (KeyHeader)
//   n, R^2 mod n, R mod n, unit(=1)           L limbs each      (R = 2^(32L))
//   e, d                                      L+4 limbs each    (zero padded)
//   p, q, R^2 mod p, R^3 mod p, R^2 mod q, R^3 mod q,
//   R mod p, R mod q, qinv = q^-1 mod p, unit  H limbs each      (R = 2^(32H))
//   dp = d mod (p-1), dq = d mod (q-1)         H+4 limbs each
// with H = L/2.  Exponent arrays carry padding so a window that straddles the
// top limb can read one limb past it.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define RSAGPU_HD __host__ __device__
#else
#define RSAGPU_HD
#endif

namespace rsagpu {

enum : uint32_t { KEY_HAS_D = 1u, KEY_HAS_CRT = 2u };

struct KeyHeader {
  uint32_t nbits, L, H, flags;
  uint32_t np_n, np_p, np_q;    // -m^-1 mod 2^32 for m = n, p, q
  uint32_t e_bits, d_bits;      // bit lengths (e_bits drives the public binary method)
  uint32_t reserved[7];
};
static_assert(sizeof(KeyHeader) == 64, "header is 16 words");

struct KeyLayout {
  uint32_t L, H;
  uint32_t n, r2n, onen, unitL, e, d;
  uint32_t p, q, r2p, r3p, r2q, r3q, onep, oneq, qinv, unitH, dp, dq;
  uint32_t total;  // words
  RSAGPU_HD constexpr explicit KeyLayout(uint32_t L_)
      : L(L_), H(L_ / 2),
        n(16), r2n(16 + L_), onen(16 + 2 * L_), unitL(16 + 3 * L_), e(16 + 4 * L_),
        d(16 + 5 * L_ + 4),
        p(16 + 6 * L_ + 8), q(p + L_ / 2), r2p(q + L_ / 2), r3p(r2p + L_ / 2), r2q(r3p + L_ / 2),
        r3q(r2q + L_ / 2), onep(r3q + L_ / 2), oneq(onep + L_ / 2), qinv(oneq + L_ / 2),
        unitH(qinv + L_ / 2), dp(unitH + L_ / 2), dq(dp + L_ / 2 + 4), total(dq + L_ / 2 + 4) {}
};

}  // namespace rsagpu
