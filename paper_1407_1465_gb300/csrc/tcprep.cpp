// tcprep.cpp -- host construction of the tensor-core operands of one prime.
//
// The tensor-core kernel (crt_tc.cu) reduces a 2048-bit product T modulo a
// 1024-bit prime m with Montgomery's method, R = 2^1024:
//     mu = (T mod R) * m' mod R,  m' = -m^-1 mod R
//     U  = (T + mu * m) / R
// Both products have one operand that is the same for every message of the
// batch (m' and m), so each is a matrix product: the per-message byte digits
// (rows) times a Toeplitz matrix built from the constant's byte digits.  This
// file builds those two matrices, as fp16 values (bytes 0..255 are exact), in
// the shared-memory layout the kernel's MMA descriptors expect.
//
//   BM (128 x 144): row n (output digit n of mu), column k < 128: m'_{n-k}
//       (0 outside 0 <= n-k < 128);  columns 128..143: 2048 (bias block)
//   BP (128 x 144): row j = output position n = 124 + j of mu * m,
//       column k < 128: m_{n-k} (0 outside 0 <= n-k < 128);  columns 128..143: 2048
//
// The bias block meets a constant A block of 2^-16 (an fp16 subnormal) in the
// kernel, so every output column starts at 16 * 2^-16 * 2048 = 1/2 and the
// per-message digits enter as d * 2^-24: a column sum w < 2^23 then reads
// back as the fp32 1/2 + w * 2^-24, whose bit pattern is 0x3F000000 + w.
#include <cstring>
#include <vector>

#include "crt_tc.h"

namespace rsagpu {
namespace tcr {

// fp16 bit pattern of an integer 0 <= x < 2048 (exact).
uint16_t f16_of_int(uint32_t x) {
  if (x == 0) return 0;
  int e = 31 - __builtin_clz(x);
  const uint32_t mant = (x << (10 - e)) & 0x3FFu;
  return (uint16_t)(((uint32_t)(e + 15) << 10) | mant);
}

// Byte offset of element (row, k) in a K-major no-swizzle core-matrix image
// with `rows` rows: [k / 8][row / 8][row % 8][k % 8].
size_t core_off(int row, int k, int rows) {
  return (size_t)(k / 8) * (size_t)(rows / 8) * 128 + (size_t)(row / 8) * 128 + (size_t)(row % 8) * 16 +
         (size_t)(k % 8) * 2;
}

// out = a * b mod 2^(32 n)
void mul_lo(const uint32_t *a, const uint32_t *b, uint32_t *out, int n) {
  std::vector<uint32_t> r(n, 0);
  for (int i = 0; i < n; ++i) {
    uint64_t carry = 0;
    for (int j = 0; i + j < n; ++j) {
      const uint64_t cur = (uint64_t)a[i] * b[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)cur;
      carry = cur >> 32;
    }
  }
  std::memcpy(out, r.data(), (size_t)n * 4);
}

// out = -m^-1 mod 2^(32 n) by Newton's iteration x <- x (2 - m x), which
// doubles the number of correct low bits; x = m is correct to 3 bits.
void neg_inverse(const uint32_t *m, uint32_t *out, int n) {
  std::vector<uint32_t> x(m, m + n), t(n), u(n);
  for (int bits = 3; bits < 32 * n; bits *= 2) {
    mul_lo(m, x.data(), t.data(), n);          // t = m x
    uint32_t borrow = 0;                       // u = 2 - t
    for (int i = 0; i < n; ++i) {
      const uint64_t sub = (uint64_t)(i == 0 ? 2u : 0u) - t[i] - borrow;
      u[i] = (uint32_t)sub;
      borrow = (uint32_t)((sub >> 32) & 1u);
    }
    mul_lo(x.data(), u.data(), t.data(), n);   // x = x (2 - m x)
    x = t;
  }
  uint32_t borrow = 0;                         // out = 0 - x
  for (int i = 0; i < n; ++i) {
    const uint64_t sub = (uint64_t)0 - x[i] - borrow;
    out[i] = (uint32_t)sub;
    borrow = (uint32_t)((sub >> 32) & 1u);
  }
}

uint32_t byte_of(const uint32_t *w, int i) { return (w[i >> 2] >> (8 * (i & 3))) & 0xFFu; }

void neg_inverse_lo(const uint32_t *m, uint32_t *out, int n) { neg_inverse(m, out, n); }

bool build_tc_image(const uint32_t *m, uint8_t *out) {
  if ((m[0] & 1u) == 0) return false;
  uint32_t mp[kH];
  neg_inverse(m, mp, kH);
  std::memset(out, 0, kImgPrime);
  uint8_t *bm = out, *bp = out + kImgBm;
  const uint16_t bias = f16_of_int(2048);
  for (int n = 0; n < kN1; ++n)
    for (int k = 0; k < kKt; ++k) {
      uint16_t h;
      if (k < kDig) {
        const int i = n - k;
        h = (i >= 0 && i < kDig) ? f16_of_int(byte_of(mp, i)) : 0;
      } else {
        h = bias;
      }
      std::memcpy(bm + core_off(n, k, kN1), &h, 2);
    }
  for (int j = 0; j < kN2; ++j)
    for (int k = 0; k < kKt; ++k) {
      uint16_t h;
      if (k < kDig) {
        const int i = kN2First + j - k;
        h = (i >= 0 && i < kDig) ? f16_of_int(byte_of(m, i)) : 0;
      } else {
        h = bias;
      }
      std::memcpy(bp + core_off(j, k, kN2), &h, 2);
    }
  return true;
}

}  // namespace tcr

namespace tc4 {

// The operands of one prime m of H limbs (H = 48 or 64) for crt_tc4.cu, where
// a Montgomery product reduces modulo m in two rounds of r = 2^(16H), with
// D = 2H byte digits per round:
//   B1 (D x (D + 16)): row n, column k < D: byte n-k of m' = -m^-1 mod 2^(16H)
//       (it depends only on m mod 2^(16H)); columns D .. D+15: 2048 (bias)
//   B2 (2D x (D + 16)): row j = output position D-4+j of mu * m, column k < D:
//       byte D-4+j-k of m (0 outside 0 .. 4H-1); columns D .. D+15: 2048
bool build_tc4_image(const uint32_t *m, int H, uint8_t *out) {
  if (!supported(H) || (m[0] & 1u) == 0) return false;
  const int D = 2 * H, Kt = D + 16, N1 = D, N2 = 2 * D, first = D - 4;
  std::vector<uint32_t> mp(H / 2);
  tcr::neg_inverse_lo(m, mp.data(), H / 2);
  std::memset(out, 0, img_prime_bytes(H));
  uint8_t *b1 = out, *b2 = out + img_b1_bytes(H);
  const uint16_t bias = tcr::f16_of_int(2048);
  for (int n = 0; n < N1; ++n)
    for (int k = 0; k < Kt; ++k) {
      uint16_t h;
      if (k < D) {
        const int i = n - k;
        h = (i >= 0 && i < D) ? tcr::f16_of_int(tcr::byte_of(mp.data(), i)) : 0;
      } else {
        h = bias;
      }
      std::memcpy(b1 + tcr::core_off(n, k, N1), &h, 2);
    }
  for (int j = 0; j < N2; ++j)
    for (int k = 0; k < Kt; ++k) {
      uint16_t h;
      if (k < D) {
        const int i = first + j - k;
        h = (i >= 0 && i < 4 * H) ? tcr::f16_of_int(tcr::byte_of(m, i)) : 0;
      } else {
        h = bias;
      }
      std::memcpy(b2 + tcr::core_off(j, k, N2), &h, 2);
    }
  return true;
}

}  // namespace tc4
}  // namespace rsagpu
