// keyprep.h -- per-key precomputation on the host (runs once per key load).
//
// Builds the device key record (keyrec.h) from (n, e, d, p, q): the Montgomery
// constants n' = -n^-1 mod 2^32, R mod n, R^2 mod n (and for p, q: R^2, R^3
// mod p|q, R mod p|q), the CRT exponents dp = d mod (p-1), dq = d mod (q-1)
// and qinv = q^-1 mod p.  The arithmetic is deliberately simple and bit-serial
// (powers of two by repeated doubling with conditional subtraction, remainders
// by shift-and-subtract, the inverse by the binary extended Euclidean method);
// it runs once per key and is independent of any other implementation.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace rsagpu {

struct KeyInput {
  uint32_t nbits = 0;
  std::vector<uint32_t> n, e, d, p, q;  // d, p, q may be empty
};

// Returns "" on success or a message; fills `rec` (words of the record) and
// `flags` (KEY_HAS_D | KEY_HAS_CRT).  Error class: 'A' argument, 'K' key,
// 'U' unsupported, reported through *err_class.
std::string build_key_record(const KeyInput &in, std::vector<uint32_t> &rec, uint32_t &flags,
                             char *err_class);

// Exposed for tests of the host arithmetic.
uint32_t neg_inv32(uint32_t n0);
void pow2_mod(std::vector<uint32_t> &out, const std::vector<uint32_t> &m, uint64_t k);
void mod_bitserial(std::vector<uint32_t> &out, const std::vector<uint32_t> &a,
                   const std::vector<uint32_t> &m);
bool inv_mod(std::vector<uint32_t> &out, const std::vector<uint32_t> &a,
             const std::vector<uint32_t> &m);

}  // namespace rsagpu
