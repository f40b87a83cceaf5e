// launch.h -- kernel lookup shared by the runtime and the instantiation units.
//
// Each instantiation unit (inst_*.cu) compiles the kernel templates for one
// limb count; the runtime finds them through these functions and launches
// them with cudaLaunchKernel.  A null return means "not instantiated".
#pragma once
#include <cstdint>

namespace rsagpu {

// Squaring variant of the private-exponent kernels: 0 = automatic (separated
// squaring where it fits in registers), 1 = CIOS squaring, 2 = separated.
// CRT decryption, half size H limbs, window W
const void *crt_kernel_fn(int H, int W, int variant = 0);
// plain private exponent mod n, L limbs, window W
const void *plain_kernel_fn(int L, int W, int variant = 0);
// public exponent (binary method), L limbs
const void *pub_kernel_fn(int L);
// public exponent, sliding windows of up to W bits (Fig. 7), L <= 64 limbs
const void *pub_slide_kernel_fn(int L, int W);
// single-limb keys (n < 2^32)
const void *toy_kernel_fn();
// T lanes per operation (T = 2, 4): CRT with half size H, public exponent with L limbs
const void *crt_kernel_t_fn(int H, int T, int W);
const void *pub_kernel_t_fn(int L, int T);
const void *plain_kernel_t_fn(int L, int T, int W);

// windows instantiated for the private-exponent kernels
constexpr int kMinWindow = 3;
constexpr int kMaxWindow = 6;

#define RSAGPU_DECLARE_UNIT(X)                      \
  const void *crt_kernel_fn_##X(int W, int variant);   \
  const void *plain_kernel_fn_##X(int W, int variant); \
  const void *pub_kernel_fn_##X();                     \
  const void *pub_slide_kernel_fn_##X(int W);

RSAGPU_DECLARE_UNIT(16)
RSAGPU_DECLARE_UNIT(32)
RSAGPU_DECLARE_UNIT(48)
RSAGPU_DECLARE_UNIT(64)

}  // namespace rsagpu
