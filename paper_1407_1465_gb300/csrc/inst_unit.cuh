// inst_unit.cuh -- body of one instantiation unit.  Before including, define
// RSAGPU_UNIT (the CRT half size H of this unit, in limbs).  The unit holds
//   crt_kernel<H, W>      for W in the instantiated window range
//   plain_kernel<2H, W>   and pub_kernel<2H>   when 2H <= 64 (register-resident A)
#include "kernels.cuh"
#include "launch.h"

#ifndef RSAGPU_UNIT
#error "define RSAGPU_UNIT"
#endif

#define RSAGPU_CAT2(a, b) a##b
#define RSAGPU_CAT(a, b) RSAGPU_CAT2(a, b)

namespace rsagpu {

namespace {
constexpr int kH = RSAGPU_UNIT;
constexpr int kL = 2 * kH;
// outer CIOS block: limbs of B per runtime iteration (fully unrolled inside).
// Measured on GB300: 8 is best up to 32-limb halves, 4 for 48/64 limbs (smaller
// loop body, fewer registers).
#ifdef RSAGPU_CIOS_BLOCK
constexpr int kU = RSAGPU_CIOS_BLOCK;
#else
constexpr int kU = (RSAGPU_UNIT <= 32) ? 8 : 4;
#endif

// separated squaring where its 2L-limb product fits in registers
constexpr bool kSqrOk = (kH <= 32);
constexpr bool kSqrOkFull = (kL <= 32);

// variant 0 (automatic) is the CIOS squaring: the separated squaring issues fewer
// products but its unrolled body overflows the instruction cache (ncu: stalls on
// "no instruction" dominate), so it is slower on GB300.
template <int W>
const void *crt_fn(int variant) {
  if (variant == 2) {
    if constexpr (kSqrOk) return reinterpret_cast<const void *>(&crt_kernel<kH, W, kU, true>);
    else return nullptr;
  }
  return reinterpret_cast<const void *>(&crt_kernel<kH, W, kU, false>);
}

template <int W>
const void *plain_fn(int variant) {
  if constexpr (kL <= 64) {
    if (variant == 2) {
      if constexpr (kSqrOkFull) return reinterpret_cast<const void *>(&plain_kernel<kL, W, kU, true>);
      else return nullptr;
    }
    return reinterpret_cast<const void *>(&plain_kernel<kL, W, kU, false>);
  }
  return nullptr;
}
}  // namespace

const void *RSAGPU_CAT(crt_kernel_fn_, RSAGPU_UNIT)(int W, int variant) {
  switch (W) {
    case 3: return crt_fn<3>(variant);
    case 4: return crt_fn<4>(variant);
    case 5: return crt_fn<5>(variant);
    case 6: return crt_fn<6>(variant);
    default: return nullptr;
  }
}

const void *RSAGPU_CAT(plain_kernel_fn_, RSAGPU_UNIT)(int W, int variant) {
  switch (W) {
    case 4: return plain_fn<4>(variant);
    case 5: return plain_fn<5>(variant);
    default: return nullptr;
  }
}

const void *RSAGPU_CAT(pub_slide_kernel_fn_, RSAGPU_UNIT)(int W) {
  if constexpr (kL <= 64) {
    switch (W) {
      case 4: return reinterpret_cast<const void *>(&pub_slide_kernel<kL, kU, 4>);
      case 5: return reinterpret_cast<const void *>(&pub_slide_kernel<kL, kU, 5>);
      case 6: return reinterpret_cast<const void *>(&pub_slide_kernel<kL, kU, 6>);
      default: return nullptr;
    }
  }
  return nullptr;
}

const void *RSAGPU_CAT(pub_kernel_fn_, RSAGPU_UNIT)() {
  if constexpr (kL <= 64) return reinterpret_cast<const void *>(&pub_kernel<kL, kU>);
  else return reinterpret_cast<const void *>(&pub_wide_kernel<kL, 4>);
}

}  // namespace rsagpu
