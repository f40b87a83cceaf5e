// inst_t.cu -- instantiations of the T-lanes-per-operation kernels (kernels_t.cuh).
#include "kernels_t.cuh"
#include "launch.h"

namespace rsagpu {

const void *crt_kernel_t_fn(int H, int T, int W) {
  if (W < 4 || W > 6) return nullptr;
#define RSAGPU_CRT_T(h, t)                                                                          \
  if (H == h && T == t)                                                                             \
    return W == 4   ? reinterpret_cast<const void *>(&crt_kernel_t<h, t, 4, (h / t >= 32 ? 4 : 8)>) \
           : W == 5 ? reinterpret_cast<const void *>(&crt_kernel_t<h, t, 5, (h / t >= 32 ? 4 : 8)>) \
                    : reinterpret_cast<const void *>(&crt_kernel_t<h, t, 6, (h / t >= 32 ? 4 : 8)>);
  RSAGPU_CRT_T(32, 2)
  RSAGPU_CRT_T(32, 4)
  RSAGPU_CRT_T(48, 2)
  RSAGPU_CRT_T(48, 4)
  RSAGPU_CRT_T(64, 2)
  RSAGPU_CRT_T(64, 4)
#undef RSAGPU_CRT_T
  return nullptr;
}

const void *pub_kernel_t_fn(int L, int T) {
#define RSAGPU_PUB_T(l, t) \
  if (L == l && T == t) return reinterpret_cast<const void *>(&pub_kernel_t<l, t, (l / t >= 32 ? 4 : 8)>);
  RSAGPU_PUB_T(64, 2)
  RSAGPU_PUB_T(64, 4)
  RSAGPU_PUB_T(96, 2)
  RSAGPU_PUB_T(96, 4)
  RSAGPU_PUB_T(128, 2)
  RSAGPU_PUB_T(128, 4)
#undef RSAGPU_PUB_T
  return nullptr;
}

const void *plain_kernel_t_fn(int L, int T, int W) {
  if (W != 4 && W != 5) return nullptr;
#define RSAGPU_PLAIN_T(l, t)                                                                     \
  if (L == l && T == t)                                                                          \
    return W == 4 ? reinterpret_cast<const void *>(&plain_kernel_t<l, t, 4, (l / t >= 32 ? 4 : 8)>) \
                  : reinterpret_cast<const void *>(&plain_kernel_t<l, t, 5, (l / t >= 32 ? 4 : 8)>);
  RSAGPU_PLAIN_T(96, 4)
  RSAGPU_PLAIN_T(128, 4)
#undef RSAGPU_PLAIN_T
  return nullptr;
}

}  // namespace rsagpu
