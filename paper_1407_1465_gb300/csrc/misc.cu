// misc.cu -- single-limb kernel (moduli below 2^32), the integer-multiply
// throughput probe, and the kernel lookup across instantiation units.
#include <cstdint>

#include "keyrec.h"
#include "kernels.cuh"
#include "launch.h"
#include "mont.cuh"

namespace rsagpu {

// ------------------------------------------------------------------ single-limb keys
__global__ void toy_kernel(ToyArgs a) {
  const KeyLayout lay(1);
  const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(a.keyrec);
  const uint32_t n = a.keyrec[lay.n];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.count; i += gridDim.x * blockDim.x) {
    const uint32_t x = a.msgs[i];
    const bool ok = x < n;
    const uint32_t r = toy_op(a.keyrec, hd, a.kind, x);
    a.out[i] = ok ? r : 0u;
    if (a.status) a.status[i] = ok ? 0 : -3;
  }
}

const void *toy_kernel_fn() { return reinterpret_cast<const void *>(&toy_kernel); }

// ------------------------------------------------------------------ lookup
const void *crt_kernel_fn(int H, int W, int variant) {
  switch (H) {
    case 16: return crt_kernel_fn_16(W, variant);
    case 32: return crt_kernel_fn_32(W, variant);
    case 48: return crt_kernel_fn_48(W, variant);
    case 64: return crt_kernel_fn_64(W, variant);
    default: return nullptr;
  }
}
const void *plain_kernel_fn(int L, int W, int variant) {
  switch (L) {
    case 32: return plain_kernel_fn_16(W, variant);
    case 64: return plain_kernel_fn_32(W, variant);
    default: return nullptr;
  }
}
const void *pub_slide_kernel_fn(int L, int W) {
  switch (L) {
    case 32: return pub_slide_kernel_fn_16(W);
    case 64: return pub_slide_kernel_fn_32(W);
    default: return nullptr;
  }
}

const void *pub_kernel_fn(int L) {
  switch (L) {
    case 32: return pub_kernel_fn_16();
    case 64: return pub_kernel_fn_32();
    case 96: return pub_kernel_fn_48();
    case 128: return pub_kernel_fn_64();
    default: return nullptr;
  }
}

// ------------------------------------------------------------------ IMAD probe
// Independent multiply-add chains: 8 accumulators, each step one mad.lo and
// one mad.hi per accumulator (16 lane-operations per thread per step).
__global__ void imad_probe_kernel(uint32_t *sink, uint32_t iters, uint32_t seed) {
  uint32_t a[8], h[8];
  const uint32_t b = seed * 2654435761u + threadIdx.x;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a[k] = seed + 17u * k + blockIdx.x;
    h[k] = seed ^ (31u * k);
  }
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(b), "r"(h[k]));
      asm volatile("mad.hi.u32 %0, %1, %2, %0;" : "+r"(h[k]) : "r"(a[k]), "r"(b));
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) x ^= a[k] ^ h[k];
  if (x == 0x9e3779b9u) sink[blockIdx.x * blockDim.x + threadIdx.x] = x;
}

// Carry chains as the kernels' product scans run them: per step one row,
// t[0..31] += b * a[0..31] with the even/odd mad.lo.cc / madc.hi.cc chains of
// mul_emit (32 word products), the lowest limb leaving.  The next row's
// multiplier is formed from that limb, the row's first result, so consecutive
// rows overlap as they do when the multipliers come from shared memory (a
// multiplier taken from the row's last carry would serialise the rows and
// understate the rate the kernels can reach).
__global__ void chain_probe_kernel(uint32_t *sink, uint32_t iters, uint32_t seed) {
  uint32_t a[32], t[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    a[j] = seed * (j + 1) + threadIdx.x;
    t[j] = 0u;
  }
  uint32_t b = seed | 1u, x = 0u;
  for (uint32_t it = 0; it < iters; ++it) {
    const uint32_t out = mul_emit<32>(t, a, b);
    x ^= out;
    b = out + it;   // data dependent, so nothing is hoisted
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) x ^= t[j];
  if (x == 0x9e3779b9u) sink[blockIdx.x * blockDim.x + threadIdx.x] = x;
}

const void *imad_probe_fn() { return reinterpret_cast<const void *>(&imad_probe_kernel); }
const void *chain_probe_fn() { return reinterpret_cast<const void *>(&chain_probe_kernel); }

}  // namespace rsagpu
