// noalloc.cu -- CRT decryption entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA graph
// capture, a plug-in living in a host process whose device memory is managed
// by someone else's pool allocator, or a service that forbids allocation after
// start-up so that it can never fail on out-of-memory mid-request.  For them,
// rsa_crt_decrypt_noalloc() runs the same CRT kernel as rsa_modexp_key()
// without a context and without allocating: its only scratch (the per-warp
// window tables of the fixed-window exponentiation) is the file-scope array
// below, which the loader reserves on every GPU that loads this library and
// keeps until the process exits.
//
// Limits and sharing rules:
//   - the array holds kNoAllocScratchBytes (32 MiB); the grid is sized so the
//     tables fit (window width 4: 16 entries per warp), which caps the call at
//     kNoAllocScratchBytes / (2 * 16 * H * 128) resident warp pairs;
//   - every call uses the same array and it keeps the previous call's
//     contents; the kernel writes every table entry before reading it, so no
//     clearing is needed;
//   - calls whose work overlaps on the GPU (different streams, or different
//     host threads without ordering) race on the array and give wrong results.
//     Order them on one stream.
//   - the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current and caches it; make that
//     first call before any stream capture begins.
//   - the cached address belongs to the device's primary context (the one the
//     CUDA runtime uses); callers that run their own driver-API contexts on the
//     same device are not supported, because the array has a separate instance
//     in each context.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>

#include "kernels.cuh"
#include "launch.h"
#include "rsa_gb300.h"
#include "runtime_internal.h"

namespace rsagpu {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
constexpr int kNoAllocWindow = 4;
constexpr int kMaxDevices = 64;

__device__ __align__(256) uint4 g_noalloc_scratch[kNoAllocScratchBytes / sizeof(uint4)];

struct DeviceSetup {
  bool ready = false;
  uint4 *scratch = nullptr;
  int sm_count = 0;
};
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

int setup_device(int dev, DeviceSetup **out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup &s = g_setup[dev];
  if (!s.ready) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-alloc scratch)");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
    s.scratch = static_cast<uint4 *>(ptr);
    s.sm_count = sms;
    s.ready = true;
  }
  *out = &s;
  return RSA_OK;
}

}  // namespace
}  // namespace rsagpu

using namespace rsagpu;

extern "C" int rsa_crt_decrypt_noalloc(const uint32_t *key_record, uint32_t nbits, uint64_t count,
                                       const uint32_t *msgs, uint32_t *out, int32_t *op_status, void *stream) {
  if (!(nbits == 1024 || nbits == 2048 || nbits == 3072 || nbits == 4096))
    return set_error(RSA_ERR_UNSUPPORTED, "no-alloc CRT entry point takes 1024-, 2048-, 3072- or 4096-bit keys");
  if (count > 0x7fffffffull) return set_error(RSA_ERR_ARG, "count exceeds 2^31 - 1");
  if (count == 0) return RSA_OK;
  if (!key_record || !msgs || !out) return set_error(RSA_ERR_ARG, "null pointer");
  if ((reinterpret_cast<uintptr_t>(key_record) | reinterpret_cast<uintptr_t>(msgs) |
       reinterpret_cast<uintptr_t>(out)) & 15u)
    return set_error(RSA_ERR_ARG, "key record, message and output rows must be 16-byte aligned");
  const int H = (int)nbits / 64;
  const size_t pair_bytes = (size_t)2 * (1u << kNoAllocWindow) * H * 128;
  if (pair_bytes > kNoAllocScratchBytes)
    return set_error(RSA_ERR_UNSUPPORTED, "key size needs more scratch than the no-alloc array holds");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(RSA_ERR_ARG, "device index out of range");
  DeviceSetup *s = nullptr;
  int rc = setup_device(dev, &s);
  if (rc) return rc;
  const void *fn = crt_kernel_fn(H, kNoAllocWindow);
  if (!fn) return set_error(RSA_ERR_UNSUPPORTED, "no CRT kernel for this key size");
  const int threads = 64;  // one warp pair per CTA
  const size_t smem = ((KeyLayout(2 * H).total + 3) / 4 * 4) * 4 + (size_t)4 * (H / 4) * 32 * 16;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  const uint64_t ntiles = (count + 31) / 32;
  const uint64_t cap_pairs = kNoAllocScratchBytes / pair_bytes;
  const uint64_t grid = std::max<uint64_t>(
      1, std::min<uint64_t>({ntiles, cap_pairs, (uint64_t)s->sm_count * (uint64_t)std::max(per_sm, 1)}));
  CrtArgs a{key_record, msgs, out, op_status, (uint32_t)count, s->scratch};
  void *args[] = {&a};
  e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(threads), args, smem, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "launch crt_kernel (no-alloc)");
  return RSA_OK;
}
