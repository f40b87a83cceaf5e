// sign.cu -- signing and verification on the modular-exponentiation kernels.
//
// The paper's primitives (Sec. 3.2-3.3) used the other way round: a signature
// is the private-exponent operation on a representative, verification the
// public-exponent operation followed by a comparison with the expected
// representative.  Hashing and padding stay with the caller.
#include <cuda_runtime.h>

#include <cstdint>

#include "keyrec.h"
#include "rsa_gb300.h"
#include "runtime_internal.h"

namespace rsagpu {

// op_status[i] stays RSA_OK only if the recovered row equals the expected one.
__global__ void verify_compare_kernel(uint64_t count, uint32_t L, const uint4 *recovered, const uint4 *expected,
                                      int32_t *op_status) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  if (op_status[i] != RSA_OK) return;   // RSA_ERR_RANGE from the exponentiation
  const uint32_t G = L / 4;
  uint32_t diff = 0;
  for (uint32_t g = 0; g < G; ++g) {
    const uint4 a = recovered[i * G + g], b = expected[i * G + g];
    diff |= (a.x ^ b.x) | (a.y ^ b.y) | (a.z ^ b.z) | (a.w ^ b.w);
  }
  if (diff) op_status[i] = RSA_ERR_VERIFY;
}

// Single-limb keys: one word per row.
__global__ void verify_compare1_kernel(uint64_t count, const uint32_t *recovered, const uint32_t *expected,
                                       int32_t *op_status) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  if (op_status[i] == RSA_OK && recovered[i] != expected[i]) op_status[i] = RSA_ERR_VERIFY;
}

}  // namespace rsagpu

using namespace rsagpu;

extern "C" {

int rsa_sign_key(rsa_ctx *ctx, int32_t key_id, uint64_t count, const uint32_t *reps, uint32_t *sigs,
                 int32_t *op_status, void *stream) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  int kind;
  {
    std::lock_guard<std::mutex> lock(c->mu);
    if (key_id < 0 || (size_t)key_id >= c->keys.size() || !c->keys[key_id].used)
      return set_error(RSA_ERR_KEY, "unknown key id " + std::to_string(key_id));
    const uint32_t flags = c->keys[key_id].flags;
    if (!(flags & KEY_HAS_D)) return set_error(RSA_ERR_KEY, "signing needs a key loaded with d");
    kind = (flags & KEY_HAS_CRT) ? RSA_EXP_PRIVATE_CRT : RSA_EXP_PRIVATE_PLAIN;
  }
  return rsa_modexp_key(ctx, key_id, kind, count, reps, sigs, op_status, stream);
}

int rsa_verify_key(rsa_ctx *ctx, int32_t key_id, uint64_t count, const uint32_t *sigs, const uint32_t *reps,
                   int32_t *op_status, void *stream) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  if (count > 0 && (!sigs || !reps || !op_status))
    return set_error(RSA_ERR_ARG, "null signature, representative or status pointer");
  if (count > 0x7fffffffull) return set_error(RSA_ERR_ARG, "count exceeds 2^31 - 1");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  const KeySlot *k = nullptr;
  int rc = c->check_key(key_id, RSA_EXP_PUBLIC, &k);
  if (rc) return rc;
  if (count == 0) return RSA_OK;
  if (k->L > 1 && ((reinterpret_cast<uintptr_t>(sigs) | reinterpret_cast<uintptr_t>(reps)) & 15u))
    return set_error(RSA_ERR_ARG, "signature and representative rows must be 16-byte aligned");
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Workspace &w = c->ws(s);
  const size_t bytes = (size_t)count * k->L * 4;
  rc = c->ensure(w.verify, bytes);
  if (rc) return rc;
  uint32_t *rec = static_cast<uint32_t *>(w.verify.ptr);
  c->stats.ops += count;
  rc = c->run_key(*k, RSA_EXP_PUBLIC, count, sigs, rec, op_status, s);
  if (rc) return rc;
  const int threads = 256;
  const unsigned blocks = (unsigned)((count + threads - 1) / threads);
  if (k->L == 1)
    verify_compare1_kernel<<<blocks, threads, 0, s>>>(count, rec, reps, op_status);
  else
    verify_compare_kernel<<<blocks, threads, 0, s>>>(count, k->L, reinterpret_cast<const uint4 *>(rec),
                                                     reinterpret_cast<const uint4 *>(reps), op_status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "launch verify_compare_kernel");
  c->stats.kernel_launches++;
  return RSA_OK;
}

}  // extern "C"
