// batch.cu -- ragged multi-key batches (rsa_modexp_batch).
#include "runtime_internal.h"

namespace rsagpu {

int Ctx::collect_device_errors(cudaStream_t s) {
  (void)s;
  return RSA_OK;
}

void Ctx::free_extra() {}

}  // namespace rsagpu

using namespace rsagpu;

extern "C" {

int rsa_modexp_batch(rsa_ctx *ctx, uint64_t count, const int32_t *key_ids, const uint8_t *exp_sel,
                     const uint64_t *limb_offsets, const uint32_t *msgs, uint32_t *out, int32_t *op_status,
                     void *stream) {
  (void)ctx; (void)count; (void)key_ids; (void)exp_sel; (void)limb_offsets; (void)msgs; (void)out;
  (void)op_status; (void)stream;
  return set_error(RSA_ERR_UNSUPPORTED, "ragged batches are not available yet");
}

int rsa_modexp_batch_host(rsa_ctx *ctx, uint64_t count, const int32_t *key_ids, const uint8_t *exp_sel,
                          const uint64_t *limb_offsets, uint64_t total_limbs, const uint32_t *msgs,
                          uint32_t *out, int32_t *op_status, void *stream) {
  (void)ctx; (void)count; (void)key_ids; (void)exp_sel; (void)limb_offsets; (void)total_limbs; (void)msgs;
  (void)out; (void)op_status; (void)stream;
  return set_error(RSA_ERR_UNSUPPORTED, "ragged batches are not available yet");
}

}  // extern "C"
