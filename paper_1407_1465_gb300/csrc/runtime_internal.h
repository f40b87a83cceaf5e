// runtime_internal.h -- library-private state behind the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rsa_gb300.h"

namespace rsagpu {

// NVTX range over a host call (named in Nsight timelines; costs nothing
// measurable without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

int set_error(int code, const std::string &msg);
int cuda_error(cudaError_t e, const char *what);

struct DevBuf {
  void *ptr = nullptr;
  size_t bytes = 0;
};

// Scratch owned per stream, so work enqueued on different streams never shares it.
struct Workspace {
  DevBuf tables;                  // window tables of the private-exponent kernels
  DevBuf io_in, io_out, io_status;  // host-buffer entry points
  DevBuf aux0, aux1, aux2, aux3;  // ragged-batch planning buffers
  DevBuf halves;                  // tensor-core CRT path: per-prime results between its two kernels
  DevBuf tc_halves[2];            // ragged batches: the same for the 3072- and 4096-bit tensor-core groups
  DevBuf verify;                  // rsa_verify_key: recovered representatives
  DevBuf gcd0, gcd1;              // rsa_batch_gcd: validity + block products, partial products
  DevBuf gcd_tree, gcd_tw;        // rsa_batch_gcd, tree form: levels and transform scratch, twiddle tables
  const void *gcd_tw_ptr = nullptr; // gcd_tw's allocation when its tables were built
  uint64_t gcd_tw_n = 0;          // ... and the transform length they were built for
  void free_all();
};

struct KeySlot {
  bool used = false;
  uint32_t nbits = 0, L = 0, flags = 0;
  uint32_t *d_rec = nullptr;      // device key record (keyrec.h)
  size_t bytes = 0;
  std::vector<uint32_t> host_rec; // host copy of the record
  void *d_tc = nullptr;           // tensor-core operand images (2048-bit keys with p, q)
  size_t tc_bytes = 0;
  void *d_tcn = nullptr;          // n's two-round tensor-core operands (2048-bit keys: public exponent)
  size_t tcn_bytes = 0;
};

struct Tune {
  int window, warps_per_cta, ctas_per_sm, variant, tpo;
  int window_big, window_tc, tc_min_ops;   // ragged batches only (rsa_tuning)
};

struct Ctx {
  int device = 0;
  int sm_count = 0;
  size_t budget = 0, used = 0;
  std::mutex mu;
  std::vector<KeySlot> keys;
  uint64_t key_epoch = 0;         // bumped on every key load/unload
  std::map<cudaStream_t, Workspace> workspaces;
  std::map<std::pair<uint32_t, int>, Tune> tuning;
  rsa_stats stats{};
  int last_grid = 0, last_threads = 0;
  // ragged-batch state (batch.cu) and the request loop (server.cu)
  void *batch_state = nullptr;
  void *server = nullptr;

  ~Ctx();
  int reserve(size_t bytes);
  void release(size_t bytes);
  int ensure(DevBuf &b, size_t need);
  Workspace &ws(cudaStream_t s);
  Tune tune_for(uint32_t nbits, int kind) const;
  int check_key(int32_t key_id, int kind, const KeySlot **out);
  int launch_grid(const void *fn, int threads, size_t smem, uint64_t units_per_cta_slot, uint64_t units,
                  int ctas_per_sm_req, int *grid_out);
  int run_key(const KeySlot &k, int kind, uint64_t count, const uint32_t *msgs, uint32_t *out,
              int32_t *status, cudaStream_t s);
  int prepare_batch(cudaStream_t s, uint64_t max_count);
  // wide: 1 runs 2048/4096-bit CRT on 4/8 lanes per operation, 0 on 1/4,
  // -1 decides by the batch's own size (at most batch_wave_ops operations)
  int run_batch(uint64_t count, const int32_t *key_ids, const uint8_t *exp_sel, const uint64_t *offsets,
                const uint32_t *msgs, uint32_t *out, int32_t *status, cudaStream_t s, int wide = -1);
  // operations one wave of the multi-lane group holds (after prepare_batch on s)
  uint64_t batch_wave_ops(cudaStream_t s);
  // an order-independent 64-bit digest of the result rows of a ragged batch
  // (after run_batch on s with the same arguments); synchronises s
  int batch_digest(uint64_t count, const int32_t *key_ids, const uint64_t *offsets, const uint32_t *out,
                   cudaStream_t s, uint64_t *digest);
  int collect_device_errors(cudaStream_t s);
  // Free everything the library keeps for stream s (its ragged-batch graph and
  // key directory, its workspace buffers) before the caller destroys s.
  // Synchronises s first.
  void release_stream(cudaStream_t s);
  void free_extra();
};

}  // namespace rsagpu
