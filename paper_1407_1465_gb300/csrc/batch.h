// batch.h -- ragged multi-key batches: shared definitions of the planning
// kernels (batch.cu) and the persistent execution kernel (batch_exec.cu).
//
// A ragged batch mixes keys of every supported size and all exponent kinds.
// Operations are grouped on the device into buckets (key id x exponent kind),
// each bucket is cut into tiles (32 operations for a CRT warp pair, 64 for the
// other kinds: one warp per 32), tiles are laid out longest-first by class
// (the cost of one operation of that size and kind) and one persistent kernel
// pulls tiles from an atomic counter until none are left.
#pragma once
#include <cstdint>

#include "crt_tc.h"
#include "keyrec.h"

namespace rsagpu {

struct KeyDirEntry {          // one per key id; rec == null for a free slot
  const uint32_t *rec;
  uint32_t L, flags, nbits, e_bits;
  const void *tc;             // tensor-core operands (2048-bit keys with p, q), else null
};

struct TileDesc {
  int32_t bucket;             // key id * 3 + exponent kind
  int32_t op_start;           // first slot in the sorted operation list
  int32_t nops;               // live operations in the tile
  int32_t cls;                // work class (below)
};

// Work classes: what the execution kernel runs for a (key size, kind) pair.
enum : int32_t {
  CLS_TOY = 0,                                   // single-limb keys, any kind
  CLS_CRT16 = 1, CLS_CRT32 = 2, CLS_CRT48 = 3, CLS_CRT64 = 4,   // CRT, half size H
  CLS_PUB32 = 5, CLS_PUB64 = 6, CLS_PUB96 = 7, CLS_PUB128 = 8,  // public exponent, L limbs
                                                                // (96, 128: four lanes per operation)
  CLS_PLAIN32 = 9, CLS_PLAIN64 = 10,             // plain private exponent, L limbs
  CLS_CRT32W = 11,                               // CRT of 2048-bit keys, four lanes per operation
  CLS_CRT64W = 12,                               // CRT of 4096-bit keys, eight lanes per operation
                                                 // (the W classes: small batches, latency over throughput)
  CLS_PLAIN96 = 13, CLS_PLAIN128 = 14,           // plain private exponent of 3072/4096-bit moduli,
                                                 // four lanes per operation
  CLS_CRT64X = 15,                               // CRT of 4096-bit keys, sixteen lanes per operation
                                                 // (small batches, when asked for instead of eight)
  CLS_COUNT = 16
};

// Window widths of the CRT classes are chosen per batch (BatchDesc::win_small
// for 1024/2048-bit keys, win_big for 3072/4096-bit keys; 4 or 5, the ragged
// autotuner sweeps them); these are the defaults (3072/4096-bit CRT: 5; with 4
// the 256-key ragged mix ran at 717 K ops/s against 732 K).  Plain private
// exponents always use kBatchWindowPlain.
constexpr int kBatchWindowSmall = 4, kBatchWindowBig = 5, kBatchWindowMax = 5;
constexpr int kBatchWindowPlain = 4;
// the tensor-core groups: window 3 (tables stay in L2) or 4 at 2048 bits; a
// 2048/3072/4096-bit CRT bucket runs there, in tiles of 128 operations, once
// it holds at least kBatchTcMinOps operations (smaller ones on the CUDA cores)
constexpr int kBatchWindowTc = 3;
constexpr uint32_t kBatchTcMinOps = 128;

// wide (nonzero): run 2048-bit CRT with four lanes per operation (CLS_CRT32W)
// and 4096-bit CRT with eight (CLS_CRT64W; wide == 2: sixteen, CLS_CRT64X)
__host__ __device__ inline int32_t batch_class(uint32_t L, int kind, uint32_t wide = 0) {
  if (L == 1) return CLS_TOY;
  if (kind == 1)
    return L == 32 ? CLS_CRT16 : L == 64 ? (wide ? CLS_CRT32W : CLS_CRT32) : L == 96 ? CLS_CRT48
           : L == 128 ? (wide == 2 ? CLS_CRT64X : wide ? CLS_CRT64W : CLS_CRT64) : -1;
  if (kind == 0) return L == 32 ? CLS_PUB32 : L == 64 ? CLS_PUB64 : L == 96 ? CLS_PUB96 : L == 128 ? CLS_PUB128 : -1;
  if (kind == 2) return L == 32 ? CLS_PLAIN32 : L == 64 ? CLS_PLAIN64 : L == 96 ? CLS_PLAIN96 : L == 128 ? CLS_PLAIN128 : -1;
  return -1;
}

// Execution groups: one persistent kernel each, so every group gets the
// register allocation its own largest class needs.  Group order is the order
// of tile ranges (longest operations first).
//   BIG   CRT of 3072/4096-bit keys (and of 2048-bit keys in small batches),
//         four lanes per operation (eight for 4096-bit keys in small batches)
//   CRT   CRT of 1024/2048-bit keys, public/plain of 1024-bit keys, toy keys
//   L64   public/plain exponents of 2048-bit moduli (one lane, 232 registers)
//   WIDE  public and plain private exponents of 3072/4096-bit moduli, four
//         lanes per operation
enum : int32_t { GRP_BIG = 0, GRP_CRT = 1, GRP_L64 = 2, GRP_WIDE = 3, GRP_COUNT = 4 };
__host__ __device__ inline int32_t batch_group(int32_t cls) {
  if (cls == CLS_CRT48 || cls == CLS_CRT64 || cls == CLS_CRT32W || cls == CLS_CRT64W || cls == CLS_CRT64X)
    return GRP_BIG;
  if (cls == CLS_PUB96 || cls == CLS_PUB128 || cls == CLS_PLAIN96 || cls == CLS_PLAIN128) return GRP_WIDE;
  if (cls == CLS_PUB64 || cls == CLS_PLAIN64) return GRP_L64;
  return GRP_CRT;
}

// Window-table scratch per warp (uint4) of an execution group: 2^w entries of
// (limbs per lane)/4 uint4 for each of the 32 lanes, for the largest class the
// group runs at the batch's windows (win_small: 1024/2048-bit CRT, win_big:
// 3072/4096-bit CRT).  The kernels index tables by BatchDesc::table_u4.
__host__ __device__ constexpr size_t batch_table_need(int w, int limbs_per_lane) {
  return ((size_t)1 << w) * (size_t)(limbs_per_lane / 4) * 32;
}
__host__ __device__ constexpr size_t batch_max(size_t a, size_t b) { return a > b ? a : b; }
__host__ __device__ constexpr size_t batch_table_u4(int group, int win_small, int win_big) {
  return group == GRP_BIG   ? batch_max(batch_table_need(win_big, 16),     // CRT H=64, four lanes (H=48: 12)
                                        batch_table_need(win_small, 8))    // CRT H=32 on four lanes
         : group == GRP_CRT ? batch_max(batch_table_need(win_small, 32),   // CRT H=32 (H=16: 16 limbs)
                                        batch_table_need(kBatchWindowPlain, 32))   // plain L=32
         : group == GRP_L64 ? batch_table_need(kBatchWindowPlain, 64)      // plain L=64
                            : batch_table_need(kBatchWindowPlain, 32);     // plain L=128, four lanes
}

// operations per tile of a class: CRT 32 (warp pair on the same 32), wide CRT 8
// (4 lanes per operation, the pair on the same 8; 4 with 8 lanes, 2 with 16), wide public and plain 16 (4
// lanes per operation, 8 per warp), others 64 (32 per warp)
__host__ __device__ constexpr int32_t batch_tile_ops(int32_t cls) {
  if (cls == CLS_CRT64X) return 2;
  if (cls == CLS_CRT64W) return 4;
  if (cls == CLS_CRT48 || cls == CLS_CRT64 || cls == CLS_CRT32W) return 8;
  if (cls == CLS_PUB96 || cls == CLS_PUB128 || cls == CLS_PLAIN96 || cls == CLS_PLAIN128) return 16;
  return (cls == CLS_CRT16 || cls == CLS_CRT32) ? 32 : 64;
}

// the smallest tile of any class (CLS_CRT64X): the tile list holds up to
// count / kMinTileOps + (buckets) + 1 descriptors, enough for every class
constexpr uint32_t kMinTileOps = 2;
__host__ __device__ constexpr bool batch_tiles_fit() {
  for (int c = 0; c < CLS_COUNT; ++c)
    if ((uint32_t)batch_tile_ops(c) < kMinTileOps) return false;
  return true;
}
static_assert(batch_tiles_fit(), "a class has tiles smaller than kMinTileOps");

struct BatchDesc {
  uint32_t count, nkeys;
  const int32_t *key_ids;
  const uint8_t *exp_sel;
  const uint64_t *offsets;
  const uint32_t *msgs;
  uint32_t *out;
  int32_t *status;
  const KeyDirEntry *dir;
  // workspace
  int32_t *op_bucket;         // [count]
  int32_t *sorted;            // [count]
  uint32_t *bcount, *bfill, *boff;  // [nkeys * 3]
  TileDesc *tiles;            // [max_tiles]
  uint32_t *ctl;              // [0] unused, [1] tile count, [2] error bits,
                              // [4+g] first tile of group g, [8+g] end, [12+g] counter (g < 4)
  uint4 *tables;              // per resident warp of the group: table_u4 uint4
  uint32_t table_u4;          // batch_table_u4(group, win_small, win_big) of the node's group
  uint32_t max_tiles;
  int32_t class_rank[CLS_COUNT];  // position of each class in the longest-first order
  uint32_t wide_crt32;        // small batch: 2048/4096-bit CRT as CLS_CRT32W / CLS_CRT64W (2: CLS_CRT64X)
  int32_t win_small, win_big; // CRT windows of 1024/2048-bit and of 3072/4096-bit keys (4 or 5)
  // tensor-core groups: CRT buckets of at least tc_min_ops operations (0:
  // none) run there in ceil(count / 128) tiles, in chunks of up to
  // batch_tc_chunk_tiles tiles of one key; max_tc_chunks bounds each chunk list
  uint32_t tc_min_ops, max_tc_chunks;
  tcr::TcChunk *tc_chunks;    // 2048-bit CRT chunks (up to tcr::kTiles tiles each)
  tcr::TcChunk *tcx_chunks[2];  // 3072- and 4096-bit CRT chunks (up to tc4::kTiles tiles each)
};

// Tensor-core groups of ragged batches: 2048-, 3072- and 4096-bit CRT buckets,
// each with its chunk list and the control words chunk count / work counter.
enum : int32_t { TCG_2048 = 0, TCG_3072 = 1, TCG_4096 = 2, TCG_COUNT = 3 };
__host__ __device__ constexpr int32_t batch_tc_ctl_word(int32_t grp) { return tcr::kCtlTcChunks + 2 * grp; }
__host__ __device__ constexpr int32_t batch_tc_chunk_tiles(int32_t grp) {
  return grp == TCG_2048 ? tcr::kTiles : tc4::kTiles;
}
// the tensor-core group of a class (-1: none): the one-lane 2048-bit CRT class
// and the four-lane 3072/4096-bit ones (the throughput shapes)
__host__ __device__ inline int32_t batch_tc_group(int32_t cls) {
  return cls == CLS_CRT32 ? TCG_2048 : cls == CLS_CRT48 ? TCG_3072 : cls == CLS_CRT64 ? TCG_4096 : -1;
}
static_assert(tcr::kCtlTcChunks + 2 * TCG_COUNT <= 30, "control words");

// operations a bucket of c sends to its tensor-core group: all of them (in
// ceil(c / 128) tiles, the last one possibly partial) once c reaches
// tc_min_ops, else none
__host__ __device__ inline uint32_t batch_tc_ops(const BatchDesc &d, int32_t cls, const KeyDirEntry &e, uint32_t c) {
  if (batch_tc_group(cls) < 0 || d.tc_min_ops == 0 || e.tc == nullptr || c < d.tc_min_ops) return 0u;
  return c;
}

const void *batch_exec_fn(int group);
size_t batch_exec_smem_bytes(int group);

}  // namespace rsagpu
