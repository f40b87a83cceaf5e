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

#include "keyrec.h"

namespace rsagpu {

struct KeyDirEntry {          // one per key id; rec == null for a free slot
  const uint32_t *rec;
  uint32_t L, flags, nbits, e_bits;
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
  CLS_COUNT = 15
};

// Window widths the execution kernel is compiled with, per class (3072/4096-bit
// CRT: 5; with 4 the 256-key ragged mix ran at 717 K ops/s against 732 K).
constexpr int kBatchWindowCrt16 = 4, kBatchWindowCrt32 = 4, kBatchWindowCrt48 = 5, kBatchWindowCrt64 = 5;
constexpr int kBatchWindowPlain = 4;

// wide: run 2048-bit CRT with four lanes per operation (CLS_CRT32W) and
// 4096-bit CRT with eight (CLS_CRT64W)
__host__ __device__ inline int32_t batch_class(uint32_t L, int kind, bool wide = false) {
  if (L == 1) return CLS_TOY;
  if (kind == 1)
    return L == 32 ? CLS_CRT16 : L == 64 ? (wide ? CLS_CRT32W : CLS_CRT32) : L == 96 ? CLS_CRT48
           : L == 128 ? (wide ? CLS_CRT64W : CLS_CRT64) : -1;
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
  if (cls == CLS_CRT48 || cls == CLS_CRT64 || cls == CLS_CRT32W || cls == CLS_CRT64W) return GRP_BIG;
  if (cls == CLS_PUB96 || cls == CLS_PUB128 || cls == CLS_PLAIN96 || cls == CLS_PLAIN128) return GRP_WIDE;
  if (cls == CLS_PUB64 || cls == CLS_PLAIN64) return GRP_L64;
  return GRP_CRT;
}

// Window-table scratch per warp (uint4) of an execution group: 2^w entries of
// (limbs per lane)/4 uint4 for each of the 32 lanes, for the largest class the
// group runs (each call site checks its own need against this at compile time).
__host__ __device__ constexpr size_t batch_table_need(int w, int limbs_per_lane) {
  return ((size_t)1 << w) * (size_t)(limbs_per_lane / 4) * 32;
}
__host__ __device__ constexpr size_t batch_table_u4(int group) {
  return group == GRP_BIG   ? batch_table_need(5, 16)   // CRT H=64, w=5, four lanes: 16 limbs per lane
         : group == GRP_CRT ? batch_table_need(4, 32)   // CRT H=32, w=4; plain L=32, w=4
         : group == GRP_L64 ? batch_table_need(4, 64)   // plain L=64, w=4
                            : batch_table_need(kBatchWindowPlain, 32);   // plain L=128, w=4, four lanes
}

// operations per tile of a class: CRT 32 (warp pair on the same 32), wide CRT 8
// (4 lanes per operation, the pair on the same 8; 4 with 8 lanes), wide public and plain 16 (4
// lanes per operation, 8 per warp), others 64 (32 per warp)
__host__ __device__ inline int32_t batch_tile_ops(int32_t cls) {
  if (cls == CLS_CRT64W) return 4;
  if (cls == CLS_CRT48 || cls == CLS_CRT64 || cls == CLS_CRT32W) return 8;
  if (cls == CLS_PUB96 || cls == CLS_PUB128 || cls == CLS_PLAIN96 || cls == CLS_PLAIN128) return 16;
  return (cls == CLS_CRT16 || cls == CLS_CRT32) ? 32 : 64;
}

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
  uint4 *tables;              // per resident warp of the group: batch_table_u4(group)
  uint32_t max_tiles;
  int32_t class_rank[CLS_COUNT];  // position of each class in the longest-first order
  uint32_t wide_crt32;        // small batch: 2048/4096-bit CRT as CLS_CRT32W / CLS_CRT64W
};

const void *batch_exec_fn(int group);
size_t batch_exec_smem_bytes(int group);

}  // namespace rsagpu
