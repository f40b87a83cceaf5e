// batch_exec.cu -- the persistent execution kernel of ragged batches.
//
// One CTA is a warp pair (64 threads).  It repeatedly takes the next tile from
// the planned list (an atomic counter; tiles are ordered longest-first, so the
// short ones fill the tail), copies the tile's key record into shared memory
// and runs the tile function of its class:
//   CRT       both warps, q half and p half (crt_tile)
//   public    L <= 64: one warp per 32 operations (pub_tile);
//             L = 96, 128: four lanes per operation, 8 operations per warp (pub_tile_t)
//   plain     one warp per 32 operations (plain_tile)
//   toy       one thread per operation (toy_op)
#include "batch.h"
#include "kernels.cuh"
#include "kernels_t.cuh"

namespace rsagpu {
namespace {

constexpr int kU = 8;
constexpr int kKeyWordsMax = (KeyLayout(128).total + 3) / 4 * 4;
// work area after the key record: the largest of
//   CRT H=64: exchange + 2 stages = 3 * 64 * 128 B; public L=64: 2 warps x 2 stages = 4 * 64 * 128 B;
//   public wide L=128: 1 warp x 2 stages = 2 * 128 * 128 B
constexpr size_t kWorkBytes = (size_t)4 * 64 * 128;
// work area each group's tile functions use (the largest of its classes):
//   BIG  four-lane CRT H=64: exchange + 2 stages of (H/4) x 8 uint4
//   CRT  public L=32: 2 warps x 2 stages of (L/4) x 32 uint4 (CRT H=32 needs 3 such stages)
//   L64  public L=64: 2 warps x 2 stages of (L/4) x 32 uint4
//   WIDE public L=128, four lanes: 2 warps x 2 stages of (L/4) x 8 uint4
__host__ __device__ constexpr size_t work_bytes(int g) {
  return g == GRP_BIG   ? (size_t)3 * (64 / 4) * 8 * 16
         : g == GRP_CRT ? (size_t)4 * (32 / 4) * 32 * 16
         : g == GRP_L64 ? (size_t)4 * (64 / 4) * 32 * 16
                        : (size_t)4 * (128 / 4) * 8 * 16;
}
static_assert(work_bytes(GRP_BIG) <= kWorkBytes && work_bytes(GRP_CRT) <= kWorkBytes &&
                  work_bytes(GRP_L64) <= kWorkBytes && work_bytes(GRP_WIDE) <= kWorkBytes,
              "work areas");
// uint4 count of the stages a tile function indexes: n_stages * kStage
__host__ __device__ constexpr size_t stage_u4(int n_stages, int limbs, int ops_per_warp) {
  return (size_t)n_stages * (limbs / 4) * ops_per_warp;
}

template <int H, int W>
__device__ __forceinline__ void run_crt(const uint32_t *ks, uint4 *work, uint4 *table_warp, int warp, int lane,
                                        const TileIO &io) {
  constexpr int kStage = (H / 4) * 32;
  uint4 *xb = work + lane;
  uint4 *stage_lane = work + kStage + warp * kStage + lane;
  crt_tile<H, W, kU, false>(ks, warp == 1, lane, stage_lane, xb, table_warp + lane, 1, io);
}

// CRT of 3072/4096-bit keys: four lanes per operation, the pair on the same 8 operations
template <int H, int W>
__device__ __forceinline__ void run_crt4(const uint32_t *ks, uint4 *work, uint4 *table_warp, int warp, int lane,
                                         const TileIO &io) {
  constexpr int kStage = (H / 4) * 8;
  const Group<4> g(lane);
  uint4 *xb = work + g.opi;
  uint4 *stage_op = work + kStage + warp * kStage + g.opi;
  crt_tile_t<H, 4, W, 8>(ks, warp == 1, g, stage_op, xb, table_warp + lane, 1, io);
}

// CRT of 4096-bit keys in small batches: eight lanes per operation, the pair on the same 4
template <int H, int W>
__device__ __forceinline__ void run_crt8(const uint32_t *ks, uint4 *work, uint4 *table_warp, int warp, int lane,
                                         const TileIO &io) {
  constexpr int kStage = (H / 4) * 4;
  const Group<8> g(lane);
  uint4 *xb = work + g.opi;
  uint4 *stage_op = work + kStage + warp * kStage + g.opi;
  crt_tile_t<H, 8, W, 8>(ks, warp == 1, g, stage_op, xb, table_warp + lane, 1, io);
}

// CRT of 4096-bit keys in small batches: sixteen lanes per operation, the pair on the same 2
template <int H, int W>
__device__ __forceinline__ void run_crt16(const uint32_t *ks, uint4 *work, uint4 *table_warp, int warp, int lane,
                                          const TileIO &io) {
  constexpr int kStage = (H / 4) * 2;
  const Group<16> g(lane);
  uint4 *xb = work + g.opi;
  uint4 *stage_op = work + kStage + warp * kStage + g.opi;
  crt_tile_t<H, 16, W, 8>(ks, warp == 1, g, stage_op, xb, table_warp + lane, 1, io);
}

template <int L>
__device__ __forceinline__ void run_pub(const uint32_t *ks, uint4 *work, int warp, int lane, const TileIO &io) {
  constexpr int kStage = (L / 4) * 32;
  uint4 *sq = work + warp * 2 * kStage + lane;
  pub_tile<L, kU>(ks, lane, sq, sq + kStage, io);
}

// wide public exponents: 4 lanes per operation, 8 operations per warp
template <int L>
__device__ __forceinline__ void run_pub_wide(const uint32_t *ks, uint4 *work, int warp, int lane, const TileIO &io) {
  constexpr int kStage = (L / 4) * 8;
  const Group<4> g(lane);
  uint4 *sq = work + warp * 2 * kStage;
  pub_tile_t<L, 4, 8>(ks, g, sq + g.opi, sq + kStage + g.opi, io);
}

// wide plain private exponents: 4 lanes per operation, 8 operations per warp
template <int L>
__device__ __forceinline__ void run_plain_wide(const uint32_t *ks, uint4 *work, uint4 *table_warp, int warp, int lane,
                                               const TileIO &io) {
  constexpr int kStage = (L / 4) * 8;
  const Group<4> g(lane);
  plain_tile_t<L, 4, kBatchWindowPlain, 4>(ks, g, work + warp * kStage + g.opi, table_warp + lane, io);
}

template <int L>
__device__ __forceinline__ void run_plain(const uint32_t *ks, uint4 *work, uint4 *table_warp, int warp, int lane,
                                          const TileIO &io) {
  constexpr int kStage = (L / 4) * 32;
  plain_tile<L, kBatchWindowPlain, kU, false>(ks, lane, work + warp * kStage + lane, table_warp + lane, io);
}

// The multi-lane CRT group needs about 12 KB of shared memory per CTA, so
// registers decide its occupancy: capped at 128 a thread (20 bytes of
// spills), 8 CTAs per SM instead of 5.  The same cap on the one-lane group
// spills in its 32-limb CRT and was not faster (728 K against 732 K ops/s).
template <int G>
__global__ void __launch_bounds__(64, G == GRP_BIG ? 8 : 1) batch_exec_kernel(BatchDesc d) {
  extern __shared__ uint4 smem4[];
  __shared__ int32_t s_tile;
  uint32_t *ks = reinterpret_cast<uint32_t *>(smem4);
  uint4 *work = smem4 + kKeyWordsMax / 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4 *table_warp = d.tables + ((size_t)blockIdx.x * 2 + warp) * d.table_u4;
  const uint32_t first = d.ctl[4 + G], end = d.ctl[8 + G];
#pragma unroll 1
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int32_t)(first + atomicAdd(&d.ctl[12 + G], 1u));
    __syncthreads();
    const uint32_t t = (uint32_t)s_tile;
    if (t >= end) break;
    const TileDesc td = d.tiles[t];
    const int32_t kid = td.bucket / 3, kind = td.bucket % 3;
    const KeyDirEntry e = d.dir[kid];
    const uint32_t words = (KeyLayout(e.L).total + 3) / 4 * 4;
    const uint4 *src = reinterpret_cast<const uint4 *>(e.rec);
    for (uint32_t i = threadIdx.x; i < words / 4; i += blockDim.x)
      smem4[i] = (i * 4 < KeyLayout(e.L).total) ? src[i] : make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    // per-warp slice of a 64-operation tile
    const int32_t wn = min(32, max(0, td.nops - 32 * warp));
    const TileIO io_pair{d.msgs, d.out, d.status, d.sorted, d.offsets, (uint32_t)td.op_start, (uint32_t)td.nops};
    const TileIO io_warp{d.msgs, d.out, d.status, d.sorted, d.offsets, (uint32_t)(td.op_start + 32 * warp),
                         (uint32_t)wn};
    if constexpr (G == GRP_BIG) {
      static_assert(stage_u4(3, 48, 8) * 16 <= work_bytes(GRP_BIG) && stage_u4(3, 64, 8) * 16 <= work_bytes(GRP_BIG) &&
                        stage_u4(3, 32, 8) * 16 <= work_bytes(GRP_BIG) && stage_u4(3, 64, 4) * 16 <= work_bytes(GRP_BIG) &&
                        stage_u4(3, 64, 2) * 16 <= work_bytes(GRP_BIG),
                    "work area of a four/eight/sixteen-lane CRT class");
      // tables: win_big entries of 16 (H=64) or 12 (H=48) limbs per lane, win_small
      // of 8 (H=32 on four lanes), win_big of 8 (H=64 on eight lanes)
      static_assert(batch_table_need(5, 48 / 4) <= batch_table_u4(GRP_BIG, 4, 5) &&
                        batch_table_need(4, 64 / 4) <= batch_table_u4(GRP_BIG, 4, 4) &&
                        batch_table_need(5, 32 / 4) <= batch_table_u4(GRP_BIG, 5, 4) &&
                        batch_table_need(5, 64 / 8) <= batch_table_u4(GRP_BIG, 4, 5),
                    "window table of a four/eight-lane CRT class");
      const bool w5big = d.win_big == 5, w5small = d.win_small == 5;
      if (td.cls == CLS_CRT48) {
        if (w5big) run_crt4<48, 5>(ks, work, table_warp, warp, lane, io_pair);
        else run_crt4<48, 4>(ks, work, table_warp, warp, lane, io_pair);
      } else if (td.cls == CLS_CRT64) {
        if (w5big) run_crt4<64, 5>(ks, work, table_warp, warp, lane, io_pair);
        else run_crt4<64, 4>(ks, work, table_warp, warp, lane, io_pair);
      } else if (td.cls == CLS_CRT32W) {
        if (w5small) run_crt4<32, 5>(ks, work, table_warp, warp, lane, io_pair);
        else run_crt4<32, 4>(ks, work, table_warp, warp, lane, io_pair);
      } else if (td.cls == CLS_CRT64W) {
        if (w5big) run_crt8<64, 5>(ks, work, table_warp, warp, lane, io_pair);
        else run_crt8<64, 4>(ks, work, table_warp, warp, lane, io_pair);
      } else if (td.cls == CLS_CRT64X) {
        if (w5big) run_crt16<64, 5>(ks, work, table_warp, warp, lane, io_pair);
        else run_crt16<64, 4>(ks, work, table_warp, warp, lane, io_pair);
      }
    } else if constexpr (G == GRP_L64) {
      static_assert(batch_table_need(kBatchWindowPlain, 64) <= batch_table_u4(GRP_L64, 4, 4), "plain L=64 table");
      static_assert(stage_u4(4, 64, 32) * 16 <= work_bytes(GRP_L64) && stage_u4(2, 64, 32) * 16 <= work_bytes(GRP_L64),
                    "work area of the L=64 classes");
      if (wn > 0) {
        if (td.cls == CLS_PUB64) run_pub<64>(ks, work, warp, lane, io_warp);
        else if (td.cls == CLS_PLAIN64) run_plain<64>(ks, work, table_warp, warp, lane, io_warp);
      }
    } else if constexpr (G == GRP_WIDE) {
      // 16-operation tiles: 8 per warp
      const int32_t wn8 = min(8, max(0, td.nops - 8 * warp));
      static_assert(stage_u4(4, 128, 8) * 16 <= work_bytes(GRP_WIDE) && stage_u4(4, 96, 8) * 16 <= work_bytes(GRP_WIDE) &&
                        stage_u4(2, 128, 8) * 16 <= work_bytes(GRP_WIDE),
                    "work area of the wide public and plain classes");
      static_assert(batch_table_need(kBatchWindowPlain, 128 / 4) <= batch_table_u4(GRP_WIDE, 4, 4) &&
                        batch_table_need(kBatchWindowPlain, 96 / 4) <= batch_table_u4(GRP_WIDE, 4, 4),
                    "window table of a wide plain class");
      const TileIO io8{d.msgs, d.out, d.status, d.sorted, d.offsets, (uint32_t)(td.op_start + 8 * warp),
                       (uint32_t)wn8};
      if (td.cls == CLS_PUB96) run_pub_wide<96>(ks, work, warp, lane, io8);
      else if (td.cls == CLS_PUB128) run_pub_wide<128>(ks, work, warp, lane, io8);
      else if (td.cls == CLS_PLAIN96) run_plain_wide<96>(ks, work, table_warp, warp, lane, io8);
      else if (td.cls == CLS_PLAIN128) run_plain_wide<128>(ks, work, table_warp, warp, lane, io8);
    } else {
      static_assert(stage_u4(3, 32, 32) * 16 <= work_bytes(GRP_CRT) && stage_u4(4, 32, 32) * 16 <= work_bytes(GRP_CRT) &&
                        stage_u4(2, 32, 32) * 16 <= work_bytes(GRP_CRT),
                    "work area of the one-lane classes");
      static_assert(batch_table_need(5, 16) <= batch_table_u4(GRP_CRT, 5, 4) &&
                        batch_table_need(5, 32) <= batch_table_u4(GRP_CRT, 5, 4) &&
                        batch_table_need(kBatchWindowPlain, 32) <= batch_table_u4(GRP_CRT, 4, 4),
                    "window table of a one-lane class");
      const KeyHeader &hd = *reinterpret_cast<const KeyHeader *>(ks);
      const bool w5 = d.win_small == 5;
      switch (td.cls) {
        case CLS_CRT16:
          if (w5) run_crt<16, 5>(ks, work, table_warp, warp, lane, io_pair);
          else run_crt<16, 4>(ks, work, table_warp, warp, lane, io_pair);
          break;
        case CLS_CRT32:
          if (w5) run_crt<32, 5>(ks, work, table_warp, warp, lane, io_pair);
          else run_crt<32, 4>(ks, work, table_warp, warp, lane, io_pair);
          break;
        case CLS_PUB32: if (wn > 0) run_pub<32>(ks, work, warp, lane, io_warp); break;
        case CLS_PLAIN32: if (wn > 0) run_plain<32>(ks, work, table_warp, warp, lane, io_warp); break;
        case CLS_TOY: {
          const int slot = (int)threadIdx.x;
          if (slot < td.nops) {
            const uint32_t op = (uint32_t)d.sorted[td.op_start + slot];
            const size_t off = (size_t)d.offsets[op];
            const uint32_t x = d.msgs[off];
            const bool ok = x < ks[KeyLayout(1).n];
            const uint32_t r = toy_op(ks, hd, kind, x);
            d.out[off] = ok ? r : 0u;
            if (d.status) d.status[op] = ok ? 0 : -3;
          }
          break;
        }
        default: break;
      }
    }
    __syncthreads();
  }
}

}  // namespace

const void *batch_exec_fn(int group) {
  switch (group) {
    case GRP_BIG: return reinterpret_cast<const void *>(&batch_exec_kernel<GRP_BIG>);
    case GRP_CRT: return reinterpret_cast<const void *>(&batch_exec_kernel<GRP_CRT>);
    case GRP_L64: return reinterpret_cast<const void *>(&batch_exec_kernel<GRP_L64>);
    case GRP_WIDE: return reinterpret_cast<const void *>(&batch_exec_kernel<GRP_WIDE>);
    default: return nullptr;
  }
}
size_t batch_exec_smem_bytes(int group) { return (size_t)kKeyWordsMax * 4 + work_bytes(group); }

}  // namespace rsagpu
