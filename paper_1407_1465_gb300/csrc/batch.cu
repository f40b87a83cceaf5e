// batch.cu -- ragged multi-key batches (rsa_modexp_batch): the device-side
// planning kernels, the per-stream CUDA graph that runs plan + execute, and
// the device error collection used by rsa_sync().
//
// Graph (built once per context and stream, kernel parameters updated every
// call): reset -> count -> tiles -> scatter -> persistent execute.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "batch.h"
#include "kernels.cuh"
#include "launch.h"
#include "runtime_internal.h"

namespace rsagpu {
namespace {

// error bits in ctl[2]: bit k set <=> some operation failed with status -k
__device__ __forceinline__ void flag_error(uint32_t *ctl, int32_t code) { atomicOr(&ctl[2], 1u << (-code)); }

__global__ void plan_reset(BatchDesc d) {
  const uint32_t nb = d.nkeys * 3;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    d.bcount[i] = 0u;
    d.bfill[i] = 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x < tcr::kCtlWords && threadIdx.x != 2) d.ctl[threadIdx.x] = 0u;  // ranges, counters
}

// classify each operation into a bucket (key id * 3 + kind); invalid ones get a status
__global__ void plan_count(BatchDesc d) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < d.count; i += gridDim.x * blockDim.x) {
    const int32_t kid = d.key_ids[i];
    const int32_t kind = d.exp_sel[i];
    int32_t err = 0, b = -1;
    if (kid < 0 || (uint32_t)kid >= d.nkeys || d.dir[kid].rec == nullptr) {
      err = -2;
    } else if (kind > 2) {
      err = -1;
    } else {
      const KeyDirEntry e = d.dir[kid];
      if (kind != 0 && !(e.flags & KEY_HAS_D)) err = -2;
      else if (kind == 1 && !(e.flags & KEY_HAS_CRT)) err = -2;
      else if (batch_class(e.L, kind, d.wide_crt32) < 0) err = -7;
      else if (e.L > 1 && (d.offsets[i] & 3u)) err = -1;   // rows must be 16-byte aligned
      else b = kid * 3 + kind;
    }
    d.op_bucket[i] = b;
    if (b >= 0) {
      atomicAdd(&d.bcount[b], 1u);
    } else {
      if (d.status) d.status[i] = err;
      flag_error(d.ctl, err);
    }
  }
}

// Block-wide exclusive scan of one value per thread (blockDim.x == 1024).
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total, uint32_t *sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = sh[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  const uint32_t before = (warp > 0 ? sh[warp - 1] : 0u) + x - v;
  *total = sh[31];
  __syncthreads();
  return before;
}

// one block of 1024 threads: bucket offsets and tile descriptors, longest class first
__global__ void __launch_bounds__(1024) plan_tiles(BatchDesc d) {
  __shared__ uint32_t sh[32];
  const uint32_t nb = d.nkeys * 3;
  const uint32_t per = (nb + blockDim.x - 1) / blockDim.x;
  const uint32_t b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
  uint32_t op_base = 0, tile_base = 0;
  int32_t group = -1;
  for (int rank = 0; rank < CLS_COUNT; ++rank) {
    // ranks are grouped: record where each execution group's tiles start and end
    int32_t g = -1;
    for (int c = 0; c < CLS_COUNT; ++c)
      if (d.class_rank[c] == rank) g = batch_group(c);
    if (g != group) {
      if (threadIdx.x == 0) {
        if (group >= 0) d.ctl[8 + group] = min(tile_base, d.max_tiles);
        d.ctl[4 + g] = min(tile_base, d.max_tiles);
      }
      group = g;
    }
    // a bucket's tensor-core tiles (if any) take all its operations, else the
    // CUDA-core tiles do
    uint32_t my_ops = 0, my_tiles = 0;
    for (uint32_t b = b0; b < b1; ++b) {
      const uint32_t c = d.bcount[b];
      if (!c) continue;
      const int32_t cls = batch_class(d.dir[b / 3].L, (int)(b % 3), d.wide_crt32);
      if (d.class_rank[cls] != rank) continue;
      const uint32_t to = (uint32_t)batch_tile_ops(cls);
      const uint32_t rest = c - batch_tc_ops(d, cls, d.dir[b / 3], c);
      my_ops += c;
      my_tiles += (rest + to - 1) / to;
    }
    uint32_t tot_ops, tot_tiles;
    uint32_t op_off = op_base + block_exclusive_scan(my_ops, &tot_ops, sh);
    uint32_t tile_off = tile_base + block_exclusive_scan(my_tiles, &tot_tiles, sh);
    for (uint32_t b = b0; b < b1; ++b) {
      const uint32_t c = d.bcount[b];
      if (!c) continue;
      const int32_t cls = batch_class(d.dir[b / 3].L, (int)(b % 3), d.wide_crt32);
      if (d.class_rank[cls] != rank) continue;
      const uint32_t to = (uint32_t)batch_tile_ops(cls);
      d.boff[b] = op_off;
      const uint32_t skip = batch_tc_ops(d, cls, d.dir[b / 3], c);
      const uint32_t rest = c - skip;
      const uint32_t nt = (rest + to - 1) / to;
      for (uint32_t j = 0; j < nt && tile_off + j < d.max_tiles; ++j)
        d.tiles[tile_off + j] =
            TileDesc{(int32_t)b, (int32_t)(op_off + skip + j * to), (int32_t)min(to, rest - j * to), cls};
      op_off += c;
      tile_off += nt;
    }
    op_base += tot_ops;
    tile_base += tot_tiles;
  }
  if (threadIdx.x == 0) {
    d.ctl[1] = min(tile_base, d.max_tiles);
    if (group >= 0) d.ctl[8 + group] = min(tile_base, d.max_tiles);
  }
  // tensor-core chunks: whole tiles of one bucket, up to the group's tiles per CTA
  if (d.tc_min_ops) {
    for (int32_t grp = 0; grp < TCG_COUNT; ++grp) {
      const uint32_t per = (uint32_t)batch_tc_chunk_tiles(grp);
      tcr::TcChunk *list = grp == TCG_2048 ? d.tc_chunks : d.tcx_chunks[grp - 1];
      uint32_t my_chunks = 0;
      for (uint32_t b = b0; b < b1; ++b) {
        const uint32_t c = d.bcount[b];
        if (!c) continue;
        const int32_t cls = batch_class(d.dir[b / 3].L, (int)(b % 3), d.wide_crt32);
        if (batch_tc_group(cls) != grp) continue;
        const uint32_t nt = (batch_tc_ops(d, cls, d.dir[b / 3], c) + tcr::kRows - 1) / tcr::kRows;
        my_chunks += (nt + per - 1) / per;
      }
      uint32_t tot_chunks;
      uint32_t ch = block_exclusive_scan(my_chunks, &tot_chunks, sh);
      for (uint32_t b = b0; b < b1; ++b) {
        const uint32_t c = d.bcount[b];
        if (!c) continue;
        const KeyDirEntry e = d.dir[b / 3];
        const int32_t cls = batch_class(e.L, (int)(b % 3), d.wide_crt32);
        if (batch_tc_group(cls) != grp) continue;
        const uint32_t nops = batch_tc_ops(d, cls, e, c);
        const uint32_t nt = (nops + tcr::kRows - 1) / tcr::kRows;
        for (uint32_t t0 = 0; t0 < nt; t0 += per, ++ch)
          if (ch < d.max_tc_chunks)
            list[ch] = tcr::TcChunk{e.rec, e.tc, (int32_t)(d.boff[b] + t0 * tcr::kRows), (int32_t)min(per, nt - t0),
                                    (int32_t)min(per * tcr::kRows, nops - t0 * tcr::kRows), 0};
      }
      if (threadIdx.x == 0) d.ctl[batch_tc_ctl_word(grp)] = min(tot_chunks, d.max_tc_chunks);
    }
  }
}

__global__ void plan_scatter(BatchDesc d) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < d.count; i += gridDim.x * blockDim.x) {
    const int32_t b = d.op_bucket[i];
    if (b < 0) continue;
    const uint32_t pos = d.boff[b] + atomicAdd(&d.bfill[b], 1u);
    d.sorted[pos] = (int32_t)i;
  }
}

// An order-independent digest of the result rows: sum over operations of a
// mix of (operation index, row words); rows of unknown keys count as empty.
__device__ __forceinline__ uint64_t digest_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__global__ void batch_digest_kernel(uint32_t count, uint32_t nkeys, const KeyDirEntry *dir, const int32_t *key_ids,
                                    const uint64_t *offsets, const uint32_t *out, unsigned long long *acc) {
  uint64_t local = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const int32_t k = key_ids[i];
    if (k < 0 || (uint32_t)k >= nkeys || dir[k].rec == nullptr) continue;
    const uint32_t L = dir[k].L;
    const uint32_t *row = out + offsets[i];
    uint64_t h = digest_mix(0x9e3779b97f4a7c15ull + i);
    for (uint32_t j = 0; j < L; ++j) h = digest_mix(h ^ row[j]);
    local += h;
  }
  atomicAdd(acc, (unsigned long long)local);
}

// Share (percent) of one wave of the four-lane group up to which a ragged
// batch runs 2048-bit CRT four lanes per operation; 0 disables it.
uint64_t ragged_wide_fraction() {
  const char *v = std::getenv("RSAGPU_RAGGED_WIDE_PCT");
  const long p = v ? std::atol(v) : 100;
  return p < 0 ? 0 : (uint64_t)p;
}

// Lanes per operation of 4096-bit CRT in the latency shapes: 16 (GB300,
// serving at 1 k req/s: 4096-bit requests p50/p99 8.8/22.7 ms against
// 12.8/27.5 ms with 8, the 256-key mix 3.5/14.9 against 4.0/17.6 ms);
// RSAGPU_RAGGED_LANES_4096=8 selects 8.
int lanes_4096() {
  const char *v = std::getenv("RSAGPU_RAGGED_LANES_4096");
  return v && std::atoi(v) == 8 ? 8 : 16;
}

// approximate word products per operation of a class, for the longest-first order
double class_cost(int32_t cls) {
  auto mm = [](double l) { return 2.0 * l * l + l; };
  switch (cls) {
    case CLS_TOY: return 1.0;
    case CLS_CRT16: return 2.0 * 660 * mm(16);
    case CLS_CRT32: return 2.0 * 1300 * mm(32);
    case CLS_CRT48: return 2.0 * 1880 * mm(48);
    case CLS_CRT64: return 2.0 * 2500 * mm(64);
    case CLS_CRT32W: return 2.0 * 1300 * mm(32) / 4;   // per lane
    case CLS_CRT64W: return 2.0 * 2500 * mm(64) / 8;
    case CLS_CRT64X: return 2.0 * 2500 * mm(64) / 16;
    case CLS_PUB32: return 19 * mm(32);
    case CLS_PUB64: return 19 * mm(64);
    case CLS_PUB96: return 19 * mm(96);
    case CLS_PUB128: return 19 * mm(128);
    case CLS_PLAIN32: return 1300 * mm(32);
    case CLS_PLAIN64: return 2600 * mm(64);
    case CLS_PLAIN96: return 3900 * mm(96) / 4;   // per lane
    case CLS_PLAIN128: return 5200 * mm(128) / 4;
    default: return 0.0;
  }
}

}  // namespace

// the tensor-core chunk lists (TCG_COUNT of them) follow the tile descriptors in the same buffer
static size_t tc_chunks_offset(uint64_t max_tiles) { return ((size_t)max_tiles * sizeof(TileDesc) + 255) / 256 * 256; }
// Chunks one tensor-core group can have in a batch of `count` operations: a
// bucket of c >= tc_min_ops operations makes at most ceil(c / 128) <= c / 128 + 1
// chunks, and there are at most count / tc_min_ops such buckets.
static uint64_t tc_chunk_cap(uint64_t count, int tc_min_ops) {
  return count / tcr::kRows + count / (uint64_t)std::max(tc_min_ops, 1) + 1;
}
// the 3072- and 4096-bit tensor-core groups: prime limbs and window (GB300:
// window 4 at 3072 bits, 3 at 4096, as for uniform batches)
static constexpr int kTcxH[2] = {48, 64};
static constexpr int kTcxWindow[2] = {4, 3};
// window tables shared by the tensor-core groups (their kernels run one after
// the other): one table per tile slot of sm_count CTAs, sized for the largest
static size_t tc_tables_shared(int grid, int window_tc) {
  size_t b = tcr::tc_tables_bytes(grid, window_tc);
  for (int x = 0; x < 2; ++x) b = std::max(b, tc4::tc4_tables_bytes(kTcxH[x], grid, kTcxWindow[x]));
  return b;
}

struct BatchState {
  cudaStream_t stream = nullptr;
  bool built = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t nodes[4 + 2 * TCG_COUNT + GRP_COUNT] = {};
  int tc_window = 0;          // window of the tensor-core node the graph was built with
  int exec_grid = 0;
  int grids_exec[GRP_COUNT] = {};
  DevBuf keydir;
  uint64_t keydir_epoch = ~0ull;
};

static std::vector<BatchState *> &batch_states(Ctx *c) {
  if (!c->batch_state) c->batch_state = new std::vector<BatchState *>();
  return *static_cast<std::vector<BatchState *> *>(c->batch_state);
}

void Ctx::free_extra() {
  if (!batch_state) return;
  for (BatchState *b : batch_states(this)) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->keydir.ptr) cudaFree(b->keydir.ptr);
    delete b;
  }
  delete static_cast<std::vector<BatchState *> *>(batch_state);
  batch_state = nullptr;
}

int Ctx::collect_device_errors(cudaStream_t s) {
  auto it = workspaces.find(s);
  if (it == workspaces.end() || !it->second.aux3.ptr) return RSA_OK;
  uint32_t bits = 0;
  uint32_t *ctl = static_cast<uint32_t *>(it->second.aux3.ptr);
  cudaError_t e = cudaMemcpy(&bits, ctl + 2, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "read device error word");
  if (!bits) return RSA_OK;
  const uint32_t zero = 0;
  cudaMemcpy(ctl + 2, &zero, 4, cudaMemcpyHostToDevice);
  for (int code : {2, 1, 7, 6, 4}) {
    if (bits & (1u << code)) {
      const char *what = code == 2 ? "operation with an unknown key or a kind its key cannot serve"
                         : code == 1 ? "operation with a bad exponent kind or a misaligned row"
                         : code == 7 ? "operation kind not supported for its key size"
                         : code == 6 ? "device-side wait timed out" : "out of memory";
      return set_error(-code, std::string("ragged batch: ") + what);
    }
  }
  return RSA_OK;
}

void Ctx::release_stream(cudaStream_t s) {
  cudaStreamSynchronize(s);
  if (batch_state) {
    std::vector<BatchState *> &v = batch_states(this);
    for (auto it = v.begin(); it != v.end(); ++it) {
      BatchState *b = *it;
      if (b->stream != s) continue;
      if (b->exec) cudaGraphExecDestroy(b->exec);
      if (b->graph) cudaGraphDestroy(b->graph);
      if (b->keydir.ptr) {
        cudaFree(b->keydir.ptr);
        release(b->keydir.bytes);
      }
      delete b;
      v.erase(it);
      break;
    }
  }
  auto it = workspaces.find(s);
  if (it != workspaces.end()) {
    Workspace &w = it->second;
    for (DevBuf *d : {&w.tables, &w.io_in, &w.io_out, &w.io_status, &w.aux0, &w.aux1, &w.aux2, &w.aux3, &w.halves,
                      &w.tc_halves[0], &w.tc_halves[1],
                      &w.verify, &w.gcd0, &w.gcd1, &w.gcd_tree, &w.gcd_tw})
      if (d->ptr) {
        cudaFree(d->ptr);
        release(d->bytes);
        d->ptr = nullptr;
        d->bytes = 0;
      }
    workspaces.erase(it);
  }
}

static BatchState *state_for(Ctx *c, cudaStream_t s) {
  for (BatchState *b : batch_states(c))
    if (b->stream == s) return b;
  BatchState *b = new BatchState();
  b->stream = s;
  batch_states(c).push_back(b);
  return b;
}

// Key directory and scratch of the ragged path on stream s, sized for batches
// of up to max_count operations.  Growing a buffer frees the old one, which
// waits for the whole device, so callers that keep batches in flight on
// several streams (the request loop) size them once up front.
int Ctx::prepare_batch(cudaStream_t s, uint64_t max_count) {
  BatchState *st = state_for(this, s);
  Workspace &w = ws(s);
  const uint32_t nkeys = (uint32_t)keys.size();
  // key directory (rebuilt when keys change)
  if (st->keydir_epoch != key_epoch || !st->keydir.ptr) {
    std::vector<KeyDirEntry> dir(std::max<uint32_t>(nkeys, 1));
    for (uint32_t i = 0; i < nkeys; ++i) {
      const KeySlot &k = keys[i];
      if (!k.used) continue;
      const KeyHeader *hd = reinterpret_cast<const KeyHeader *>(k.host_rec.data());
      dir[i] = KeyDirEntry{k.d_rec, k.L, k.flags, k.nbits, hd->e_bits, k.d_tc};
    }
    int rc = ensure(st->keydir, dir.size() * sizeof(KeyDirEntry));
    if (rc) return rc;
    cudaError_t e = cudaMemcpy(st->keydir.ptr, dir.data(), dir.size() * sizeof(KeyDirEntry), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "upload key directory");
    st->keydir_epoch = key_epoch;
  }
  const uint32_t nb = std::max<uint32_t>(nkeys, 1) * 3;
  const uint64_t max_tiles = max_count / kMinTileOps + nb + 1;   // tiles of at least kMinTileOps operations
  const Tune tr = tune_for(0, RSA_TUNE_RAGGED);
  const uint64_t chunk_cap = tc_chunk_cap(max_count, tr.tc_min_ops);
  int rc;
  if ((rc = ensure(w.aux0, (size_t)max_count * 8)) ||                  // op_bucket + sorted
      (rc = ensure(w.aux1, (size_t)nb * 12)) ||                        // bcount, bfill, boff
      (rc = ensure(w.aux2, tc_chunks_offset(max_tiles) + TCG_COUNT * chunk_cap * sizeof(tcr::TcChunk))) ||
      (rc = ensure(w.aux3, tcr::kCtlWords * 4)))
    return rc;
  const bool tc_possible = tr.variant != 1;
  if (tc_possible) {
    // the tensor-core groups: one CTA per SM, the whole shared memory of an SM
    const void *fn = tcr::ragged_tc_half_fn(tr.window_tc);
    if (!fn) return set_error(RSA_ERR_ARG, "no tensor-core kernel for this window");
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcr::tc_smem_bytes());
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(ragged tensor-core kernel)");
    if ((rc = ensure(w.halves, tcr::tc_halves_bytes((uint32_t)max_count)))) return rc;
    for (int x = 0; x < 2; ++x) {
      const int H = kTcxH[x];
      e = cudaFuncSetAttribute(tc4::ragged_tc4_half_fn(H, kTcxWindow[x]), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tc4::tc4_smem_bytes(H));
      if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(ragged tensor-core kernel)");
      if ((rc = ensure(w.tc_halves[x], tc4::tc4_halves_bytes(H, (uint32_t)max_count)))) return rc;
    }
  }
  int max_grid = 0;
  for (int g = 0; g < GRP_COUNT; ++g) {
    const void *fn = batch_exec_fn(g);
    const size_t sm = batch_exec_smem_bytes(g);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(batch_exec)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 64, sm);
    if (e != cudaSuccess) return cuda_error(e, "occupancy(batch_exec)");
    const Tune t = tune_for(0, RSA_TUNE_RAGGED);
    if (t.ctas_per_sm > 0) per_sm = std::min(per_sm, t.ctas_per_sm);
    st->grids_exec[g] = std::max(1, per_sm) * sm_count;
    max_grid = std::max(max_grid, st->grids_exec[g]);
  }
  st->exec_grid = max_grid;
  // window tables: one per resident warp of each group (groups run concurrently),
  // each the size its group's largest class needs
  size_t table_u4 = 0;
  for (int gi = 0; gi < GRP_COUNT; ++gi)
    table_u4 += (size_t)st->grids_exec[gi] * 2 * batch_table_u4(gi, tr.window, tr.window_big);
  // then the tensor-core groups' tables (one per tile slot of their sm_count
  // CTAs; the groups run one after the other and share them)
  const size_t tc_bytes = tc_possible ? tc_tables_shared(sm_count, tr.window_tc) : 0;
  return ensure(w.tables, std::max<size_t>(table_u4 * 16 + tc_bytes, 16));
}

int Ctx::batch_digest(uint64_t count, const int32_t *key_ids, const uint64_t *offsets, const uint32_t *out,
                      cudaStream_t s, uint64_t *digest) {
  BatchState *st = state_for(this, s);
  Workspace &w = ws(s);
  if (!st->keydir.ptr || !w.aux3.ptr) return set_error(RSA_ERR_ARG, "batch_digest before a ragged batch");
  // the digest word sits in the control block's last word pair, after the planner's words
  unsigned long long *acc = reinterpret_cast<unsigned long long *>(static_cast<uint32_t *>(w.aux3.ptr) + 30);
  cudaError_t e = cudaMemsetAsync(acc, 0, 8, s);
  if (e != cudaSuccess) return cuda_error(e, "digest reset");
  const uint32_t nkeys = std::max<uint32_t>((uint32_t)keys.size(), 1);
  const int grid = (int)std::min<uint64_t>((count + 255) / 256, (uint64_t)sm_count * 4);
  batch_digest_kernel<<<std::max(grid, 1), 256, 0, s>>>((uint32_t)count, nkeys,
                                                         static_cast<const KeyDirEntry *>(st->keydir.ptr), key_ids,
                                                         offsets, out, acc);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "digest kernel");
  unsigned long long h = 0;
  if ((e = cudaMemcpyAsync(&h, acc, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_error(e, "digest read");
  *digest = h;
  return RSA_OK;
}

uint64_t Ctx::batch_wave_ops(cudaStream_t s) {
  const BatchState *st = state_for(this, s);
  return (uint64_t)8 * (uint64_t)st->grids_exec[GRP_BIG] * ragged_wide_fraction() / 100;
}

int Ctx::run_batch(uint64_t count, const int32_t *key_ids, const uint8_t *exp_sel, const uint64_t *offsets,
                   const uint32_t *msgs, uint32_t *out, int32_t *status, cudaStream_t s, int wide) {
  if (count == 0) return RSA_OK;
  NvtxRange range("rsa_modexp_batch");
  int rc = prepare_batch(s, count);
  if (rc) return rc;
  BatchState *st = state_for(this, s);
  Workspace &w = ws(s);
  const uint32_t nkeys = (uint32_t)keys.size();
  const uint32_t nb = std::max<uint32_t>(nkeys, 1) * 3;
  const uint32_t max_tiles = (uint32_t)(count / kMinTileOps + nb + 1);
  int grids_exec[GRP_COUNT];
  for (int g = 0; g < GRP_COUNT; ++g) grids_exec[g] = st->grids_exec[g];

  BatchDesc d{};
  d.count = (uint32_t)count;
  d.nkeys = std::max<uint32_t>(nkeys, 1);
  d.key_ids = key_ids;
  d.exp_sel = exp_sel;
  d.offsets = offsets;
  d.msgs = msgs;
  d.out = out;
  d.status = status;
  d.dir = static_cast<const KeyDirEntry *>(st->keydir.ptr);
  d.op_bucket = static_cast<int32_t *>(w.aux0.ptr);
  d.sorted = d.op_bucket + count;
  d.bcount = static_cast<uint32_t *>(w.aux1.ptr);
  d.bfill = d.bcount + nb;
  d.boff = d.bfill + nb;
  d.tiles = static_cast<TileDesc *>(w.aux2.ptr);
  d.ctl = static_cast<uint32_t *>(w.aux3.ptr);
  d.tables = static_cast<uint4 *>(w.tables.ptr);
  d.max_tiles = max_tiles;
  d.tc_chunks = reinterpret_cast<tcr::TcChunk *>(static_cast<char *>(w.aux2.ptr) + tc_chunks_offset(max_tiles));
  d.max_tc_chunks = (uint32_t)tc_chunk_cap(count, tune_for(0, RSA_TUNE_RAGGED).tc_min_ops);
  d.tcx_chunks[0] = d.tc_chunks + d.max_tc_chunks;
  d.tcx_chunks[1] = d.tc_chunks + 2 * d.max_tc_chunks;
  // Small batches run 2048-bit CRT with four lanes per operation and 4096-bit
  // CRT with eight: each operation finishes sooner (about 2.2x at 2048 bits),
  // and while the batch fits in one wave of the multi-lane group (8 operations
  // per resident warp pair) the GPU has idle SMs anyway.  Larger batches keep
  // one (four) lanes per operation, which has the higher throughput.
  // lanes per operation of the long CRT sizes: the caller's choice, else the
  // tuned one (threads_per_op 1: one/four lanes, 4: four/eight), else by size
  if (wide < 0) {
    const int tpo = tune_for(0, RSA_TUNE_RAGGED).tpo;
    wide = tpo == 4 ? 1 : tpo == 1 ? 0 : (count <= batch_wave_ops(s) ? 1 : 0);
  }
  // lanes per operation of 4096-bit CRT in the latency shapes (lanes_4096)
  d.wide_crt32 = wide != 0 ? (lanes_4096() == 16 ? 2u : 1u) : 0u;
  // windows of the CRT classes and the tensor-core group (the ragged tuning):
  // the group takes 2048-bit CRT buckets in the throughput shapes, unless the
  // tuning keeps every operation on the CUDA cores (variant 1) or asks for it
  // in every shape (variant 3)
  const Tune tr = tune_for(0, RSA_TUNE_RAGGED);
  d.win_small = tr.window;
  d.win_big = tr.window_big;
  const bool tc_on = tr.variant == 3 || (tr.variant == 0 && !d.wide_crt32);
  d.tc_min_ops = tc_on ? (uint32_t)std::max(tr.tc_min_ops, 1) : 0u;
  {
    std::vector<int32_t> order(CLS_COUNT);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [](int32_t a, int32_t b) {
      if (batch_group(a) != batch_group(b)) return batch_group(a) < batch_group(b);
      return class_cost(a) > class_cost(b);
    });
    for (int r = 0; r < CLS_COUNT; ++r) d.class_rank[order[r]] = r;
  }
  const int g_ops = (int)std::min<uint64_t>((count + 255) / 256, (uint64_t)sm_count * 8);
  const int g_nb = (int)std::min<uint32_t>((nb + 255) / 256, (uint32_t)sm_count * 8);
  // nodes: reset -> count -> tiles -> scatter -> {the tensor-core groups
  // (4096-, 3072-, 2048-bit CRT exponentiation kernels in a chain, each
  // followed by its Garner kernel), one persistent kernel per CUDA-core group}
  // (run concurrently).  The tensor-core kernels need whole SMs (all registers,
  // ~210 KB of shared memory), so they are scheduled first (see the graph
  // build); without tensor-core work their CTAs leave at once.
  constexpr int kNodes = 4 + 2 * TCG_COUNT + GRP_COUNT;
  constexpr int kTcNode = 4, kGroup0 = 4 + 2 * TCG_COUNT;   // tensor-core group x: 4 + 2x, its Garner 5 + 2x
  const void *tc_fn = tcr::ragged_tc_half_fn(tr.window_tc);
  if (!tc_fn) return set_error(RSA_ERR_ARG, "no tensor-core kernel for this window");
  const void *fns[kNodes] = {reinterpret_cast<const void *>(&plan_reset), reinterpret_cast<const void *>(&plan_count),
                             reinterpret_cast<const void *>(&plan_tiles), reinterpret_cast<const void *>(&plan_scatter),
                             tc_fn, tcr::ragged_tc_garner_fn(),
                             tc4::ragged_tc4_half_fn(kTcxH[0], kTcxWindow[0]), tc4::ragged_tc4_garner_fn(kTcxH[0]),
                             tc4::ragged_tc4_half_fn(kTcxH[1], kTcxWindow[1]), tc4::ragged_tc4_garner_fn(kTcxH[1]),
                             batch_exec_fn(0), batch_exec_fn(1), batch_exec_fn(2), batch_exec_fn(3)};
  dim3 grids[kNodes] = {dim3(std::max(1, g_nb)), dim3(g_ops), dim3(1), dim3(g_ops),
                        dim3(sm_count), dim3(sm_count * 4), dim3(sm_count), dim3(sm_count * 4),
                        dim3(sm_count), dim3(sm_count * 4)};
  dim3 blocks[kNodes] = {dim3(256), dim3(256), dim3(1024), dim3(256), dim3(tcr::kThreads),
                         dim3(tcr::kRaggedGarnerThreads), dim3(tc4::kThreads), dim3(128), dim3(tc4::kThreads),
                         dim3(128)};
  size_t smems[kNodes] = {0, 0, 0, 0, tcr::tc_smem_bytes(), tcr::ragged_tc_garner_smem(),
                          tc4::tc4_smem_bytes(kTcxH[0]), tc4::ragged_tc4_garner_smem(kTcxH[0]),
                          tc4::tc4_smem_bytes(kTcxH[1]), tc4::ragged_tc4_garner_smem(kTcxH[1])};
  BatchDesc dg[kNodes];
  void *args[kNodes][1];
  for (int i = 0; i < kNodes; ++i) {
    dg[i] = d;
    args[i][0] = &dg[i];
  }
  // the tensor-core nodes take their own argument blocks
  size_t group_table_u4 = 0;
  for (int gi = 0; gi < GRP_COUNT; ++gi)
    group_table_u4 += (size_t)grids_exec[gi] * 2 * batch_table_u4(gi, d.win_small, d.win_big);
  tcr::RaggedTcArgs ra[TCG_COUNT];
  for (int x = 0; x < TCG_COUNT; ++x) {
    ra[x] = tcr::RaggedTcArgs{};
    ra[x].chunks = x == TCG_2048 ? d.tc_chunks : d.tcx_chunks[x - 1];
    ra[x].ctl = d.ctl;
    ra[x].sorted = d.sorted;
    ra[x].offsets = offsets;
    ra[x].msgs = msgs;
    ra[x].out = out;
    ra[x].status = status;
    ra[x].tables = d.tables + group_table_u4;
    ra[x].halves = x == TCG_2048 ? w.halves.ptr : w.tc_halves[x - 1].ptr;
    ra[x].count = (uint32_t)count;
    ra[x].wait_polls = tcr::kDefaultWaitPolls;
    if (const char *ev = std::getenv("RSAGPU_TC_WAIT_POLLS")) ra[x].wait_polls = (uint32_t)std::strtoul(ev, nullptr, 10);
    ra[x].ctl_word = (uint32_t)batch_tc_ctl_word(x);
    args[kTcNode + 2 * x][0] = &ra[x];
    args[kTcNode + 2 * x + 1][0] = &ra[x];
  }
  if (tc_on && (!w.halves.ptr || w.halves.bytes < tcr::tc_halves_bytes((uint32_t)count) ||
                w.tc_halves[0].bytes < tc4::tc4_halves_bytes(kTcxH[0], (uint32_t)count) ||
                w.tc_halves[1].bytes < tc4::tc4_halves_bytes(kTcxH[1], (uint32_t)count) ||
                w.tables.bytes < group_table_u4 * 16 + tc_tables_shared(sm_count, tr.window_tc)))
    return set_error(RSA_ERR_NOMEM, "tensor-core workspace of the ragged batch is missing");
  // each group's warps index their own slice of the table scratch
  size_t slot_off = 0;
  // a batch with few tiles launches only the CTAs it can use (at most one
  // per tile: count / smallest tile + one partial tile per bucket), so that
  // its tiles start on separate SMs instead of wherever the first CTAs landed
  const uint64_t tile_min[GRP_COUNT] = {d.wide_crt32 == 2 ? 2u : d.wide_crt32 ? 4u : 8u, 32u, 32u, 16u};
  static_assert(GRP_BIG == 0 && GRP_CRT == 1 && GRP_L64 == 2 && GRP_WIDE == 3, "tile_min order");
  for (int gi = 0; gi < GRP_COUNT; ++gi) {
    const uint64_t useful = count / tile_min[gi] + std::min<uint64_t>(nb, count) + 1;
    grids[kGroup0 + gi] = dim3((unsigned)std::min<uint64_t>((uint64_t)grids_exec[gi], useful));
    blocks[kGroup0 + gi] = dim3(64);
    smems[kGroup0 + gi] = batch_exec_smem_bytes(gi);
    dg[kGroup0 + gi].tables = d.tables + slot_off;
    dg[kGroup0 + gi].table_u4 = (uint32_t)batch_table_u4(gi, d.win_small, d.win_big);
    slot_off += (size_t)grids_exec[gi] * 2 * dg[kGroup0 + gi].table_u4;
  }
  cudaError_t e;
  auto params = [&](int i) {
    cudaKernelNodeParams p{};
    p.func = const_cast<void *>(fns[i]);
    p.gridDim = grids[i];
    p.blockDim = blocks[i];
    p.sharedMemBytes = (unsigned)smems[i];
    p.kernelParams = args[i];
    return p;
  };
  if (st->built && st->tc_window != tr.window_tc) {
    // the tensor-core node's kernel changed with its window: build the graph anew
    cudaGraphExecDestroy(st->exec);
    cudaGraphDestroy(st->graph);
    st->exec = nullptr;
    st->graph = nullptr;
    st->built = false;
  }
  if (!st->built) {
    if ((e = cudaGraphCreate(&st->graph, 0)) != cudaSuccess) return cuda_error(e, "cudaGraphCreate");
    // The CUDA-core groups start with the tensor-core kernel rather than after
    // it; that kernel gets the highest scheduling priority, so its CTAs take
    // empty SMs first and the groups' CTAs fill the SMs its last wave leaves
    // (GB300, 256-key mix: 779 K against 767 K ops/s with the groups after it).
    // RSAGPU_RAGGED_TC_OVERLAP=0 runs the groups after the tensor-core kernel.
    const char *ov = std::getenv("RSAGPU_RAGGED_TC_OVERLAP");
    const bool overlap = !ov || std::atoi(ov) != 0;
    // The tensor-core kernels run one after the other, longest chunks first
    // (4096, 3072, then 2048 bits): each takes whole SMs, and the shorter
    // chunks of the later kernels fill the SMs the earlier ones leave (GB300,
    // 256-key mix: 971 K ops/s, against 946 K in the opposite order and 911 K
    // with the three as siblings, which hold every SM before the CUDA-core
    // groups get any).  Nodes are added so that each follows its dependences.
    int order[kNodes], n = 0;
    for (int i = 0; i < kTcNode; ++i) order[n++] = i;
    for (int x = TCG_COUNT - 1; x >= 0; --x) order[n++] = kTcNode + 2 * x;
    for (int x = TCG_COUNT - 1; x >= 0; --x) order[n++] = kTcNode + 2 * x + 1;
    for (int i = kGroup0; i < kNodes; ++i) order[n++] = i;
    constexpr int kLastTc = kTcNode + 2 * (TCG_COUNT - 1);   // the 4096-bit kernel, first in the chain
    for (int k = 0; k < kNodes; ++k) {
      const int i = order[k];
      cudaKernelNodeParams p = params(i);
      // planning in sequence; the tensor-core chain after the scatter, each
      // Garner after its kernel; the CUDA-core groups after the scatter
      // (without overlap: after the last kernel of the chain, the 2048-bit one)
      cudaGraphNode_t dep = nullptr;
      if (i >= 1 && i <= 3) dep = st->nodes[i - 1];
      else if (i >= kTcNode && i < kGroup0 && ((i - kTcNode) & 1)) dep = st->nodes[i - 1];
      else if (i >= kTcNode && i < kGroup0) dep = st->nodes[i < kLastTc ? i + 2 : 3];
      else if (i >= kGroup0) dep = st->nodes[overlap ? 3 : kTcNode];
      e = cudaGraphAddKernelNode(&st->nodes[i], st->graph, dep ? &dep : nullptr, dep ? 1 : 0, &p);
      if (e != cudaSuccess) return cuda_error(e, "cudaGraphAddKernelNode");
    }
    if (overlap) {
      int least = 0, greatest = 0;
      if ((e = cudaDeviceGetStreamPriorityRange(&least, &greatest)) != cudaSuccess)
        return cuda_error(e, "cudaDeviceGetStreamPriorityRange");
      cudaLaunchAttributeValue v{};
      v.priority = greatest;
      for (int x = 0; x < TCG_COUNT; ++x)
        if ((e = cudaGraphKernelNodeSetAttribute(st->nodes[kTcNode + 2 * x], cudaLaunchAttributePriority, &v)) !=
            cudaSuccess)
          return cuda_error(e, "cudaGraphKernelNodeSetAttribute(priority)");
    }
    if ((e = cudaGraphInstantiate(&st->exec, st->graph, 0)) != cudaSuccess)
      return cuda_error(e, "cudaGraphInstantiate");
    st->built = true;
    st->tc_window = tr.window_tc;
  } else {
    for (int i = 0; i < kNodes; ++i) {
      cudaKernelNodeParams p = params(i);
      e = cudaGraphExecKernelNodeSetParams(st->exec, st->nodes[i], &p);
      if (e != cudaSuccess) return cuda_error(e, "cudaGraphExecKernelNodeSetParams");
    }
  }
  if ((e = cudaGraphLaunch(st->exec, s)) != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
  stats.graph_launches++;
  stats.kernel_launches += kNodes;
  return RSA_OK;
}

}  // namespace rsagpu

using namespace rsagpu;

extern "C" {

int rsa_modexp_batch(rsa_ctx *ctx, uint64_t count, const int32_t *key_ids, const uint8_t *exp_sel,
                     const uint64_t *limb_offsets, const uint32_t *msgs, uint32_t *out, int32_t *op_status,
                     void *stream) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  if (count > 0x7fffffffull) return set_error(RSA_ERR_ARG, "count exceeds 2^31 - 1");
  if (count > 0 && (!key_ids || !exp_sel || !limb_offsets || !msgs || !out))
    return set_error(RSA_ERR_ARG, "null pointer");
  if ((reinterpret_cast<uintptr_t>(msgs) | reinterpret_cast<uintptr_t>(out)) & 15u)
    return set_error(RSA_ERR_ARG, "message and output buffers must be 16-byte aligned");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  cudaSetDevice(c->device);
  c->stats.ops += count;
  return c->run_batch(count, key_ids, exp_sel, limb_offsets, msgs, out, op_status, static_cast<cudaStream_t>(stream));
}

int rsa_modexp_batch_host(rsa_ctx *ctx, uint64_t count, const int32_t *key_ids, const uint8_t *exp_sel,
                          const uint64_t *limb_offsets, uint64_t total_limbs, const uint32_t *msgs, uint32_t *out,
                          int32_t *op_status, void *stream) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  if (count > 0x7fffffffull) return set_error(RSA_ERR_ARG, "count exceeds 2^31 - 1");
  if (count == 0) return RSA_OK;
  if (!key_ids || !exp_sel || !limb_offsets || !msgs || !out) return set_error(RSA_ERR_ARG, "null pointer");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Workspace &w = c->ws(s);
  // layout of io_in: [key_ids | exp_sel (padded to 8) | offsets | msgs], io_out: out, io_status: status
  const size_t kb = (size_t)count * 4, eb = ((size_t)count + 7) / 8 * 8, ob = (size_t)count * 8;
  const size_t mb = (size_t)total_limbs * 4;
  const size_t head = (kb + eb + ob + 255) / 256 * 256;
  int rc;
  if ((rc = c->ensure(w.io_in, head + mb)) || (rc = c->ensure(w.io_out, mb)) ||
      (op_status && (rc = c->ensure(w.io_status, (size_t)count * 4))))
    return rc;
  char *base = static_cast<char *>(w.io_in.ptr);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(base, key_ids, kb, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + kb, exp_sel, (size_t)count, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + kb + eb, limb_offsets, ob, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + head, msgs, mb, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_error(e, "cudaMemcpyAsync H2D");
  c->stats.ops += count;
  rc = c->run_batch(count, reinterpret_cast<const int32_t *>(base), reinterpret_cast<const uint8_t *>(base + kb),
                    reinterpret_cast<const uint64_t *>(base + kb + eb), reinterpret_cast<const uint32_t *>(base + head),
                    static_cast<uint32_t *>(w.io_out.ptr),
                    op_status ? static_cast<int32_t *>(w.io_status.ptr) : nullptr, s);
  if (rc) return rc;
  if ((e = cudaMemcpyAsync(out, w.io_out.ptr, mb, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_error(e, "cudaMemcpyAsync D2H");
  if (op_status &&
      (e = cudaMemcpyAsync(op_status, w.io_status.ptr, (size_t)count * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_error(e, "cudaMemcpyAsync D2H status");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  return c->collect_device_errors(s);
}

}  // extern "C"
