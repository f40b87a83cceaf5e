// runtime.cu -- the C ABI (include/rsa_gb300.h): contexts, the device-resident
// key table, per-stream workspace, launch sizing and dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "crt_tc.h"
#include "keyprep.h"
#include "keyrec.h"
#include "kernels.cuh"
#include "launch.h"
#include "rsa_gb300.h"
#include "runtime_internal.h"

namespace rsagpu {

thread_local std::string g_last_error;

int set_error(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

int cuda_error(cudaError_t e, const char *what) {
  return set_error(RSA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

const void *imad_probe_fn();
const void *chain_probe_fn();

// ------------------------------------------------------------------ workspace
int Ctx::reserve(size_t bytes) {
  if (used + bytes > budget)
    return set_error(RSA_ERR_NOMEM, "memory budget exceeded (" + std::to_string(used + bytes) +
                                        " > " + std::to_string(budget) + " bytes)");
  used += bytes;
  return RSA_OK;
}
void Ctx::release(size_t bytes) { used -= std::min(used, bytes); }

int Ctx::ensure(DevBuf &b, size_t need) {
  if (need <= b.bytes) return RSA_OK;
  size_t want = std::max(need, b.bytes + b.bytes / 2);
  if (used - b.bytes + want > budget) want = need;
  if (b.ptr) {
    cudaFree(b.ptr);
    release(b.bytes);
    b.ptr = nullptr;
    b.bytes = 0;
  }
  int rc = reserve(want);
  if (rc) return rc;
  cudaError_t e = cudaMalloc(&b.ptr, want);
  if (e != cudaSuccess) {
    release(want);
    cudaGetLastError();
    return set_error(RSA_ERR_NOMEM, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e));
  }
  b.bytes = want;
  return RSA_OK;
}

Workspace &Ctx::ws(cudaStream_t s) { return workspaces[s]; }

Ctx::~Ctx() {
  cudaSetDevice(device);
  cudaDeviceSynchronize();
  for (auto &k : keys) {
    if (k.d_rec) cudaFree(k.d_rec);
    if (k.d_tc) cudaFree(k.d_tc);
    if (k.d_tcn) cudaFree(k.d_tcn);
  }
  for (auto &kv : workspaces) kv.second.free_all();
  free_extra();
}

void Workspace::free_all() {
  for (DevBuf *b : {&tables, &io_in, &io_out, &io_status, &aux0, &aux1, &aux2, &aux3, &halves, &tc_halves[0],
                    &tc_halves[1], &verify, &gcd0, &gcd1, &gcd_tree, &gcd_tw}) {
    if (b->ptr) cudaFree(b->ptr);
    b->ptr = nullptr;
    b->bytes = 0;
  }
  gcd_tw_ptr = nullptr;
  gcd_tw_n = 0;
}

// ------------------------------------------------------------------ tuning
// Window width, from sweeps on GB300: the constant-time table read costs 2^w
// entries per window, so the smaller table wins although it needs a few more
// multiplications (RSA-2048 CRT: w = 4 1.25 M/s, w = 5 1.18 M/s, w = 6 0.97 M/s;
// RSA-4096 CRT: 128 K/s, 127 K/s, 118 K/s).
// Public exponents longer than this use sliding windows (variant 0).
constexpr uint32_t kSlideMinBits = 64;
// the public exponent of 2048-bit keys goes to the tensor cores from this many operations
constexpr uint64_t kPubTcMinCount = 4096;
// Smallest RSA-3072 / RSA-4096 CRT batch the automatic tuning sends to the
// tensor cores (where the CUDA-core kernel's time reaches one tensor-core
// launch's: GB300, 285 K/s against ~33 ms, 149 K/s against ~83 ms).
static uint64_t tc4_auto_min_count(uint32_t L) { return L == 96 ? 8192 : 12288; }

static int default_window(uint32_t L, int kind) {
  (void)L;
  (void)kind;
  return 4;
}

Tune Ctx::tune_for(uint32_t nbits, int kind) const {
  Tune t{0, 0, 0, 0, 0, 0, 0, 0};
  auto it = tuning.find({nbits, kind});
  if (it != tuning.end()) t = it->second;
  const uint32_t L = nbits / 32;
  // RSA-2048 and RSA-4096 CRT: the Montgomery reduction on the tensor cores
  // (GB300, w = 3: 2.14 M/s against 1.25 M/s for the CUDA-core CIOS kernel at
  // 2048 bits; 196 K/s against 149 K/s for the four-lane kernel at 4096 bits)
  // (only when nothing else was asked for: windows 3/4, one lane per operation)
  if (!t.variant && kind == RSA_EXP_PRIVATE_CRT && (L == 2 * (uint32_t)tcr::kH || tc4::supported((int)L / 2)) &&
      t.tpo <= 1 && (t.window == 0 || t.window == 3 || t.window == 4))
    t.variant = 3;
  // tensor-core path: window 3 keeps the tables in L2 at 2048 and 4096 bits;
  // at 3072 bits window 4 is faster (GB300: 502 K against 480 K decrypts/s)
  if (!t.window) t.window = (t.variant == 3) ? (L == 96 ? 4 : 3) : (kind == RSA_EXP_PUBLIC ? 5 : default_window(L, kind));
  if (!t.warps_per_cta) t.warps_per_cta = 4;
  // lanes per operation (GB300 sweeps): four for 3072/4096-bit keys -- CRT halves of
  // 48/64 limbs need 255 registers on one lane and 128 on four (RSA-4096 CRT:
  // 127 K/s -> 145 K/s), and the one-lane public exponent of those sizes spills --
  // one lane otherwise (RSA-2048 CRT: 1.24 M/s on one lane, 1.10 M on two).
  if (kind == RSA_TUNE_RAGGED) {
    // ragged batches: CRT windows 4 (1024/2048-bit) and 5 (3072/4096-bit),
    // tensor-core groups (2048 bits at window 3) for buckets of at least 128 operations;
    // the lanes-per-operation policy and the variant stay automatic (0)
    if (!t.window) t.window = 4;
    if (!t.window_big) t.window_big = 5;
    if (!t.window_tc) t.window_tc = 3;
    if (!t.tc_min_ops) t.tc_min_ops = 128;
    return t;
  }
  if (!t.tpo) t.tpo = L > 64 ? 4 : 1;
  return t;
}

// ------------------------------------------------------------------ launch helpers
static size_t crt_smem_bytes(int H, int P) {
  const size_t key_words = (KeyLayout(2 * H).total + 3) / 4 * 4;
  const size_t stage = (size_t)(H / 4) * 32 * 16;
  return key_words * 4 + (size_t)P * 2 * stage + (size_t)2 * P * stage;
}
static size_t crt_t_smem_bytes(int H, int T, int P) {
  const size_t key_words = (KeyLayout(2 * H).total + 3) / 4 * 4;
  const size_t stage = (size_t)(H / 4) * (32 / T) * 16;
  return key_words * 4 + (size_t)P * 2 * stage + (size_t)2 * P * stage;
}
static size_t pub_t_smem_bytes(int L, int T, int warps) {
  const size_t key_words = (KeyLayout(L).total + 3) / 4 * 4;
  return key_words * 4 + (size_t)warps * 2 * (L / 4) * (32 / T) * 16;
}
static size_t exp_smem_bytes(int L, int warps) {
  const size_t key_words = (KeyLayout(L).total + 3) / 4 * 4;
  const size_t stage = (size_t)(L / 4) * 32 * 16;
  return key_words * 4 + (size_t)warps * 2 * stage;
}

int Ctx::launch_grid(const void *fn, int threads, size_t smem, uint64_t units_per_cta_slot,
                     uint64_t units, int ctas_per_sm_req, int *grid_out) {
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (per_sm <= 0) return set_error(RSA_ERR_UNSUPPORTED, "kernel does not fit on an SM with this launch shape");
  if (ctas_per_sm_req > 0) per_sm = std::min(per_sm, ctas_per_sm_req);
  const uint64_t need = (units + units_per_cta_slot - 1) / units_per_cta_slot;
  *grid_out = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)sm_count * per_sm));
  return RSA_OK;
}

int Ctx::run_key(const KeySlot &k, int kind, uint64_t count, const uint32_t *msgs, uint32_t *out,
                 int32_t *status, cudaStream_t s) {
  if (count == 0) return RSA_OK;
  Workspace &w = ws(s);
  const uint32_t L = k.L;
  cudaError_t e;
  if (L == 1) {
    ToyArgs a{k.d_rec, msgs, out, status, (uint32_t)count, kind};
    const void *fn = toy_kernel_fn();
    int grid = (int)std::min<uint64_t>((count + 255) / 256, (uint64_t)sm_count * 8);
    void *args[] = {&a};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(256), args, 0, s);
    if (e != cudaSuccess) return cuda_error(e, "launch toy_kernel");
    stats.kernel_launches++;
    return RSA_OK;
  }
  Tune t = tune_for(k.nbits, kind);
  // At 3072/4096 bits a tensor-core launch costs a whole tile's exponentiation
  // (~80 ms at 4096 bits on GB300) however few operations it carries, while
  // the four-lane CUDA-core kernel's time grows with the count (6.7 us per
  // 4096-bit operation at full occupancy): the automatic choice takes the
  // tensor cores from tc4_auto_min_count operations up (an explicit variant 3
  // always does).
  if (t.variant == 3 && tc4::supported((int)L / 2) && count < tc4_auto_min_count(L)) {
    auto it = tuning.find({k.nbits, kind});
    if (it == tuning.end() || it->second.variant == 0) {
      t.variant = 0;
      t.tpo = 4;
      if (it == tuning.end() || it->second.window == 0) t.window = 5;
    }
  }
  // The public exponent of 2048-bit keys on the tensor cores (crt_tc4.cu): n has
  // the shape of an RSA-4096 prime, so each Montgomery product mod n runs the
  // same two reduction rounds.  variant 3 asks for it; automatically it takes
  // exponents up to kSlideMinBits bits (the binary method) in batches of at
  // least kPubTcMinCount operations.
  if (kind == RSA_EXP_PUBLIC && L == (uint32_t)tc4::kPubH && k.d_tcn) {
    const uint32_t e_bits = k.host_rec.size() > 7 ? k.host_rec[7] : 0u;
    if (t.variant == 3 || (t.variant == 0 && t.tpo <= 1 && e_bits <= kSlideMinBits && count >= kPubTcMinCount)) {
      if (count > 0xFFFFFFFFull) return set_error(RSA_ERR_ARG, "count out of range");
      const int grid = tc4::pub_tc4_grid((uint32_t)count, sm_count);
      int rc = ensure(w.tables, tc4::pub_tc4_tables_bytes(grid));
      if (rc) return rc;
      uint32_t polls = tcr::kDefaultWaitPolls;
      if (const char *ev = std::getenv("RSAGPU_TC_WAIT_POLLS")) polls = (uint32_t)std::strtoul(ev, nullptr, 10);
      e = tc4::launch_pub_tc4(k.d_rec, k.d_tcn, msgs, out, status, (uint32_t)count, grid, w.tables.ptr, polls, s);
      if (e != cudaSuccess) return cuda_error(e, "launch pub_tc4 kernel");
      stats.kernel_launches += 1;
      last_grid = grid;
      last_threads = tc4::kThreads;
      return RSA_OK;
    }
  }
  if (kind == RSA_EXP_PRIVATE_CRT && t.variant == 3 && tc4::supported((int)L / 2)) {
    // RSA-3072/4096: the Montgomery reduction on the tensor cores in two rounds (crt_tc4.cu)
    const int H = (int)L / 2;
    if (!k.d_tc) return set_error(RSA_ERR_UNSUPPORTED, "the tensor-core CRT path needs a key with p and q");
    if (count > 0xFFFFFFFFull) return set_error(RSA_ERR_ARG, "count out of range");
    if (t.window != 3 && t.window != 4)
      return set_error(RSA_ERR_UNSUPPORTED, "the tensor-core CRT path has windows 3 and 4");
    const int grid = tc4::tc4_grid((uint32_t)count, sm_count);
    int rc = ensure(w.tables, tc4::tc4_tables_bytes(H, grid, t.window));
    if (rc) return rc;
    rc = ensure(w.halves, tc4::tc4_halves_bytes(H, (uint32_t)count));
    if (rc) return rc;
    uint32_t polls = tcr::kDefaultWaitPolls;
    if (const char *ev = std::getenv("RSAGPU_TC_WAIT_POLLS")) polls = (uint32_t)std::strtoul(ev, nullptr, 10);
    e = tc4::launch_crt_tc4(H, k.d_rec, k.d_tc, msgs, out, status, (uint32_t)count, grid, t.window, w.tables.ptr,
                            w.halves.ptr, polls, s);
    if (e != cudaSuccess) return cuda_error(e, "launch crt_tc4 kernels");
    stats.kernel_launches += 2;
    last_grid = grid;
    last_threads = tc4::kThreads;
    return RSA_OK;
  }
  if (kind == RSA_EXP_PRIVATE_CRT && t.variant == 3) {
    // Montgomery reduction on the tensor cores (crt_tc.cu): 2048-bit keys
    if (L != 2 * (uint32_t)tcr::kH || !k.d_tc)
      return set_error(RSA_ERR_UNSUPPORTED, "the tensor-core CRT path needs a 2048- or 4096-bit key with p and q");
    if (count > 0xFFFFFFFFull) return set_error(RSA_ERR_ARG, "count out of range");
    if (t.window != 3 && t.window != 4)
      return set_error(RSA_ERR_UNSUPPORTED, "the tensor-core CRT path has windows 3 and 4");
    const int grid = tcr::tc_grid((uint32_t)count, sm_count);
    const int win = t.window;
    int rc = ensure(w.tables, tcr::tc_tables_bytes(grid, win));
    if (rc) return rc;
    rc = ensure(w.halves, tcr::tc_halves_bytes((uint32_t)count));
    if (rc) return rc;
    // RSAGPU_TC_WAIT_POLLS overrides the poll budget of the kernel's bounded
    // waits (0: every wait gives up at once), to exercise the timeout path
    uint32_t polls = tcr::kDefaultWaitPolls;
    if (const char *ev = std::getenv("RSAGPU_TC_WAIT_POLLS")) polls = (uint32_t)std::strtoul(ev, nullptr, 10);
    e = tcr::launch_crt_tc(k.d_rec, k.d_tc, msgs, out, status, (uint32_t)count, grid, win, w.tables.ptr,
                           w.halves.ptr, polls, s);
    if (e != cudaSuccess) return cuda_error(e, "launch crt_tc kernels");
    stats.kernel_launches += 2;
    last_grid = grid;
    last_threads = tcr::kThreads;
    return RSA_OK;
  }
  if (t.tpo > 1 && kind == RSA_EXP_PRIVATE_CRT) {
    const int H = (int)L / 2, T = t.tpo;
    const void *fn = crt_kernel_t_fn(H, T, t.window);
    if (!fn) return set_error(RSA_ERR_UNSUPPORTED, "no CRT kernel for this size / window / lanes per operation");
    const int P = std::max(1, t.warps_per_cta / 2);
    const int threads = 64 * P;
    const size_t smem = crt_t_smem_bytes(H, T, P);
    const uint64_t ntiles = (count + 32 / T - 1) / (32 / T);
    int grid = 0;
    int rc = launch_grid(fn, threads, smem, (uint64_t)P, ntiles, t.ctas_per_sm, &grid);
    if (rc) return rc;
    const size_t tbytes = (size_t)grid * 2 * P * ((size_t)1 << t.window) * (H / T) * 128;
    rc = ensure(w.tables, tbytes);
    if (rc) return rc;
    CrtArgs a{k.d_rec, msgs, out, status, (uint32_t)count, static_cast<uint4 *>(w.tables.ptr)};
    void *args[] = {&a};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
    if (e != cudaSuccess) return cuda_error(e, "launch crt_kernel_t");
    stats.kernel_launches++;
    last_grid = grid;
    last_threads = threads;
    return RSA_OK;
  }
  if (t.tpo > 1 && kind == RSA_EXP_PUBLIC) {
    const int T = t.tpo;
    const void *fn = pub_kernel_t_fn((int)L, T);
    if (!fn) return set_error(RSA_ERR_UNSUPPORTED, "no public kernel for this size / lanes per operation");
    const int warps = std::max(1, t.warps_per_cta);
    const int threads = 32 * warps;
    const size_t smem = pub_t_smem_bytes((int)L, T, warps);
    const uint64_t ntiles = (count + 32 / T - 1) / (32 / T);
    int grid = 0;
    int rc = launch_grid(fn, threads, smem, (uint64_t)warps, ntiles, t.ctas_per_sm, &grid);
    if (rc) return rc;
    ExpArgs a{k.d_rec, msgs, out, status, (uint32_t)count, nullptr};
    void *args[] = {&a};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
    if (e != cudaSuccess) return cuda_error(e, "launch pub_kernel_t");
    stats.kernel_launches++;
    last_grid = grid;
    last_threads = threads;
    return RSA_OK;
  }
  if (t.tpo > 1 && kind == RSA_EXP_PRIVATE_PLAIN) {
    // d mod n on T lanes per operation (3072/4096-bit moduli; window 4 or 5)
    const int T = t.tpo;
    const void *fn = plain_kernel_t_fn((int)L, T, t.window);
    if (!fn) return set_error(RSA_ERR_UNSUPPORTED, "no plain-exponent kernel for this size / window / lanes per operation");
    const int warps = std::max(1, t.warps_per_cta);
    const int threads = 32 * warps;
    const size_t smem = (KeyLayout(L).total + 3) / 4 * 4 * 4 + (size_t)warps * (L / 4) * (32 / T) * 16;
    const uint64_t ntiles = (count + 32 / T - 1) / (32 / T);
    int grid = 0;
    int rc = launch_grid(fn, threads, smem, (uint64_t)warps, ntiles, t.ctas_per_sm, &grid);
    if (rc) return rc;
    const size_t tbytes = (size_t)grid * warps * ((size_t)1 << t.window) * (L / T) * 128;
    rc = ensure(w.tables, tbytes);
    if (rc) return rc;
    ExpArgs a{k.d_rec, msgs, out, status, (uint32_t)count, static_cast<uint4 *>(w.tables.ptr)};
    void *args[] = {&a};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
    if (e != cudaSuccess) return cuda_error(e, "launch plain_kernel_t");
    stats.kernel_launches++;
    last_grid = grid;
    last_threads = threads;
    return RSA_OK;
  }
  if (kind == RSA_EXP_PRIVATE_CRT) {
    const int H = (int)L / 2;
    const void *fn = crt_kernel_fn(H, t.window, t.variant);
    if (!fn) return set_error(RSA_ERR_UNSUPPORTED, "no CRT kernel for this key size / window");
    const int P = std::max(1, t.warps_per_cta / 2);
    const int threads = 64 * P;
    const size_t smem = crt_smem_bytes(H, P);
    const uint64_t ntiles = (count + 31) / 32;
    int grid = 0;
    int rc = launch_grid(fn, threads, smem, (uint64_t)P, ntiles, t.ctas_per_sm, &grid);
    if (rc) return rc;
    const size_t tbytes = (size_t)grid * 2 * P * ((size_t)1 << t.window) * H * 128;
    rc = ensure(w.tables, tbytes);
    if (rc) return rc;
    CrtArgs a{k.d_rec, msgs, out, status, (uint32_t)count, static_cast<uint4 *>(w.tables.ptr)};
    void *args[] = {&a};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
    if (e != cudaSuccess) return cuda_error(e, "launch crt_kernel");
    stats.kernel_launches++;
    last_grid = grid;
    last_threads = threads;
    return RSA_OK;
  }
  const bool pub = (kind == RSA_EXP_PUBLIC);
  // public exponents: sliding windows (Fig. 7) for long exponents, where they
  // save multiplications; the binary method (Fig. 5) for short ones such as
  // 65537, where the window table would cost more than it saves
  const uint32_t e_bits = k.host_rec.size() > 7 ? k.host_rec[7] : 0u;
  const bool slide = pub && L <= 64 && (t.variant == 2 || (t.variant == 0 && e_bits > kSlideMinBits));
  const void *fn = pub ? (slide ? pub_slide_kernel_fn((int)L, t.window) : pub_kernel_fn((int)L))
                       : plain_kernel_fn((int)L, t.window, t.variant);
  if (!fn) return set_error(RSA_ERR_UNSUPPORTED, "no kernel for this key size / exponent kind / window");
  const int warps = std::max(1, t.warps_per_cta);
  const int threads = 32 * warps;
  const size_t smem = exp_smem_bytes((int)L, warps);
  const uint64_t ntiles = (count + 31) / 32;
  int grid = 0;
  int rc = launch_grid(fn, threads, smem, (uint64_t)warps, ntiles, t.ctas_per_sm, &grid);
  if (rc) return rc;
  uint4 *tables = nullptr;
  if (!pub || slide) {
    const size_t entries = slide ? ((size_t)1 << (t.window - 1)) : ((size_t)1 << t.window);
    const size_t tbytes = (size_t)grid * warps * entries * L * 128;
    rc = ensure(w.tables, tbytes);
    if (rc) return rc;
    tables = static_cast<uint4 *>(w.tables.ptr);
  }
  ExpArgs a{k.d_rec, msgs, out, status, (uint32_t)count, tables};
  void *args[] = {&a};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
  if (e != cudaSuccess) return cuda_error(e, pub ? "launch public-exponent kernel" : "launch plain_kernel");
  stats.kernel_launches++;
  last_grid = grid;
  last_threads = threads;
  return RSA_OK;
}

int Ctx::check_key(int32_t key_id, int kind, const KeySlot **out) {
  if (key_id < 0 || (size_t)key_id >= keys.size() || !keys[key_id].used)
    return set_error(RSA_ERR_KEY, "unknown key id " + std::to_string(key_id));
  const KeySlot &k = keys[key_id];
  if (kind != RSA_EXP_PUBLIC && kind != RSA_EXP_PRIVATE_CRT && kind != RSA_EXP_PRIVATE_PLAIN)
    return set_error(RSA_ERR_ARG, "bad exp_sel " + std::to_string(kind));
  if (kind != RSA_EXP_PUBLIC && !(k.flags & KEY_HAS_D))
    return set_error(RSA_ERR_KEY, "private operation on a key loaded without d");
  if (kind == RSA_EXP_PRIVATE_CRT && !(k.flags & KEY_HAS_CRT))
    return set_error(RSA_ERR_KEY, "CRT operation on a key loaded without p, q");
  *out = &k;
  return RSA_OK;
}

}  // namespace rsagpu

using namespace rsagpu;

// ====================================================================== C ABI
extern "C" {

int rsa_ctx_create(rsa_ctx **out, int device, size_t mem_budget_bytes) {
  if (!out) return set_error(RSA_ERR_ARG, "out is null");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return set_error(RSA_ERR_ARG, "no such CUDA device");
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  Ctx *c = new Ctx();
  c->device = device;
  c->budget = mem_budget_bytes ? mem_budget_bytes : ((size_t)2 << 30);
  e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_error(e, "cudaDeviceGetAttribute");
  }
  *out = reinterpret_cast<rsa_ctx *>(c);
  return RSA_OK;
}

int rsa_ctx_destroy(rsa_ctx *ctx) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  if (reinterpret_cast<Ctx *>(ctx)->server) rsa_server_stop(ctx);
  delete reinterpret_cast<Ctx *>(ctx);
  return RSA_OK;
}

static int make_record(uint32_t nbits, const uint32_t *n, const uint32_t *e, uint32_t e_limbs,
                       const uint32_t *d, const uint32_t *p, const uint32_t *q, std::vector<uint32_t> &rec,
                       uint32_t &flags) {
  if (!n || !e) return set_error(RSA_ERR_ARG, "null argument");
  if ((p == nullptr) != (q == nullptr)) return set_error(RSA_ERR_ARG, "p and q must both be given or both be null");
  if (nbits % 32 != 0 || nbits == 0 || nbits > 4096) return set_error(RSA_ERR_UNSUPPORTED, "unsupported key size");
  const uint32_t L = nbits / 32;
  if (e_limbs == 0 || e_limbs > L) return set_error(RSA_ERR_ARG, "e_limbs must be in 1..L");
  KeyInput in;
  in.nbits = nbits;
  in.n.assign(n, n + L);
  in.e.assign(e, e + e_limbs);
  if (d) in.d.assign(d, d + L);
  const uint32_t hl = (L == 1) ? 1u : L / 2;
  if (p) {
    in.p.assign(p, p + hl);
    in.q.assign(q, q + hl);
  }
  char cls = 0;
  std::string msg = build_key_record(in, rec, flags, &cls);
  if (!msg.empty())
    return set_error(cls == 'U' ? RSA_ERR_UNSUPPORTED : cls == 'A' ? RSA_ERR_ARG : RSA_ERR_KEY, msg);
  return RSA_OK;
}

int rsa_tc_round_operand_image(uint32_t prime_bits, const uint32_t *m, void *out, size_t out_bytes) {
  if (!m || !out) return set_error(RSA_ERR_ARG, "null pointer");
  if (prime_bits != 1536 && prime_bits != 2048) return set_error(RSA_ERR_ARG, "prime_bits must be 1536 or 2048");
  const int H = (int)prime_bits / 32;
  if (out_bytes < tc4::img_prime_bytes(H)) return set_error(RSA_ERR_ARG, "output buffer too small");
  if (!tc4::build_tc4_image(m, H, static_cast<uint8_t *>(out))) return set_error(RSA_ERR_ARG, "modulus must be odd");
  return RSA_OK;
}

int rsa_tc_operand_image(const uint32_t *m, void *out, size_t out_bytes) {
  if (!m || !out) return set_error(RSA_ERR_ARG, "null argument");
  if (out_bytes < tcr::kImgPrime) return set_error(RSA_ERR_ARG, "output buffer too small");
  if (!tcr::build_tc_image(m, static_cast<uint8_t *>(out))) return set_error(RSA_ERR_ARG, "modulus must be odd");
  return RSA_OK;
}

int rsa_key_record(uint32_t nbits, const uint32_t *n, const uint32_t *e, uint32_t e_limbs, const uint32_t *d,
                   const uint32_t *p, const uint32_t *q, uint32_t *rec, size_t rec_capacity_words,
                   size_t *rec_words) {
  std::vector<uint32_t> r;
  uint32_t flags = 0;
  int rc = make_record(nbits, n, e, e_limbs, d, p, q, r, flags);
  if (rc) return rc;
  if (rec_words) *rec_words = r.size();
  if (!rec) return RSA_OK;
  if (rec_capacity_words < r.size()) return set_error(RSA_ERR_ARG, "record buffer too small");
  std::copy(r.begin(), r.end(), rec);
  return RSA_OK;
}

int rsa_keyload(rsa_ctx *ctx, uint32_t nbits, const uint32_t *n, const uint32_t *e, uint32_t e_limbs,
                const uint32_t *d, const uint32_t *p, const uint32_t *q, int32_t *key_id_out) {
  if (!ctx || !key_id_out) return set_error(RSA_ERR_ARG, "null argument");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  std::vector<uint32_t> rec;
  uint32_t flags = 0;
  int rc0 = make_record(nbits, n, e, e_limbs, d, p, q, rec, flags);
  if (rc0) return rc0;
  const uint32_t L = nbits / 32;
  const size_t bytes = rec.size() * 4;
  int rc = c->reserve(bytes);
  if (rc) return rc;
  cudaSetDevice(c->device);
  uint32_t *dptr = nullptr;
  cudaError_t ce = cudaMalloc(&dptr, bytes);
  if (ce != cudaSuccess) {
    c->release(bytes);
    cudaGetLastError();
    return set_error(RSA_ERR_NOMEM, std::string("cudaMalloc key record: ") + cudaGetErrorString(ce));
  }
  ce = cudaMemcpy(dptr, rec.data(), bytes, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    cudaFree(dptr);
    c->release(bytes);
    return cuda_error(ce, "cudaMemcpy key record");
  }
  // tensor-core operand images of q and p for the RSA-2048 and RSA-4096 CRT paths
  void *dtc = nullptr;
  size_t tc_bytes = 0;
  const int Hk = (int)L / 2;
  if ((L == 2 * (uint32_t)tcr::kH || tc4::supported(Hk)) && (flags & KEY_HAS_CRT)) {
    const bool rounds = tc4::supported(Hk);
    const KeyLayout lay(L);
    std::vector<uint8_t> img(rounds ? tc4::img_key_bytes(Hk) : tcr::kImgKey);
    const bool ok = rounds ? tc4::build_tc4_image(rec.data() + lay.q, Hk, img.data()) &&
                                 tc4::build_tc4_image(rec.data() + lay.p, Hk, img.data() + tc4::img_prime_bytes(Hk))
                           : tcr::build_tc_image(rec.data() + lay.q, img.data()) &&
                                 tcr::build_tc_image(rec.data() + lay.p, img.data() + tcr::kImgPrime);
    int rc2 = ok ? c->reserve(img.size()) : set_error(RSA_ERR_KEY, "p and q must be odd");
    if (rc2 == RSA_OK) {
      if (cudaMalloc(&dtc, img.size()) == cudaSuccess &&
          cudaMemcpy(dtc, img.data(), img.size(), cudaMemcpyHostToDevice) == cudaSuccess) {
        tc_bytes = img.size();
      } else {
        if (dtc) cudaFree(dtc);
        dtc = nullptr;
        cudaGetLastError();
        c->release(img.size());
        rc2 = set_error(RSA_ERR_NOMEM, "device allocation of the tensor-core operands failed");
      }
    }
    if (rc2 != RSA_OK) {
      cudaFree(dptr);
      c->release(bytes);
      return rc2;
    }
  }
  // n's two-round tensor-core operands: the public exponent of 2048-bit keys
  void *dtcn = nullptr;
  size_t tcn_bytes = 0;
  if (L == (uint32_t)tc4::kPubH) {
    const KeyLayout lay(L);
    std::vector<uint8_t> img(tc4::img_prime_bytes(tc4::kPubH));
    int rc3 = tc4::build_tc4_image(rec.data() + lay.n, tc4::kPubH, img.data()) ? c->reserve(img.size())
                                                                              : set_error(RSA_ERR_KEY, "n must be odd");
    if (rc3 == RSA_OK) {
      if (cudaMalloc(&dtcn, img.size()) == cudaSuccess &&
          cudaMemcpy(dtcn, img.data(), img.size(), cudaMemcpyHostToDevice) == cudaSuccess) {
        tcn_bytes = img.size();
      } else {
        if (dtcn) cudaFree(dtcn);
        dtcn = nullptr;
        cudaGetLastError();
        c->release(img.size());
        rc3 = set_error(RSA_ERR_NOMEM, "device allocation of the tensor-core operands failed");
      }
    }
    if (rc3 != RSA_OK) {
      if (dtc) {
        cudaFree(dtc);
        c->release(tc_bytes);
      }
      cudaFree(dptr);
      c->release(bytes);
      return rc3;
    }
  }
  int32_t id = -1;
  for (size_t i = 0; i < c->keys.size(); ++i)
    if (!c->keys[i].used) {
      id = (int32_t)i;
      break;
    }
  if (id < 0) {
    id = (int32_t)c->keys.size();
    c->keys.emplace_back();
  }
  KeySlot &k = c->keys[id];
  k.used = true;
  k.nbits = nbits;
  k.L = L;
  k.flags = flags;
  k.d_rec = dptr;
  k.bytes = bytes;
  k.host_rec = rec;
  k.d_tc = dtc;
  k.tc_bytes = tc_bytes;
  k.d_tcn = dtcn;
  k.tcn_bytes = tcn_bytes;
  c->key_epoch++;
  *key_id_out = id;
  return RSA_OK;
}

int rsa_keyunload(rsa_ctx *ctx, int32_t key_id) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  if (key_id < 0 || (size_t)key_id >= c->keys.size() || !c->keys[key_id].used)
    return set_error(RSA_ERR_KEY, "unknown key id");
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  KeySlot &k = c->keys[key_id];
  cudaFree(k.d_rec);
  c->release(k.bytes);
  if (k.d_tc) {
    cudaFree(k.d_tc);
    c->release(k.tc_bytes);
  }
  if (k.d_tcn) {
    cudaFree(k.d_tcn);
    c->release(k.tcn_bytes);
  }
  k = KeySlot();
  c->key_epoch++;
  return RSA_OK;
}

int rsa_key_info(rsa_ctx *ctx, int32_t key_id, uint32_t *nbits, int32_t *has_d, int32_t *has_crt) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  if (key_id < 0 || (size_t)key_id >= c->keys.size() || !c->keys[key_id].used)
    return set_error(RSA_ERR_KEY, "unknown key id");
  const KeySlot &k = c->keys[key_id];
  if (nbits) *nbits = k.nbits;
  if (has_d) *has_d = (k.flags & KEY_HAS_D) ? 1 : 0;
  if (has_crt) *has_crt = (k.flags & KEY_HAS_CRT) ? 1 : 0;
  return RSA_OK;
}

int rsa_modexp_key(rsa_ctx *ctx, int32_t key_id, int32_t exp_sel, uint64_t count, const uint32_t *msgs,
                   uint32_t *out, int32_t *op_status, void *stream) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  if (count > 0 && (!msgs || !out)) return set_error(RSA_ERR_ARG, "null message or output pointer");
  if (count > 0x7fffffffull) return set_error(RSA_ERR_ARG, "count exceeds 2^31 - 1");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  const KeySlot *k = nullptr;
  int rc = c->check_key(key_id, exp_sel, &k);
  if (rc) return rc;
  if (k->L > 1 && ((reinterpret_cast<uintptr_t>(msgs) | reinterpret_cast<uintptr_t>(out)) & 15u))
    return set_error(RSA_ERR_ARG, "message and output rows must be 16-byte aligned");
  cudaSetDevice(c->device);
  c->stats.ops += count;
  NvtxRange range("rsa_modexp_key");
  return c->run_key(*k, exp_sel, count, msgs, out, op_status, static_cast<cudaStream_t>(stream));
}

int rsa_modexp_key_host(rsa_ctx *ctx, int32_t key_id, int32_t exp_sel, uint64_t count, const uint32_t *msgs,
                        uint32_t *out, int32_t *op_status, void *stream) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  if (count > 0 && (!msgs || !out)) return set_error(RSA_ERR_ARG, "null message or output pointer");
  if (count > 0x7fffffffull) return set_error(RSA_ERR_ARG, "count exceeds 2^31 - 1");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  const KeySlot *k = nullptr;
  int rc = c->check_key(key_id, exp_sel, &k);
  if (rc) return rc;
  if (count == 0) return RSA_OK;
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Workspace &w = c->ws(s);
  const size_t bytes = (size_t)count * k->L * 4;
  if ((rc = c->ensure(w.io_in, bytes)) || (rc = c->ensure(w.io_out, bytes))) return rc;
  if (op_status && (rc = c->ensure(w.io_status, (size_t)count * 4))) return rc;
  cudaError_t e = cudaMemcpyAsync(w.io_in.ptr, msgs, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync H2D");
  c->stats.ops += count;
  rc = c->run_key(*k, exp_sel, count, static_cast<uint32_t *>(w.io_in.ptr), static_cast<uint32_t *>(w.io_out.ptr),
                  op_status ? static_cast<int32_t *>(w.io_status.ptr) : nullptr, s);
  if (rc) return rc;
  e = cudaMemcpyAsync(out, w.io_out.ptr, bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync D2H");
  if (op_status) {
    e = cudaMemcpyAsync(op_status, w.io_status.ptr, (size_t)count * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync D2H status");
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  return RSA_OK;
}

int rsa_sync(rsa_ctx *ctx, void *stream) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  cudaSetDevice(c->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  std::lock_guard<std::mutex> lock(c->mu);
  return c->collect_device_errors(static_cast<cudaStream_t>(stream));
}

const char *rsa_last_error(void) { return g_last_error.c_str(); }

int rsa_set_tuning(rsa_ctx *ctx, uint32_t nbits, int32_t exp_sel, const rsa_tuning *t) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  if (!t) {
    c->tuning.erase({nbits, exp_sel});
    return RSA_OK;
  }
  if (t->window && (t->window < kMinWindow || t->window > kMaxWindow))
    return set_error(RSA_ERR_ARG, "window out of range");
  if (t->warps_per_cta < 0 || t->warps_per_cta > 8 || t->ctas_per_sm < 0)
    return set_error(RSA_ERR_ARG, "bad launch shape");
  if (t->variant < 0 || t->variant > 3) return set_error(RSA_ERR_ARG, "variant must be 0 .. 3");
  if (!(t->threads_per_op == 0 || t->threads_per_op == 1 || t->threads_per_op == 2 || t->threads_per_op == 4))
    return set_error(RSA_ERR_ARG, "threads_per_op must be 0, 1, 2 or 4");
  if (exp_sel == RSA_TUNE_RAGGED) {
    if (t->threads_per_op == 2)
      return set_error(RSA_ERR_ARG, "ragged batches: threads_per_op must be 0 (automatic), 1 or 4");
    if (!(t->window == 0 || t->window == 4 || t->window == 5) || !(t->window_big == 0 || t->window_big == 4 ||
                                                                   t->window_big == 5))
      return set_error(RSA_ERR_ARG, "ragged batches: CRT windows must be 0 (automatic), 4 or 5");
    if (!(t->window_tc == 0 || t->window_tc == 3 || t->window_tc == 4))
      return set_error(RSA_ERR_ARG, "ragged batches: the tensor-core window must be 0 (automatic), 3 or 4");
    if (!(t->variant == 0 || t->variant == 1 || t->variant == 3))
      return set_error(RSA_ERR_ARG, "ragged batches: variant must be 0 (automatic), 1 or 3");
    if (t->tc_min_ops < 0) return set_error(RSA_ERR_ARG, "ragged batches: tc_min_ops must be >= 0");
  } else if (t->window_big || t->window_tc || t->tc_min_ops) {
    return set_error(RSA_ERR_ARG, "window_big, window_tc and tc_min_ops apply to RSA_TUNE_RAGGED only");
  }
  if (exp_sel == RSA_EXP_PRIVATE_CRT && (t->warps_per_cta & 1))
    return set_error(RSA_ERR_ARG, "CRT kernels run warp pairs: warps_per_cta must be even");
  c->tuning[{nbits, exp_sel}] = Tune{t->window,     t->warps_per_cta, t->ctas_per_sm, t->variant,
                                     t->threads_per_op, t->window_big, t->window_tc,  t->tc_min_ops};
  return RSA_OK;
}

int rsa_get_tuning(rsa_ctx *ctx, uint32_t nbits, int32_t exp_sel, rsa_tuning *t) {
  if (!ctx || !t) return set_error(RSA_ERR_ARG, "null argument");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  Tune x = c->tune_for(nbits, exp_sel);
  t->window = x.window;
  t->warps_per_cta = x.warps_per_cta;
  t->ctas_per_sm = x.ctas_per_sm;
  t->variant = x.variant;
  t->threads_per_op = x.tpo;
  t->window_big = x.window_big;
  t->window_tc = x.window_tc;
  t->tc_min_ops = x.tc_min_ops;
  return RSA_OK;
}

int rsa_get_stats(rsa_ctx *ctx, rsa_stats *s) {
  if (!ctx || !s) return set_error(RSA_ERR_ARG, "null argument");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  *s = c->stats;
  s->bytes_resident = c->used;
  return RSA_OK;
}

double rsa_products_per_op(uint32_t nbits, int32_t exp_sel, uint32_t e_bits, uint32_t e_weight, int32_t window) {
  const double L = nbits / 32.0;
  auto mm = [](double l) { return 2.0 * l * l + l; };
  const int W = window > 0 ? window : 5;
  if (exp_sel == RSA_EXP_PUBLIC) {
    if (e_bits == 0) return 0.0;
    const double mults = 2.0 + (e_bits - 1) + (e_weight > 0 ? e_weight - 1 : 0);
    return mults * mm(L);
  }
  if (exp_sel == RSA_EXP_PRIVATE_PLAIN) {
    const double nwin = std::ceil(32.0 * L / W);
    const double mults = 2.0 + ((1 << W) - 2) + (nwin - 1) * (W + 1);
    return mults * mm(L);
  }
  const double H = L / 2.0;
  const double nwin = std::ceil(32.0 * H / W);
  const double per_half = 2.0 + ((1 << W) - 2) + (nwin - 1) * (W + 1);
  return (2.0 * per_half + 3.0) * mm(H) + H * H;
}

int rsa_imad_probe(int device, double *imad_lanes_per_s, double *chain_products_per_s) {
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  uint32_t *sink = nullptr;
  const int threads = 256, blocks = sms * 8;
  e = cudaMalloc(&sink, (size_t)threads * blocks * 4);
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc probe");
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto run = [&](const void *fn, uint32_t iters, int nblocks, int nthreads, float *ms) -> cudaError_t {
    uint32_t seed = 12345u;
    void *args[] = {&sink, &iters, &seed};
    cudaError_t r = cudaLaunchKernel(fn, dim3(nblocks), dim3(nthreads), args, 0, nullptr);  // warm-up
    if (r != cudaSuccess) return r;
    cudaEventRecord(a);
    r = cudaLaunchKernel(fn, dim3(nblocks), dim3(nthreads), args, 0, nullptr);
    if (r != cudaSuccess) return r;
    cudaEventRecord(b);
    r = cudaEventSynchronize(b);
    cudaEventElapsedTime(ms, a, b);
    return r;
  };
  float ms1 = 0;
  const uint32_t it1 = 20000, it2 = 4000;
  e = run(imad_probe_fn(), it1, blocks, threads, &ms1);
  // the carry-chain rows at two occupancies (as many CTAs of 256 threads as
  // fit; 16 warps per SM), the faster counts
  double chain = 0.0;
  const int shapes[2][2] = {{blocks, threads}, {sms, 512}};
  for (const auto &sh : shapes) {
    if (e != cudaSuccess) break;
    float ms2 = 0;
    e = run(chain_probe_fn(), it2, sh[0], sh[1], &ms2);
    if (e == cudaSuccess) chain = std::max(chain, (double)sh[0] * sh[1] * it2 * 32.0 / (ms2 * 1e-3));
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_error(e, "probe kernel");
  const double thr = (double)threads * blocks;
  if (imad_lanes_per_s) *imad_lanes_per_s = thr * it1 * 16.0 / (ms1 * 1e-3);
  if (chain_products_per_s) *chain_products_per_s = chain;
  return RSA_OK;
}

}  // extern "C"
