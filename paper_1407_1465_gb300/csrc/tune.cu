// tune.cu -- rsa_autotune: times launch shapes of the uniform kernels and
// keeps the fastest, with a small text cache keyed by GPU and problem class.
//
// Cache lines: "<gpu name>|<sm count>|<nbits>|<kind>|<log2 count bucket> window warps ctas variant tpo ms"
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <iomanip>
#include <sstream>
#include <string>
#include <vector>

#include "runtime_internal.h"

namespace rsagpu {
namespace {

std::string cache_key(int device, int sms, uint32_t nbits, int kind, uint64_t count) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, device);
  std::string name(prop.name);
  for (char &c : name)
    if (c == '|' || c == ' ') c = '_';
  const int bucket = count ? (int)std::floor(std::log2((double)count)) : 0;
  std::ostringstream os;
  os << name << "|" << sms << "|" << nbits << "|" << kind << "|" << bucket;
  return os.str();
}

bool cache_lookup(const std::string &path, const std::string &key, Tune *t, double *ms) {
  std::ifstream f(path);
  if (!f) return false;
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string k;
    Tune x{};
    double m = 0;
    if (!(is >> k >> x.window >> x.warps_per_cta >> x.ctas_per_sm >> x.variant >> x.tpo >> m)) continue;
    if (k == key) {
      *t = x;
      *ms = m;
      found = true;  // last entry wins
    }
  }
  return found;
}

}  // namespace
}  // namespace rsagpu

using namespace rsagpu;

extern "C" int rsa_autotune(rsa_ctx *ctx, int32_t key_id, int32_t exp_sel, uint64_t count, const char *cache_path,
                            rsa_tuning *best, double *best_ms) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  if (count == 0 || count > (1u << 24)) return set_error(RSA_ERR_ARG, "count must be in 1..2^24");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::unique_lock<std::mutex> lock(c->mu);
  const KeySlot *k = nullptr;
  int rc = c->check_key(key_id, exp_sel, &k);
  if (rc) return rc;
  if (k->L == 1) return set_error(RSA_ERR_UNSUPPORTED, "single-limb keys have no launch parameters to tune");
  const uint32_t nbits = k->nbits, L = k->L;
  const std::string path = cache_path ? cache_path : (std::getenv("RSA_TUNE_CACHE") ? std::getenv("RSA_TUNE_CACHE") : "");
  const std::string key = cache_key(c->device, c->sm_count, nbits, exp_sel, count);
  Tune chosen{};
  double chosen_ms = 0;
  if (!path.empty() && cache_lookup(path, key, &chosen, &chosen_ms)) {
    c->tuning[{nbits, exp_sel}] = chosen;
  } else {
    cudaSetDevice(c->device);
    const size_t bytes = (size_t)count * L * 4;
    DevBuf in, out;
    if ((rc = c->ensure(in, bytes)) || (rc = c->ensure(out, bytes))) {
      if (in.ptr) { cudaFree(in.ptr); c->release(in.bytes); }
      return rc;
    }
    // messages 0x01010101...: below any modulus of full bit length
    cudaMemset(in.ptr, 0x01, bytes);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const Tune saved = c->tune_for(nbits, exp_sel);
    const bool priv = exp_sel != RSA_EXP_PUBLIC;
    std::vector<int> windows = priv ? std::vector<int>{3, 4, 5, 6} : std::vector<int>{0};
    std::vector<int> warps = exp_sel == RSA_EXP_PRIVATE_CRT ? std::vector<int>{2, 4, 8} : std::vector<int>{1, 2, 4, 8};
    std::vector<int> variants = priv ? std::vector<int>{1, 2} : std::vector<int>{0};
    if (exp_sel == RSA_EXP_PRIVATE_CRT && k->d_tc) variants.push_back(3);
    double best_t = 1e30;
    int err = RSA_OK;
    for (int tpo : {1, 2, 4})
    for (int v : variants)
      for (int w : windows)
        for (int wp : warps)
          for (int cps : {0, 1, 2}) {
            if (tpo > 1 && v == 2) continue;  // not offered (shapes without a kernel fail below and are skipped)
            // the tensor-core path has its own fixed launch shape and windows 3, 4
            if (v == 3 && (tpo != 1 || wp != warps[0] || cps != 0 || (w != 3 && w != 4))) continue;
            c->tuning[{nbits, exp_sel}] = Tune{w, wp, cps, v, tpo};
            // warm-up, then the median of three timed runs
            if (c->run_key(*k, exp_sel, count, static_cast<uint32_t *>(in.ptr), static_cast<uint32_t *>(out.ptr),
                           nullptr, s) != RSA_OK)
              continue;  // shape not available (kernel not instantiated or does not fit)
            float t3[3];
            for (int r = 0; r < 3; ++r) {
              cudaEventRecord(a, s);
              c->run_key(*k, exp_sel, count, static_cast<uint32_t *>(in.ptr), static_cast<uint32_t *>(out.ptr),
                         nullptr, s);
              cudaEventRecord(b, s);
              cudaError_t e = cudaEventSynchronize(b);
              if (e != cudaSuccess) {
                err = cuda_error(e, "autotune run");
                break;
              }
              cudaEventElapsedTime(&t3[r], a, b);
            }
            if (err) break;
            std::sort(t3, t3 + 3);
            if (t3[1] < best_t) {
              best_t = t3[1];
              chosen = Tune{w, wp, cps, v, tpo};
            }
          }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    c->release_stream(s);
    cudaStreamDestroy(s);
    cudaFree(in.ptr);
    c->release(in.bytes);
    cudaFree(out.ptr);
    c->release(out.bytes);
    if (err) {
      c->tuning[{nbits, exp_sel}] = saved;
      return err;
    }
    if (best_t >= 1e29) {
      c->tuning[{nbits, exp_sel}] = saved;
      return set_error(RSA_ERR_UNSUPPORTED, "no launch shape ran for this key size and kind");
    }
    chosen_ms = best_t;
    c->tuning[{nbits, exp_sel}] = chosen;
    if (!path.empty()) {
      std::ofstream f(path, std::ios::app);
      f.precision(17);
      f << key << " " << chosen.window << " " << chosen.warps_per_cta << " " << chosen.ctas_per_sm << " "
        << chosen.variant << " " << chosen.tpo << " " << chosen_ms << "\n";
    }
  }
  if (best) {
    best->window = chosen.window;
    best->warps_per_cta = chosen.warps_per_cta;
    best->ctas_per_sm = chosen.ctas_per_sm;
    best->variant = chosen.variant;
    best->threads_per_op = chosen.tpo;
  }
  if (best_ms) *best_ms = chosen_ms;
  return RSA_OK;
}

// Ragged batches: coordinate descent over the RSA_TUNE_RAGGED tuning on the
// caller's own batch.  Each parameter in turn takes every value it may have
// while the others keep their best values so far: the lanes-per-operation
// policy of the long CRT sizes, the tensor-core group (off / on, the smallest
// bucket it takes, its window), the CRT windows of 1024/2048-bit and of
// 3072/4096-bit keys, and the cap on resident CTAs per SM of the persistent
// groups.  A candidate is the median of three timed runs after a warm-up; its
// results must equal the first candidate's (a digest of every output row), or
// the candidate is not taken.
extern "C" int rsa_autotune_batch(rsa_ctx *ctx, uint64_t count, const int32_t *key_ids, const uint8_t *exp_sel,
                                  const uint64_t *limb_offsets, const uint32_t *msgs, uint32_t *out,
                                  rsa_tuning *best, double *best_ms) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  if (count == 0 || count > 0x7fffffffull) return set_error(RSA_ERR_ARG, "count must be in 1..2^31-1");
  if (!key_ids || !exp_sel || !limb_offsets || !msgs || !out) return set_error(RSA_ERR_ARG, "null pointer");
  if ((reinterpret_cast<uintptr_t>(msgs) | reinterpret_cast<uintptr_t>(out)) & 15u)
    return set_error(RSA_ERR_ARG, "message and output buffers must be 16-byte aligned");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  std::lock_guard<std::mutex> lock(c->mu);
  cudaSetDevice(c->device);
  const std::pair<uint32_t, int> tk{0u, RSA_TUNE_RAGGED};
  const bool had = c->tuning.count(tk) != 0;
  const Tune saved = had ? c->tuning[tk] : Tune{};
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_error(e, "autotune stream");
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  int err = RSA_OK;
  bool have_ref = false;
  uint64_t ref_digest = 0;
  int mismatches = 0;
  // time one candidate: the median of three runs (infinite if it does not run or disagrees)
  auto measure = [&](const Tune &cand) -> double {
    c->tuning[tk] = cand;
    if (c->run_batch(count, key_ids, exp_sel, limb_offsets, msgs, out, nullptr, s) != RSA_OK) return 1e30;
    uint64_t dg = 0;
    if ((err = c->batch_digest(count, key_ids, limb_offsets, out, s, &dg))) return 1e30;
    if (!have_ref) {
      have_ref = true;
      ref_digest = dg;
    } else if (dg != ref_digest) {
      ++mismatches;
      return 1e30;
    }
    float t3[3];
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(a, s);
      if ((err = c->run_batch(count, key_ids, exp_sel, limb_offsets, msgs, out, nullptr, s))) return 1e30;
      cudaEventRecord(b, s);
      if ((e = cudaEventSynchronize(b)) != cudaSuccess) {
        err = cuda_error(e, "autotune batch run");
        return 1e30;
      }
      cudaEventElapsedTime(&t3[r], a, b);
    }
    std::sort(t3, t3 + 3);
    return t3[1];
  };
  struct Dim {
    int Tune::*field;
    std::vector<int> values;
  };
  const Dim dims[] = {{&Tune::tpo, {1, 4}},          {&Tune::variant, {0, 1, 3}},    {&Tune::tc_min_ops, {128, 512}},
                      {&Tune::window_tc, {3, 4}},     {&Tune::window, {4, 5}},        {&Tune::window_big, {5, 4}},
                      {&Tune::ctas_per_sm, {0, 2, 4}}};
  Tune chosen{};
  chosen.window = 4;
  chosen.window_big = 5;
  chosen.window_tc = 3;
  chosen.tc_min_ops = 128;
  chosen.tpo = 1;
  double best_t = measure(chosen);
  int candidates = 1;
  for (const Dim &d : dims) {
    if (err) break;
    const int incumbent = chosen.*(d.field);
    for (int v : d.values) {
      if (v == incumbent) continue;
      Tune cand = chosen;
      cand.*(d.field) = v;
      const double t = measure(cand);
      ++candidates;
      if (err) break;
      if (t < best_t) {
        best_t = t;
        chosen = cand;
      }
    }
  }
  // operations the batch itself rejects leave error bits on the stream: read
  // and clear them so they do not surface at the caller's next rsa_sync
  if (!err) err = c->collect_device_errors(s);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  c->release_stream(s);
  cudaStreamDestroy(s);
  if (err || best_t >= 1e29) {
    if (had) c->tuning[tk] = saved;
    else c->tuning.erase(tk);
    return err ? err : set_error(RSA_ERR_UNSUPPORTED, "no launch shape ran for this batch");
  }
  if (mismatches)
    return set_error(RSA_ERR_CUDA, "ragged autotuner: " + std::to_string(mismatches) + " of " +
                                       std::to_string(candidates) + " configurations gave different results");
  c->tuning[tk] = chosen;
  if (best) {
    best->window = chosen.window;
    best->warps_per_cta = 0;
    best->ctas_per_sm = chosen.ctas_per_sm;
    best->variant = chosen.variant;
    best->threads_per_op = chosen.tpo;
    best->window_big = chosen.window_big;
    best->window_tc = chosen.window_tc;
    best->tc_min_ops = chosen.tc_min_ops;
  }
  if (best_ms) *best_ms = best_t;
  return RSA_OK;
}
