// server.cu -- the request loop (rsa_server_*): arrival replay, admission by
// device-memory budget, continuous batching over several streams, latency
// accounting.  Host code; the GPU work of each batch is rsa_modexp_batch's
// graph (batch.cu) on the slot's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "keyrec.h"
#include "runtime_internal.h"

namespace rsagpu {
namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Req {
  uint64_t ticket = 0;
  int32_t key_id = 0, exp_sel = 0;
  uint32_t count = 0, L = 0;
  const uint32_t *msgs = nullptr;
  uint32_t *out = nullptr;
  int32_t *status = nullptr;
  uint64_t arrive = 0;   // steady-clock ns
  int32_t state = 0;     // 0 queued, 1 in flight, 2 done, < 0 failed
  uint64_t done = 0;
};

// First-fit allocator over the byte range [0, size) of the in-flight arenas
// (host-side bookkeeping only); ranges are multiples of 256 bytes and freed
// ranges merge with their neighbours.
class Arena {
 public:
  void init(size_t size) {
    free_.clear();
    size_ = size / 256 * 256;
    if (size_) free_[0] = size_;
  }
  size_t size() const { return size_; }
  size_t largest() const {
    size_t m = 0;
    for (const auto &kv : free_) m = std::max(m, kv.second);
    return m;
  }
  bool alloc(size_t n, size_t *off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      *off = it->first;
      const size_t rest = it->second - n;
      const size_t at = it->first + n;
      free_.erase(it);
      if (rest) free_[at] = rest;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t n) {
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + n == next->first) {
      n += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += n;
        return;
      }
    }
    free_[off] = n;
  }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Bytes a batch of `ops` operations and `limbs` message limbs takes in the
// arenas: key ids, kinds, row offsets and statuses (each 256-byte aligned),
// then messages and results of `limbs` limbs each (rounded up to 4 limbs).
size_t batch_bytes(uint64_t ops, uint64_t limbs) {
  const uint64_t l4 = (limbs + 3) / 4 * 4;
  return align256(ops * 4) + align256(ops) + align256(ops * 8) + align256(ops * 4) + align256(l4 * 4) * 2;
}

// one in-flight batch: a stream, its range of the arenas and the requests it carries
struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  size_t off = 0, len = 0;              // the batch's range of the arenas
  // views into the pinned host arena and the device arena at [off, off + len)
  int32_t *h_keys = nullptr;
  uint8_t *h_sel = nullptr;
  uint64_t *h_off = nullptr;
  uint32_t *h_msgs = nullptr, *h_out = nullptr;
  int32_t *h_status = nullptr;
  int32_t *d_keys = nullptr;
  uint8_t *d_sel = nullptr;
  uint64_t *d_off = nullptr;
  uint32_t *d_msgs = nullptr, *d_out = nullptr;
  int32_t *d_status = nullptr;
  std::vector<Req *> reqs;
  std::vector<uint64_t> req_off;        // first limb of each request in the staging buffers
  uint32_t ops = 0;
};

}  // namespace

struct Server {
  Ctx *ctx = nullptr;
  rsa_server_cfg cfg{};
  std::thread thr;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  bool stop = false;
  uint64_t epoch = 0;
  uint64_t next_ticket = 1;
  std::deque<Req *> queue;                      // not yet admitted, in submission order
  std::unordered_map<uint64_t, Req *> all;      // every request not yet retired
  std::vector<Slot> slots;
  // in-flight requests live in two arenas of mem_budget_bytes at the same
  // offsets: device memory (messages, results, metadata) and pinned host
  // staging for the copies
  void *d_arena = nullptr, *h_arena = nullptr;
  size_t arena_reserved = 0;
  Arena arena;
  uint64_t inflight_bytes = 0, peak_bytes = 0;
  uint64_t inflight_ops = 0, wave_ops = 0;       // operations on the GPU; one multi-lane wave
  size_t busy_cap = 3;                           // batches in flight once a wave is full
  uint64_t pending = 0;                         // submitted and not finished
  // statistics
  std::vector<double> lat_us;
  uint64_t submitted = 0, completed = 0, rejected = 0, ops_completed = 0, batches = 0;
  uint64_t first_arrive = 0, last_done = 0;
  int fatal = 0;

  int init();
  void release();
  void loop();
  bool launch(Slot &s, std::vector<Req *> &batch, uint64_t ops, uint64_t limbs);
  void finish(Slot &s);
};

int Server::init() {
  const int n = cfg.max_inflight_batches;
  if (const char *v = std::getenv("RSAGPU_SERVER_BUSY_CAP")) busy_cap = (size_t)std::max(1, std::atoi(v));
  const size_t budget = (size_t)cfg.mem_budget_bytes / 256 * 256;
  if (budget < batch_bytes(1, 128)) return set_error(RSA_ERR_ARG, "memory budget too small for one request");
  cudaError_t e;
  int rc = ctx->reserve(budget);
  if (rc) return rc;
  arena_reserved = budget;
  if ((e = cudaMalloc(&d_arena, budget)) != cudaSuccess)
    return set_error(RSA_ERR_NOMEM, std::string("server device arena: ") + cudaGetErrorString(e));
  if ((e = cudaMallocHost(&h_arena, budget)) != cudaSuccess) return cuda_error(e, "server pinned arena");
  arena.init(budget);
  slots.resize(n);
  for (Slot &s : slots) {
    if ((e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_error(e, "server stream/event");
    // the ragged path's scratch on this slot's stream, sized for the largest
    // batch now, so no buffer grows (and waits for the device) later
    std::lock_guard<std::mutex> lock(ctx->mu);
    rc = ctx->prepare_batch(s.stream, (uint64_t)cfg.max_batch_ops);
    if (rc) return rc;
    wave_ops = ctx->batch_wave_ops(s.stream);
  }
  return RSA_OK;
}

void Server::release() {
  for (Slot &s : slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.stream) {
      {
        std::lock_guard<std::mutex> lock(ctx->mu);
        ctx->release_stream(s.stream);   // the slot's ragged scratch leaves the budget
      }
      cudaStreamDestroy(s.stream);
    }
  }
  slots.clear();
  if (d_arena) cudaFree(d_arena);
  if (h_arena) cudaFreeHost(h_arena);
  d_arena = h_arena = nullptr;
  if (arena_reserved) ctx->release(arena_reserved);
  arena_reserved = 0;
  for (auto &kv : all) delete kv.second;
  all.clear();
  queue.clear();
}

// Lay the batch out in its arena range [s.off, s.off + s.len), pack it into
// the pinned staging and enqueue copies + the ragged batch on the slot's stream.
bool Server::launch(Slot &s, std::vector<Req *> &batch, uint64_t nops, uint64_t nlimbs) {
  NvtxRange range("server batch");
  {
    char *h = static_cast<char *>(h_arena) + s.off, *d = static_cast<char *>(d_arena) + s.off;
    size_t at = 0;
    auto carve = [&](size_t bytes, void **hp, void **dp) {
      *hp = h + at;
      *dp = d + at;
      at += align256(bytes);
    };
    const uint64_t l4 = (nlimbs + 3) / 4 * 4;
    carve(nops * 4, (void **)&s.h_keys, (void **)&s.d_keys);
    carve(nops, (void **)&s.h_sel, (void **)&s.d_sel);
    carve(nops * 8, (void **)&s.h_off, (void **)&s.d_off);
    carve(nops * 4, (void **)&s.h_status, (void **)&s.d_status);
    carve(l4 * 4, (void **)&s.h_msgs, (void **)&s.d_msgs);
    carve(l4 * 4, (void **)&s.h_out, (void **)&s.d_out);
  }
  uint32_t op = 0;
  uint64_t limb = 0;
  s.reqs = batch;
  s.req_off.clear();
  for (Req *r : s.reqs) {
    const uint32_t step = r->L == 1 ? 1u : r->L;
    limb = r->L == 1 ? limb : (limb + 3) / 4 * 4;
    s.req_off.push_back(limb);
    std::memcpy(s.h_msgs + limb, r->msgs, (size_t)r->count * r->L * 4);
    for (uint32_t i = 0; i < r->count; ++i) {
      s.h_keys[op] = r->key_id;
      s.h_sel[op] = (uint8_t)r->exp_sel;
      s.h_off[op] = limb + (uint64_t)i * step;
      ++op;
    }
    limb += (uint64_t)r->count * r->L;
    r->state = 1;
  }
  cudaStream_t st = s.stream;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(s.d_keys, s.h_keys, (size_t)op * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(s.d_sel, s.h_sel, op, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(s.d_off, s.h_off, (size_t)op * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(s.d_msgs, s.h_msgs, limb * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
    fatal = cuda_error(e, "server H2D");
    return false;
  }
  int rc;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    // the multi-lane (lower latency) shapes while everything in flight fits in
    // one wave of the GPU; past that, the higher-throughput shapes
    const int tuned = ctx->tune_for(0, RSA_TUNE_RAGGED).tpo;
    const int wide = tuned == 4 ? 1 : tuned == 1 ? 0 : (inflight_ops + op <= wave_ops ? 1 : 0);
    rc = ctx->run_batch(op, s.d_keys, s.d_sel, s.d_off, s.d_msgs, s.d_out, s.d_status, st, wide);
  }
  if (rc) {
    fatal = rc;
    return false;
  }
  if ((e = cudaMemcpyAsync(s.h_out, s.d_out, limb * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(s.h_status, s.d_status, (size_t)op * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaEventRecord(s.ev, st)) != cudaSuccess) {
    fatal = cuda_error(e, "server D2H");
    return false;
  }
  s.busy = true;
  s.ops = op;
  inflight_ops += op;
  batches++;
  return true;
}

// Copy results of a completed slot back to the requests' buffers.
void Server::finish(Slot &s) {
  uint32_t op = 0;
  const uint64_t t = now_ns();
  for (size_t k = 0; k < s.reqs.size(); ++k) {
    Req *r = s.reqs[k];
    std::memcpy(r->out, s.h_out + s.req_off[k], (size_t)r->count * r->L * 4);
    int32_t worst = 0;
    for (uint32_t i = 0; i < r->count; ++i) {
      const int32_t v = s.h_status[op + i];
      if (r->status) r->status[i] = v;
      if (v != 0 && worst == 0) worst = v;
    }
    op += r->count;
    r->done = t;
    r->state = 2;
    lat_us.push_back((double)(t - r->arrive) / 1e3);
    completed++;
    ops_completed += r->count;
    last_done = t;
    pending--;
  }
  arena.release(s.off, s.len);
  inflight_bytes -= s.len;
  inflight_ops -= s.ops;
  s.ops = 0;
  s.len = 0;
  s.reqs.clear();
  s.busy = false;
}

void Server::loop() {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lock(mu);
  std::vector<Req *> batch;
  while (true) {
    // 1. retire finished batches
    for (Slot &s : slots) {
      if (s.busy && cudaEventQuery(s.ev) == cudaSuccess) finish(s);
    }
    // on stop, requests whose arrival time has not come are cancelled: never
    // launched, RSA_ERR_TIMEOUT in each of their status entries
    if (stop) {
      const uint64_t now = now_ns();
      for (auto it = queue.begin(); it != queue.end();) {
        Req *r = *it;
        if (r->arrive <= now) {
          ++it;
          continue;
        }
        r->state = RSA_ERR_TIMEOUT;
        if (r->status)
          for (uint32_t i = 0; i < r->count; ++i) r->status[i] = RSA_ERR_TIMEOUT;
        pending--;
        it = queue.erase(it);
      }
    }
    if (pending == 0) done_cv.notify_all();
    if (stop && queue.empty() && std::none_of(slots.begin(), slots.end(), [](const Slot &s) { return s.busy; }))
      break;
    // 2. form a batch for a free slot from requests that have arrived; it is
    //    admitted when its bytes fit in a free range of the in-flight arena
    //    (otherwise it waits for batches in flight to finish)
    // Once the work in flight fills a wave of the GPU, at most busy_cap
    // batches run at once: waiting requests then accumulate into larger
    // batches, whose per-key buckets reach the tensor-core groups; below that,
    // every slot takes a batch at once (low latency).  GB300, the 256-key mix:
    // cap 3 against no cap (16 slots) at 20 k req/s p50/p99 93/164 ms against
    // 157/264, 30 k req/s 751 K ops/s sustained against 658 K, 100 k 1.03 M
    // against 0.97 M; 1 k-10 k req/s unchanged; cap 2 and 4 measured worse.
    const size_t busy_now = (size_t)std::count_if(slots.begin(), slots.end(), [](const Slot &x) { return x.busy; });
    const size_t cap = inflight_ops >= wave_ops ? std::min(busy_cap, slots.size()) : slots.size();
    Slot *free_slot = nullptr;
    if (busy_now < cap)
      for (Slot &s : slots)
        if (!s.busy) {
          free_slot = &s;
          break;
        }
    const uint64_t t = now_ns();
    bool launched = false;
    if (free_slot && !queue.empty() && queue.front()->arrive <= t && !fatal) {
      // A batch carries one modulus size: the oldest waiting request fixes it
      // and requests of other sizes wait for another slot, so a batch finishes
      // at its own size's latency instead of the slowest size's.  Wait
      // (briefly) after that request's arrival for more, unless the batch is
      // full (operations or the largest free range of the arena).
      const uint64_t window = (uint64_t)cfg.batch_window_us * 1000ull;
      const uint64_t first = queue.front()->arrive;
      const uint32_t cls = queue.front()->L;
      const bool mixed = (cfg.flags & RSA_SERVER_MIX_SIZES) != 0;
      const size_t room = arena.largest();
      const uint64_t max_ops = (uint64_t)cfg.max_batch_ops;
      // requests (in queue order) that make up the batch, and whether one more would not fit
      auto gather = [&](std::vector<size_t> *picked, uint64_t *ops_out, uint64_t *limbs_out) {
        uint64_t ops = 0, limbs = 0;
        bool full = false;
        for (size_t qi = 0; qi < queue.size(); ++qi) {
          Req *r = queue[qi];
          if (r->arrive > t) break;
          if (!mixed && r->L != cls) continue;
          const uint64_t l = (r->L == 1 ? limbs : (limbs + 3) / 4 * 4) + (uint64_t)r->count * r->L;
          if (ops + r->count > max_ops || batch_bytes(ops + r->count, l) > room) {
            full = true;
            break;
          }
          ops += r->count;
          limbs = l;
          if (picked) picked->push_back(qi);
        }
        *ops_out = ops;
        *limbs_out = limbs;
        return full;
      };
      uint64_t ops = 0, limbs = 0;
      const bool full = gather(nullptr, &ops, &limbs);
      if (ops > 0 && (full || t >= first + window || stop)) {
        std::vector<size_t> picked;
        gather(&picked, &ops, &limbs);
        // one pass: the picked requests leave the queue in order, the rest keep theirs
        batch.clear();
        std::deque<Req *> rest;
        size_t k = 0;
        for (size_t qi = 0; qi < queue.size(); ++qi) {
          if (k < picked.size() && picked[k] == qi) {
            batch.push_back(queue[qi]);
            ++k;
          } else {
            rest.push_back(queue[qi]);
          }
        }
        queue.swap(rest);
        const size_t need = batch_bytes(ops, limbs);
        size_t off = 0;
        if (!arena.alloc(need, &off)) {
          // cannot happen: `room` is a free range at least this large
          for (Req *r : batch) {
            r->state = RSA_ERR_NOMEM;
            pending--;
          }
          fatal = set_error(RSA_ERR_NOMEM, "server arena allocation failed");
        } else {
          free_slot->off = off;
          free_slot->len = need;
          inflight_bytes += need;
          peak_bytes = std::max(peak_bytes, inflight_bytes);
          lock.unlock();
          const bool ok = launch(*free_slot, batch, ops, limbs);
          lock.lock();
          if (!ok) {
            for (Req *r : batch) {
              r->state = fatal ? fatal : RSA_ERR_CUDA;
              pending--;
            }
            arena.release(off, need);
            inflight_bytes -= need;
            free_slot->len = 0;
          }
        }
        launched = true;
      }
    }
    if (!launched) {
      // sleep until the next arrival, the end of the batching window, or a completion check
      uint64_t wait_ns = 20000;  // poll in-flight events every 20 us
      if (!queue.empty() && queue.front()->arrive > t) wait_ns = std::min<uint64_t>(wait_ns, queue.front()->arrive - t);
      cv.wait_for(lock, std::chrono::nanoseconds(wait_ns));
    }
  }
}

}  // namespace rsagpu

using namespace rsagpu;

static Server *server_of(rsa_ctx *ctx) {
  return ctx ? static_cast<Server *>(reinterpret_cast<Ctx *>(ctx)->server) : nullptr;
}

extern "C" {

int rsa_server_start(rsa_ctx *ctx, const rsa_server_cfg *cfg) {
  if (!ctx) return set_error(RSA_ERR_ARG, "ctx is null");
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (c->server) return set_error(RSA_ERR_ARG, "a server is already running on this context");
  Server *s = new Server();
  s->ctx = c;
  if (cfg) s->cfg = *cfg;
  if (s->cfg.max_inflight_batches <= 0) s->cfg.max_inflight_batches = 16;
  if (s->cfg.batch_window_us <= 0) s->cfg.batch_window_us = 200;
  if (s->cfg.max_batch_ops <= 0) s->cfg.max_batch_ops = 65536;
  if (s->cfg.mem_budget_bytes == 0) s->cfg.mem_budget_bytes = (uint64_t)2 << 30;
  cudaSetDevice(c->device);
  int rc = s->init();
  if (rc) {
    s->release();
    delete s;
    return rc;
  }
  s->epoch = now_ns();
  c->server = s;
  s->thr = std::thread([s] { s->loop(); });
  return RSA_OK;
}

int rsa_server_submit(rsa_ctx *ctx, const rsa_request *req, uint64_t *ticket) {
  Server *s = server_of(ctx);
  if (!s) return set_error(RSA_ERR_ARG, "no server running on this context");
  if (!req || !ticket || (req->count > 0 && (!req->msgs || !req->out)))
    return set_error(RSA_ERR_ARG, "null request field");
  Ctx *c = s->ctx;
  uint32_t L = 0;
  {
    std::lock_guard<std::mutex> lock(c->mu);
    const KeySlot *k = nullptr;
    int rc = c->check_key(req->key_id, req->exp_sel, &k);
    if (rc) return rc;
    L = k->L;
  }
  if (req->count > (uint32_t)s->cfg.max_batch_ops ||
      batch_bytes(req->count, (uint64_t)req->count * L) > s->arena.size()) {
    std::lock_guard<std::mutex> lock(s->mu);
    s->rejected++;
    return set_error(RSA_ERR_NOMEM, "request exceeds the memory budget for requests in flight (or max_batch_ops)");
  }
  Req *r = new Req();
  r->key_id = req->key_id;
  r->exp_sel = req->exp_sel;
  r->count = req->count;
  r->L = L;
  r->msgs = req->msgs;
  r->out = req->out;
  r->status = req->status;
  std::lock_guard<std::mutex> lock(s->mu);
  r->arrive = req->arrive_ns ? s->epoch + req->arrive_ns : now_ns();
  r->ticket = s->next_ticket++;
  if (!s->first_arrive || r->arrive < s->first_arrive) s->first_arrive = r->arrive;
  if (req->count == 0) {
    r->state = 2;
    r->done = r->arrive;
  } else {
    s->queue.push_back(r);
    s->pending++;
  }
  s->all[r->ticket] = r;
  s->submitted++;
  *ticket = r->ticket;
  s->cv.notify_one();
  return RSA_OK;
}

int rsa_server_submit_many(rsa_ctx *ctx, const rsa_request *reqs, uint32_t n, uint64_t *tickets,
                           uint32_t *accepted) {
  if (accepted) *accepted = 0;
  if (!reqs && n) return set_error(RSA_ERR_ARG, "null request array");
  for (uint32_t i = 0; i < n; ++i) {
    uint64_t t = 0;
    const int rc = rsa_server_submit(ctx, &reqs[i], &t);
    if (rc) return rc;
    if (tickets) tickets[i] = t;
    if (accepted) *accepted = i + 1;
  }
  return RSA_OK;
}

int rsa_server_clock(rsa_ctx *ctx, uint64_t *ns) {
  Server *s = server_of(ctx);
  if (!s || !ns) return set_error(RSA_ERR_ARG, "no server or null argument");
  *ns = now_ns() - s->epoch;
  return RSA_OK;
}

int rsa_server_poll(rsa_ctx *ctx, uint64_t ticket, int32_t *done) {
  Server *s = server_of(ctx);
  if (!s || !done) return set_error(RSA_ERR_ARG, "no server or null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return set_error(RSA_ERR_ARG, "unknown ticket");
  const int32_t st = it->second->state;
  *done = st == 2 ? 1 : st < 0 ? st : 0;
  if (st == 2 || st < 0) {
    delete it->second;
    s->all.erase(it);
  }
  return RSA_OK;
}

int rsa_server_drain(rsa_ctx *ctx, int32_t timeout_ms) {
  Server *s = server_of(ctx);
  if (!s) return set_error(RSA_ERR_ARG, "no server running on this context");
  std::unique_lock<std::mutex> lock(s->mu);
  s->cv.notify_one();
  auto pred = [s] { return s->pending == 0; };
  if (timeout_ms <= 0) {
    s->done_cv.wait(lock, pred);
  } else if (!s->done_cv.wait_for(lock, std::chrono::milliseconds(timeout_ms), pred)) {
    return set_error(RSA_ERR_TIMEOUT, "requests still pending after the timeout");
  }
  return s->fatal ? s->fatal : RSA_OK;
}

int rsa_server_get_stats(rsa_ctx *ctx, rsa_server_stats *st, int32_t reset) {
  Server *s = server_of(ctx);
  if (!s || !st) return set_error(RSA_ERR_ARG, "no server or null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->rejected = s->rejected;
  st->ops_completed = s->ops_completed;
  st->batches = s->batches;
  st->peak_bytes = s->peak_bytes;
  if (!s->lat_us.empty()) {
    std::vector<double> v = s->lat_us;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    st->p50_us = pct(0.50);
    st->p99_us = pct(0.99);
    st->max_us = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    st->mean_us = sum / v.size();
  }
  if (s->last_done > s->first_arrive) st->span_s = (double)(s->last_done - s->first_arrive) / 1e9;
  if (reset) {
    s->lat_us.clear();
    s->submitted = s->completed = s->rejected = s->ops_completed = s->batches = 0;
    s->peak_bytes = s->inflight_bytes;
    s->first_arrive = s->last_done = 0;
  }
  return RSA_OK;
}

int rsa_server_stop(rsa_ctx *ctx) {
  Server *s = server_of(ctx);
  if (!s) return set_error(RSA_ERR_ARG, "no server running on this context");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_one();
  if (s->thr.joinable()) s->thr.join();
  s->release();
  reinterpret_cast<Ctx *>(ctx)->server = nullptr;
  delete s;
  return RSA_OK;
}

}  // extern "C"
